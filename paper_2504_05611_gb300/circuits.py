"""Circuit generator for distributed transversal operations.

Builds the noisy Clifford op lists that the sampler consumes: rotated
surface-code (SC) and bivariate-bicycle (BB) code blocks, their syndrome
extraction rounds, the non-local transversal CNOT (gate teleportation through
ebit pairs) and logical teleportation across three blocks, with the paper's
circuit-level noise model.

Paper sections this module restates (arXiv 2504.05611):
  * Supplementary Note 1 (symplectic Pauli encoding, CSS check matrices).
  * Supplementary "Surface Codes" (rotated d x d lattice, weight-4 bulk and
    weight-2 boundary plaquettes, weight-d logical strings).
  * Supplementary "Bivariate Bicycle Codes" (x = S_l (x) I_m, y = I_l (x) S_m,
    H_X = [A|B], H_Z = [B^T|A^T]) and Supplementary Table S1 (parameters).
  * Methods "Simulation" (noise model), "Non-local CNOT circuit",
    "State teleportation circuit", Fig. 1(b,c).

This module is an input generator: it emits op lists and holds none of the
sampling arithmetic (frames, noise draws, parities). Both the CUDA sampler
and the CPU oracle consume what it produces.

Op-list conventions (shared with the C ABI):
  * targets are qubit ids; CX and DEPOLARIZE2 take (a, b) pairs;
  * M / MX append one measurement record per target, in target order;
  * DETECTOR and OBSERVABLE targets are absolute record indices;
    OBSERVABLE's ``arg`` is the observable id;
  * XFEED / ZFEED take (record, qubit) pairs: a classically conditioned
    X (resp. Z) on ``qubit`` when ``record`` reads 1;
  * TICK is a layer hint with no effect.
"""

from __future__ import annotations

import dataclasses
import math
import re
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

OPCODES: Tuple[str, ...] = (
    "R", "RX", "H", "S", "CX", "M", "MX",
    "X_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2",
    "XFEED", "ZFEED", "DETECTOR", "OBSERVABLE", "TICK",
    "PAULI_CHANNEL_1",
)
OPCODE_ID: Dict[str, int] = {name: i for i, name in enumerate(OPCODES)}
NOISE_OPS = frozenset({"X_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2", "PAULI_CHANNEL_1"})
PAIR_OPS = frozenset({"CX", "DEPOLARIZE2", "XFEED", "ZFEED"})
QUBIT_OPS = frozenset({"R", "RX", "H", "S", "CX", "M", "MX",
                       "X_ERROR", "Z_ERROR", "DEPOLARIZE1", "DEPOLARIZE2", "PAULI_CHANNEL_1"})


def pauli_channel_thresholds(px: float, py: float, pz: float) -> Tuple[float, int, int]:
    """PAULI_CHANNEL_1(px, py, pz) as (p, t1, t2): an event happens with
    probability p = px + py + pz; its Pauli is X if w < t1, Y if w < t2, else
    Z, for a uniform 32-bit word w, with t1 = floor(2^32 px / p) and
    t2 = floor(2^32 (px + py) / p) (both capped at 2^32 - 1), i.e. the
    conditional split is quantised to 2^-32."""
    for v in (px, py, pz):
        if not (0.0 <= v <= 1.0):
            raise ValueError("PAULI_CHANNEL_1 probabilities must lie in [0, 1]")
    p = px + py + pz
    if p > 1.0 + 1e-12:
        raise ValueError("PAULI_CHANNEL_1 probabilities sum above 1")
    p = min(p, 1.0)
    if p == 0.0:
        return 0.0, 0, 0
    cap = 2 ** 32 - 1
    t1 = min(cap, int(math.floor(2.0 ** 32 * px / p)))
    t2 = min(cap, int(math.floor(2.0 ** 32 * (px + py) / p)))
    return p, t1, t2


@dataclasses.dataclass
class Op:
    """One instruction of an op list.

    ``tag`` is generator bookkeeping ("gate", "prep", "readout", "noise",
    "ebit", "init", ...); it is not part of the C ABI and has no effect on
    sampling.
    """

    name: str
    targets: np.ndarray
    p: float = 0.0
    arg: int = 0
    tag: str = ""
    arg2: int = 0
    channel: Optional[Tuple[float, float, float]] = None  # PAULI_CHANNEL_1 (px, py, pz)


class Circuit:
    """An op list plus running counts of qubits, records, detectors and
    observables."""

    def __init__(self) -> None:
        self.ops: List[Op] = []
        self.n_qubits = 0
        self.n_meas = 0
        self.n_det = 0
        self.n_obs = 0
        self.meta: Dict[str, object] = {}

    # -- construction -------------------------------------------------------
    def append(self, name: str, targets: Iterable[int] = (), p=0.0,
               arg: int = 0, tag: str = "") -> np.ndarray:
        """Append one op; returns the record indices an M/MX op creates
        (empty otherwise). PAULI_CHANNEL_1 takes p = (px, py, pz)."""
        if name not in OPCODE_ID:
            raise ValueError(f"unknown op {name!r}")
        channel = None
        arg2 = 0
        if name == "PAULI_CHANNEL_1":
            channel = tuple(float(v) for v in p)
            if len(channel) != 3:
                raise ValueError("PAULI_CHANNEL_1 needs (px, py, pz)")
            p, arg, arg2 = pauli_channel_thresholds(*channel)
        t = np.asarray(list(targets) if not isinstance(targets, np.ndarray) else targets,
                       dtype=np.int64).ravel()
        if t.size and t.min() < 0:
            raise ValueError(f"{name}: negative target")
        if name in PAIR_OPS and t.size % 2:
            raise ValueError(f"{name}: odd number of targets")
        if name in NOISE_OPS and not (0.0 <= p <= 1.0):
            raise ValueError(f"{name}: probability {p} outside [0, 1]")
        if name in ("DETECTOR", "OBSERVABLE") and t.size and t.max() >= self.n_meas:
            raise ValueError(f"{name}: record index beyond {self.n_meas}")
        if name in ("XFEED", "ZFEED") and t.size and t[0::2].max() >= self.n_meas:
            raise ValueError(f"{name}: record index beyond {self.n_meas}")
        t = t.astype(np.uint32)
        self.ops.append(Op(name, t, float(p), int(arg), tag, int(arg2), channel))
        if name in QUBIT_OPS and t.size:
            self.n_qubits = max(self.n_qubits, int(t.max()) + 1)
        if name in ("XFEED", "ZFEED") and t.size:
            self.n_qubits = max(self.n_qubits, int(t[1::2].max()) + 1)
        recs = np.empty(0, dtype=np.int64)
        if name in ("M", "MX"):
            recs = np.arange(self.n_meas, self.n_meas + t.size, dtype=np.int64)
            self.n_meas += t.size
        elif name == "DETECTOR":
            self.n_det += 1
        elif name == "OBSERVABLE":
            self.n_obs = max(self.n_obs, int(arg) + 1)
        return recs

    # -- text format --------------------------------------------------------
    def to_text(self) -> str:
        """Project text format: ``NAME[(p)] t0 t1 ...`` per line;
        OBSERVABLE carries its id in the parentheses."""
        lines = []
        for op in self.ops:
            head = op.name
            if op.name == "PAULI_CHANNEL_1":
                head += "(" + ",".join(repr(v) for v in op.channel) + ")"
            elif op.name in NOISE_OPS:
                head += f"({op.p!r})"
            elif op.name == "OBSERVABLE":
                head += f"({op.arg})"
            body = " ".join(str(int(x)) for x in op.targets)
            lines.append(f"{head} {body}".rstrip())
        return "\n".join(lines) + "\n"

    @staticmethod
    def from_text(text: str) -> "Circuit":
        c = Circuit()
        pat = re.compile(r"^([A-Z_0-9]+)(?:\(([^)]*)\))?\s*(.*)$")
        for lineno, raw in enumerate(text.splitlines(), 1):
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            m = pat.match(line)
            if not m:
                raise ValueError(f"line {lineno}: cannot parse {raw!r}")
            name, par, rest = m.group(1), m.group(2), m.group(3)
            targets = [int(x) for x in rest.split()] if rest else []
            p, arg = 0.0, 0
            if par is not None:
                if name == "OBSERVABLE":
                    arg = int(par)
                elif name == "PAULI_CHANNEL_1":
                    p = tuple(float(v) for v in par.split(","))
                else:
                    p = float(par)
            c.append(name, targets, p=p, arg=arg)
        return c

    def __len__(self) -> int:
        return len(self.ops)


# ---------------------------------------------------------------------------
# GF(2) linear algebra (code construction only)
# ---------------------------------------------------------------------------

def gf2_rref(m: np.ndarray) -> Tuple[np.ndarray, List[int]]:
    """Reduced row echelon form over GF(2); returns (rref, pivot columns)."""
    a = (np.asarray(m, dtype=np.uint8) & 1).copy()
    rows, cols = a.shape
    pivots: List[int] = []
    r = 0
    for c in range(cols):
        if r >= rows:
            break
        nz = np.nonzero(a[r:, c])[0]
        if nz.size == 0:
            continue
        pr = r + int(nz[0])
        if pr != r:
            a[[r, pr]] = a[[pr, r]]
        others = np.nonzero(a[:, c])[0]
        others = others[others != r]
        if others.size:
            a[others] ^= a[r]
        pivots.append(c)
        r += 1
    return a[:r], pivots


def gf2_rank(m: np.ndarray) -> int:
    if np.asarray(m).size == 0:
        return 0
    return len(gf2_rref(m)[1])


def gf2_nullspace(m: np.ndarray) -> np.ndarray:
    """Basis (rows) of {v : m v = 0} over GF(2)."""
    m = np.asarray(m, dtype=np.uint8) & 1
    cols = m.shape[1]
    r, piv = gf2_rref(m)
    free = [c for c in range(cols) if c not in set(piv)]
    basis = np.zeros((len(free), cols), dtype=np.uint8)
    for i, f in enumerate(free):
        basis[i, f] = 1
        for row, pc in enumerate(piv):
            if r[row, f]:
                basis[i, pc] = 1
    return basis


def logical_basis(h_comm: np.ndarray, h_stab: np.ndarray) -> List[np.ndarray]:
    """Independent representatives of ker(h_comm) / rowspace(h_stab).

    For Z logicals pass (H_X, H_Z): Z-type operators that commute with every
    X check and are not products of Z checks (Supplementary Note 1).
    The basis is chosen greedily from the RREF null-space basis in column
    order, so it is deterministic; it is not unique.
    """
    null = gf2_nullspace(h_comm)
    chosen: List[np.ndarray] = []
    base = np.asarray(h_stab, dtype=np.uint8) & 1
    cur_rank = gf2_rank(base)
    for v in null:
        trial = np.vstack([base] + chosen + [v[None, :]]) if chosen else np.vstack([base, v[None, :]])
        rk = gf2_rank(trial)
        if rk > cur_rank:
            chosen.append(v[None, :])
            cur_rank = rk
    return [np.nonzero(v.ravel())[0].astype(np.int64) for v in chosen]


# ---------------------------------------------------------------------------
# Codes
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class CSSCode:
    """A CSS code with a syndrome-extraction CX schedule.

    ``x_layers[t]`` lists (x_check, data) pairs whose CX (ancilla -> data)
    runs in CX layer t of the X sub-schedule; ``z_layers[t]`` lists
    (z_check, data) pairs whose CX (data -> ancilla) runs in layer t of the
    Z sub-schedule. ``interleaved`` runs X layer t and Z layer t together.
    """

    name: str
    n: int
    d: int
    hx: np.ndarray
    hz: np.ndarray
    x_layers: List[List[Tuple[int, int]]]
    z_layers: List[List[Tuple[int, int]]]
    interleaved: bool
    z_logicals: List[np.ndarray]
    x_logicals: List[np.ndarray]

    @property
    def k(self) -> int:
        return self.n - gf2_rank(self.hx) - gf2_rank(self.hz)

    @property
    def n_xchecks(self) -> int:
        return self.hx.shape[0]

    @property
    def n_zchecks(self) -> int:
        return self.hz.shape[0]

    def z_support(self, i: int) -> np.ndarray:
        return np.nonzero(self.hz[i])[0]


def rotated_surface_code(d: int) -> CSSCode:
    """Rotated surface code [[d^2, 1, d]] (Supplementary "Surface Codes").

    Data qubit (x, y) has index y*d + x. A plaquette with north-west corner
    (x, y), x, y in [-1, d-1], touches the data corners NW (x,y), NE (x+1,y),
    SW (x,y+1), SE (x+1,y+1) that lie on the lattice. Bulk plaquettes are
    Z-type when x+y is even and X-type otherwise; weight-2 plaquettes are
    kept only on the top/bottom edges for X type and on the left/right edges
    for Z type. Z_L is the top row, X_L the left column (weight d each).

    CX order (hook-avoiding, an assumption: the paper defers the schedule to
    Stim's generated circuits): X checks visit NW, NE, SW, SE ("Z" shape),
    so a mid-schedule ancilla X fault leaves a horizontal XX pair,
    perpendicular to the vertical X_L; Z checks visit NW, SW, NE, SE ("N"
    shape), leaving a vertical ZZ pair, perpendicular to the horizontal Z_L.
    """
    if d < 3 or d % 2 == 0:
        raise ValueError("rotated surface code needs odd d >= 3")
    n = d * d
    idx = lambda x, y: y * d + x  # noqa: E731
    xchecks: List[List[Optional[int]]] = []
    zchecks: List[List[Optional[int]]] = []
    for y in range(-1, d):
        for x in range(-1, d):
            corners = [(x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1)]
            inside = [idx(cx, cy) if (0 <= cx < d and 0 <= cy < d) else None
                      for cx, cy in corners]
            w = sum(c is not None for c in inside)
            typ = "Z" if (x + y) % 2 == 0 else "X"
            if w == 4:
                pass
            elif w == 2:
                top_bottom = y in (-1, d - 1)
                if top_bottom and typ != "X":
                    continue
                if not top_bottom and typ != "Z":
                    continue
            else:
                continue
            (xchecks if typ == "X" else zchecks).append(inside)
    hx = np.zeros((len(xchecks), n), dtype=np.uint8)
    hz = np.zeros((len(zchecks), n), dtype=np.uint8)
    for i, cs in enumerate(xchecks):
        for q in cs:
            if q is not None:
                hx[i, q] = 1
    for i, cs in enumerate(zchecks):
        for q in cs:
            if q is not None:
                hz[i, q] = 1
    x_order = (0, 1, 2, 3)  # NW, NE, SW, SE
    z_order = (0, 2, 1, 3)  # NW, SW, NE, SE
    x_layers = [[(i, cs[c]) for i, cs in enumerate(xchecks) if cs[c] is not None] for c in x_order]
    z_layers = [[(i, cs[c]) for i, cs in enumerate(zchecks) if cs[c] is not None] for c in z_order]
    zl = [np.array([idx(x, 0) for x in range(d)], dtype=np.int64)]
    xl = [np.array([idx(0, y) for y in range(d)], dtype=np.int64)]
    return CSSCode(f"SC[[{n},1,{d}]]", n, d, hx, hz, x_layers, z_layers, True, zl, xl)


Monomial = Tuple[int, int]  # (power of x, power of y)

# Supplementary Table S1: (l, m, a(x,y), b(x,y)) with nominal distance.
BB_TABLE_S1: Dict[str, Tuple[int, int, Tuple[Monomial, ...], Tuple[Monomial, ...], int]] = {
    "bb18": (3, 3, ((0, 0), (1, 0), (0, 1)), ((0, 0), (2, 0), (0, 2)), 4),
    "bb36": (3, 6, ((1, 0), (0, 2), (0, 3)), ((0, 0), (2, 0), (0, 1)), 6),
    "bb54": (3, 9, ((1, 0), (0, 1), (0, 3)), ((0, 0), (2, 0), (0, 2)), 8),
    "bb90": (15, 3, ((9, 0), (0, 1), (0, 2)), ((0, 0), (2, 0), (7, 0)), 10),
    "bb144": (12, 6, ((3, 0), (0, 1), (0, 2)), ((1, 0), (2, 0), (0, 3)), 12),
}


def bb_code(l: int, m: int, a: Sequence[Monomial], b: Sequence[Monomial],
            d: int = 0, name: str = "") -> CSSCode:
    """Bivariate bicycle code (Supplementary "Bivariate Bicycle Codes").

    x = S_l (x) I_m and y = I_l (x) S_m with S_j the cyclic shift
    (S_j[i, i+1 mod j] = 1); A = a(x, y), B = b(x, y); H_X = [A|B],
    H_Z = [B^T|A^T]. Data index r1*m + r2 for the left (A) half, lm + that
    for the right (B) half; check index r1*m + r2.

    Schedule (the paper's depth-8 interleaving from Bravyi et al. is not
    reproduced; this is this project's own valid schedule): each monomial of
    A and B is a permutation, so the X sub-round is 6 CX layers, one per
    monomial (A terms on the left half, then B terms on the right half), and
    the Z sub-round is 6 more (B^T terms on the left, then A^T terms on the
    right). X and Z sub-rounds run one after the other.
    """
    lm = l * m

    def shift(r: int, mono: Monomial, sign: int) -> int:
        r1, r2 = divmod(r, m)
        return ((r1 + sign * mono[0]) % l) * m + (r2 + sign * mono[1]) % m

    def mat(poly: Sequence[Monomial]) -> np.ndarray:
        out = np.zeros((lm, lm), dtype=np.uint8)
        for mono in poly:
            for r in range(lm):
                out[r, shift(r, mono, +1)] ^= 1
        return out

    A, B = mat(a), mat(b)
    hx = np.hstack([A, B])
    hz = np.hstack([B.T, A.T])
    x_layers = [[(r, shift(r, mono, +1)) for r in range(lm)] for mono in a]
    x_layers += [[(r, lm + shift(r, mono, +1)) for r in range(lm)] for mono in b]
    z_layers = [[(r, shift(r, mono, -1)) for r in range(lm)] for mono in b]
    z_layers += [[(r, lm + shift(r, mono, -1)) for r in range(lm)] for mono in a]
    zl = logical_basis(hx, hz)
    xl = logical_basis(hz, hx)
    n = 2 * lm
    code = CSSCode(name or f"BB[[{n},{len(zl)},{d}]]", n, d, hx, hz,
                   x_layers, z_layers, False, zl, xl)
    return code


def bb_from_table(key: str) -> CSSCode:
    l, m, a, b, d = BB_TABLE_S1[key]
    code = bb_code(l, m, a, b, d=d)
    code.name = f"BB[[{code.n},{code.k},{d}]]"
    return code


def code_by_name(name: str) -> CSSCode:
    """``sc<d>`` (rotated surface code) or a key of Supplementary Table S1."""
    if name.startswith("sc"):
        return rotated_surface_code(int(name[2:]))
    if name in BB_TABLE_S1:
        return bb_from_table(name)
    raise ValueError(f"unknown code {name!r}")


# ---------------------------------------------------------------------------
# Circuit builder
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Block:
    code: CSSCode
    data: np.ndarray
    xanc: np.ndarray
    zanc: np.ndarray
    name: str = ""


@dataclasses.dataclass
class Decoherence:
    """Ebit decoherence while ebits wait for use (Methods "Decoherence").

    Each ebit is aged by the time between its generation and the end of
    generation of all n ebits, and both of its halves get
    PAULI_CHANNEL_1(p_X, p_Y, p_Z) with p_X = p_Y = (1 - e^{-t/T1}) / 4 and
    p_Z = (1 - e^{-t/T2}) / 2 - (1 - e^{-t/T1}) / 4 (the paper takes
    T1 = T2). Schedules:
      * "serial": one ebit per time step t_gen; ebit j (1..n) has age
        (n - j) t_gen;
      * "lines": ``lines`` ebits per time step (default: d for surface codes,
        the divisor of n closest to d for BB codes); the L = ceil(n / f)
        lines are generated in order and line l (1..L) has age (L - l) t_gen.
        (The text's formula for this case repeats the serial one; this is the
        reading used here.)
    Ages are in units of T1 through ``t_gen_over_t1``.
    """

    t_gen_over_t1: float
    t2_over_t1: float = 1.0
    schedule: str = "serial"
    lines: int = 0


def decoherence_paulis(t_over_t1: float, t_over_t2: float) -> Tuple[float, float, float]:
    """(p_X, p_Y, p_Z) of an idle period t (Methods "Decoherence")."""
    a = -math.expm1(-t_over_t1)
    b = -math.expm1(-t_over_t2)
    return a / 4.0, a / 4.0, b / 2.0 - a / 4.0


def line_width(code: "CSSCode", n: int) -> int:
    """Ebits generated per time step in the line schedule: d for the surface
    code; for BB codes the divisor of n closest to d (ties: the smaller)."""
    if code.name.startswith("SC"):
        return max(1, code.d)
    divs = [f for f in range(1, n + 1) if n % f == 0]
    return min(divs, key=lambda f: (abs(f - code.d), f))


def ebit_ages(code: "CSSCode", n: int, dec: Decoherence) -> List[int]:
    """Age of ebit j (index 0..n-1) in units of t_gen."""
    if dec.schedule == "serial":
        return [n - 1 - j for j in range(n)]
    if dec.schedule == "lines":
        f = dec.lines or line_width(code, n)
        L = (n + f - 1) // f
        return [L - 1 - j // f for j in range(n)]
    raise ValueError(f"unknown ebit schedule {dec.schedule!r}")


@dataclasses.dataclass
class NoiseModel:
    """Methods "Simulation": p on gates, resets and measurements; p_ebit on
    freshly prepared ebit pairs.

    Readings where the paper is silent or garbled:
      * every R is followed by X_ERROR(p) and every RX by Z_ERROR(p) (block
        qubits only; ebit preparation is perfect);
      * measurement flips are X_ERROR(p) before M and Z_ERROR(p) before MX,
        on block qubits and ebits;
      * DEPOLARIZE1(p) after every noisy H, DEPOLARIZE2(p) after every noisy
        CX (including the ebit-data CX);
      * classically conditioned Paulis are noiseless unless ``feed_noise``;
      * idle DEPOLARIZE1(p) on block qubits untouched by a CX layer only when
        ``idle`` is set (off by default).
    """

    p: float = 1e-3
    p_ebit: float = 1e-2
    idle: bool = False
    feed_noise: bool = False
    decoherence: Optional[Decoherence] = None


class Builder:
    def __init__(self, noise: NoiseModel):
        self.c = Circuit()
        self.noise = noise
        self.nq = 0

    def qubits(self, count: int) -> np.ndarray:
        ids = np.arange(self.nq, self.nq + count, dtype=np.int64)
        self.nq += count
        return ids

    def block(self, code: CSSCode, name: str = "") -> Block:
        data = self.qubits(code.n)
        xanc = self.qubits(code.n_xchecks)
        zanc = self.qubits(code.n_zchecks)
        return Block(code, data, xanc, zanc, name)

    def op(self, name: str, targets, p: float = 0.0, arg: int = 0, tag: str = "gate") -> np.ndarray:
        return self.c.append(name, np.asarray(targets, dtype=np.int64), p=p, arg=arg, tag=tag)

    def err(self, name: str, targets, p: float, tag: str = "noise") -> None:
        targets = np.asarray(targets, dtype=np.int64)
        if targets.size and p > 0.0:
            self.c.append(name, targets, p=p, tag=tag)

    # -- pieces -------------------------------------------------------------
    def reset_data(self, blocks: Sequence[Block]) -> None:
        data = np.concatenate([b.data for b in blocks])
        self.op("R", data, tag="init")
        self.err("X_ERROR", data, self.noise.p)

    def syndrome_round(self, blocks: Sequence[Block]) -> Dict[int, np.ndarray]:
        """One syndrome-extraction round on ``blocks`` (run in parallel).

        Returns, per block position, the record indices of its Z checks in
        check order."""
        p = self.noise.p
        zanc = np.concatenate([b.zanc for b in blocks])
        xanc = np.concatenate([b.xanc for b in blocks])
        self.op("R", zanc, tag="reset")
        self.op("RX", xanc, tag="reset")
        self.err("X_ERROR", zanc, p)
        self.err("Z_ERROR", xanc, p)
        code = blocks[0].code
        if code.interleaved:
            layers = [(code.x_layers[t], code.z_layers[t]) for t in range(len(code.x_layers))]
        else:
            layers = [(xl, []) for xl in code.x_layers] + [([], zl) for zl in code.z_layers]
        for xl, zl in layers:
            pairs = []
            for b in blocks:
                for chk, dq in xl:
                    pairs += [b.xanc[chk], b.data[dq]]
                for chk, dq in zl:
                    pairs += [b.data[dq], b.zanc[chk]]
            self.op("TICK", [], tag="tick")
            self.op("CX", pairs, tag="gate")
            self.err("DEPOLARIZE2", pairs, p)
            if self.noise.idle:
                busy = set(int(q) for q in pairs)
                allq = np.concatenate([np.concatenate([b.data, b.xanc, b.zanc]) for b in blocks])
                idle = [int(q) for q in allq if int(q) not in busy]
                self.err("DEPOLARIZE1", idle, p, tag="idle")
        self.op("TICK", [], tag="tick")
        self.err("X_ERROR", zanc, p)
        self.err("Z_ERROR", xanc, p)
        recs = self.op("M", zanc, tag="meas")
        self.op("MX", xanc, tag="meas")
        out: Dict[int, np.ndarray] = {}
        off = 0
        for i, b in enumerate(blocks):
            out[i] = recs[off:off + b.code.n_zchecks]
            off += b.code.n_zchecks
        return out

    def round_detectors(self, block: Block, recs: np.ndarray, prev: Optional[np.ndarray],
                        extra: Optional[List[List[int]]]) -> None:
        for i in range(block.code.n_zchecks):
            t = [int(recs[i])]
            if prev is not None:
                t.append(int(prev[i]))
            if extra is not None:
                t += extra[i]
            self.op("DETECTOR", t, tag="det")

    def final_detectors(self, block: Block, data_recs: np.ndarray, prev: Optional[np.ndarray],
                        extra: Optional[List[List[int]]]) -> None:
        for i in range(block.code.n_zchecks):
            t = [int(data_recs[j]) for j in block.code.z_support(i)]
            if prev is not None:
                t.append(int(prev[i]))
            if extra is not None:
                t += extra[i]
            self.op("DETECTOR", t, tag="det")

    def observables(self, block: Block, data_recs: np.ndarray, first_id: int) -> int:
        for j, zl in enumerate(block.code.z_logicals):
            self.op("OBSERVABLE", [int(data_recs[q]) for q in zl], arg=first_id + j, tag="obs")
        return first_id + len(block.code.z_logicals)

    def measure_data(self, blocks: Sequence[Block], tag: str) -> List[np.ndarray]:
        data = np.concatenate([b.data for b in blocks])
        self.err("X_ERROR", data, self.noise.p)
        recs = self.op("M", data, tag=tag)
        out, off = [], 0
        for b in blocks:
            out.append(recs[off:off + b.code.n])
            off += b.code.n
        return out

    def nonlocal_cnot_core(self, ctrl: Block, targ: Block) -> None:
        """Methods "Non-local CNOT circuit" and Fig. 1(b): gate teleportation
        of a transversal CNOT ctrl -> targ through n ebit pairs.

        Ebits (e_A on the control's module, e_B on the target's) are prepared
        perfectly as Bell pairs and then depolarized with p_ebit. Then:
        CX(ctrl_k -> e_A_k); measure e_A_k (Z); X on e_B_k conditioned on it;
        CX(e_B_k -> targ_k); H on e_B_k; measure e_B_k (Z); Z on ctrl_k
        conditioned on it. The conditioned Z is placed on the control side,
        as in the standard gate-teleported CNOT (the text names the other
        block; for Z-basis detectors and readout the two are equivalent when
        the conditioned Paulis are noiseless).
        """
        nz = self.noise
        n = ctrl.code.n
        ea = self.qubits(n)
        eb = self.qubits(n)
        bell = np.stack([ea, eb], axis=1).ravel()
        self.op("R", np.concatenate([ea, eb]), tag="prep")
        self.op("H", ea, tag="prep")
        self.op("CX", bell, tag="prep")
        self.err("DEPOLARIZE2", bell, nz.p_ebit, tag="ebit")
        if nz.decoherence is not None:
            dec = nz.decoherence
            ages = ebit_ages(ctrl.code, n, dec)
            for age in sorted(set(ages), reverse=True):
                if age == 0:
                    continue
                t = age * dec.t_gen_over_t1
                ch = decoherence_paulis(t, t / dec.t2_over_t1)
                js = [j for j in range(n) if ages[j] == age]
                qs = np.concatenate([ea[js], eb[js]])
                self.c.append("PAULI_CHANNEL_1", qs, p=ch, tag="ebit")
        self.op("TICK", [], tag="tick")
        pairs1 = np.stack([ctrl.data, ea], axis=1).ravel()
        self.op("CX", pairs1, tag="gate")
        self.err("DEPOLARIZE2", pairs1, nz.p)
        self.err("X_ERROR", ea, nz.p)
        ra = self.op("M", ea, tag="meas")
        self.op("XFEED", np.stack([ra, eb], axis=1).ravel(), tag="gate")
        if nz.feed_noise:
            self.err("DEPOLARIZE1", eb, nz.p)
        self.op("TICK", [], tag="tick")
        pairs2 = np.stack([eb, targ.data], axis=1).ravel()
        self.op("CX", pairs2, tag="gate")
        self.err("DEPOLARIZE2", pairs2, nz.p)
        self.op("H", eb, tag="gate")
        self.err("DEPOLARIZE1", eb, nz.p)
        self.err("X_ERROR", eb, nz.p)
        rb = self.op("M", eb, tag="meas")
        self.op("ZFEED", np.stack([rb, ctrl.data], axis=1).ravel(), tag="gate")
        if nz.feed_noise:
            self.err("DEPOLARIZE1", ctrl.data, nz.p)
        self.op("TICK", [], tag="tick")


def nonlocal_cnot_circuit(code: CSSCode, rounds_before: int = 4, rounds_after: int = 3,
                          noise: Optional[NoiseModel] = None) -> Circuit:
    """Methods "Non-local CNOT circuit": noisy |0_L> init of CB1 and CB2,
    ``rounds_before`` rounds on both, the non-local transversal CNOT
    CB1 -> CB2, ``rounds_after`` rounds on both, Z-basis readout.

    Detectors are on Z checks only (Methods). The first CB2 detector after
    the CNOT also takes CB1's last pre-CNOT record of the same check: under
    the transversal CNOT a target Z check maps to the product of itself and
    the control's check. Observables: Z_L of every logical of CB1, then of
    CB2 (2k in total, Methods "Decoding").
    """
    noise = noise or NoiseModel()
    b = Builder(noise)
    cb1, cb2 = b.block(code, "CB1"), b.block(code, "CB2")
    b.reset_data([cb1, cb2])
    prev: List[Optional[np.ndarray]] = [None, None]
    extra: List[Optional[List[List[int]]]] = [None, None]
    for _ in range(rounds_before):
        recs = b.syndrome_round([cb1, cb2])
        for i, blk in enumerate((cb1, cb2)):
            b.round_detectors(blk, recs[i], prev[i], extra[i])
            prev[i], extra[i] = recs[i], None
    b.nonlocal_cnot_core(cb1, cb2)
    if prev[0] is not None:
        extra[1] = [[int(prev[0][i])] for i in range(code.n_zchecks)]
    for _ in range(rounds_after):
        recs = b.syndrome_round([cb1, cb2])
        for i, blk in enumerate((cb1, cb2)):
            b.round_detectors(blk, recs[i], prev[i], extra[i])
            prev[i], extra[i] = recs[i], None
    d1, d2 = b.measure_data([cb1, cb2], tag="readout")
    b.final_detectors(cb1, d1, prev[0], extra[0])
    b.final_detectors(cb2, d2, prev[1], extra[1])
    nxt = b.observables(cb1, d1, 0)
    b.observables(cb2, d2, nxt)
    b.c.meta.update(op="nl", code=code.name, rounds=(rounds_before, rounds_after),
                    p=noise.p, p_ebit=noise.p_ebit, n=code.n, k=code.k)
    return b.c


def teleport_circuit(code: CSSCode, rounds_before: int = 4, rounds_after: int = 3,
                     noise: Optional[NoiseModel] = None) -> Circuit:
    """Methods "State teleportation circuit" and Fig. 1(c).

    CB1, CB2, CB3 are noisily initialised in |0_L>; ``rounds_before`` rounds
    on all three; transversal H on CB2; non-local CNOT CB2 -> CB3 (logical
    Bell pairs); logical Bell measurement of CB1 with CB2 (transversal CX
    CB1 -> CB2, transversal H on CB1, Z-basis measurement of both);
    transversal corrections on CB3: X on qubit k conditioned on CB2's
    qubit-k outcome and Z on qubit k conditioned on CB1's qubit-k outcome
    (n conditioned gates each, matching the paper's 7n single-qubit count);
    ``rounds_after`` rounds on CB3; Z-basis readout of CB3.

    No rounds run on CB1 or CB2 after the first H (Methods
    "Transversality"), so they carry no final-layer detectors. The first CB3
    detector after the corrections is m_CB3,post + m_CB3,pre + m_CB1,pre:
    propagating CB3's check backwards, the non-local CNOT contributes CB2's
    (random) check parity, the conditioned X corrections contribute the CB2
    outcomes on the support, and those outcomes equal CB1's check parity plus
    the same CB2 parity (transversal CX CB1 -> CB2), so only CB1's last
    record remains. Observables: Z_L of each logical of CB3 (k in total).
    """
    noise = noise or NoiseModel()
    b = Builder(noise)
    cb1, cb2, cb3 = b.block(code, "CB1"), b.block(code, "CB2"), b.block(code, "CB3")
    blocks = [cb1, cb2, cb3]
    b.reset_data(blocks)
    prev: List[Optional[np.ndarray]] = [None, None, None]
    for _ in range(rounds_before):
        recs = b.syndrome_round(blocks)
        for i, blk in enumerate(blocks):
            b.round_detectors(blk, recs[i], prev[i], None)
            prev[i] = recs[i]
    p = noise.p
    b.op("H", cb2.data, tag="gate")
    b.err("DEPOLARIZE1", cb2.data, p)
    b.nonlocal_cnot_core(cb2, cb3)
    pairs = np.stack([cb1.data, cb2.data], axis=1).ravel()
    b.op("CX", pairs, tag="gate")
    b.err("DEPOLARIZE2", pairs, p)
    b.op("H", cb1.data, tag="gate")
    b.err("DEPOLARIZE1", cb1.data, p)
    m1, m2 = b.measure_data([cb1, cb2], tag="meas")
    b.op("XFEED", np.stack([m2, cb3.data], axis=1).ravel(), tag="gate")
    b.op("ZFEED", np.stack([m1, cb3.data], axis=1).ravel(), tag="gate")
    if noise.feed_noise:
        b.err("DEPOLARIZE1", cb3.data, p)
    b.op("TICK", [], tag="tick")
    extra3: Optional[List[List[int]]] = None
    if prev[0] is not None:
        extra3 = [[int(prev[0][i])] for i in range(code.n_zchecks)]
    prev3 = prev[2]
    for _ in range(rounds_after):
        recs = b.syndrome_round([cb3])
        b.round_detectors(cb3, recs[0], prev3, extra3)
        prev3, extra3 = recs[0], None
    (d3,) = b.measure_data([cb3], tag="readout")
    b.final_detectors(cb3, d3, prev3, extra3)
    b.observables(cb3, d3, 0)
    b.c.meta.update(op="teleport", code=code.name, rounds=(rounds_before, rounds_after),
                    p=noise.p, p_ebit=noise.p_ebit, n=code.n, k=code.k)
    return b.c


# Methods "Pauli string compute": local (0) / non-local (1) pattern of the
# chain CX_{1->2}, ..., CX_{(w-1)->w} for each string weight w.
CHAIN_PATTERNS: Dict[int, str] = {2: "1", 3: "10", 4: "101", 5: "1010", 6: "10101"}


def pauli_string_circuit(code: CSSCode, w: int, pattern: Optional[str] = None, rounds_before: int = 4,
                         noise: Optional[NoiseModel] = None) -> Circuit:
    """Methods "Pauli string compute" (Eq. chain-compute): the parity of w
    code blocks is computed onto an ancilla block by the chain
    CX_{1->2}, ..., CX_{(w-1)->w}, CX_{w->a}.

    w + 1 blocks are noisily initialised in |0_L>; ``rounds_before`` rounds
    run on all of them; each chain CNOT is local (transversal CX with
    DEPOLARIZE2(p) on every pair) or non-local (the gate-teleported CNOT of
    ``Builder.nonlocal_cnot_core``) as ``pattern`` says (default: the
    paper's pattern for w); the final CX_{w->a} is local. After each chain
    CNOT between blocks m and m+1 one syndrome round runs on those two blocks
    only; then every block, ancilla included, is measured in the Z basis.

    Readings: the text sends non-local CNOTs through "Fig. 1(c)" with ebit
    noise equal to the physical error rate; this uses the non-local CNOT of
    Fig. 1(b) and leaves p_ebit to the noise model (set p_ebit = p to match).
    The round after a CNOT also follows the final CX_{w->a}.

    Detectors: as in the non-local CNOT, a target block's first check after
    a CNOT also takes the control block's last record of the same check.
    Observables: Z_L of every logical of every block, block order
    1..w then the ancilla.
    """
    if w < 1:
        raise ValueError("string weight must be >= 1")
    pattern = pattern if pattern is not None else CHAIN_PATTERNS.get(w, "")
    if len(pattern) != w - 1 or any(ch not in "01" for ch in pattern):
        raise ValueError(f"pattern must have {w - 1} symbols in {{0, 1}}")
    noise = noise or NoiseModel()
    b = Builder(noise)
    blocks = [b.block(code, f"CB{i + 1}") for i in range(w)] + [b.block(code, "ANC")]
    b.reset_data(blocks)
    prev: List[Optional[np.ndarray]] = [None] * len(blocks)
    extra: List[Optional[List[List[int]]]] = [None] * len(blocks)
    for _ in range(rounds_before):
        recs = b.syndrome_round(blocks)
        for i, blk in enumerate(blocks):
            b.round_detectors(blk, recs[i], prev[i], extra[i])
            prev[i], extra[i] = recs[i], None
    links = [(m, m + 1, pattern[m] == "1") for m in range(w - 1)] + [(w - 1, w, False)]
    for m, t, nonlocal_ in links:
        if nonlocal_:
            b.nonlocal_cnot_core(blocks[m], blocks[t])
        else:
            pairs = np.stack([blocks[m].data, blocks[t].data], axis=1).ravel()
            b.op("CX", pairs, tag="gate")
            b.err("DEPOLARIZE2", pairs, noise.p)
            b.op("TICK", [], tag="tick")
        if prev[m] is not None:
            extra[t] = [[int(prev[m][i])] + (extra[t][i] if extra[t] else []) for i in range(code.n_zchecks)]
        recs = b.syndrome_round([blocks[m], blocks[t]])
        for j, bi in enumerate((m, t)):
            b.round_detectors(blocks[bi], recs[j], prev[bi], extra[bi])
            prev[bi], extra[bi] = recs[j], None
    data_recs = b.measure_data(blocks, tag="readout")
    nxt = 0
    for i, blk in enumerate(blocks):
        b.final_detectors(blk, data_recs[i], prev[i], extra[i])
    for i, blk in enumerate(blocks):
        nxt = b.observables(blk, data_recs[i], nxt)
    b.c.meta.update(op="pauli_string", code=code.name, w=w, pattern=pattern, rounds=(rounds_before, 1),
                    p=noise.p, p_ebit=noise.p_ebit, n=code.n, k=code.k)
    return b.c


def memory_circuit(code: CSSCode, rounds: int, noise: Optional[NoiseModel] = None) -> Circuit:
    """Single-block Z-basis memory experiment (test fixture; not a paper
    workload): |0_L> init, ``rounds`` rounds, readout, Z detectors,
    Z_L observables."""
    noise = noise or NoiseModel()
    b = Builder(noise)
    blk = b.block(code, "CB")
    b.reset_data([blk])
    prev = None
    for _ in range(rounds):
        recs = b.syndrome_round([blk])
        b.round_detectors(blk, recs[0], prev, None)
        prev = recs[0]
    (dr,) = b.measure_data([blk], tag="readout")
    b.final_detectors(blk, dr, prev, None)
    b.observables(blk, dr, 0)
    b.c.meta.update(op="memory", code=code.name, rounds=(rounds, 0), p=noise.p, n=code.n, k=code.k)
    return b.c


def gate_counts(c: Circuit) -> Dict[str, int]:
    """Counts in the convention of Table III (gate counts and PCM rows).

    1q = targets of noisy H / S gates plus conditioned-Pauli gates (one per
    (record, qubit) pair); 2q = CX pairs of noisy CX gates (ebit Bell-pair
    preparation is perfect and not counted); M = every measurement except
    the final readout of the blocks measured at the end; rows = detectors.
    """
    one = two = meas = 0
    for op in c.ops:
        if op.tag != "gate" and op.tag != "meas":
            continue
        if op.name in ("H", "S"):
            one += op.targets.size
        elif op.name in ("XFEED", "ZFEED"):
            one += op.targets.size // 2
        elif op.name == "CX":
            two += op.targets.size // 2
        elif op.name in ("M", "MX"):
            meas += op.targets.size
    return {"1q": one, "2q": two, "M": meas, "rows": c.n_det}


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    """A named sampling workload: circuit recipe plus shots and seed."""

    name: str
    code: str
    op: str
    rounds_before: int
    rounds_after: int
    p: float
    p_ebit: float
    shots: int
    seed: int = 1
    decoherence: Optional[Decoherence] = None

    def circuit(self) -> Circuit:
        code = code_by_name(self.code)
        nz = NoiseModel(p=self.p, p_ebit=self.p_ebit, decoherence=self.decoherence)
        if self.op == "nl":
            return nonlocal_cnot_circuit(code, self.rounds_before, self.rounds_after, nz)
        if self.op == "teleport":
            return teleport_circuit(code, self.rounds_before, self.rounds_after, nz)
        if self.op.startswith("pauli"):
            return pauli_string_circuit(code, int(self.op[5:]), rounds_before=self.rounds_before, noise=nz)
        raise ValueError(self.op)


WORKLOADS: Dict[str, Workload] = {
    # distance-3 SC non-local CNOT, 3 rounds before/after, 1e4 shots
    "nl_sc3": Workload("nl_sc3", "sc3", "nl", 3, 3, 1e-3, 1e-2, 10_000),
    # distance-11 SC non-local CNOT, 11 rounds before/after, 1e7 shots
    "nl_sc11": Workload("nl_sc11", "sc11", "nl", 11, 11, 1e-3, 1e-2, 10_000_000),
    # BB [[144,12,12]] teleportation, 12 rounds per stage, 1e7 shots
    "tp_bb144": Workload("tp_bb144", "bb144", "teleport", 12, 12, 1e-3, 1e-2, 10_000_000),
    # distance-29 SC non-local CNOT, 29 rounds before/after, 1e7 shots
    "nl_sc29": Workload("nl_sc29", "sc29", "nl", 29, 29, 1e-3, 1e-2, 10_000_000),
    "nl_sc29_p1e-4": Workload("nl_sc29_p1e-4", "sc29", "nl", 29, 29, 1e-4, 1e-3, 10_000_000),
    # Pauli-string compute, weight 4 (pattern 101), BB[[144,12,12]], p = p_ebit
    "ps4_bb144": Workload("ps4_bb144", "bb144", "pauli4", 4, 1, 5e-4, 5e-4, 1_000_000),
    # distance-11 SC non-local CNOT with line-generated ebits decohering
    # (t_gen / T1 = 1e-4, T1 = T2), p = p_ebit = 1e-3
    "nl_sc11_deco": Workload("nl_sc11_deco", "sc11", "nl", 11, 11, 1e-3, 1e-3, 10_000_000,
                             decoherence=Decoherence(1e-4, schedule="lines")),
}


def batch_mix(n_jobs: int = 64, seed: int = 1) -> List[Workload]:
    """Seeded mix of uneven jobs: code uniform over SC d = 3..29 (odd) and
    BB[[144,12,12]]; op uniform over {NL, teleport}; p uniform over
    {1e-4, 3e-4, 1e-3} with p_ebit = 10 p; shots log-uniform in
    [1e4, 1e7]; rounds = d before and after for SC, 12 per stage for BB."""
    rng = np.random.default_rng(seed)
    codes = [f"sc{d}" for d in range(3, 30, 2)] + ["bb144"]
    out = []
    for j in range(n_jobs):
        code = codes[int(rng.integers(len(codes)))]
        op = ("nl", "teleport")[int(rng.integers(2))]
        p = (1e-4, 3e-4, 1e-3)[int(rng.integers(3))]
        shots = int(round(10 ** rng.uniform(4, 7)))
        r = 12 if code == "bb144" else int(code[2:])
        out.append(Workload(f"job{j}", code, op, r, r, p, 10 * p, shots, seed=j + 1))
    return out
