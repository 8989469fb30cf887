"""Brute-force state-vector simulator for tiny circuits -- TEST INFRASTRUCTURE.

Pins the gate semantics of the frame oracle and of the tableau oracle on
circuits of at most ~12 qubits: a noiseless op list is executed on an explicit
2^n amplitude vector with textbook gate matrices (|0>,|1> computational
basis, qubit q = bit q of the basis index).

Measurements resolve a random outcome (probability strictly between 0 and 1)
to 0, like the reference sample; a deterministic outcome is taken as it is.
Conditioned Paulis (XFEED/ZFEED) act on the outcome actually recorded.
Noise ops are ignored; explicit Pauli faults can be injected after any op.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

_EPS = 1e-9


class StateVector:
    def __init__(self, n: int):
        if n > 16:
            raise ValueError("state-vector oracle is for tiny circuits only")
        self.n = n
        self.psi = np.zeros(1 << n, dtype=np.complex128)
        self.psi[0] = 1.0
        self.idx = np.arange(1 << n, dtype=np.int64)

    def _bit(self, q: int) -> np.ndarray:
        return (self.idx >> q) & 1

    def x(self, q: int) -> None:
        self.psi = self.psi[self.idx ^ (1 << q)]

    def z(self, q: int) -> None:
        self.psi = self.psi * np.where(self._bit(q) == 1, -1.0, 1.0)

    def y(self, q: int) -> None:
        # Y = i X Z
        self.z(q)
        self.x(q)
        self.psi = self.psi * 1j

    def h(self, q: int) -> None:
        b = self._bit(q)
        partner = self.psi[self.idx ^ (1 << q)]
        self.psi = (np.where(b == 0, self.psi + partner, partner - self.psi)) / np.sqrt(2.0)

    def s(self, q: int) -> None:
        self.psi = self.psi * np.where(self._bit(q) == 1, 1j, 1.0)

    def cx(self, c: int, t: int) -> None:
        src = np.where(self._bit(c) == 1, self.idx ^ (1 << t), self.idx)
        self.psi = self.psi[src]

    def prob1(self, q: int) -> float:
        return float(np.sum(np.abs(self.psi[self._bit(q) == 1]) ** 2))

    def measure_z(self, q: int) -> int:
        p1 = self.prob1(q)
        out = 1 if p1 > 1.0 - _EPS else 0
        keep = self._bit(q) == out
        self.psi = np.where(keep, self.psi, 0.0)
        self.psi /= np.linalg.norm(self.psi)
        return out

    def pauli(self, q: int, p: int) -> None:
        """p: bit0 = X part, bit1 = Z part (X=1, Z=2, Y=3), up to phase."""
        if p & 2:
            self.z(q)
        if p & 1:
            self.x(q)


def run(circuit, faults: Sequence[Tuple[int, int, int]] = ()) -> Dict[str, np.ndarray]:
    """Execute ``circuit`` noiselessly; ``faults`` = (op index, qubit, pauli)
    applied right after that op. Returns measurement record, detector and
    observable parities (absolute values, not flips)."""
    sv = StateVector(circuit.n_qubits)
    rec: List[int] = []
    det: List[int] = []
    obs = np.zeros(circuit.n_obs, dtype=np.uint8)
    by_op: Dict[int, List[Tuple[int, int]]] = {}
    for op_i, q, p in faults:
        by_op.setdefault(int(op_i), []).append((int(q), int(p)))
    for i, op in enumerate(circuit.ops):
        t = [int(v) for v in op.targets]
        name = op.name
        if name == "R":
            for q in t:
                if sv.measure_z(q):
                    sv.x(q)
        elif name == "RX":
            for q in t:
                if sv.measure_z(q):
                    sv.x(q)
                sv.h(q)
        elif name == "H":
            for q in t:
                sv.h(q)
        elif name == "S":
            for q in t:
                sv.s(q)
        elif name == "CX":
            for a in range(0, len(t), 2):
                sv.cx(t[a], t[a + 1])
        elif name == "M":
            for q in t:
                rec.append(sv.measure_z(q))
        elif name == "MX":
            for q in t:
                sv.h(q)
                rec.append(sv.measure_z(q))
                sv.h(q)
        elif name == "XFEED":
            for a in range(0, len(t), 2):
                if rec[t[a]]:
                    sv.x(t[a + 1])
        elif name == "ZFEED":
            for a in range(0, len(t), 2):
                if rec[t[a]]:
                    sv.z(t[a + 1])
        elif name == "DETECTOR":
            det.append(int(np.bitwise_xor.reduce([rec[r] for r in t])) if t else 0)
        elif name == "OBSERVABLE":
            if t:
                obs[op.arg] ^= int(np.bitwise_xor.reduce([rec[r] for r in t]))
        for q, p in by_op.get(i, ()):
            sv.pauli(q, p)
    return {"rec": np.array(rec, dtype=np.uint8), "det": np.array(det, dtype=np.uint8), "obs": obs}


def outcome_distribution(circuit) -> Dict[Tuple[int, ...], float]:
    """Exact probability of every measurement-record string of a noiseless
    circuit (Born rule), by branching the state vector at every measurement
    and reset; conditioned Paulis follow each branch's outcomes."""
    out: Dict[Tuple[int, ...], float] = {}

    def measure_branch(sv: StateVector, q: int, outcome: int):
        keep = sv._bit(q) == outcome
        psi = np.where(keep, sv.psi, 0.0)
        p = float(np.sum(np.abs(psi) ** 2))
        if p < 1e-12:
            return None, 0.0
        nsv = StateVector(sv.n)
        nsv.psi = psi / np.sqrt(p)
        return nsv, p

    def run_from(sv: StateVector, op_i: int, t_i: int, rec: Tuple[int, ...], prob: float):
        ops = circuit.ops
        while op_i < len(ops):
            op = ops[op_i]
            t = [int(v) for v in op.targets]
            name = op.name
            if name in ("M", "MX", "R", "RX") and t_i < len(t):
                q = t[t_i]
                if name == "MX":
                    sv.h(q)
                for outcome in (0, 1):
                    nsv, p = measure_branch(sv, q, outcome)
                    if nsv is None:
                        continue
                    nrec = rec
                    if name in ("M", "MX"):
                        nrec = rec + (outcome,)
                        if name == "MX":
                            nsv.h(q)
                    else:
                        if outcome:
                            nsv.x(q)
                        if name == "RX":
                            nsv.h(q)
                    run_from(nsv, op_i, t_i + 1, nrec, prob * p)
                return
            if name not in ("M", "MX", "R", "RX"):
                if name == "H":
                    for q in t:
                        sv.h(q)
                elif name == "S":
                    for q in t:
                        sv.s(q)
                elif name == "CX":
                    for a in range(0, len(t), 2):
                        sv.cx(t[a], t[a + 1])
                elif name == "XFEED":
                    for a in range(0, len(t), 2):
                        if rec[t[a]]:
                            sv.x(t[a + 1])
                elif name == "ZFEED":
                    for a in range(0, len(t), 2):
                        if rec[t[a]]:
                            sv.z(t[a + 1])
            op_i, t_i = op_i + 1, 0
        out[rec] = out.get(rec, 0.0) + prob

    run_from(StateVector(circuit.n_qubits), 0, 0, (), 1.0)
    return out
