"""Exhaustive single-fault detector error model -- TEST INFRASTRUCTURE.

Restates what the paper takes from its simulator's detector error model
(Methods "Decoding"; Table III "rows" and "cols"): every elementary fault
(one non-identity Pauli of one noise channel at one site) is injected alone
into the noiseless circuit and the detectors and observables it flips are
recorded (its signature). Rows are detectors, columns distinct signatures.

Because the frame is linear over GF(2) and each (noise op, target unit) is
an independent channel whose Paulis are mutually exclusive, every detector
parity is the XOR of independent channel contributions, so its flip
probability is exactly (1 - prod_c (1 - 2 P_c)) / 2 with P_c the total
probability of the channel's Paulis that flip it.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Tuple

import numpy as np

from . import Marshalled, propagate64

# Pauli index -> (first, second) single-qubit Paulis; bit0 = X, bit1 = Z.
_K = {"X_ERROR": 1, "Z_ERROR": 1, "DEPOLARIZE1": 3, "DEPOLARIZE2": 15, "PAULI_CHANNEL_1": 3}


def fault_list(circuit) -> List[Tuple[int, int, List[Tuple[int, int]], float]]:
    """(op index, channel id, [(qubit, pauli), ...], probability) for every
    elementary fault of every noise channel with p > 0, in the order noise op,
    target unit, Pauli index k = 1..K."""
    out = []
    ch = 0
    for i, op in enumerate(circuit.ops):
        if op.name not in _K or op.p <= 0.0:
            continue
        t = [int(v) for v in op.targets]
        K = _K[op.name]
        units = len(t) // 2 if op.name == "DEPOLARIZE2" else len(t)
        for u in range(units):
            for k in range(1, K + 1):
                if op.name == "PAULI_CHANNEL_1":
                    px, py, pz = op.channel
                    out.append((i, ch, [(t[u], k)], {1: px, 2: pz, 3: py}[k]))
                    continue
                if op.name == "X_ERROR":
                    inj = [(t[u], 1)]
                elif op.name == "Z_ERROR":
                    inj = [(t[u], 2)]
                elif op.name == "DEPOLARIZE1":
                    inj = [(t[u], k)]
                else:
                    inj = [(t[2 * u], k >> 2), (t[2 * u + 1], k & 3)]
                inj = [(q, p) for q, p in inj if p]
                out.append((i, ch, inj, op.p / K))
            ch += 1
    return out


def signatures(circuit):
    """Per elementary fault: detector signature and observable signature as
    Python int bitmasks, plus channel id and probability."""
    m = Marshalled(circuit)
    faults = fault_list(circuit)
    dets: List[int] = []
    obss: List[int] = []
    for base in range(0, len(faults), 64):
        grp = faults[base:base + 64]
        io, it, ip, il = [], [], [], []
        for lane, (op_i, _, inj, _) in enumerate(grp):
            for q, p in inj:
                io.append(op_i); it.append(q); ip.append(p); il.append(lane)
        dw, ow = propagate64(circuit, io, it, ip, il, marshalled=m)
        dbits = ((dw[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint8)
        obits = ((ow[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.uint8)
        for lane in range(len(grp)):
            dets.append(_mask(np.nonzero(dbits[:, lane])[0]))
            obss.append(_mask(np.nonzero(obits[:, lane])[0]))
    chans = [f[1] for f in faults]
    probs = [f[3] for f in faults]
    return dets, obss, chans, probs


def _mask(idx) -> int:
    v = 0
    for i in idx:
        v |= 1 << int(i)
    return v


def _bits(mask: int) -> List[int]:
    out = []
    i = 0
    while mask:
        if mask & 1:
            out.append(i)
        mask >>= 1
        i += 1
    return out


def flip_probabilities(circuit) -> Tuple[np.ndarray, np.ndarray]:
    """Exact P(detector j flips) and P(observable o flips)."""
    dets, obss, chans, probs = signatures(circuit)
    pd: Dict[Tuple[int, int], float] = {}
    po: Dict[Tuple[int, int], float] = {}
    for dm, om, c, p in zip(dets, obss, chans, probs):
        for j in _bits(dm):
            pd[(c, j)] = pd.get((c, j), 0.0) + p
        for j in _bits(om):
            po[(c, j)] = po.get((c, j), 0.0) + p
    prod_d = np.ones(circuit.n_det)
    prod_o = np.ones(circuit.n_obs)
    for (c, j), p in pd.items():
        prod_d[j] *= 1.0 - 2.0 * p
    for (c, j), p in po.items():
        prod_o[j] *= 1.0 - 2.0 * p
    return (1.0 - prod_d) / 2.0, (1.0 - prod_o) / 2.0


def pair_flip_probability(circuit, a: int, b: int) -> float:
    """Exact P(detector a XOR detector b = 1)."""
    dets, _, chans, probs = signatures(circuit)
    pc: Dict[int, float] = {}
    for dm, c, p in zip(dets, chans, probs):
        if ((dm >> a) & 1) ^ ((dm >> b) & 1):
            pc[c] = pc.get(c, 0.0) + p
    prod = 1.0
    for p in pc.values():
        prod *= 1.0 - 2.0 * p
    return (1.0 - prod) / 2.0


def columns(circuit) -> List[Tuple[int, int]]:
    """Distinct non-empty (detector mask, observable mask) signatures: the
    columns of the space-time parity-check matrix."""
    dets, obss, _, _ = signatures(circuit)
    return sorted({(d, o) for d, o in zip(dets, obss) if d or o})


def column_probabilities(circuit) -> Dict[Tuple[int, int], Tuple[float, int]]:
    """Per distinct non-empty signature (detector mask, observable mask): the
    probability that an odd number of its elementary faults occur in a shot,
    and how many faults it merges. Faults of one channel (noise op, target
    unit) exclude one another, so they add within the channel; channels are
    independent, so a signature's parity over channels XOR-combines:
    P = (1 - prod_channels (1 - 2 P_channel)) / 2."""
    dets, obss, chans, probs = signatures(circuit)
    per: Dict[Tuple[int, int], Dict[int, float]] = {}
    count: Dict[Tuple[int, int], int] = {}
    for d, o, c, p in zip(dets, obss, chans, probs):
        if not (d or o):
            continue
        key = (d, o)
        per.setdefault(key, {})
        per[key][c] = per[key].get(c, 0.0) + p
        count[key] = count.get(key, 0) + 1
    out = {}
    for key, by_chan in per.items():
        prod = 1.0
        for p in by_chan.values():
            prod *= 1.0 - 2.0 * p
        out[key] = ((1.0 - prod) / 2.0, count[key])
    return out


def circuit_distance(circuit, max_weight: int = 3) -> int:
    """Smallest number of elementary faults whose combined signature flips no
    detector but some observable (brute force up to ``max_weight``; returns
    max_weight + 1 if none is found)."""
    cols = columns(circuit)
    if any(d == 0 and o for d, o in cols):
        return 1
    by_det: Dict[int, set] = {}
    for d, o in cols:
        by_det.setdefault(d, set()).add(o)
    if max_weight >= 2:
        for d, os_ in by_det.items():
            if len(os_) > 1:
                return 2
    if max_weight >= 3:
        for (d1, o1), (d2, o2) in itertools.combinations(cols, 2):
            want = d1 ^ d2
            for o3 in by_det.get(want, ()):
                if o1 ^ o2 ^ o3:
                    return 3
    if max_weight >= 4:
        pair_obs: Dict[int, set] = {}
        for (d1, o1), (d2, o2) in itertools.combinations(cols, 2):
            pair_obs.setdefault(d1 ^ d2, set()).add(o1 ^ o2)
        for d, os_ in pair_obs.items():
            if len(os_) > 1:
                return 4
    return max_weight + 1
