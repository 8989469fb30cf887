"""Pins of the oracle's raw measurement sampler (gauge-randomised frames).

* Born rule: on tiny random Clifford circuits with mid-circuit measurements,
  resets and conditioned Paulis, the empirical distribution of record
  strings matches the exact distribution from exhaustive state-vector
  branching (chi-square), so the gauge Paulis randomise exactly the
  non-deterministic outcomes and nothing else.
* With noise, detector parities recomputed from the sampled records equal
  the detector sampler's output bit for bit (same noise streams).
"""
import math

import numpy as np
import pytest

import oracle
from circuit_gen import random_noisy_circuit
from oracle import statevector, tableau
from paper_2504_05611_gb300 import circuits as C
from paper_2504_05611_gb300.circuits import Circuit


def random_measured(rng, n, steps):
    c = Circuit()
    c.append("R", list(range(n)))
    for _ in range(steps):
        u = rng.random()
        if u < 0.45:
            kind = int(rng.integers(3))
            if kind == 0:
                c.append("H", [int(rng.integers(n))])
            elif kind == 1:
                c.append("S", [int(rng.integers(n))])
            else:
                a, b = rng.choice(n, 2, replace=False)
                c.append("CX", [int(a), int(b)])
        elif u < 0.6:
            c.append("M", [int(rng.integers(n))])
        elif u < 0.7:
            c.append("MX", [int(rng.integers(n))])
        elif u < 0.77:
            c.append("R", [int(rng.integers(n))])
        elif u < 0.84:
            c.append("RX", [int(rng.integers(n))])
        elif c.n_meas:
            c.append("XFEED" if rng.random() < 0.5 else "ZFEED",
                     [int(rng.integers(c.n_meas)), int(rng.integers(n))])
    c.append("M", list(range(n)))
    return c


@pytest.mark.parametrize("trial", range(12))
def test_measurement_records_follow_born_rule(trial):
    rng = np.random.default_rng(600 + trial)
    c = random_measured(rng, int(rng.integers(2, 4)), 14)
    if c.n_meas > 9:
        pytest.skip("too many outcomes to enumerate")
    dist = statevector.outcome_distribution(c)
    shots = 64 * 600
    recs = oracle.unpack_bits(oracle.sample_measurements(c, shots, seed=trial + 1, threads=4), shots)
    keys = [tuple(int(v) for v in recs[:, s]) for s in range(shots)]
    counts = {}
    for k in keys:
        counts[k] = counts.get(k, 0) + 1
    assert set(counts) <= set(dist)   # never an impossible record string
    chi2, dof = 0.0, 0
    for k, p in dist.items():
        e = p * shots
        chi2 += (counts.get(k, 0) - e) ** 2 / e
        dof += 1
    dof -= 1
    assert chi2 < dof + 6 * math.sqrt(2 * max(dof, 1)) + 10


def test_deterministic_circuit_reproduces_reference():
    c = C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.0, 0.0))
    ref = tableau.reference_sample(c)["rec"]
    recs = oracle.unpack_bits(oracle.sample_measurements(c, 640, seed=3), 640)
    # every detector's records XOR to its reference parity in every shot
    for op in c.ops:
        if op.name == "DETECTOR":
            t = [int(v) for v in op.targets]
            par = np.bitwise_xor.reduce(recs[t], axis=0)
            assert np.all(par == np.bitwise_xor.reduce(ref[t]))
    # random outcomes (X-check ancillas of the first round) are fair coins
    frac = recs.mean(axis=1)
    assert frac.max() > 0.3 and np.all((frac < 0.01) | (frac > 0.35))


@pytest.mark.parametrize("trial", range(3))
def test_detectors_from_records_equal_detector_sampler(trial):
    rng = np.random.default_rng(50 + trial)
    if trial == 0:
        c = C.teleport_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.02, 0.05))
    else:
        c = random_noisy_circuit(rng, 6, 30)
    shots = 64 * 20 + 13
    ref = tableau.reference_sample(c)["rec"]
    recs = oracle.unpack_bits(oracle.sample_measurements(c, shots, seed=77, reference=ref), shots)
    det, _ = oracle.sample(c, shots, seed=77)
    dbits = oracle.unpack_bits(det, shots)
    k = 0
    for op in c.ops:
        if op.name == "DETECTOR":
            t = [int(v) for v in op.targets]
            par = np.bitwise_xor.reduce(recs[t], axis=0) ^ np.bitwise_xor.reduce(ref[t]) if t else 0
            assert np.array_equal(par, dbits[k]), k
            k += 1
