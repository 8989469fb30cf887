"""Pins of the single-fault DEM enumeration and the oracle sampler's
whole-circuit statistics.

* Table I: the distance-3 surface-code non-local CNOT and teleportation
  circuits have circuit-level distance exactly 3 (no undetectable logical
  fault set of weight <= 2 exists, one of weight 3 does).
* Exact detector and observable flip marginals, computed from the DEM
  (independent channels, XOR of contributions), agree with oracle samples
  within 5 sigma; so does one pair of adjacent-round detectors.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import golden_rows
from oracle import dem
from paper_2504_05611_gb300 import circuits as C

TABLE_I = {r[0]: (int(r[1]), int(r[2])) for r in golden_rows("table_i_distance.txt")}


def test_circuit_distance_table_i():
    code = C.code_by_name("sc3")
    nl, tp = TABLE_I["sc3"]
    assert dem.circuit_distance(C.nonlocal_cnot_circuit(code, 4, 3), max_weight=3) == nl
    assert dem.circuit_distance(C.teleport_circuit(code, 4, 3), max_weight=3) == tp


def test_memory_distance_sc5_at_least_5():
    """A d=5 memory circuit has no undetectable logical fault set of weight
    <= 4 (the hook-avoiding schedule keeps the circuit distance at d)."""
    c = C.memory_circuit(C.code_by_name("sc5"), 2)
    assert dem.circuit_distance(c, max_weight=4) == 5


@pytest.mark.parametrize("kind", ["nl", "teleport"])
def test_marginals_match_samples(kind):
    code = C.code_by_name("sc3")
    nz = C.NoiseModel(p=0.01, p_ebit=0.05)
    fn = C.nonlocal_cnot_circuit if kind == "nl" else C.teleport_circuit
    c = fn(code, 2, 2, nz)
    pd, po = dem.flip_probabilities(c)
    shots = 64 * 1600
    det, obs = oracle.sample(c, shots, seed=2024, threads=8)
    bd = oracle.unpack_bits(det, shots).astype(np.float64)
    bo = oracle.unpack_bits(obs, shots).astype(np.float64)
    sd = np.sqrt(pd * (1 - pd) / shots)
    assert np.all(np.abs(bd.mean(1) - pd) < 5.5 * sd + 1e-9)
    sdo = np.sqrt(po * (1 - po) / shots)
    assert np.all(np.abs(bo.mean(1) - po) < 5.5 * sdo + 1e-9)
    a, b = 0, code.n_zchecks * (2 if kind == "nl" else 3)   # same check, next round
    pab = dem.pair_flip_probability(c, a, b)
    emp = np.mean(np.logical_xor(bd[a], bd[b]))
    assert abs(emp - pab) < 5.5 * math.sqrt(pab * (1 - pab) / shots)


def test_column_probabilities_closed_forms():
    """Column probabilities against closed forms: one X_ERROR(p) before M is
    one column of probability p; DEPOLARIZE1(p) before M has X and Y flip the
    record (one column, mutually exclusive faults: 2p/3); two independent
    X_ERROR sites with the same signature XOR-combine to 2p(1-p); Z_ERROR
    before M flips nothing (no column)."""
    from paper_2504_05611_gb300.circuits import Circuit
    p = 0.1
    c = Circuit()
    c.append("R", [0, 1, 2, 3])
    c.append("X_ERROR", [0], p=p)
    c.append("DEPOLARIZE1", [1], p=p)
    c.append("X_ERROR", [2], p=p)
    c.append("X_ERROR", [2], p=p)
    c.append("Z_ERROR", [3], p=p)
    c.append("M", [0, 1, 2, 3])
    for r in range(4):
        c.append("DETECTOR", [r])
    cols = dem.column_probabilities(c)
    assert set(cols) == {(1, 0), (2, 0), (4, 0)}
    assert abs(cols[(1, 0)][0] - p) < 1e-15 and cols[(1, 0)][1] == 1
    assert abs(cols[(2, 0)][0] - 2 * p / 3) < 1e-15 and cols[(2, 0)][1] == 2
    assert abs(cols[(4, 0)][0] - 2 * p * (1 - p)) < 1e-15 and cols[(4, 0)][1] == 2
