"""Pins of the frame-update rules and of the reference tableau.

* The state-vector simulator itself is checked on textbook identities
  (H|0> is balanced, a Bell pair is perfectly ZZ-correlated, HSSH = X,
  CX flips the target only when the control is 1).
* Frame propagation (the oracle's 64-lane propagator, which shares its
  update rules with the one-shot sampler) against brute-force state vectors:
  random Clifford circuits U U^-1 on |0>/|+> inputs, with a Pauli fault
  injected at a random point and, in half the cases, a mid-circuit
  measurement feeding conditioned X/Z gates. Every outcome is deterministic,
  and the frame must predict exactly which ones the fault flips
  (Supplementary Note 1's symplectic encoding).
* The one-shot sampler's update rules against the propagator: with a
  probability-1 X_ERROR placed where the fault was, its records equal the
  propagator's.
* The CHP tableau against the state vector on random circuits with random
  mid-circuit measurements (random outcomes resolved to 0 on both sides).
"""
import numpy as np
import pytest

import oracle
from oracle import statevector, tableau
from paper_2504_05611_gb300.circuits import Circuit


def test_statevector_textbook_identities():
    sv = statevector.StateVector(2)
    sv.h(0)
    assert abs(sv.prob1(0) - 0.5) < 1e-12
    sv.cx(0, 1)
    amp = np.abs(sv.psi) ** 2
    assert abs(amp[0] - 0.5) < 1e-12 and abs(amp[3] - 0.5) < 1e-12
    sv = statevector.StateVector(1)
    for g in (sv.h, sv.s, sv.s, sv.h):
        g(0)
    assert abs(sv.prob1(0) - 1.0) < 1e-12
    sv = statevector.StateVector(2)
    sv.cx(0, 1)
    assert abs(sv.prob1(1)) < 1e-12
    sv.x(0)
    sv.cx(0, 1)
    assert abs(sv.prob1(1) - 1.0) < 1e-12


def random_unitary_ops(rng, n, depth):
    ops = []
    for _ in range(depth):
        kind = rng.integers(3)
        if kind == 0:
            ops.append(("H", [int(rng.integers(n))]))
        elif kind == 1:
            ops.append(("S", [int(rng.integers(n))]))
        else:
            a, b = rng.choice(n, 2, replace=False)
            ops.append(("CX", [int(a), int(b)]))
    return ops


def inverse_ops(ops):
    inv = []
    for name, t in reversed(ops):
        if name == "S":
            inv += [("S", t)] * 3
        else:
            inv.append((name, t))
    return inv


def build_identity_circuit(rng, n, depth, with_feed):
    c = Circuit()
    xbasis = [q for q in range(n) if rng.random() < 0.5]
    zbasis = [q for q in range(n) if q not in xbasis]
    if zbasis:
        c.append("R", zbasis)
    if xbasis:
        c.append("RX", xbasis)
    body = random_unitary_ops(rng, n, depth)
    for name, t in body + inverse_ops(body):
        c.append(name, t)
    anc = n
    if with_feed:
        # measure an ancilla that copies the x-frame of qubit 0 (in Z basis or
        # not, its outcome is deterministic only if qubit 0 is Z-basis)
        q0 = zbasis[0] if zbasis else None
        if q0 is not None:
            c.append("R", [anc])
            c.append("CX", [q0, anc])
            r = c.append("M", [anc])
            tgt = int(rng.integers(n))
            c.append("XFEED" if rng.random() < 0.5 else "ZFEED", [int(r[0]), tgt])
    if zbasis:
        c.append("M", zbasis)
    if xbasis:
        c.append("MX", xbasis)
    for r in range(c.n_meas):
        c.append("DETECTOR", [r])
    return c


@pytest.mark.parametrize("trial", range(60))
def test_frame_rules_match_statevector(trial):
    rng = np.random.default_rng(1000 + trial)
    n = int(rng.integers(2, 6))
    c = build_identity_circuit(rng, n, int(rng.integers(3, 14)), with_feed=trial % 2 == 1)
    ref = statevector.run(c)
    assert not ref["rec"].any()
    # inject one random Pauli after a random op (qubits only, not after feeds)
    ops_ok = [i for i, op in enumerate(c.ops) if op.name in ("R", "RX", "H", "S", "CX")]
    i = int(rng.choice(ops_ok))
    q = int(rng.integers(n))
    pauli = int(rng.integers(1, 4))
    faulty = statevector.run(c, faults=[(i, q, pauli)])
    det, _ = oracle.propagate64(c, [i], [q], [pauli], [5])
    frame_flips = ((det >> np.uint64(5)) & np.uint64(1)).astype(np.uint8)
    assert np.array_equal(frame_flips, faulty["det"] ^ ref["det"])


@pytest.mark.parametrize("trial", range(10))
def test_one_shot_sampler_matches_propagator(trial):
    rng = np.random.default_rng(77 + trial)
    n = 4
    c0 = build_identity_circuit(rng, n, 10, with_feed=True)
    ops_ok = [i for i, op in enumerate(c0.ops) if op.name in ("R", "RX", "H", "S", "CX")]
    i = int(rng.choice(ops_ok))
    q = int(rng.integers(n))
    # rebuild with a certain X error right after op i
    c = Circuit()
    for j, op in enumerate(c0.ops):
        c.append(op.name, op.targets, p=op.p, arg=op.arg)
        if j == i:
            c.append("X_ERROR", [q], p=1.0)
    det_s, _ = oracle.sample(c, 64, seed=3)
    det_p, _ = oracle.propagate64(c0, [i], [q], [1], [0])
    want = (det_p & np.uint64(1)).astype(bool)
    got_all = det_s[:, 0]
    assert np.array_equal(got_all == np.uint64(0xFFFFFFFFFFFFFFFF), want)
    assert np.all((got_all == 0) | (got_all == np.uint64(0xFFFFFFFFFFFFFFFF)))


def random_measured_circuit(rng, n, steps):
    c = Circuit()
    c.append("R", list(range(n)))
    for _ in range(steps):
        u = rng.random()
        if u < 0.5:
            for name, t in random_unitary_ops(rng, n, 1):
                c.append(name, t)
        elif u < 0.65:
            c.append("M", [int(rng.integers(n))])
        elif u < 0.75:
            c.append("MX", [int(rng.integers(n))])
        elif u < 0.82:
            c.append("R", [int(rng.integers(n))])
        elif u < 0.88:
            c.append("RX", [int(rng.integers(n))])
        elif c.n_meas:
            c.append("XFEED" if rng.random() < 0.5 else "ZFEED",
                     [int(rng.integers(c.n_meas)), int(rng.integers(n))])
    c.append("M", list(range(n)))
    return c


@pytest.mark.parametrize("trial", range(40))
def test_tableau_matches_statevector(trial):
    rng = np.random.default_rng(5000 + trial)
    n = int(rng.integers(2, 7))
    c = random_measured_circuit(rng, n, 40)
    a = tableau.reference_sample(c)["rec"]
    b = statevector.run(c)["rec"]
    assert np.array_equal(a, b)
