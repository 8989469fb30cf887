"""Invariants of the oracle sampler (definition-level properties).

* No noise: every detector and observable is 0 for every shot.
* Output is a function of (seed, global chunk) only: a sub-range sampled
  with ``first_chunk`` equals the matching columns of a full run, and the
  thread count does not matter.
* Shots that are not a multiple of 64 leave pad bits zero and do not change
  the bits of real shots.
* Different seeds give different samples.
"""
import numpy as np

import oracle
from paper_2504_05611_gb300 import circuits as C


def circ(p=1e-2):
    return C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(p=p, p_ebit=5 * p))


def test_noiseless_is_all_zero():
    c = circ(p=0.0)
    det, obs = oracle.sample(c, 640, seed=9)
    assert not det.any() and not obs.any()


def test_chunk_keyed_and_thread_invariant():
    c = circ()
    full_d, full_o = oracle.sample(c, 64 * 12, seed=123, threads=1)
    par_d, par_o = oracle.sample(c, 64 * 12, seed=123, threads=5)
    assert np.array_equal(full_d, par_d) and np.array_equal(full_o, par_o)
    sub_d, sub_o = oracle.sample(c, 64 * 4, seed=123, first_chunk=5)
    assert np.array_equal(sub_d, full_d[:, 5:9]) and np.array_equal(sub_o, full_o[:, 5:9])


def test_ragged_shots():
    c = circ(p=0.05)
    d1, o1 = oracle.sample(c, 64 * 3, seed=4)
    d2, o2 = oracle.sample(c, 64 * 2 + 37, seed=4)
    mask = np.uint64((1 << 37) - 1)
    assert np.array_equal(d2[:, :2], d1[:, :2]) and np.array_equal(d2[:, 2], d1[:, 2] & mask)
    assert np.array_equal(o2[:, 2], o1[:, 2] & mask)


def test_seed_changes_output():
    c = circ(p=0.05)
    a, _ = oracle.sample(c, 640, seed=1)
    b, _ = oracle.sample(c, 640, seed=2)
    assert not np.array_equal(a, b)
