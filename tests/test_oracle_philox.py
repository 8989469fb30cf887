"""Pins of the oracle's Philox4x32-10 and gap tables.

Philox4x32-10 (Salmon et al., SC'11) is pinned three ways: (1) the
known-answer vectors published with the generator's reference library
(``tests/golden/philox4x32_10_kat.txt``), which fix every output word for
three counter/key pairs; (2) the round structure is inverted (the
multipliers are odd, so each low product is invertible mod 2^32) and the
inverse of the oracle's output must return the counter, so a wrong
multiplier, key schedule or output wiring breaks the round trip; (3) output
statistics. An independent implementation, cuRAND's device Philox4x32-10, is
compared with the oracle on many random counter/key pairs in
``tests/test_gpu_rng.py``.

The gap table is pinned by the distribution it induces: P(G >= g) read off
the table must equal the geometric tail (1-p)^g to within the 2^-32
quantisation.
"""
import math

import numpy as np
import pytest

import oracle

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox_inverse(out, key):
    inv0, inv1 = pow(M0, -1, 1 << 32), pow(M1, -1, 1 << 32)
    keys = [((key[0] + r * W0) & MASK, (key[1] + r * W1) & MASK) for r in range(10)]
    n0, n1, n2, n3 = out
    for r in reversed(range(10)):
        k0, k1 = keys[r]
        c2 = (n1 * inv1) & MASK
        c0 = (n3 * inv0) & MASK
        hi1 = (M1 * c2) >> 32
        hi0 = (M0 * c0) >> 32
        c1 = n0 ^ hi1 ^ k0
        c3 = n2 ^ hi0 ^ k1
        n0, n1, n2, n3 = c0, c1, c2, c3
    return (n0, n1, n2, n3)


def test_philox_known_answer_vectors():
    from conftest import golden_rows
    rows = golden_rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_philox_is_the_published_bijection():
    rng = np.random.default_rng(5)
    for _ in range(200):
        ctr = tuple(int(v) for v in rng.integers(0, 1 << 32, 4, dtype=np.uint64))
        key = tuple(int(v) for v in rng.integers(0, 1 << 32, 2, dtype=np.uint64))
        out = oracle.philox4x32_10(ctr, key)
        assert philox_inverse(out, key) == ctr
    assert oracle.philox4x32_10((0, 0, 0, 0), (0, 0)) != (0, 0, 0, 0)


def test_philox_output_statistics():
    outs = np.array([oracle.philox4x32_10((j, 7, 3, 1), (12345, 0)) for j in range(20000)],
                    dtype=np.uint64)
    bits = ((outs[:, :, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)
    frac = bits.mean(axis=0)
    # every output bit is balanced: |mean - 1/2| < 5 sigma
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / math.sqrt(outs.shape[0]))
    # byte histogram of all words is uniform (chi-square, 255 dof)
    b = outs.astype(np.uint32).view(np.uint8).ravel()
    h = np.bincount(b, minlength=256)
    e = b.size / 256
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    # consecutive counters are uncorrelated in word 0
    w = outs[:, 0].astype(np.float64)
    r = np.corrcoef(w[:-1], w[1:])[0, 1]
    assert abs(r) < 5 / math.sqrt(w.size)


@pytest.mark.parametrize("p", [1e-4, 1e-3, 1e-2, 0.1, 0.5, 0.9])
def test_gap_table_induces_geometric_tails(p):
    """P(G >= g) = T[g] / 2^32 must equal (1-p)^g, the geometric tail, to
    within the 2^-32 quantisation (plus double rounding of the power)."""
    t = oracle.gap_table(p).astype(np.int64)
    g = np.arange(1, 4097, dtype=np.float64)
    want = np.array([(1 - p) ** int(v) for v in g])
    assert np.all(np.abs(t / 2.0 ** 32 - want) <= 2.0 ** -31 + 1e-12 * want)
    assert np.all(np.diff(t) <= 0)


def test_gap_table_edge_probabilities():
    assert not oracle.gap_table(1.0).any()          # p = 1: every trial is an event
    t = oracle.gap_table(1e-12)                       # tiny p: G reaches the 4096 cap
    assert t[-1] > 0xFFFF0000
