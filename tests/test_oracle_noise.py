"""Closed-form flip rates of the paper's noise channels (Methods
"Simulation"), sampled with the oracle and compared within 5 sigma.

* X_ERROR(p) before M: the record flips with probability p.
* DEPOLARIZE1(p): X, Y, Z each with p/3; read out (x, z) through two copy
  CNOTs, the joint distribution is (1-p, p/3, p/3, p/3).
* DEPOLARIZE2(p): the 15 non-identity two-qubit Paulis each with p/15; the
  4-bit (x1, z1, x2, z2) readout is uniform over the 15 non-zero values.
* Bell pair + DEPOLARIZE2(p_ebit) + ZZ parity: 8 p_ebit / 15.
* XOR of N independent X_ERROR(p) sites: (1 - (1 - 2p)^N) / 2.
* Per-site rates and independence over many targets (several 64-unit
  segments with a ragged last one); p = 0 never fires, p = 1 always does.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2504_05611_gb300.circuits import Circuit


def bits(c, shots, seed=11):
    det, obs = oracle.sample(c, shots, seed, threads=4)
    return oracle.unpack_bits(det, shots)


def close(k, n, p, sig=5.0):
    sd = math.sqrt(max(p * (1 - p), 1e-12) / n)
    return abs(k / n - p) <= sig * sd + 1e-12


@pytest.mark.parametrize("p", [1e-3, 0.05, 0.3])
def test_x_error_before_measure(p):
    c = Circuit()
    c.append("R", [0])
    c.append("X_ERROR", [0], p=p)
    c.append("M", [0])
    c.append("DETECTOR", [0])
    n = 400_000
    assert close(bits(c, n).sum(), n, p)


def readout_xz(c, q, a, b):
    """Copy x_q onto ancilla a (CX q->a, M a) and z_q onto b (RX b, CX b->q, MX b)."""
    c.append("CX", [q, a])
    c.append("CX", [b, q])


def test_depolarize1_pauli_distribution():
    p = 0.3
    c = Circuit()
    c.append("R", [0, 1])
    c.append("RX", [2])
    c.append("DEPOLARIZE1", [0], p=p)
    readout_xz(c, 0, 1, 2)
    c.append("M", [1])
    c.append("MX", [2])
    c.append("DETECTOR", [0])
    c.append("DETECTOR", [1])
    n = 300_000
    b = bits(c, n)
    code = b[0] + 2 * b[1]
    h = np.bincount(code, minlength=4)
    assert close(h[0], n, 1 - p)
    for k in (1, 2, 3):
        assert close(h[k], n, p / 3)


def test_depolarize2_pauli_distribution():
    p = 0.45
    c = Circuit()
    c.append("R", [0, 1, 2, 4])
    c.append("RX", [3, 5])
    c.append("DEPOLARIZE2", [0, 1], p=p)
    readout_xz(c, 0, 2, 3)
    readout_xz(c, 1, 4, 5)
    c.append("M", [2, 4])
    c.append("MX", [3, 5])
    for r in range(4):
        c.append("DETECTOR", [r])
    n = 300_000
    b = bits(c, n)
    x1, x2, z1, z2 = b[0], b[1], b[2], b[3]
    code = x1 + 2 * z1 + 4 * x2 + 8 * z2
    h = np.bincount(code, minlength=16)
    assert close(h[0], n, 1 - p)
    e = n * p / 15
    chi2 = ((h[1:] - e) ** 2 / e).sum()
    assert chi2 < 14 + 6 * math.sqrt(28)
    # marginal x1 flip: 8 of 15 Paulis carry X or Y on the first qubit
    assert close(x1.sum(), n, 8 * p / 15)


def test_bell_pair_zz_parity():
    pe = 0.2
    c = Circuit()
    c.append("R", [0, 1])
    c.append("H", [0])
    c.append("CX", [0, 1])
    c.append("DEPOLARIZE2", [0, 1], p=pe)
    c.append("M", [0, 1])
    c.append("DETECTOR", [0, 1])
    n = 300_000
    assert close(bits(c, n).sum(), n, 8 * pe / 15)


@pytest.mark.parametrize("N,p", [(7, 0.02), (130, 0.003)])
def test_xor_of_independent_sites(N, p):
    c = Circuit()
    c.append("R", list(range(N + 1)))
    c.append("X_ERROR", list(range(N)), p=p)
    c.append("CX", [v for q in range(N) for v in (q, N)])
    c.append("M", [N])
    c.append("DETECTOR", [0])
    n = 300_000
    assert close(bits(c, n).sum(), n, (1 - (1 - 2 * p) ** N) / 2)


def test_many_targets_rates_and_independence():
    """200 targets = segments of 64, 64, 64 and 8 units."""
    T, p = 200, 0.02
    c = Circuit()
    c.append("R", list(range(T)))
    c.append("X_ERROR", list(range(T)), p=p)
    c.append("M", list(range(T)))
    for q in range(T):
        c.append("DETECTOR", [q])
    n = 64 * 1500
    b = bits(c, n).astype(np.float64)
    rates = b.mean(axis=1)
    sd = math.sqrt(p * (1 - p) / n)
    assert np.all(np.abs(rates - p) < 5.5 * sd)
    z = (b.sum() / (T * n) - p) / math.sqrt(p * (1 - p) / (T * n))
    assert abs(z) < 5
    # neighbouring targets and neighbouring shots are independent
    cov_t = np.mean(b[:-1] * b[1:]) - p * p
    assert abs(cov_t) < 6 * p / math.sqrt((T - 1) * n)
    cov_s = np.mean(b[:, :-1] * b[:, 1:]) - p * p
    assert abs(cov_s) < 6 * p / math.sqrt(T * (n - 1))
    # per (segment, chunk) event counts are Binomial(64 * units, p)
    counts = b[:64].reshape(64, n // 64, 64).sum(axis=(0, 2))
    assert abs(counts.mean() - 4096 * p) < 5 * math.sqrt(4096 * p * (1 - p) / counts.size)
    assert abs(counts.var() / (4096 * p * (1 - p)) - 1) < 0.2


def test_probability_zero_and_one():
    c = Circuit()
    c.append("R", [0, 1])
    c.append("X_ERROR", [0], p=0.0)
    c.append("X_ERROR", [1], p=1.0)
    c.append("M", [0, 1])
    c.append("DETECTOR", [0])
    c.append("DETECTOR", [1])
    b = bits(c, 1000)
    assert not b[0].any() and b[1].all()


def test_pauli_channel_1_distribution():
    """PAULI_CHANNEL_1(px, py, pz) (Methods "Decoherence"): X, Y, Z with the
    given probabilities, read out through x/z copy CNOTs."""
    px, py, pz = 0.05, 0.12, 0.2
    c = Circuit()
    c.append("R", [0, 1])
    c.append("RX", [2])
    c.append("PAULI_CHANNEL_1", [0], p=(px, py, pz))
    readout_xz(c, 0, 1, 2)
    c.append("M", [1])
    c.append("MX", [2])
    c.append("DETECTOR", [0])
    c.append("DETECTOR", [1])
    n = 300_000
    b = bits(c, n)
    h = np.bincount(b[0] + 2 * b[1], minlength=4)
    assert close(h[1], n, px) and close(h[3], n, py) and close(h[2], n, pz)
    assert close(h[0], n, 1 - px - py - pz)


def test_pauli_channel_1_edges():
    c = Circuit()
    c.append("R", [0, 1, 2])
    c.append("PAULI_CHANNEL_1", [0], p=(0.0, 0.0, 0.0))
    c.append("PAULI_CHANNEL_1", [1], p=(1.0, 0.0, 0.0))
    c.append("PAULI_CHANNEL_1", [2], p=(0.0, 0.0, 1.0))
    c.append("M", [0, 1, 2])
    for r in range(3):
        c.append("DETECTOR", [r])
    b = bits(c, 640)
    assert not b[0].any() and b[1].sum() >= 639 and not b[2].any()


def test_pauli_channel_1_thresholds_oracle_vs_generator():
    """The oracle derives PAULI_CHANNEL_1's event probability and X/Y
    thresholds from (px, py, pz) itself; the op-list generator computes the
    copies the library receives (op.p, op.arg, op.arg2). The two must agree
    exactly, or the oracle and the CUDA sampler would split X/Y/Z differently.
    The split itself is pinned by test_pauli_channel_1_distribution."""
    from paper_2504_05611_gb300.circuits import pauli_channel_thresholds
    rng = np.random.default_rng(77)
    cases = [(0.0, 0.0, 0.0), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (0.1, 0.2, 0.7),
             (1 / 3, 1 / 3, 1 / 3), (1e-9, 1e-9, 1e-9), (0.25, 0.25, 0.5), (2.5e-5, 2.5e-5, 4.9e-5)]
    for _ in range(2000):
        v = rng.random(3) * rng.choice([1e-6, 1e-3, 0.1, 0.33])
        cases.append(tuple(float(x) for x in v))
    for ch in cases:
        assert oracle.pauli_channel(*ch) == pauli_channel_thresholds(*ch), ch
    # PAULI_CHANNEL_1 with p = 1 and a pure X split: every word is below t1
    p, t1, t2 = oracle.pauli_channel(1.0, 0.0, 0.0)
    assert p == 1.0 and t1 == t2 == 2 ** 32 - 1
    with pytest.raises(ValueError):
        oracle.pauli_channel(0.6, 0.6, 0.0)


def test_oracle_reads_channel_not_generator_copy():
    """Planted mismatch: an op whose generator copies (p, arg, arg2) are
    wrong still samples with the oracle's own derivation from (px, py, pz)."""
    def circ(corrupt):
        c = Circuit()
        c.append("R", [0, 1])
        c.append("RX", [2])
        c.append("PAULI_CHANNEL_1", [0], p=(0.3, 0.0, 0.0))
        if corrupt:
            op = c.ops[-1]
            op.p, op.arg, op.arg2 = 0.9, 0, 0    # would mean "Z with probability 0.9"
        readout_xz(c, 0, 1, 2)
        c.append("M", [1])
        c.append("MX", [2])
        c.append("DETECTOR", [0])
        c.append("DETECTOR", [1])
        return c
    assert np.array_equal(bits(circ(False), 2000), bits(circ(True), 2000))
