"""Detector error model on the GPU (single-fault injection, one fault per
lane): every fault's signature equals the oracle's noiseless propagation of
that fault, and the number of distinct signatures reproduces the "cols" of
Table III for the surface-code circuits."""
import numpy as np
import pytest

from conftest import golden_rows
from paper_2504_05611_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_05611_gb300 import tmcs  # noqa: E402
from circuit_gen import random_noisy_circuit  # noqa: E402

T3 = {r[0]: [int(v) for v in r[1:]] for r in golden_rows("table_iii_counts.txt")}


def gpu_signatures(circ):
    s = tmcs.Sampler(circ)
    n = tmcs.tmcs_fault_count(s.handle)
    cols = (n + 63) // 64
    det = torch.empty((circ.n_det, cols), dtype=torch.int64, device="cuda")
    obs = torch.empty((max(circ.n_obs, 1), cols), dtype=torch.int64, device="cuda")
    tmcs.tmcs_fault_signatures(s.handle, 0, n, det, obs if circ.n_obs else None)
    torch.cuda.synchronize()
    d = np.unpackbits(det.cpu().numpy().view(np.uint8).reshape(circ.n_det, -1), axis=1, bitorder="little")[:, :n]
    o = np.unpackbits(obs.cpu().numpy().view(np.uint8).reshape(max(circ.n_obs, 1), -1), axis=1,
                      bitorder="little")[: circ.n_obs, :n]
    s.close()
    return d, o


def oracle_signatures(circ):
    from oracle import dem
    dets, obss, _, _ = dem.signatures(circ)
    n = len(dets)
    d = np.zeros((circ.n_det, n), dtype=np.uint8)
    o = np.zeros((circ.n_obs, n), dtype=np.uint8)
    for f, (dm, om) in enumerate(zip(dets, obss)):
        for j in range(circ.n_det):
            if (dm >> j) & 1:
                d[j, f] = 1
        for j in range(circ.n_obs):
            if (om >> j) & 1:
                o[j, f] = 1
    return d, o


@pytest.mark.parametrize("case", ["nl_sc3", "tp_sc3", "nl_bb18", "deco_sc5"])
def test_signatures_equal_oracle(case):
    if case == "nl_sc3":
        circ = C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2)
    elif case == "tp_sc3":
        circ = C.teleport_circuit(C.code_by_name("sc3"), 2, 2)
    elif case == "nl_bb18":
        circ = C.nonlocal_cnot_circuit(C.code_by_name("bb18"), 1, 1)
    else:
        circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 1, 1,
                                       C.NoiseModel(1e-3, 1e-2, decoherence=C.Decoherence(1e-3, schedule="lines")))
    gd, go = gpu_signatures(circ)
    od, oo = oracle_signatures(circ)
    assert gd.shape == od.shape
    assert np.array_equal(gd, od) and np.array_equal(go, oo)


@pytest.mark.parametrize("trial", range(4))
def test_signatures_random_circuits(trial):
    rng = np.random.default_rng(70 + trial)
    circ = random_noisy_circuit(rng, int(rng.integers(3, 9)), int(rng.integers(10, 40)))
    gd, go = gpu_signatures(circ)
    od, oo = oracle_signatures(circ)
    assert np.array_equal(gd, od) and np.array_equal(go, oo)


@pytest.mark.parametrize("key", ["sc3", "sc5", "sc7", "sc9", "sc11"])
def test_table_iii_columns_on_gpu(key):
    """Distinct single-fault signatures found by fault injection on the GPU
    (one fault per lane, tmcs_fault_signatures) are exactly the columns of
    tmcs_dem_columns, and their number is Table III's "cols" for the
    4/3-round circuits (non-local CNOT and teleportation)."""
    code = C.code_by_name(key)
    for fn, idx in ((C.nonlocal_cnot_circuit, 4), (C.teleport_circuit, 9)):
        circ = fn(code, 4, 3)
        d, o = gpu_signatures(circ)
        sigs = np.concatenate([d, o], axis=0).T
        nonempty = sigs[sigs.any(axis=1)]
        gpu_cols = {tuple(np.nonzero(r)[0]) for r in np.unique(nonempty, axis=0)}
        h = tmcs.tmcs_circuit_build(circ)
        cols, _, _ = tmcs.tmcs_dem_columns(h)
        tmcs.tmcs_circuit_free(h)
        lib_cols = {tuple(dd) + tuple(circ.n_det + ob for ob in oo) for dd, oo in cols}
        assert gpu_cols == lib_cols
        assert len(lib_cols) == T3[key][idx]


@pytest.mark.parametrize("case", ["nl_sc5", "tp_bb18"])
def test_gpu_marginals_match_exact_dem(case):
    """Whole-circuit statistics of 4e6 GPU shots: every detector's and
    observable's flip frequency is within 6 standard errors of the exact
    probability from the oracle's single-fault DEM, (1 - prod(1 - 2 P_c)) / 2,
    and so is the parity of detector pairs that share a fault."""
    from oracle import dem
    if case == "nl_sc5":
        circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 3, 3, C.NoiseModel(0.002, 0.02))
    else:
        circ = C.teleport_circuit(C.code_by_name("bb18"), 2, 2, C.NoiseModel(0.002, 0.02))
    shots = 4_000_000
    s = tmcs.Sampler(circ)
    det, obs = s.sample(shots, seed=2024)
    torch.cuda.synchronize()
    d = det.cpu().numpy().view(np.uint64)
    o = obs.cpu().numpy().view(np.uint64)
    s.close()

    def freq(words):
        bits = np.unpackbits(words.view(np.uint8).reshape(words.shape[0], -1), axis=1, bitorder="little")
        return bits[:, :shots].sum(axis=1) / shots

    pd, po = dem.flip_probabilities(circ)
    for f, p in ((freq(d), pd), (freq(o), po)):
        se = np.sqrt(np.maximum(p * (1 - p), 1e-12) / shots)
        assert np.all(np.abs(f - p) <= 6 * se + 1e-9), np.max(np.abs(f - p) / se)
    # detector pairs: first detector with each of the next few
    bits = np.unpackbits(d.view(np.uint8).reshape(d.shape[0], -1), axis=1, bitorder="little")[:, :shots]
    for a, b in ((0, 1), (0, 5), (3, 9), (10, 11)):
        p = dem.pair_flip_probability(circ, a, b)
        f = np.mean(bits[a] ^ bits[b])
        assert abs(f - p) <= 6 * np.sqrt(max(p * (1 - p), 1e-12) / shots) + 1e-9, (a, b, f, p)
