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
    """Distinct single-fault signatures of the 4/3-round circuits equal the
    'cols' of Table III (non-local CNOT and teleportation)."""
    code = C.code_by_name(key)
    for fn, idx in ((C.nonlocal_cnot_circuit, 4), (C.teleport_circuit, 9)):
        s = tmcs.Sampler(fn(code, 4, 3))
        assert len(tmcs.dem_columns(s)) == T3[key][idx]
        s.close()
