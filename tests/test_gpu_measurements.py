"""Raw measurement sampling on the GPU (tmcs_sample_measurements).

* Every record bit equals the oracle's gauge-randomised sampler on the same
  seed and chunk range (bit-exact), on circuits with every op kind, ragged
  tails and nonzero first chunks.
* Detector parities recomputed from the GPU records, XORed with their values
  on the reference record, equal tmcs_sample_range's detector bits: the two
  programs share their noise draws.
* At the non-local CNOT size the bench runs, sampled columns of one large
  call equal the oracle's columns computed alone, up to the reference bit
  of each record row.
"""
import numpy as np
import pytest

import oracle
from oracle import tableau
from paper_2504_05611_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_05611_gb300 import tmcs  # noqa: E402
from circuit_gen import random_noisy_circuit  # noqa: E402
from test_oracle_measurements import random_measured  # noqa: E402


def gpu_records(circ, shots, seed, first_chunk=0, flags=0, handle=None):
    h = handle if handle is not None else tmcs.tmcs_circuit_build(circ, flags)
    try:
        cols = (shots + 63) // 64
        meas = torch.full((max(circ.n_meas, 1), cols), -1, dtype=torch.int64, device="cuda")
        tmcs.tmcs_sample_measurements(h, first_chunk, shots, seed, meas)
        torch.cuda.synchronize()
        tmcs.tmcs_check_device()
        return meas[: circ.n_meas].cpu().numpy().view(np.uint64)
    finally:
        if handle is None:
            tmcs.tmcs_circuit_free(h)


def cases():
    out = [
        ("nl_sc3", C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.01, 0.05)), 0),
        ("tp_bb18", C.teleport_circuit(C.code_by_name("bb18"), 1, 1, C.NoiseModel(0.004, 0.03)), 0),
        ("mem_sc5", C.memory_circuit(C.code_by_name("sc5"), 3, C.NoiseModel(0.02, 0.02)), 0),
        ("ps4_sc3", C.pauli_string_circuit(C.code_by_name("sc3"), 4, rounds_before=1, noise=C.NoiseModel(0.003, 0.02)), 0),
        ("deco_sc3", C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2,
                                             C.NoiseModel(0.003, 0.02, decoherence=C.Decoherence(0.05))), 0),
    ]
    for t in range(4):
        rng = np.random.default_rng(900 + t)
        out.append((f"rand{t}", random_noisy_circuit(rng, int(rng.integers(2, 9)), int(rng.integers(4, 40))), 0))
    for t in range(3):
        rng = np.random.default_rng(950 + t)
        # random outcomes and conditioned Paulis: no deterministic detectors
        out.append((f"meas{t}", random_measured(rng, int(rng.integers(2, 7)), 30), tmcs.TMCS_FLAG_NO_AUDIT))
    return out


CASES = cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("shots,first_chunk", [(64 * 37 + 13, 5), (64 * 3, 0), (1, 1000)])
def test_records_equal_oracle(case, shots, first_chunk):
    _, circ, flags = case
    got = gpu_records(circ, shots, seed=77, first_chunk=first_chunk, flags=flags)
    want = oracle.sample_measurements(circ, shots, seed=77, first_chunk=first_chunk, threads=8)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def detector_words(circ, rec_words):
    """Detector parities (per detector, per column) from record rows."""
    out = []
    for op in circ.ops:
        if op.name == "DETECTOR":
            v = np.zeros(rec_words.shape[1], dtype=np.uint64)
            for r in op.targets:
                v ^= rec_words[int(r)]
            out.append(v)
    return np.array(out, dtype=np.uint64).reshape(len(out), rec_words.shape[1])


@pytest.mark.parametrize("name", ["nl_sc5", "tp_bb18"])
def test_detectors_from_records_equal_detector_sampler(name):
    if name == "nl_sc5":
        circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 3, 3, C.NoiseModel(0.005, 0.05))
    else:
        circ = C.teleport_circuit(C.code_by_name("bb18"), 2, 2, C.NoiseModel(0.005, 0.05))
    shots, first_chunk, seed = 64 * 500 + 17, 9, 1234
    h = tmcs.tmcs_circuit_build(circ)
    try:
        rec = gpu_records(circ, shots, seed, first_chunk, handle=h)
        cols = rec.shape[1]
        det = torch.empty((circ.n_det, cols), dtype=torch.int64, device="cuda")
        obs = torch.empty((max(circ.n_obs, 1), cols), dtype=torch.int64, device="cuda")
        tmcs.tmcs_sample_range(h, first_chunk, shots, seed, det, obs)
        torch.cuda.synchronize()
        det = det.cpu().numpy().view(np.uint64)
    finally:
        tmcs.tmcs_circuit_free(h)
    ref = tableau.reference_sample(circ)["rec"].astype(np.uint64)
    ref_words = np.where(ref[:, None] == 1, ~np.uint64(0), np.uint64(0)) * np.ones((1, cols), dtype=np.uint64)
    mask = np.full(cols, ~np.uint64(0), dtype=np.uint64)
    mask[-1] = np.uint64((1 << (shots % 64)) - 1) if shots % 64 else ~np.uint64(0)
    got = (detector_words(circ, rec) ^ detector_words(circ, ref_words)) & mask[None, :]
    assert np.array_equal(got, det)
    assert det.any()


def test_full_size_sampled_columns():
    """NL(29) at the error rates of the sampling throughput workload, one
    large call. The oracle runs the sampled chunks alone with an all-zero
    reference (its Python tableau is too slow at 5044 qubits), so GPU XOR
    oracle must be one constant per record row -- the reference bit -- across
    every lane of the start, middle and ragged-end columns; that constant
    row is the library's host reference record."""
    circ = C.WORKLOADS["nl_sc29"].circuit()
    shots = 64 * 1024 + 33
    h = tmcs.tmcs_circuit_build(circ)
    try:
        got = gpu_records(circ, shots, seed=5, handle=h)
        ref = tmcs.tmcs_reference_sample(h).astype(np.uint64)
    finally:
        tmcs.tmcs_circuit_free(h)
    cols = got.shape[1]
    zero_ref = np.zeros(circ.n_meas, dtype=np.uint8)
    for c0 in (0, 517, cols - 1):
        n = 64 if c0 < cols - 1 else 33
        mask = np.uint64((1 << n) - 1) if n < 64 else ~np.uint64(0)
        want = oracle.sample_measurements(circ, n, seed=5, first_chunk=c0, threads=8, reference=zero_ref)
        diff = got[:, c0] ^ want[:, 0]
        assert np.all((diff == 0) | (diff == mask)), c0
        assert np.array_equal((diff != 0).astype(np.uint64), ref), c0
