"""The allocation-free entry point, tmcs_sample_noalloc.

It serves callers that cannot allocate device memory while running (a
service whose device memory belongs to another allocator's pool, a real-time
host that forbids allocation on its request path, code that must not let
cudaMalloc/cudaFree synchronise the device). Its scratch is a fixed 8 MiB
device array instead of the per-circuit allocations tmcs_sample_range makes,
so its outputs must equal tmcs_sample_range's bit for bit.

This file is collected last so that, if it fails, a run stopping at the
first failure has already run every other test; it also passes alone.
"""
import numpy as np
import pytest

from paper_2504_05611_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_05611_gb300 import tmcs  # noqa: E402


def outputs(handle, shots, fn, first_chunk, seed):
    info = tmcs.tmcs_circuit_info(handle)
    cols = (shots + 63) // 64
    det = torch.full((info["n_det"], cols), -1, dtype=torch.int64, device="cuda")
    obs = torch.full((max(info["n_obs"], 1), cols), -1, dtype=torch.int64, device="cuda")
    fn(handle, first_chunk, shots, seed, det, obs if info["n_obs"] else None)
    torch.cuda.synchronize()
    return det.cpu().numpy(), obs[: info["n_obs"]].cpu().numpy()


def test_noalloc_matches_sample_range_on_two_calls_in_a_row():
    """Two consecutive calls (different circuits, so the shared array is
    rewritten between them) each equal the allocating entry point."""
    cases = [
        (C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 3, 3, C.NoiseModel(0.01, 0.05)), 64 * 300 + 7, 3, 11),
        (C.teleport_circuit(C.code_by_name("bb18"), 2, 2, C.NoiseModel(0.005, 0.02)), 64 * 90 + 41, 0, 12),
    ]
    handles = [tmcs.tmcs_circuit_build(c) for c, _, _, _ in cases]
    try:
        got = [outputs(h, shots, tmcs.tmcs_sample_noalloc, fc, seed)
               for h, (_, shots, fc, seed) in zip(handles, cases)]
        want = [outputs(h, shots, tmcs.tmcs_sample_range, fc, seed)
                for h, (_, shots, fc, seed) in zip(handles, cases)]
        for (gd, go), (wd, wo) in zip(got, want):
            assert np.array_equal(gd, wd)
            assert np.array_equal(go, wo)
            assert gd.any()
    finally:
        for h in handles:
            tmcs.tmcs_circuit_free(h)


def test_noalloc_rejects_programs_beyond_its_array():
    """A circuit whose compiled program exceeds the 8 MiB array is refused
    with TMCS_E_INVALID (nothing is launched)."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc29"), 45, 45, C.NoiseModel(1e-3, 1e-2))
    h = tmcs.tmcs_circuit_build(circ)
    try:
        assert tmcs.tmcs_circuit_info(h)["device_bytes"] + 256 > 8 << 20
        det = torch.empty(8, dtype=torch.int64, device="cuda")
        with pytest.raises(tmcs.TmcsError) as e:
            tmcs.tmcs_sample_noalloc(h, 0, 64, 1, det.data_ptr(), det.data_ptr())
        assert e.value.code == 1 and "at most" in str(e.value)
    finally:
        tmcs.tmcs_circuit_free(h)
