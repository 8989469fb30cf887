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


def test_noalloc_distance29_headline_circuit():
    """The documented use case: the distance-29 non-local CNOT (29/29 rounds),
    whose compiled program (about 6 MiB) fits the array, against the
    allocating entry point over several CTA tiles and a ragged last chunk."""
    circ = C.WORKLOADS["nl_sc29"].circuit()
    h = tmcs.tmcs_circuit_build(circ)
    try:
        assert tmcs.tmcs_circuit_info(h)["device_bytes"] + 256 <= 8 << 20
        shots, fc, seed = 64 * 152 * 2 + 17, 1000, 1
        gd, go = outputs(h, shots, tmcs.tmcs_sample_noalloc, fc, seed)
        wd, wo = outputs(h, shots, tmcs.tmcs_sample_range, fc, seed)
        assert np.array_equal(gd, wd) and np.array_equal(go, wo)
        assert gd.any()
    finally:
        tmcs.tmcs_circuit_free(h)


@pytest.mark.parametrize("env", [{"TMCS_KERNEL": "3", "TMCS_TILE_K": "2", "TMCS_THREADS": "128"},
                                 {"TMCS_KERNEL": "4", "TMCS_WARPS": "3", "TMCS_GROUP": "2"},
                                 {"TMCS_KERNEL": "4", "TMCS_TILE_K": "2", "TMCS_WARPS": "4"}])
def test_noalloc_forced_shapes_and_side_stream(monkeypatch, env):
    """Forced frame-kernel launch shapes, on a non-default stream, equal the
    allocating entry point's default output."""
    circ = C.teleport_circuit(C.code_by_name("sc5"), 2, 2, C.NoiseModel(0.01, 0.05))
    h = tmcs.tmcs_circuit_build(circ)
    try:
        shots, fc, seed = 64 * 53 + 17, 5, 21
        wd, wo = outputs(h, shots, tmcs.tmcs_sample_range, fc, seed)
        info = tmcs.tmcs_circuit_info(h)
        cols = (shots + 63) // 64
        side = torch.cuda.Stream()
        with monkeypatch.context() as m:
            for k, v in env.items():
                m.setenv(k, v)
            with torch.cuda.stream(side):
                det = torch.full((info["n_det"], cols), -1, dtype=torch.int64, device="cuda")
                obs = torch.full((info["n_obs"], cols), -1, dtype=torch.int64, device="cuda")
                tmcs.tmcs_sample_noalloc(h, fc, shots, seed, det, obs, stream=side)
        side.synchronize()
        assert np.array_equal(det.cpu().numpy(), wd) and np.array_equal(obs.cpu().numpy(), wo)
    finally:
        tmcs.tmcs_circuit_free(h)


def test_noalloc_expired_wait_is_reported(monkeypatch):
    """A bounded device-side wait that expired in an allocation-free call
    marks the array's status word; tmcs_check_device reports it as
    TMCS_E_TIMEOUT and clears it (the mark is planted by the host here, as a
    kernel that gave up would set it)."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.01, 0.05))
    h = tmcs.tmcs_circuit_build(circ)
    try:
        tmcs.tmcs_check_device()
        with monkeypatch.context() as m:
            m.setenv("TMCS_TEST_NOALLOC_EXPIRED", "1")
            outputs(h, 640, tmcs.tmcs_sample_noalloc, 0, 3)
        # a later call does not clear it
        outputs(h, 640, tmcs.tmcs_sample_noalloc, 0, 3)
        with pytest.raises(tmcs.TmcsError) as e:
            tmcs.tmcs_check_device()
        assert e.value.code == 5
        tmcs.tmcs_check_device()
    finally:
        tmcs.tmcs_circuit_free(h)
