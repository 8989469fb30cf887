"""The continuous-batching server: every request's result equals a solo
tmcs_sample of the same circuit, shots and seed, whether it ran alone or
overlapped with other requests, and requests wait for arena space instead
of failing (admission by HBM footprint)."""
import threading
import time

import numpy as np
import pytest

from paper_2504_05611_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_05611_gb300 import tmcs  # noqa: E402


def solo(sampler, shots, seed):
    det, obs = sampler.sample(shots, seed)
    torch.cuda.synchronize()
    return det.cpu().numpy().view(np.uint64), obs.cpu().numpy().view(np.uint64)


def mix():
    rng = np.random.default_rng(4)
    out = []
    for j in range(14):
        code = C.code_by_name(["sc3", "sc5", "sc7", "bb18", "sc11"][j % 5])
        nz = C.NoiseModel(0.005, 0.02)
        circ = C.nonlocal_cnot_circuit(code, 2, 2, nz) if j % 2 == 0 else C.teleport_circuit(code, 2, 2, nz)
        out.append((tmcs.Sampler(circ), int(rng.integers(1, 64 * 700)), 500 + j))
    return out


def test_alone_and_in_the_mix_equal_solo():
    jobs = mix()
    srv = tmcs.Server(arena_bytes=1 << 30, n_streams=4, slice_chunks=96)
    try:
        # alone: one request at a time
        s, n, seed = jobs[0]
        rid = srv.submit(s, n, seed)
        d, o = srv.fetch(rid)
        sd, so = solo(s, n, seed)
        assert np.array_equal(d, sd) and np.array_equal(o, so)
        # in the mix: all submitted at once, from two client threads
        ids = [None] * len(jobs)

        def submit(lo, hi):
            for i in range(lo, hi):
                s, n, seed = jobs[i]
                ids[i] = srv.submit(s, n, seed)
                time.sleep(0.001)

        ts = [threading.Thread(target=submit, args=(0, 7)), threading.Thread(target=submit, args=(7, 14))]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        for i in reversed(range(len(jobs))):
            s, n, seed = jobs[i]
            d, o = srv.fetch(ids[i])
            sd, so = solo(s, n, seed)
            assert np.array_equal(d, sd), i
            assert np.array_equal(o, so), i
        st = srv.stats()
        assert st["completed"] == len(jobs) + 1 and st["failed"] == 0
        assert st["latency_p99_s"] >= st["latency_p50_s"] > 0
        assert st["arena_in_use"] == 0
    finally:
        srv.close()
        for s, _, _ in jobs:
            s.close()


def test_admission_waits_for_arena_space():
    """An arena that holds one request at a time still completes all of them."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 2, 2, C.NoiseModel(0.01, 0.03))
    s = tmcs.Sampler(circ)
    shots = 64 * 300
    need = (s.info["n_det"] + s.info["n_obs"]) * 300 * 8
    srv = tmcs.Server(arena_bytes=need + need // 2, n_streams=2, slice_chunks=64)
    try:
        ids = [srv.submit(s, shots, 900 + i) for i in range(5)]
        assert srv.stats()["queued"] >= 3
        for i, rid in enumerate(ids):
            d, o = srv.fetch(rid)
            sd, so = solo(s, shots, 900 + i)
            assert np.array_equal(d, sd) and np.array_equal(o, so)
        with pytest.raises(tmcs.TmcsError):
            srv.submit(s, 64 * 10000, 1)   # larger than the arena: refused at once
    finally:
        srv.close()
        s.close()


def test_measured_peaks_are_plausible():
    """The shared-memory and integer-pipe microbenchmarks give rates in the
    range a Blackwell part can reach (per SM: at most one 128-byte shared
    wavefront and 128 LOP3 lane-operations per clock at <= 3 GHz)."""
    p = tmcs.tmcs_measure_peaks()
    sms = p["sms"]
    assert sms > 0
    assert 0.1e12 * sms / 152 < p["smem_load_bytes_per_s"] <= sms * 128 * 3e9
    assert 1e9 < p["smem_atomic_lanes_per_s"] <= sms * 32 * 3e9
    assert 1e12 < p["lop3_lanes_per_s"] <= sms * 128 * 3e9
