"""GPU parity: the CUDA sampler (through the C ABI) against the CPU oracle.

Every comparison is bit-exact: both sides implement the same sampling
specification, so detector and observable words must be identical,
including zero pad bits. Sizes span several CTA tiles and a ragged last
chunk; the full-size workloads are checked on sampled chunks the oracle
recomputes one by one (``first_chunk`` keying).
"""
import numpy as np
import pytest

import oracle
from paper_2504_05611_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_05611_gb300 import tmcs  # noqa: E402
from circuit_gen import random_noisy_circuit  # noqa: E402


def gpu_sample(circ, shots, seed, first_chunk=0, flags=0):
    s = tmcs.Sampler(circ, flags)
    det, obs = s.sample(shots, seed, first_chunk=first_chunk)
    torch.cuda.synchronize()
    out = det.cpu().numpy().view(np.uint64), obs.cpu().numpy().view(np.uint64)
    s.close()
    return out


def assert_parity(circ, shots, seed, first_chunk=0, flags=0, threads=8):
    gd, go = gpu_sample(circ, shots, seed, first_chunk, flags)
    od, oo = oracle.sample(circ, shots, seed, first_chunk=first_chunk, threads=threads)
    assert gd.shape == od.shape and go.shape == oo.shape
    bad = np.argwhere(gd != od)
    assert bad.size == 0, f"{len(bad)} detector words differ, first at {bad[:3].tolist()}"
    assert np.array_equal(go, oo)
    return gd, go


def test_config_nl_sc3_full():
    """Distance-3 SC non-local CNOT, 3/3 rounds, p=1e-3, p_ebit=1e-2, 1e4 shots, seed 1."""
    w = C.WORKLOADS["nl_sc3"]
    gd, _ = assert_parity(w.circuit(), w.shots, w.seed)
    assert gd.any()


@pytest.mark.parametrize("kind", ["nl", "teleport", "memory"])
@pytest.mark.parametrize("code", ["sc3", "sc5", "bb18"])
def test_protocols_high_noise(kind, code):
    cc = C.code_by_name(code)
    nz = C.NoiseModel(p=0.02, p_ebit=0.05)
    if kind == "nl":
        circ = C.nonlocal_cnot_circuit(cc, 2, 2, nz)
    elif kind == "teleport":
        circ = C.teleport_circuit(cc, 2, 2, nz)
    else:
        circ = C.memory_circuit(cc, 3, nz)
    assert_parity(circ, 64 * 37 + 5, seed=7)


def test_config_nl_sc11_reduced_shots():
    w = C.WORKLOADS["nl_sc11"]
    assert_parity(w.circuit(), 64 * 160 + 29, w.seed)


def test_config_tp_bb144_reduced_shots():
    w = C.WORKLOADS["tp_bb144"]
    assert_parity(w.circuit(), 64 * 40 + 3, w.seed)


def test_idle_and_feed_noise_variants():
    nz = C.NoiseModel(p=0.01, p_ebit=0.03, idle=True, feed_noise=True)
    assert_parity(C.teleport_circuit(C.code_by_name("bb18"), 2, 2, nz), 64 * 20 + 1, seed=3)


@pytest.mark.parametrize("shots", [1, 63, 64, 65, 127, 1000])
def test_ragged_shot_counts(shots):
    assert_parity(C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 1, 1, C.NoiseModel(0.05, 0.1)),
                  shots, seed=99)


def test_first_chunk_sharding_concatenates():
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 2, 2, C.NoiseModel(0.01, 0.05))
    full_d, full_o = gpu_sample(circ, 64 * 50, 5)
    a_d, a_o = gpu_sample(circ, 64 * 20, 5, first_chunk=0)
    b_d, b_o = gpu_sample(circ, 64 * 30, 5, first_chunk=20)
    assert np.array_equal(np.concatenate([a_d, b_d], 1), full_d)
    assert np.array_equal(np.concatenate([a_o, b_o], 1), full_o)
    assert_parity(circ, 64 * 3 + 7, seed=5, first_chunk=123456)


def test_pruning_is_exact():
    """Liveness pruning only removes work: the unpruned program gives the same bits."""
    circ = C.teleport_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.02, 0.05))
    a = gpu_sample(circ, 64 * 30, 11)
    b = gpu_sample(circ, 64 * 30, 11, flags=tmcs.TMCS_FLAG_NO_PRUNE)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_noiseless_is_zero_and_certain_noise():
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.0, 0.0))
    d, o = gpu_sample(circ, 640, 1)
    assert not d.any() and not o.any()
    c = C.Circuit()
    c.append("R", [0, 1])
    c.append("X_ERROR", [1], p=1.0)
    c.append("M", [0, 1])
    c.append("DETECTOR", [0])
    c.append("DETECTOR", [1])
    c.append("OBSERVABLE", [1], arg=0)
    c.append("OBSERVABLE", [0, 1], arg=0)   # accumulates: obs = r1 ^ r0 ^ r1 = r0
    d, o = assert_parity(c, 100, 1)
    assert not d[0].any() and (d[1][0] == np.uint64(2 ** 64 - 1)) and not o.any()


@pytest.mark.parametrize("trial", range(12))
def test_random_circuits(trial):
    rng = np.random.default_rng(900 + trial)
    circ = random_noisy_circuit(rng, int(rng.integers(2, 9)), int(rng.integers(4, 40)))
    assert_parity(circ, 64 * 9 + int(rng.integers(1, 64)), seed=int(rng.integers(1, 2 ** 62)))


def _batch(jobs, kernel, monkeypatch):
    """Batched launch; kernel "frame" forces the frame-kernel batch path."""
    if kernel == "frame":
        with monkeypatch.context() as m:
            m.setenv("TMCS_KERNEL", "3")
            tmcs.tmcs_batch_sample(jobs)
    else:
        tmcs.tmcs_batch_sample(jobs)


@pytest.mark.parametrize("kernel", ["signature", "frame"])
def test_batch_equals_solo(kernel, monkeypatch):
    """Batched launch (event-signature or frame-kernel path) equals each job's
    solo call (default path)."""
    circs = [C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.01, 0.1)),
             C.teleport_circuit(C.code_by_name("bb18"), 1, 1, C.NoiseModel(0.003, 0.03)),
             C.memory_circuit(C.code_by_name("sc5"), 3, C.NoiseModel(0.02, 0.02))]
    samplers = [tmcs.Sampler(c) for c in circs]
    shots = [64 * 7 + 3, 1000, 64 * 33]
    outs = [s.alloc(n) for s, n in zip(samplers, shots)]
    jobs = [(s.handle, n, 40 + i, d, o) for i, (s, n, (d, o)) in enumerate(zip(samplers, shots, outs))]
    _batch(jobs, kernel, monkeypatch)
    torch.cuda.synchronize()
    for i, (circ, n) in enumerate(zip(circs, shots)):
        d, o = outs[i]
        sd, so = gpu_sample(circ, n, 40 + i)
        assert np.array_equal(d.cpu().numpy().view(np.uint64), sd)
        assert np.array_equal(o[: circ.n_obs].cpu().numpy().view(np.uint64), so)
    for s in samplers:
        s.close()


@pytest.mark.parametrize("capture", [False, True])
def test_batch_with_gpu_filling_job(capture):
    """A job of at least 16 chunks per SM runs as its own tuned call inside
    tmcs_batch_sample; every job still equals its solo call, also when the
    batch is captured in a CUDA graph and replayed."""
    circs = [C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 3, 3, C.NoiseModel(0.003, 0.03)),
             C.teleport_circuit(C.code_by_name("bb18"), 1, 1, C.NoiseModel(0.003, 0.03)),
             C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.01, 0.1))]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    shots = [64 * 16 * sms + 5, 64 * 20 + 7, 999]
    samplers = [tmcs.Sampler(c) for c in circs]
    outs = [s.alloc(n) for s, n in zip(samplers, shots)]
    jobs = [(s.handle, n, 60 + i, d, o) for i, (s, n, (d, o)) in enumerate(zip(samplers, shots, outs))]
    tmcs.tmcs_batch_sample(jobs)
    torch.cuda.synchronize()
    if capture:
        for d, o in outs:
            d.zero_()
            o.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            tmcs.tmcs_batch_sample(jobs)
        g.replay()
        torch.cuda.synchronize()
    for i, (circ, n) in enumerate(zip(circs, shots)):
        d, o = outs[i]
        sd, so = gpu_sample(circ, n, 60 + i)
        assert np.array_equal(d.cpu().numpy().view(np.uint64), sd)
        assert np.array_equal(o[: circ.n_obs].cpu().numpy().view(np.uint64), so)
    for s in samplers:
        s.close()


def test_headline_full_size_sampled_chunks():
    """Distance-29 SC non-local CNOT, 29/29 rounds, 1e7 shots: sampled chunks
    (first, middle, last with its ragged tail) against the oracle."""
    w = C.WORKLOADS["nl_sc29"]
    circ = w.circuit()
    shots = w.shots
    s = tmcs.Sampler(circ)
    det, obs = s.sample(shots, w.seed)
    torch.cuda.synchronize()
    cols = (shots + 63) // 64
    for col in (0, cols // 2, cols - 1):
        n = min(64, shots - 64 * col)
        od, oo = oracle.sample(circ, n, w.seed, first_chunk=col, threads=8)
        assert np.array_equal(det[:, col].cpu().numpy().view(np.uint64), od[:, 0])
        assert np.array_equal(obs[:, col].cpu().numpy().view(np.uint64), oo[:, 0])
    # every detector word has zero pad bits (shots is a multiple of 64 here)
    assert shots % 64 == 0
    s.close()


def test_device_status_clean_after_sampling():
    """No kernel gave up on a bounded wait during the runs above."""
    tmcs.tmcs_check_device()


@pytest.mark.parametrize("kernel,tile_k,threads,warps,group", [
    (3, 1, 128, 0, 0), (3, 1, 256, 0, 0), (3, 2, 256, 0, 0), (3, 4, 512, 0, 0), (3, 8, 256, 0, 0),
    (3, 16, 512, 0, 0), (4, 1, 0, 1, 1), (4, 1, 0, 5, 1), (4, 1, 0, 15, 1), (4, 2, 0, 3, 1), (4, 2, 0, 15, 1),
    (4, 1, 0, 3, 2), (4, 1, 0, 8, 2), (4, 2, 0, 4, 4), (4, 1, 0, 2, 8)])
def test_every_launch_shape_is_bit_exact(monkeypatch, kernel, tile_k, threads, warps, group):
    """Launch shape (kernel, chunks per CTA or per warp, CTA size, warps)
    changes only the schedule: every forced shape reproduces the oracle,
    ragged tail included."""
    monkeypatch.setenv("TMCS_KERNEL", str(kernel))
    monkeypatch.setenv("TMCS_TILE_K", str(tile_k))
    if threads:
        monkeypatch.setenv("TMCS_THREADS", str(threads))
    if warps:
        monkeypatch.setenv("TMCS_WARPS", str(warps))
    if group:
        monkeypatch.setenv("TMCS_GROUP", str(group))
    circ = C.teleport_circuit(C.code_by_name("sc5"), 2, 2, C.NoiseModel(0.01, 0.05))
    assert_parity(circ, 64 * 53 + 17, seed=21)


@pytest.mark.parametrize("tile_k,threads", [(1, 256), (1, 1024), (2, 512), (4, 256), (4, 1024), (8, 512),
                                           (16, 1024), (16, 512)])
@pytest.mark.parametrize("window", [0, 1024])
def test_signature_kernel_shapes_are_bit_exact(monkeypatch, tile_k, threads, window):
    """The event-signature kernel under every chunks-per-CTA / CTA-size
    choice, with the default detector ring and with a 1024-detector ring that
    splits the circuit into several flush steps, reproduces the oracle."""
    monkeypatch.setenv("TMCS_KERNEL", "5")
    monkeypatch.setenv("TMCS_TILE_K", str(tile_k))
    monkeypatch.setenv("TMCS_THREADS", str(threads))
    if window:
        monkeypatch.setenv("TMCS_SIG_WINDOW", str(window))
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc9"), 9, 9, C.NoiseModel(0.004, 0.03))
    h = tmcs.tmcs_circuit_build(circ)
    st = tmcs.tmcs_circuit_stats(h)
    tmcs.tmcs_circuit_free(h)
    assert st["sig_ok"] == 1 and (window == 0 or st["sig_steps"] > 1)
    assert_parity(circ, 64 * 41 + 29, seed=23, first_chunk=7)


@pytest.mark.parametrize("sched", [0, 1, 2])
@pytest.mark.parametrize("tile_k,threads", [(4, 1024), (8, 512), (2, 256)])
def test_signature_schedules_are_bit_exact(monkeypatch, sched, tile_k, threads):
    """Every ring-window schedule of the program (4096, 2048 and 1024
    detectors for this circuit) reproduces the oracle."""
    monkeypatch.setenv("TMCS_KERNEL", "5")
    monkeypatch.setenv("TMCS_SIG_SCHED", str(sched))
    monkeypatch.setenv("TMCS_TILE_K", str(tile_k))
    monkeypatch.setenv("TMCS_THREADS", str(threads))
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc11"), 11, 11, C.NoiseModel(0.003, 0.02))
    h = tmcs.tmcs_circuit_build(circ)
    st = tmcs.tmcs_circuit_stats(h)
    tmcs.tmcs_circuit_free(h)
    assert st["sig_schedules"] == 3
    assert_parity(circ, 64 * 19 + 45, seed=29, first_chunk=3)


@pytest.mark.parametrize("sched", range(6))
@pytest.mark.parametrize("tile_k,threads", [(4, 1024), (8, 512), (1, 256), (2, 128), (16, 1024)])
def test_pipelined_kernel_is_bit_exact(monkeypatch, sched, tile_k, threads):
    """The pipelined event-signature kernel under each of its schedules (step
    window x steps in flight) and launch shapes reproduces the oracle: ragged
    tail, nonzero first chunk, many flush steps per tile."""
    monkeypatch.setenv("TMCS_KERNEL", "6")
    monkeypatch.setenv("TMCS_SIG_SCHED", str(sched))
    monkeypatch.setenv("TMCS_TILE_K", str(tile_k))
    monkeypatch.setenv("TMCS_THREADS", str(threads))
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc11"), 11, 11, C.NoiseModel(0.003, 0.02))
    h = tmcs.tmcs_circuit_build(circ)
    st = tmcs.tmcs_circuit_stats(h)
    tmcs.tmcs_circuit_free(h)
    assert st["sig_pipe_schedules"] == 6
    assert_parity(circ, 64 * 19 + 45, seed=29, first_chunk=3)


@pytest.mark.parametrize("sched", range(3))
@pytest.mark.parametrize("tile_k,threads,shots", [(1, 1024, 64 * 1000 + 37), (2, 512, 64 * 1000 + 37),
                                                  (2, 512, 64 * 1000), (4, 256, 64 * 2002 - 5)])
def test_pipelined_kernel_many_tiles_per_cta(monkeypatch, sched, tile_k, threads, shots):
    """Several tiles per CTA: the ring offset and the observable buffer of
    each tile alternate while steps of two tiles are in flight. Odd and even
    column counts take the scalar and the 16-byte output paths."""
    monkeypatch.setenv("TMCS_KERNEL", "6")
    monkeypatch.setenv("TMCS_SIG_SCHED", str(sched))
    monkeypatch.setenv("TMCS_TILE_K", str(tile_k))
    monkeypatch.setenv("TMCS_THREADS", str(threads))
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 6, 6, C.NoiseModel(0.01, 0.05))
    h = tmcs.tmcs_circuit_build(circ)
    st = tmcs.tmcs_circuit_stats(h)
    tmcs.tmcs_circuit_free(h)
    assert st["sig_pipe_schedules"] == 3
    gd, go = assert_parity(circ, shots, seed=41, first_chunk=11)
    assert gd.any() and go.any()


_NL7_CACHE = {}


def _nl7_oracle(shots, seed, first_chunk):
    """NL(7), 7/7 rounds (720 detectors): five pipelined schedules, lags 2 to
    4; the oracle's output is computed once per (shots, seed, chunk)."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc7"), 7, 7, C.NoiseModel(0.005, 0.03))
    key = (shots, seed, first_chunk)
    if key not in _NL7_CACHE:
        _NL7_CACHE[key] = oracle.sample(circ, shots, seed, first_chunk=first_chunk, threads=8)
    return circ, _NL7_CACHE[key]


@pytest.mark.parametrize("sched", range(5))
@pytest.mark.parametrize("tile_k,threads", [(1, 1024), (2, 512)])
def test_pipelined_kernel_every_lag_many_tiles(monkeypatch, sched, tile_k, threads):
    """Every pipelined schedule of NL(7) (lags 2, 3 and 4) over several
    tiles per CTA, so runs of `lag` steps cross tile boundaries."""
    monkeypatch.setenv("TMCS_KERNEL", "6")
    monkeypatch.setenv("TMCS_SIG_SCHED", str(sched))
    monkeypatch.setenv("TMCS_TILE_K", str(tile_k))
    monkeypatch.setenv("TMCS_THREADS", str(threads))
    shots, seed, first_chunk = 64 * 1000 + 37, 53, 5
    circ, (od, oo) = _nl7_oracle(shots, seed, first_chunk)
    h = tmcs.tmcs_circuit_build(circ)
    st = tmcs.tmcs_circuit_stats(h)
    tmcs.tmcs_circuit_free(h)
    assert st["sig_pipe_schedules"] == 5
    gd, go = gpu_sample(circ, shots, seed, first_chunk)
    assert np.array_equal(gd, od) and np.array_equal(go, oo)


@pytest.mark.parametrize("queue", [1, 64])
def test_pipelined_kernel_small_queue(monkeypatch, queue):
    """The smallest queue slices (64 events per walker warp) under heavy
    noise: the queue is applied almost every iteration."""
    monkeypatch.setenv("TMCS_KERNEL", "6")
    monkeypatch.setenv("TMCS_SIG_QUEUE", str(queue))
    circ = C.teleport_circuit(C.code_by_name("bb18"), 2, 2, C.NoiseModel(0.03, 0.1))
    assert_parity(circ, 64 * 23 + 5, seed=31)


def test_pipelined_kernel_observables_only(monkeypatch):
    """No detectors: the pipelined kernel writes every observable word."""
    monkeypatch.setenv("TMCS_KERNEL", "6")
    circ = C.Circuit()
    circ.append("R", [0, 1, 2])
    circ.append("X_ERROR", [0, 1, 2], p=0.2)
    circ.append("CX", [0, 1])
    circ.append("DEPOLARIZE2", [0, 1], p=0.1)
    circ.append("M", [0, 1, 2])
    circ.append("OBSERVABLE", [0, 2], arg=0)
    circ.append("OBSERVABLE", [1], arg=1)
    _, go = assert_parity(circ, 64 * 300 + 3, seed=3)
    assert go.any()


def test_pipelined_kernel_long_detector_span(monkeypatch):
    """A fault flipping detectors 1501 apart: the pipelined schedules size
    their ring for it."""
    from test_abi import _long_span_circuit
    monkeypatch.setenv("TMCS_KERNEL", "6")
    circ = _long_span_circuit(1500)
    gd, _ = assert_parity(circ, 64 * 9 + 3, seed=8)
    assert gd.any()


@pytest.mark.parametrize("queue", [1, 64])
def test_signature_kernel_queue_overflow(monkeypatch, queue):
    """Events that find the shared event queue full are applied directly:
    a tiny queue under heavy noise still reproduces the oracle."""
    monkeypatch.setenv("TMCS_KERNEL", "5")
    monkeypatch.setenv("TMCS_SIG_QUEUE", str(queue))
    circ = C.teleport_circuit(C.code_by_name("bb18"), 2, 2, C.NoiseModel(0.03, 0.1))
    assert_parity(circ, 64 * 23 + 5, seed=31)


@pytest.mark.parametrize("window", [1024, 2048])
def test_long_detector_span(monkeypatch, window):
    """A fault that flips the first and the last of 1502 detectors: with a
    1024-detector ring the signature program is refused and sampling runs on
    the frame kernels, with a 2048 ring on the signature kernel; both equal
    the oracle."""
    from test_abi import _long_span_circuit
    monkeypatch.setenv("TMCS_SIG_WINDOW", str(window))
    circ = _long_span_circuit(1500)
    h = tmcs.tmcs_circuit_build(circ)
    assert tmcs.tmcs_circuit_stats(h)["sig_ok"] == (1 if window == 2048 else 0)
    tmcs.tmcs_circuit_free(h)
    gd, _ = assert_parity(circ, 64 * 9 + 3, seed=8)
    assert gd.any()


def test_signature_kernel_observables_only():
    """No detectors at all: the kernel still writes every observable word."""
    circ = C.Circuit()
    circ.append("R", [0, 1, 2])
    circ.append("X_ERROR", [0, 1, 2], p=0.2)
    circ.append("CX", [0, 1])
    circ.append("DEPOLARIZE2", [0, 1], p=0.1)
    circ.append("M", [0, 1, 2])
    circ.append("OBSERVABLE", [0, 2], arg=0)
    circ.append("OBSERVABLE", [1], arg=1)
    _, go = assert_parity(circ, 64 * 5 + 3, seed=3)
    assert go.any()


def test_autotuned_large_call_matches_forced_shape(monkeypatch):
    """A call large enough to trigger the autotuner equals a forced-shape call."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 3, 3, C.NoiseModel(0.003, 0.03))
    shots = 64 * 152 * 40 + 9
    a = gpu_sample(circ, shots, 77)
    monkeypatch.setenv("TMCS_KERNEL", "3")
    monkeypatch.setenv("TMCS_TILE_K", "1")
    monkeypatch.setenv("TMCS_THREADS", "128")
    b = gpu_sample(circ, shots, 77)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _batch_case(n_jobs, seed):
    """Uneven jobs: SC d = 3..9 NL/teleport/memory and BB[[18,4,4]], varied
    noise and shot counts (ragged tails included)."""
    rng = np.random.default_rng(seed)
    circs, shots = [], []
    for j in range(n_jobs):
        code = C.code_by_name(["sc3", "sc5", "sc7", "sc9", "bb18"][int(rng.integers(5))])
        nz = C.NoiseModel(p=float(rng.choice([3e-3, 1e-2])), p_ebit=float(rng.choice([1e-2, 3e-2])))
        kind = int(rng.integers(3))
        r = int(rng.integers(1, 4))
        circs.append(C.nonlocal_cnot_circuit(code, r, r, nz) if kind == 0 else
                     C.teleport_circuit(code, r, r, nz) if kind == 1 else C.memory_circuit(code, r + 1, nz))
        shots.append(int(rng.integers(1, 64 * 400)))
    return circs, shots


@pytest.mark.parametrize("kernel", ["signature", "frame"])
def test_batch_many_uneven_jobs_two_launches(kernel, monkeypatch):
    """More jobs than one launch holds (96): every job still equals its solo run."""
    circs, shots = _batch_case(110, 5)
    samplers = [tmcs.Sampler(c) for c in circs]
    outs = [s.alloc(n) for s, n in zip(samplers, shots)]
    jobs = [(s.handle, n, 1000 + i, d, o) for i, (s, n, (d, o)) in enumerate(zip(samplers, shots, outs))]
    _batch(jobs, kernel, monkeypatch)
    torch.cuda.synchronize()
    for i in range(0, len(circs), 7):
        sd, so = gpu_sample(circs[i], shots[i], 1000 + i)
        d, o = outs[i]
        assert np.array_equal(d.cpu().numpy().view(np.uint64), sd)
        assert np.array_equal(o[: circs[i].n_obs].cpu().numpy().view(np.uint64), so)
    for s in samplers:
        s.close()


def test_batch_mixed_sizes_against_oracle():
    """Both size classes of the batched signature launch (d=3..11 and BB18
    in the 8-chunk class, d=29 in the 4-chunk class) in one call: jobs
    checked against the oracle directly."""
    circs = [C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.01, 0.05)),
             C.WORKLOADS["nl_sc29"].circuit(),
             C.teleport_circuit(C.code_by_name("bb18"), 1, 1, C.NoiseModel(0.004, 0.03)),
             C.nonlocal_cnot_circuit(C.code_by_name("sc11"), 3, 3, C.NoiseModel(0.002, 0.02))]
    shots = [64 * 40 + 9, 64 * 3 + 5, 64 * 21, 64 * 11 + 63]
    samplers = [tmcs.Sampler(c) for c in circs]
    outs = [s.alloc(n) for s, n in zip(samplers, shots)]
    jobs = [(s.handle, n, 300 + i, d, o) for i, (s, n, (d, o)) in enumerate(zip(samplers, shots, outs))]
    tmcs.tmcs_batch_sample(jobs)
    torch.cuda.synchronize()
    for i, (circ, n) in enumerate(zip(circs, shots)):
        od, oo = oracle.sample(circ, n, 300 + i, threads=8)
        d, o = outs[i]
        assert np.array_equal(d.cpu().numpy().view(np.uint64), od), i
        assert np.array_equal(o[: circ.n_obs].cpu().numpy().view(np.uint64), oo), i
    for s in samplers:
        s.close()


def test_batch_replays_under_cuda_graph():
    """A batched launch captured in a CUDA graph replays to the same bits."""
    circs, shots = _batch_case(12, 9)
    samplers = [tmcs.Sampler(c) for c in circs]
    outs = [s.alloc(n) for s, n in zip(samplers, shots)]
    jobs = [(s.handle, n, 77 + i, d, o) for i, (s, n, (d, o)) in enumerate(zip(samplers, shots, outs))]
    tmcs.tmcs_batch_sample(jobs)          # first call: uploads programs, allocates the queue
    torch.cuda.synchronize()
    ref = [(d.clone(), o.clone()) for d, o in outs]
    for d, o in outs:
        d.zero_()
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        tmcs.tmcs_batch_sample(jobs)
    for _ in range(2):
        for d, o in outs:
            d.zero_()
        g.replay()
        torch.cuda.synchronize()
        for (d, o), (rd, ro) in zip(outs, ref):
            assert torch.equal(d, rd) and torch.equal(o, ro)
    for s in samplers:
        s.close()


@pytest.mark.parametrize("code,w", [("sc3", 2), ("sc3", 4), ("sc3", 6), ("bb18", 3), ("sc5", 5)])
def test_pauli_string_chain(code, w):
    circ = C.pauli_string_circuit(C.code_by_name(code), w, rounds_before=2, noise=C.NoiseModel(0.01, 0.01))
    assert_parity(circ, 64 * 29 + 11, seed=31)


def test_pauli_string_bb144_full_size_sampled_chunks():
    """Weight-4 chain on BB[[144,12,12]] blocks at its bench size (1e6 shots):
    sampled chunks against the oracle."""
    w = C.WORKLOADS["ps4_bb144"]
    circ = w.circuit()
    s = tmcs.Sampler(circ)
    det, obs = s.sample(w.shots, w.seed)
    torch.cuda.synchronize()
    cols = (w.shots + 63) // 64
    for col in (0, cols // 3, cols - 1):
        n = min(64, w.shots - 64 * col)
        od, oo = oracle.sample(circ, n, w.seed, first_chunk=col, threads=8)
        assert np.array_equal(det[:, col].cpu().numpy().view(np.uint64), od[:, 0])
        assert np.array_equal(obs[:, col].cpu().numpy().view(np.uint64), oo[:, 0])
    s.close()


@pytest.mark.parametrize("code,schedule", [("sc5", "serial"), ("sc5", "lines"), ("bb18", "lines")])
def test_ebit_decoherence(code, schedule):
    """Methods "Decoherence": aged ebits get PAULI_CHANNEL_1 noise."""
    nz = C.NoiseModel(0.003, 0.01, decoherence=C.Decoherence(2e-3, schedule=schedule))
    circ = C.nonlocal_cnot_circuit(C.code_by_name(code), 2, 2, nz)
    assert_parity(circ, 64 * 41 + 3, seed=8)


def test_ebit_decoherence_workload_sampled_chunks():
    w = C.WORKLOADS["nl_sc11_deco"]
    circ = w.circuit()
    s = tmcs.Sampler(circ)
    shots = 64 * 152 * 20
    det, obs = s.sample(shots, w.seed)
    torch.cuda.synchronize()
    for col in (0, 777, shots // 64 - 1):
        od, oo = oracle.sample(circ, 64, w.seed, first_chunk=col, threads=8)
        assert np.array_equal(det[:, col].cpu().numpy().view(np.uint64), od[:, 0])
        assert np.array_equal(obs[:, col].cpu().numpy().view(np.uint64), oo[:, 0])
    s.close()
