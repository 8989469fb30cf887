"""GPU parity of the decoupled event-signature kernel (walker and applier
warps joined by a shared-memory event arena) against the CPU oracle.

The kernel changes only the execution order of the event-signature sampler
(Methods "Simulation": detector flips are XORs of the sampled events' output
lists), so every launch shape must reproduce the oracle bit for bit: chunks
per tile, applier warps, CTA size, ring schedule, several tiles per CTA, a
ragged last chunk, a nonzero first chunk, and the path where an event does
not fit its step's arena region (forced here with tiny capacities).
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


def gpu_sample(circ, shots, seed, first_chunk=0):
    s = tmcs.Sampler(circ)
    det, obs = s.sample(shots, seed, first_chunk=first_chunk)
    torch.cuda.synchronize()
    out = det.cpu().numpy().view(np.uint64), obs.cpu().numpy().view(np.uint64)
    s.close()
    return out


_ORACLE = {}


def oracle_sample(circ, key, shots, seed, first_chunk):
    k = (key, shots, seed, first_chunk)
    if k not in _ORACLE:
        _ORACLE[k] = oracle.sample(circ, shots, seed, first_chunk=first_chunk, threads=8)
    return _ORACLE[k]


def assert_flow_parity(monkeypatch, circ, key, shots, seed, first_chunk=0, **env):
    monkeypatch.setenv("TMCS_KERNEL", "7")
    for k, v in env.items():
        monkeypatch.setenv(k, str(v))
    gd, go = gpu_sample(circ, shots, seed, first_chunk)
    od, oo = oracle_sample(circ, key, shots, seed, first_chunk)
    assert gd.shape == od.shape and go.shape == oo.shape
    bad = np.argwhere(gd != od)
    assert bad.size == 0, f"{len(bad)} detector words differ, first at {bad[:3].tolist()}"
    assert np.array_equal(go, oo)
    tmcs.tmcs_check_device()
    return gd, go


def nl11():
    return C.nonlocal_cnot_circuit(C.code_by_name("sc11"), 11, 11, C.NoiseModel(0.003, 0.02))


# (schedule, chunks per tile, applier warps, CTA size): the ring of K x window
# words must fit shared memory next to the arena, so larger windows (schedule
# 0: 4096 detectors, 1: 2048, 2: 1024) take fewer chunks per tile
FLOW_SHAPES = [(0, 1, 8, 1024), (0, 2, 4, 1024), (0, 4, 8, 1024), (0, 4, 1, 1024), (0, 2, 2, 512), (0, 1, 1, 256),
               (1, 8, 4, 1024), (1, 4, 8, 1024), (1, 8, 8, 1024), (1, 2, 1, 256), (2, 16, 8, 1024), (2, 8, 4, 1024),
               (2, 4, 2, 512), (2, 1, 8, 1024), (2, 16, 2, 256), (1, 8, 16, 1024), (1, 8, 20, 1024),
               (2, 8, 24, 1024), (2, 4, 20, 1024)]


@pytest.mark.parametrize("sched,tile_k,appliers,threads", FLOW_SHAPES)
def test_flow_shapes_are_bit_exact(monkeypatch, sched, tile_k, appliers, threads):
    """Every ring schedule (4096, 2048, 1024 detectors) x chunks per tile x
    applier warps x CTA size, ragged tail, nonzero first chunk."""
    circ = nl11()
    gd, go = assert_flow_parity(monkeypatch, circ, "nl11", 64 * 19 + 45, 29, first_chunk=3,
                                TMCS_SIG_SCHED=sched, TMCS_TILE_K=tile_k, TMCS_FLOW_APPLIERS=appliers,
                                TMCS_THREADS=threads)
    assert gd.any() and go.any()


@pytest.mark.parametrize("tile_k,shots", [(1, 64 * 1000 + 37), (2, 64 * 1000 + 37), (2, 64 * 1000),
                                          (4, 64 * 2002 - 5), (8, 64 * 2002 - 5)])
def test_flow_many_tiles_per_cta(monkeypatch, tile_k, shots):
    """Several tiles per CTA: walkers run into the next tile's steps while
    the appliers finish this one's. Odd and even column counts take the
    scalar and the 16-byte output stores."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 6, 6, C.NoiseModel(0.01, 0.05))
    gd, go = assert_flow_parity(monkeypatch, circ, "nl5", shots, 41, first_chunk=11, TMCS_TILE_K=tile_k)
    assert gd.any() and go.any()


@pytest.mark.parametrize("cap", [1, 3, 17, 200])
@pytest.mark.parametrize("tile_k", [2, 8])
def test_flow_region_overflow_is_exact(monkeypatch, cap, tile_k):
    """Events beyond their step's arena region are held by their lane and
    XORed into the ring once that step is being applied: with capacities of
    a few events nearly every event takes that path, and the output is still
    the oracle's."""
    circ = nl11()
    assert_flow_parity(monkeypatch, circ, "nl11", 64 * 19 + 45, 29, first_chunk=3, TMCS_TILE_K=tile_k,
                       TMCS_SIG_SCHED=1 if tile_k == 8 else 0, TMCS_TEST_FLOW_CAP=cap)


@pytest.mark.parametrize("arena", [1024, 2048])
def test_flow_small_arena(monkeypatch, arena):
    """An arena smaller than a step's expected events: steps are gated on
    the appliers and regions are clamped to the arena, so events overflow."""
    circ = nl11()
    assert_flow_parity(monkeypatch, circ, "nl11", 64 * 19 + 45, 29, first_chunk=3, TMCS_TILE_K=8,
                       TMCS_SIG_SCHED=1, TMCS_FLOW_ARENA=arena)


@pytest.mark.parametrize("kind", ["nl", "teleport", "memory"])
@pytest.mark.parametrize("code", ["sc3", "sc5", "bb18"])
def test_flow_protocols_high_noise(monkeypatch, kind, code):
    cc = C.code_by_name(code)
    nz = C.NoiseModel(p=0.02, p_ebit=0.05)
    circ = {"nl": C.nonlocal_cnot_circuit(cc, 2, 2, nz), "teleport": C.teleport_circuit(cc, 2, 2, nz),
            "memory": C.memory_circuit(cc, 3, nz)}[kind]
    assert_flow_parity(monkeypatch, circ, f"{kind}-{code}", 64 * 37 + 5, 7)


@pytest.mark.parametrize("trial", range(8))
def test_flow_random_circuits(monkeypatch, trial):
    """Random Clifford circuits with every noise kind (PAULI_CHANNEL_1
    included), feedback and observables."""
    rng = np.random.default_rng(1900 + trial)
    circ = random_noisy_circuit(rng, int(rng.integers(2, 9)), int(rng.integers(4, 40)))
    assert_flow_parity(monkeypatch, circ, f"rand{trial}", 64 * 9 + int(rng.integers(1, 64)),
                       int(rng.integers(1, 2 ** 62)), TMCS_TILE_K=int(rng.choice([1, 2, 4, 8])))


def test_flow_ebit_decoherence(monkeypatch):
    """Methods "Decoherence": aged ebits carry PAULI_CHANNEL_1 noise."""
    w = C.WORKLOADS["nl_sc11_deco"]
    assert_flow_parity(monkeypatch, w.circuit(), "deco", 64 * 23 + 9, w.seed, first_chunk=5, TMCS_TILE_K=4)


def test_flow_teleport_bb144(monkeypatch):
    """BB[[144,12,12]] teleportation, 12 observables, reduced shots."""
    w = C.WORKLOADS["tp_bb144"]
    assert_flow_parity(monkeypatch, w.circuit(), "tp144", 64 * 40 + 3, w.seed, TMCS_TILE_K=4)


@pytest.mark.parametrize("window", [2, 3, 4])
@pytest.mark.parametrize("tile_k,cap", [(8, 0), (2, 5)])
def test_flow_walker_windows(monkeypatch, window, tile_k, cap):
    """Walker windows of 2 to 4 Philox calls per iteration (streams longer
    than a window continue in the next), with and without region overflow."""
    circ = nl11()
    env = dict(TMCS_TILE_K=tile_k, TMCS_SIG_SCHED=1 if tile_k == 8 else 0, TMCS_FLOW_WINDOW=window)
    if cap:
        env["TMCS_TEST_FLOW_CAP"] = cap
    assert_flow_parity(monkeypatch, circ, "nl11", 64 * 19 + 45, 29, first_chunk=3, **env)


@pytest.mark.parametrize("slice_tiles,tile_k", [(1, 2), (7, 4), (150, 2)])
def test_flow_sliced_launches(monkeypatch, slice_tiles, tile_k):
    """A call too large for one launch's 32-bit stream counters runs as
    several launches over column slices; forced small slices here (ragged
    tail in the last slice, odd slice starts, nonzero first chunk)."""
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 6, 6, C.NoiseModel(0.01, 0.05))
    gd, go = assert_flow_parity(monkeypatch, circ, "nl5", 64 * 1000 + 37, 41, first_chunk=11, TMCS_TILE_K=tile_k,
                                TMCS_TEST_FLOW_SLICE_TILES=slice_tiles)
    assert gd.any() and go.any()


@pytest.mark.parametrize("sched,tile_k,appliers,garena,cap", [(1, 8, 12, 0, 0), (2, 16, 8, 0, 0), (0, 4, 8, 1024, 0),
                                                               (1, 8, 8, 0, 3), (0, 2, 4, 2048, 0)])
def test_flow_global_arena(monkeypatch, sched, tile_k, appliers, garena, cap):
    """The event arena in a global scratch buffer (one L2-resident slice per
    CTA) instead of shared memory: same bits, also with a small arena
    (steps gated on the appliers) and with forced region overflow."""
    env = dict(TMCS_SIG_SCHED=sched, TMCS_TILE_K=tile_k, TMCS_FLOW_APPLIERS=appliers, TMCS_FLOW_GLOBAL_ARENA=1)
    if garena:
        env["TMCS_FLOW_GARENA"] = garena
    if cap:
        env["TMCS_TEST_FLOW_CAP"] = cap
    gd, go = assert_flow_parity(monkeypatch, nl11(), "nl11", 64 * 19 + 45, 29, first_chunk=3, **env)
    assert gd.any() and go.any()


def test_flow_global_arena_many_tiles(monkeypatch):
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 6, 6, C.NoiseModel(0.01, 0.05))
    assert_flow_parity(monkeypatch, circ, "nl5", 64 * 2002 - 5, 41, first_chunk=11, TMCS_TILE_K=8,
                       TMCS_FLOW_GLOBAL_ARENA=1, TMCS_FLOW_GARENA=4096)


@pytest.mark.parametrize("sched,tile_k,rows,appliers", [(1, 8, 16, 12), (1, 8, 2, 8), (0, 2, 8, 8), (0, 4, 4, 1),
                                                        (2, 16, 1, 8), (2, 16, 64, 2), (0, 4, 256, 8), (1, 8, 0, 12)])
def test_flow_tensor_store_flush(monkeypatch, sched, tile_k, rows, appliers):
    """Detector rows leave the ring as 2D tensor stores (boxes of rows x K
    chunk words, head and tail rows around the aligned boxes by plain
    stores): same bits for any box height, with the ring wrapping under the
    boxes, several tiles per CTA and the last tile partly outside the output
    (its columns past the call's end are clipped). rows = 0 turns the tensor
    stores off."""
    env = dict(TMCS_SIG_SCHED=sched, TMCS_TILE_K=tile_k, TMCS_FLOW_APPLIERS=appliers)
    env["TMCS_FLOW_TMA"] = 1 if rows else 0
    if rows:
        env["TMCS_FLOW_TMA_ROWS"] = rows
    # 20 columns: the last tile of K = 8 or 16 holds 4 columns
    gd, go = assert_flow_parity(monkeypatch, nl11(), "nl11", 64 * 19 + 45, 29, first_chunk=3, **env)
    assert gd.any() and go.any()
    circ = C.nonlocal_cnot_circuit(C.code_by_name("sc5"), 6, 6, C.NoiseModel(0.01, 0.05))
    assert_flow_parity(monkeypatch, circ, "nl5", 64 * 2002 - 5, 41, first_chunk=11, **env)


@pytest.mark.parametrize("offset_words", [1, 2])
def test_flow_flush_unaligned_outputs(monkeypatch, offset_words):
    """An output buffer that does not start on a 16-byte boundary (one word
    in) cannot be a tensor map: the flush falls back to plain stores; two
    words in (16-byte aligned) it uses the tensor stores."""
    monkeypatch.setenv("TMCS_KERNEL", "7")
    monkeypatch.setenv("TMCS_TILE_K", "4")
    monkeypatch.setenv("TMCS_FLOW_TMA", "1")
    circ = nl11()
    shots, seed, first = 64 * 19 + 45, 29, 3
    s = tmcs.Sampler(circ)
    try:
        n_det, n_obs, cols = s.info["n_det"], s.info["n_obs"], (shots + 63) // 64
        flat = torch.full((n_det * cols + offset_words,), -1, dtype=torch.int64, device="cuda")
        det = flat[offset_words:].view(n_det, cols)
        obs = torch.empty((max(n_obs, 1), cols), dtype=torch.int64, device="cuda")
        s.sample(shots, seed, first_chunk=first, out=(det, obs))
        torch.cuda.synchronize()
        tmcs.tmcs_check_device()
        od, oo = oracle_sample(circ, "nl11", shots, seed, first)
        assert np.array_equal(det.cpu().numpy().view(np.uint64), od)
        assert np.array_equal(obs[:n_obs].cpu().numpy().view(np.uint64), oo)
        assert int(flat[:offset_words].eq(-1).sum()) == offset_words  # nothing written before the buffer
    finally:
        s.close()


def _mostly_silent_circuit(n=150):
    """Z-basis readout of n qubits after two-qubit depolarizing noise on
    pairs, a Z-heavy PAULI_CHANNEL_1 and Z flips: only the X parts of the
    noise flip a detector, so most Pauli indices of every noise op flip
    nothing (the Z_ERROR op flips nothing at all and has no walked item)."""
    c = C.Circuit()
    q = list(range(n))
    c.append("R", q)
    c.append("DEPOLARIZE2", [t for i in range(0, n - 1, 2) for t in (i, i + 1)], p=0.04)
    c.append("PAULI_CHANNEL_1", q, p=(0.005, 0.0, 0.1))
    c.append("Z_ERROR", q, p=0.2)
    c.append("CX", [t for i in range(0, n - 1, 2) for t in (i, i + 1)])
    recs = c.append("M", q)
    for r in recs:
        c.append("DETECTOR", [int(r)])
    c.append("OBSERVABLE", [int(recs[0]), int(recs[n - 1])], arg=0)
    return c


@pytest.mark.parametrize("tile_k,cap", [(8, None), (8, 2), (2, None), (1, 5)])
def test_flow_events_that_flip_nothing(monkeypatch, tile_k, cap):
    """Walkers mark events whose Pauli index flips nothing in their segment
    (the segment's live-Pauli mask) so that the appliers skip them; on a
    circuit where most drawn events are such, including the events a lane
    holds back when its step's region is full, the output is the oracle's."""
    circ = _mostly_silent_circuit()
    env = {"TMCS_TILE_K": tile_k}
    if cap is not None:
        env["TMCS_TEST_FLOW_CAP"] = cap
    gd, go = assert_flow_parity(monkeypatch, circ, "silent", 64 * 23 + 9, 77, first_chunk=5, **env)
    assert gd.any() and go.any()
