"""Full-size parity: every benchmarked workload at its full shot count, in
the launch shape the autotuner keeps (the shape the benchmark times),
against the CPU oracle on sampled columns.

For each workload the test makes the benchmark's own call sequence on a
fresh circuit (tmcs_sample over the whole workload: the first such call
times the candidate shapes and keeps the fastest), reads the kept shape,
and compares at least 64 output columns (64-shot chunks) with the oracle,
chosen where a wrong index would show: both sides of several tile
boundaries of that shape, the first and last tiles of the first CTAs, the
second tile of a CTA (the persistent grid's wrap), the last tiles of the
call and its last column; then a call with a ragged shot count (same kept
shape) checks the last column's pad bits. Workloads: Methods "Non-local
CNOT circuit" at distances 11 and 29 (p = 1e-3 and 1e-4) and "State
teleportation circuit" for BB[[144,12,12]].
"""
import os
import zlib
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2504_05611_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_05611_gb300 import tmcs  # noqa: E402

SIGNATURE_MODES = {5, 6, 7}


def probe_columns(n_cols, K, sms, rng, extra=64):
    """Columns on tile boundaries of K-chunk tiles for persistent grids of
    sms and 2*sms CTAs (CTA b owns tiles b, b + grid, ...), plus random ones."""
    n_tiles = (n_cols + K - 1) // K
    cols = {0, n_cols - 1}
    for grid in (sms, 2 * sms):
        for tile in (0, 1, grid - 1, grid, grid + 1, 2 * grid - 1, 2 * grid, n_tiles // 2, n_tiles - grid - 1,
                     n_tiles - grid, n_tiles - 2, n_tiles - 1):
            if 0 <= tile < n_tiles:
                lo = tile * K
                cols.update({lo, lo + 1, lo + K - 1})
    cols = {c for c in cols if 0 <= c < n_cols}
    while len(cols) < extra + 16:
        cols.add(int(rng.integers(0, n_cols)))
    return sorted(cols)


def check_columns(circ, det, obs, shots, seed, cols):
    """det/obs: device tensors [rows][n_cols]; compares the given columns
    with the oracle one chunk at a time (first_chunk keying)."""
    idx = torch.tensor(cols, device=det.device)
    gd = det.index_select(1, idx).cpu().numpy().view(np.uint64)
    go = obs.index_select(1, idx).cpu().numpy().view(np.uint64)
    m = oracle.Marshalled(circ)

    def one(col):
        # the oracle's C call releases the GIL: columns run on all host cores
        return oracle.sample(circ, min(64, shots - 64 * col), seed, first_chunk=col, threads=1, marshalled=m)

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        want = list(ex.map(one, cols))
    for j, (col, (od, oo)) in enumerate(zip(cols, want)):
        assert np.array_equal(gd[:, j], od[:, 0]), f"column {col}: detector words differ"
        assert np.array_equal(go[: circ.n_obs, j], oo[:, 0]), f"column {col}: observable words differ"


@pytest.mark.parametrize("name", ["nl_sc11", "tp_bb144", "nl_sc29", "nl_sc29_p1e-4"])
def test_full_size_workload_in_the_tuned_shape(name):
    w = C.WORKLOADS[name]
    circ = w.circuit()
    shots = w.shots
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    s = tmcs.Sampler(circ)
    try:
        det, obs = s.alloc(shots)
        s.sample(shots, w.seed, out=(det, obs))
        torch.cuda.synchronize()
        shape = tmcs.tmcs_launch_shape(s.handle)
        # the benchmark's shape is a signature kernel with several tiles per CTA
        assert shape["mode"] in SIGNATURE_MODES, shape
        K = shape["chunks"]
        n_cols = (shots + 63) // 64
        assert n_cols // K >= 4 * sms
        # the timed call: same shape, outputs overwritten
        det.fill_(-1)
        obs.fill_(-1)
        s.sample(shots, w.seed, out=(det, obs))
        torch.cuda.synchronize()
        tmcs.tmcs_check_device()
        assert tmcs.tmcs_launch_shape(s.handle) == shape
        rng = np.random.default_rng(zlib.crc32(name.encode()))
        cols = probe_columns(n_cols, K, sms, rng)
        assert len(cols) >= 64
        check_columns(circ, det, obs[: max(circ.n_obs, 1)], shots, w.seed, cols)
        # ragged tail in the same kept shape: the last column's pad bits are 0
        ragged = shots - 37
        del det, obs
        det, obs = s.alloc(ragged)
        s.sample(ragged, w.seed, out=(det, obs))
        torch.cuda.synchronize()
        assert tmcs.tmcs_launch_shape(s.handle) == shape
        rc = (ragged + 63) // 64
        check_columns(circ, det, obs[: max(circ.n_obs, 1)], ragged, w.seed, [rc - 2, rc - 1])
        last = det[:, rc - 1].cpu().numpy().view(np.uint64)
        assert not np.any(last & ~np.uint64((1 << (ragged % 64)) - 1))
    finally:
        s.close()
