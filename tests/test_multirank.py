"""The N-GPU path's host logic, on CPU with two gloo ranks.

Each rank samples its own global chunk range (bench.py's weak-scaling
split) with the oracle; gathered in rank order, the ranks' columns equal one
single-process run over the whole range, and the step-time reduction takes
the largest rank's time. No data-path collective is involved: the gather
here only brings the results together for the check.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2504_05611_gb300 import circuits as C  # noqa: E402
from paper_2504_05611_gb300.shard import max_over_ranks, rank_chunk_range  # noqa: E402

SHOTS_PER_RANK = 64 * 5 + 21
SEED = 17


def _circuit():
    return C.nonlocal_cnot_circuit(C.code_by_name("sc3"), 2, 2, C.NoiseModel(0.01, 0.05))


def _rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        circ = _circuit()
        first_chunk, shots = rank_chunk_range(rank, world, SHOTS_PER_RANK)
        det, obs = oracle.sample(circ, shots, SEED, first_chunk=first_chunk, threads=1)
        got = [None] * world
        dist.all_gather_object(got, (first_chunk, det, obs))
        slowest = max_over_ranks(1.0 + rank)
        if rank == 0:
            np.save(os.path.join(out_dir, "det.npy"), np.concatenate([g[1] for g in got], axis=1))
            np.save(os.path.join(out_dir, "obs.npy"), np.concatenate([g[2] for g in got], axis=1))
            np.save(os.path.join(out_dir, "first.npy"), np.array([g[0] for g in got]))
            np.save(os.path.join(out_dir, "slowest.npy"), np.array([slowest]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_concatenate_to_one_run(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    import oracle
    circ = _circuit()
    cols = (SHOTS_PER_RANK + 63) // 64
    first = np.load(tmp_path / "first.npy")
    assert list(first) == [0, cols]
    det = np.load(tmp_path / "det.npy")
    obs = np.load(tmp_path / "obs.npy")
    # one process, both ranges: rank 0's columns, then rank 1's
    d0, o0 = oracle.sample(circ, SHOTS_PER_RANK, SEED, first_chunk=0, threads=1)
    d1, o1 = oracle.sample(circ, SHOTS_PER_RANK, SEED, first_chunk=cols, threads=1)
    assert np.array_equal(det, np.concatenate([d0, d1], axis=1))
    assert np.array_equal(obs, np.concatenate([o0, o1], axis=1))
    # the step-time reduction reports the slowest rank (rank r reported 1 + r)
    assert float(np.load(tmp_path / "slowest.npy")[0]) == 2.0


def test_contiguous_ranges_equal_one_long_run():
    """With whole-chunk shot counts the ranks' ranges tile one long run."""
    import oracle
    circ = _circuit()
    per = 64 * 4
    parts = []
    for r in range(3):
        fc, n = rank_chunk_range(r, 3, per)
        parts.append(oracle.sample(circ, n, SEED, first_chunk=fc, threads=1)[0])
    whole = oracle.sample(circ, 3 * per, SEED, first_chunk=0, threads=1)[0]
    assert np.array_equal(np.concatenate(parts, axis=1), whole)


def test_rank_chunk_range_rejects_bad_arguments():
    with pytest.raises(ValueError):
        rank_chunk_range(2, 2, 64)
    with pytest.raises(ValueError):
        rank_chunk_range(0, 2, 0)
