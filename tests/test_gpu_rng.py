"""The oracle's Philox4x32-10 against an independent implementation:
cuRAND's device generator ``curand_Philox4x32_10`` (counter, key) -> four
words, run on the GPU by a small test kernel (``tests/curand_philox.cu``,
built here with nvcc).

The noise streams of the sampling specification (Methods "Simulation" noise
channels drawn from Philox4x32-10, Salmon et al. SC'11) rest on this
generator; a shared misreading of the round structure by the oracle and the
CUDA sampler would pass every parity test, but not this comparison.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = tempfile.mkdtemp(prefix="curand_philox_")
    so = os.path.join(out, "libcurand_philox.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    "-o", so, os.path.join(HERE, "curand_philox.cu")], check=True)
    L = ctypes.CDLL(so)
    L.curand_philox_batch.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    L.curand_philox_batch.restype = ctypes.c_int
    yield L
    shutil.rmtree(out, ignore_errors=True)


def test_oracle_philox_equals_curand(curand_lib):
    rng = np.random.default_rng(2024)
    n = 4096
    ctr = rng.integers(0, 1 << 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 1 << 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # the counters the sampler uses: small call index, chunk, op, segment
    ctr[:64] = np.stack([np.arange(64), np.full(64, 7), np.full(64, 3), np.arange(64) % 5], 1)
    ctr[64:96] = np.stack([np.zeros(32), np.arange(32), np.full(32, 11), np.full(32, 0x80000000)], 1)
    key[:96] = [1, 0]
    out = np.zeros((n, 4), dtype=np.uint32)
    rc = curand_lib.curand_philox_batch(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, n)
    assert rc == 0, f"CUDA error {rc}"
    want = np.array([oracle.philox4x32_10(tuple(int(v) for v in c), tuple(int(v) for v in k))
                     for c, k in zip(ctr, key)], dtype=np.uint32)
    bad = np.nonzero((want != out).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} of {n} outputs differ, first at {bad[:3].tolist()}"
