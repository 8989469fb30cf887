"""Bounded device waits: an expired wait is reported, and the context stays
usable.

The pipelined event-signature kernel's flusher waits, for at most 2 s of
wall time, until the walkers have published every stream of a step. The
testing knob TMCS_TEST_STALL_FLUSH=1 makes it wait for one stream more than
step 0 has, a count nothing reaches: the wait expires, the flusher sets the
abort flag and the device status word, every warp leaves, and
tmcs_check_device raises TMCS_E_TIMEOUT. No fault, trap or unbounded wait is
involved. A normal call afterwards reproduces the oracle.
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


def test_pipelined_flush_wait_expires_and_is_reported(monkeypatch):
    monkeypatch.setenv("TMCS_KERNEL", "6")
    circ = C.teleport_circuit(C.code_by_name("bb18"), 2, 2, C.NoiseModel(0.01, 0.05))
    shots, seed = 64 * 41 + 9, 17
    tmcs.tmcs_check_device()  # start from a clear status word
    s = tmcs.Sampler(circ)
    try:
        monkeypatch.setenv("TMCS_TEST_STALL_FLUSH", "1")
        s.sample(shots, seed)
        torch.cuda.synchronize()
        with pytest.raises(tmcs.TmcsError) as err:
            tmcs.tmcs_check_device()
        assert err.value.code == 5  # TMCS_E_TIMEOUT
        tmcs.tmcs_check_device()  # the check cleared the flag
        monkeypatch.delenv("TMCS_TEST_STALL_FLUSH")
        det, obs = s.sample(shots, seed)
        torch.cuda.synchronize()
        tmcs.tmcs_check_device()
        od, oo = oracle.sample(circ, shots, seed, threads=8)
        assert np.array_equal(det.cpu().numpy().view(np.uint64), od)
        assert np.array_equal(obs[: circ.n_obs].cpu().numpy().view(np.uint64), oo)
    finally:
        s.close()
