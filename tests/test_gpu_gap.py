"""The device gap counts against their definition.

The gap between noise events of a segment is G = #{g in 1..4096 : w < T[g]}
for a uniform 32-bit word w and the table T[g] = floor(2^32 (1-p)^g)
(geometric sampling of independent noise events, Methods "Simulation").
The kernels find G from a floating-point estimate of log(w) / log(1-p)
followed by table reads; this test runs every device route on the words
where a wrong estimate would show -- each table entry T[g] and its two
neighbours, the ends of the word range -- plus random words, over
probabilities from 1 down to 1e-6 (both sides of the one-read route's
limit, |1/log2(1-p)| < 32768, near p = 2.1e-5), and compares with the count
taken from the oracle's table by binary search.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_05611_gb300 import tmcs  # noqa: E402

PROBS = [1.0, 0.75, 0.5, 0.2, 0.1, 0.03, 0.01, 3e-3, 1e-3, 6.7e-4, 3e-4, 1e-4, 5e-5, 3e-5, 2.2e-5, 2.1e-5, 2e-5,
         1e-5, 3e-6, 1e-6]


def expected_counts(table, words):
    asc = table[::-1].astype(np.int64)  # T is non-increasing
    return (len(table) - np.searchsorted(asc, words.astype(np.int64), side="right")).astype(np.int32)


def boundary_words(table, rng, n_random=1 << 20):
    t = table.astype(np.int64)
    w = np.concatenate([t - 1, t, t + 1, np.array([0, 1, 2, 3, 1 << 24, (1 << 24) + 1, (1 << 32) - 129, (1 << 32) - 128,
                                                   (1 << 32) - 2, (1 << 32) - 1]),
                        rng.integers(0, 1 << 32, n_random, dtype=np.int64),
                        # words near 2^32, where small p puts its short gaps
                        (1 << 32) - 1 - rng.integers(0, 1 << 22, n_random // 4, dtype=np.int64)])
    return np.unique(np.clip(w, 0, (1 << 32) - 1)).astype(np.uint32)


@pytest.mark.parametrize("p", PROBS)
@pytest.mark.parametrize("method", [0, 1, 2])
def test_device_gap_counts_match_definition(p, method):
    table = oracle.gap_table(p)
    rng = np.random.default_rng(int(p * 1e9) + method)
    words = boundary_words(table, rng)
    want = expected_counts(table, words)
    dw = torch.from_numpy(words.view(np.int32)).cuda()
    got = tmcs.tmcs_debug_gap_counts(p, dw, method).cpu().numpy()
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (f"{bad.size} counts differ, first: w={words[bad[:4]].tolist()} "
                           f"got {got[bad[:4]].tolist()} want {want[bad[:4]].tolist()}")
    # the routine sees every count from 0 to 4096 where p allows it
    assert want.min() == 0


def test_gap_counts_reject_bad_arguments():
    dw = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(tmcs.TmcsError):
        tmcs.tmcs_debug_gap_counts(0.0, dw, 0)
    with pytest.raises(tmcs.TmcsError):
        tmcs.tmcs_debug_gap_counts(0.1, dw, 3)
