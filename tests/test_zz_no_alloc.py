"""The allocation-free overlap-count entry point.

mlpg_overlap_counts_noalloc serves callers that cannot allocate device memory
(stream capture, fixed memory budgets, real-time loops): it keeps its scratch
in one static device array.  Its counts must equal the row lengths of the
overlap pattern that the allocating path (mlpg_integrate) builds, exactly
(integer output), on consecutive calls that reuse the same scratch.

This file is collected last so that a stop-at-first-failure run has already
run every other test before it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import mlpg_inputs as mi  # noqa: E402
import paper_2008_02205_gb300 as pkg  # noqa: E402


def _reference_counts(prob):
    with pkg.TransportProblem.from_problem(prob) as tp:
        tp.integrate()
        rowptr, _ = tp.neighbors()
    return np.diff(rowptr).astype(np.int32)


def _noalloc(prob, fill):
    x = torch.tensor(prob.x, dtype=torch.float64, device="cuda")
    R = torch.tensor(prob.R, dtype=torch.float64, device="cuda")
    out = torch.full((prob.n,), fill, dtype=torch.int32, device="cuda")
    st = pkg.mlpg_overlap_counts_noalloc(2, prob.n, x.data_ptr(), R.data_ptr(), (0.0, 0.0), (1.0, 1.0),
                                         out.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == 0
    return out.cpu().numpy()


def test_counts_match_allocating_path_on_consecutive_calls():
    big = mi.two_region_2d(n_per_dim=96, sn=4)
    small = mi.small_2d(20, sn=4, seed=1007)
    ref_big, ref_small = _reference_counts(big), _reference_counts(small)
    # two calls in a row on the same problem, then a different size, then again
    for prob, ref, fill in ((big, ref_big, -7), (big, ref_big, 12345), (small, ref_small, -1), (big, ref_big, 0)):
        got = _noalloc(prob, fill)
        assert np.array_equal(got, ref)


def test_rejects_sizes_beyond_the_static_scratch():
    n = 262145   # one more than the largest size the static scratch serves
    x = torch.full((n, 2), 0.5, dtype=torch.float64, device="cuda")
    R = torch.full((n,), 0.01, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = pkg.mlpg_overlap_counts_noalloc(2, n, x.data_ptr(), R.data_ptr(), (0.0, 0.0), (1.0, 1.0),
                                         out.data_ptr(), None)
    assert st == -1
