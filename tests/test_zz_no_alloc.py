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
import oracle.mlpg_oracle as O  # noqa: E402


def _reference_counts(prob):
    with pkg.TransportProblem.from_problem(prob) as tp:
        tp.integrate()
        rowptr, _ = tp.neighbors()
    return np.diff(rowptr).astype(np.int32)


def _noalloc(x_host, R_host, lo, hi, fill):
    n, dim = x_host.shape
    x = torch.tensor(x_host, dtype=torch.float64, device="cuda")
    R = torch.tensor(R_host, dtype=torch.float64, device="cuda")
    out = torch.full((n,), fill, dtype=torch.int32, device="cuda")
    st = pkg.mlpg_overlap_counts_noalloc(dim, n, x.data_ptr(), R.data_ptr(), tuple(lo), tuple(hi),
                                         out.data_ptr(), None)
    torch.cuda.synchronize()
    assert st == 0
    return out.cpu().numpy()


def _run(prob, fill):
    return _noalloc(prob.x, prob.R, prob.lo[:prob.dim], prob.hi[:prob.dim], fill)


def test_counts_match_allocating_path_on_consecutive_calls():
    big = mi.two_region_2d(n_per_dim=96, sn=4)
    small = mi.small_2d(20, sn=4, seed=1007)
    ref_big, ref_small = _reference_counts(big), _reference_counts(small)
    # two calls in a row on the same problem, then a different size, then again
    for prob, ref, fill in ((big, ref_big, -7), (big, ref_big, 12345), (small, ref_small, -1), (big, ref_big, 0)):
        got = _run(prob, fill)
        assert np.array_equal(got, ref)


def test_counts_3d_match_allocating_path_on_consecutive_calls():
    """The 3D binning (z bins, the 27-bin stencil) against the pattern that
    mlpg_integrate builds, twice in a row and after a 2D call."""
    p3 = mi.lognormal_3d(7, sn=4, seed=3011)
    ref3 = _reference_counts(p3)
    assert ref3.max() > 100            # interior rows reach the full 3D stencil
    flat = mi.small_2d(16, sn=4, seed=1009)
    ref2 = _reference_counts(flat)
    for prob, ref, fill in ((p3, ref3, -3), (p3, ref3, 777), (flat, ref2, 5), (p3, ref3, 0)):
        assert np.array_equal(_run(prob, fill), ref)


def test_tiny_extents_count_only_the_point_itself():
    """Extents of 1e-30 on the unit square: every point overlaps only itself.
    The bin size is bounded below by the box, so the grid still fits the
    static scratch; the counts equal the oracle's brute-force pattern."""
    rng = np.random.default_rng(4242)
    x = rng.random((3000, 2))
    R = np.full(3000, 1e-30)
    rowptr, _ = O.neighbors(x, R)
    ref = np.diff(rowptr).astype(np.int32)
    assert np.all(ref == 1)
    for fill in (-9, 99):
        assert np.array_equal(_noalloc(x, R, (0.0, 0.0), (1.0, 1.0), fill), ref)


def test_rejects_sizes_beyond_the_static_scratch_and_bad_boxes():
    n = 262145   # one more than the largest size the static scratch serves
    x = torch.full((n, 2), 0.5, dtype=torch.float64, device="cuda")
    R = torch.full((n,), 0.01, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = pkg.mlpg_overlap_counts_noalloc(2, n, x.data_ptr(), R.data_ptr(), (0.0, 0.0), (1.0, 1.0),
                                         out.data_ptr(), None)
    assert st == -1
    for lo, hi in (((0.0, 0.0), (float("inf"), 1.0)), ((float("nan"), 0.0), (1.0, 1.0)), ((0.0, 0.0), (0.0, 1.0))):
        st = pkg.mlpg_overlap_counts_noalloc(2, 100, x.data_ptr(), R.data_ptr(), lo, hi, out.data_ptr(), None)
        assert st == -1
