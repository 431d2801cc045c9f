"""Pins of the oracle's kernel and reproducing-kernel functions (Sec. 2.1-2.2)."""
import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O


def _setup(n=12, jitter=0.2, seed=3):
    x, h = mi.jittered_lattice(n, 2, seed, jitter=jitter)
    d = O.Discretization(x, np.full(len(x), 2 * h))
    return d


def _sums(d, pts, owner):
    sptr, sidx, U, dU = O.rk_at_points(d.x, d.R, d.V, d.rowptr, d.col, pts, owner)
    rows = np.repeat(np.arange(len(pts)), np.diff(sptr))
    N = U * d.V[sidx]
    dN = dU * d.V[sidx][:, None]
    s0 = np.bincount(rows, N, minlength=len(pts))
    s1 = np.stack([np.bincount(rows, N * d.x[sidx, b], minlength=len(pts)) for b in range(2)], 1)
    g0 = np.stack([np.bincount(rows, dN[:, g], minlength=len(pts)) for g in range(2)], 1)
    g1 = np.stack([[np.bincount(rows, dN[:, g] * d.x[sidx, b], minlength=len(pts))
                    for b in range(2)] for g in range(2)])
    return s0, s1, g0, g1, (sptr, sidx, U, dU)


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_linear_reproduction_at_quadrature_points(jitter):
    d = _setup(jitter=jitter)
    s0, s1, g0, g1, _ = _sums(d, d.vq.x, d.vq.owner)
    assert np.abs(s0 - 1).max() < 1e-12                       # sum_j N_j = 1
    assert np.abs(s1 - d.vq.x).max() < 1e-12                  # sum_j N_j x_j = x
    hinv = 1.0 / d.h.min()
    assert np.abs(g0).max() < 1e-11 * hinv                    # sum_j dN_j = 0
    assert np.abs(g1 - np.eye(2)[:, :, None]).max() < 1e-11 * hinv  # sum_j d_g N_j x_j^b = delta


def test_reproduction_at_centres_and_boundary():
    d = _setup()
    for pts, ow in ((d.x, np.arange(d.n, dtype=np.int32)), (d.bq.x, d.bq.owner)):
        s0, s1, g0, g1, _ = _sums(d, pts, ow)
        assert np.abs(s0 - 1).max() < 1e-12
        assert np.abs(s1 - pts).max() < 1e-12


def test_gradient_matches_finite_difference():
    d = _setup()
    rng = np.random.default_rng(0)
    i = d.n // 2 + 3
    p = d.x[i] + 0.2 * d.h[i] * rng.uniform(-1, 1, 2)
    eps = 1e-6 * d.h[i]
    base = O.rk_at_points(d.x, d.R, d.V, d.rowptr, d.col, p[None], np.array([i], np.int32))
    for g in range(2):
        e = np.zeros(2); e[g] = eps
        up = O.rk_at_points(d.x, d.R, d.V, d.rowptr, d.col, (p + e)[None], np.array([i], np.int32))
        dn = O.rk_at_points(d.x, d.R, d.V, d.rowptr, d.col, (p - e)[None], np.array([i], np.int32))
        assert np.array_equal(up[1], base[1]) and np.array_equal(dn[1], base[1])
        fd = (up[2] - dn[2]) / (2 * eps)
        assert np.abs(fd - base[3][:, g]).max() < 1e-6 * np.abs(base[3]).max()


def test_support_is_strict_radius():
    d = _setup()
    sptr, sidx, U, dU = O.rk_at_points(d.x, d.R, d.V, d.rowptr, d.col, d.vq.x[:500], d.vq.owner[:500])
    rows = np.repeat(np.arange(500), np.diff(sptr))
    r = np.linalg.norm(d.vq.x[rows] - d.x[sidx], axis=1)
    assert np.all(r < d.R[sidx])
    # nothing inside the support is missing
    for p in range(0, 500, 37):
        inside = np.where(np.linalg.norm(d.x - d.vq.x[p], axis=1) < d.R)[0]
        assert set(inside) == set(sidx[sptr[p]:sptr[p + 1]])


def test_partition_of_unity_changes_with_scale_only_by_rounding():
    # U does not depend on the common basis scale s (here: owner h); compare a
    # point evaluated from two different owners that both see its support.
    d = _setup()
    q = 100
    o1 = d.vq.owner[q]
    nb = d.col[d.rowptr[o1]:d.rowptr[o1 + 1]]
    dist = np.linalg.norm(d.x[nb] - d.vq.x[q], axis=1)
    o2 = nb[np.argsort(dist)[1]]
    a = O.rk_at_points(d.x, d.R, d.V, d.rowptr, d.col, d.vq.x[q:q + 1], np.array([o1], np.int32))
    b = O.rk_at_points(d.x, d.R, d.V, d.rowptr, d.col, d.vq.x[q:q + 1], np.array([o2], np.int32))
    if np.array_equal(a[1], b[1]):
        assert np.allclose(a[2], b[2], rtol=1e-12, atol=1e-12)


def test_singular_moment_matrix_reported():
    # two points only: the linear moment matrix at a point is rank deficient
    x = np.array([[0.3, 0.5], [0.7, 0.5]])
    R = np.full(2, 0.3)
    V = np.full(2, 0.5)
    rowptr = np.array([0, 2, 4], np.int64)
    col = np.array([0, 1, 0, 1], np.int32)
    with pytest.raises(FloatingPointError):
        O.rk_at_points(x, R, V, rowptr, col, np.array([[0.5, 0.5]]), np.array([0], np.int32))
