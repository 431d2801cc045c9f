"""Pins of the oracle's connectivity (Sec. 3.4) and cells (Sec. 3.1)."""
import os

import numpy as np
import pytest
from scipy.spatial import Voronoi, cKDTree

import mlpg_inputs as mi
import oracle.mlpg_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _pts(n, jitter=0.2, seed=11):
    x, h = mi.jittered_lattice(n, 2, seed, jitter=jitter)
    return x, np.full(len(x), 2 * h), h


def test_neighbors_match_kdtree():
    x, R, h = _pts(20)
    rowptr, col = O.neighbors(x, R)
    tree = cKDTree(x)
    for i in range(len(x)):
        ref = sorted(j for j in tree.query_ball_point(x[i], 4 * h * (1 + 1e-12))
                     if np.linalg.norm(x[i] - x[j]) < R[i] + R[j])
        assert list(col[rowptr[i]:rowptr[i + 1]]) == ref


def test_overlap_count_matches_paper():
    # Sec. 5: a sampling radius of 4 neighbours gives about 50 overlap
    # neighbours per point in 2D (continuum count pi * 4^2).
    table = dict(np.loadtxt(os.path.join(GOLDEN, "overlap_neighbors.txt"), dtype=int))
    x, R, h = _pts(48)
    rowptr, col = O.neighbors(x, R)
    cnt = np.diff(rowptr)
    interior = np.all((x > 4 * h) & (x < 1 - 4 * h), axis=1)
    assert abs(cnt[interior].mean() - table[2]) / table[2] < 0.03


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_cells_partition_domain(jitter):
    x, R, h = _pts(16, jitter)
    rowptr, col = O.neighbors(x, R)
    cptr, verts, labels, V = O.cells_2d(x, R, np.zeros(2), np.ones(2), rowptr, col)
    assert abs(V.sum() - 1.0) < 1e-13
    assert np.all(V > 0)
    if jitter == 0.0:
        assert np.allclose(V, h * h, rtol=1e-12)


def test_cells_equal_scipy_voronoi_interior():
    x, R, h = _pts(16)
    rowptr, col = O.neighbors(x, R)
    cptr, verts, labels, V = O.cells_2d(x, R, np.zeros(2), np.ones(2), rowptr, col)
    vor = Voronoi(x)
    interior = np.where(np.all((x > 3 * h) & (x < 1 - 3 * h), axis=1))[0]
    for i in interior:
        reg = vor.regions[vor.point_region[i]]
        assert -1 not in reg
        p = vor.vertices[reg]
        c = p.mean(0)
        p = p[np.argsort(np.arctan2(p[:, 1] - c[1], p[:, 0] - c[0]))]
        area = 0.5 * abs(np.sum(p[:, 0] * np.roll(p[:, 1], -1) - np.roll(p[:, 0], -1) * p[:, 1]))
        assert abs(area - V[i]) < 1e-14


def test_cells_contain_generator_and_are_ccw():
    x, R, h = _pts(12)
    rowptr, col = O.neighbors(x, R)
    cptr, verts, labels, V = O.cells_2d(x, R, np.zeros(2), np.ones(2), rowptr, col)
    for i in range(len(x)):
        P = verts[cptr[i]:cptr[i + 1]]
        Q = np.roll(P, -1, axis=0)
        cross = (P[:, 0] - x[i, 0]) * (Q[:, 1] - x[i, 1]) - (P[:, 1] - x[i, 1]) * (Q[:, 0] - x[i, 0])
        assert np.all(cross >= -1e-18)


def test_quadrature_points_cover_domain():
    x, R, h = _pts(10)
    d = O.Discretization(x, R)
    assert abs(d.vq.w.sum() - 1.0) < 1e-13
    assert abs(d.bq.w.sum() - 4.0) < 1e-13
    for f in range(4):
        assert abs(d.bq.w[d.bq.face == f].sum() - 1.0) < 1e-13
    # int x dV = 1/2, int x y dV = 1/4 (polynomials: exact with the degree-9 rule)
    assert abs(np.sum(d.vq.w * d.vq.x[:, 0]) - 0.5) < 1e-14
    assert abs(np.sum(d.vq.w * d.vq.x[:, 0] * d.vq.x[:, 1] ** 3) - 1 / 8) < 1e-14
    # boundary points lie on their face
    on = np.array([d.bq.x[d.bq.face == f][:, f // 2] for f in range(4)], dtype=object)
    for f in range(4):
        assert np.allclose(on[f], float(f % 2), atol=0)
