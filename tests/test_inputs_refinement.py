"""Pins of the hierarchical octant quadrature and its selective refinement
(Sec. 4.3, Alg. 2): exact spherical areas, additivity across levels, the
goal ordinates that hit the object kept, the extreme cases (nothing hits:
the coarsest rule; everything hits: the goal rule), and weights summing to
4 pi."""
import math

import numpy as np
import pytest

import mlpg_inputs as mi


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_levels_partition_the_sphere(level):
    om, w = mi._tri_ordinates(mi._octant_triangles(level))
    assert len(w) == 8 * 4 ** level
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    assert np.allclose(np.linalg.norm(om, axis=1), 1.0)
    if level == 0:
        assert np.allclose(w, math.pi / 2)   # an octant
    # each triangle's area is the sum of its four children's
    _, wc = mi._tri_ordinates(mi._octant_triangles(level + 1))
    assert np.allclose(wc.reshape(-1, 4).sum(1), w, rtol=1e-13, atol=0)


def test_area_against_monte_carlo():
    a, b, c = mi._octant_triangles(1)[3]   # the middle child of the first octant
    _, w = mi._tri_ordinates([(a, b, c)])
    rng = np.random.default_rng(3)
    v = rng.normal(size=(400000, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    M = np.linalg.inv(np.array([a, b, c]).T)   # barycentric-cone coordinates
    inside = np.all(v @ M.T >= 0, axis=1)
    est = 4 * math.pi * inside.mean()
    assert abs(est - w[0]) < 5 * math.sqrt(w[0] * 4 * math.pi / 400000)


def test_refinement_keeps_hitting_goal_ordinates():
    hits = mi.cone_hits((1.0, 0.0, 0.0), 15.0)
    om, w = mi.refined_quadrature(1, 4, hits)
    gom, gw = mi._tri_ordinates(mi._octant_triangles(4))
    goal_hits = np.array([hits(o) for o in gom])
    for o in gom[goal_hits]:
        assert np.min(np.linalg.norm(om - o, axis=1)) < 1e-15
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    assert len(w) < len(gw)


def test_refinement_extremes():
    om, w = mi.refined_quadrature(1, 3, lambda o: False)
    lom, lw = mi._tri_ordinates(mi._octant_triangles(1))
    assert np.allclose(om, lom) and np.allclose(w, lw)
    om, w = mi.refined_quadrature(1, 3, lambda o: True)
    gom, gw = mi._tri_ordinates(mi._octant_triangles(3))
    assert np.allclose(om, gom) and np.allclose(w, gw)


def test_configuration_direction_count():
    p = mi.lognormal_3d(4, refine=(1, 5, 15.0))
    assert p.m == 272 and abs(p.w.sum() - 4 * math.pi) < 1e-12
    inside = p.omega[:, 0] >= math.cos(math.radians(15.0))
    assert inside.sum() == 168
