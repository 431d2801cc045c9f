"""Pins of the oracle's reference rules (Sec. 3.2, App. A) and angular sets."""
import math

import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    t, w = O.gauss_jacobi(n, 0.0, 0.0)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * t ** k) - exact) < 1e-14
    # and not beyond: degree 2n is integrated with an error
    assert abs(np.sum(w * t ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("a,b", [(1.0, 0.0), (2.0, 0.0), (0.5, 1.5)])
def test_gauss_jacobi_weight(a, b):
    # int_{-1}^{1} (1-t)^a (1+t)^b t^k dt against scipy's independent rule
    from scipy.special import roots_jacobi
    n = 5
    t, w = O.gauss_jacobi(n, a, b)
    t2, w2 = roots_jacobi(n, a, b)
    assert np.allclose(np.sort(t), np.sort(t2), atol=1e-14)
    assert np.allclose(w[np.argsort(t)], w2[np.argsort(t2)], rtol=1e-13)


def test_triangle_rule_degree_9():
    xi, w = O.triangle_rule(5)
    assert abs(w.sum() - 0.5) < 1e-15
    for a in range(12):
        for b in range(12 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b)
            if a + b <= 9:
                assert abs(got - exact) < 1e-15
    # degree 10 is not exact in u
    assert abs(np.sum(w * xi[:, 0] ** 10) - math.factorial(10) / math.factorial(12)) > 1e-9
    assert np.all(w > 0) and np.all(xi >= 0) and np.all(xi.sum(1) <= 1)


@pytest.mark.parametrize("order,dim,count", [(4, 2, 12), (8, 2, 40), (12, 2, 84), (4, 3, 24), (8, 3, 80)])
def test_level_symmetric_moments(order, dim, count):
    om, w = mi.level_symmetric(order, dim)
    assert om.shape == (count, 3)
    assert np.all(w > 0)
    assert abs(w.sum() - 4 * math.pi) < 1e-13
    assert np.allclose(np.linalg.norm(om, axis=1), 1.0, atol=1e-15)
    d = dim
    first = (w[:, None] * om[:, :d]).sum(0)
    assert np.abs(first).max() < 1e-13
    second = np.einsum("m,ma,mb->ab", w, om, om)
    assert np.abs(second - 4 * math.pi / 3 * np.eye(3)).max() < 1e-13
    # fourth moment int mu^4 = 4 pi / 5 (matched by construction for N >= 4)
    assert abs(np.sum(w * om[:, 0] ** 4) - 4 * math.pi / 5) < 1e-12


def test_s4_mu1_closed_form():
    # S4: 2 mu1^4 + (1 - 2 mu1^2)^2 = 3/5  ->  mu1^2 = (4 - sqrt(6.4)) / 12
    om, _ = mi.level_symmetric(4, 3)
    mu1 = math.sqrt((4 - math.sqrt(6.4)) / 12)
    assert abs(np.abs(om).min() - mu1) < 1e-12
