"""The request stream of the serving configuration (input generation only):
Poisson arrivals, the dimension / size / angular-set / material / step-count
draws, and reproducibility from the seed."""
import math

import numpy as np
import pytest

import mlpg_inputs as mi


@pytest.fixture(scope="module")
def stream():
    return mi.serving_stream(count=200, rate=4.0, seed=5100, n_range=(64, 1024))


def test_arrivals_are_a_poisson_process(stream):
    t = np.array([a for _, a in stream])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps of mean 1 / rate: mean within 4 standard errors, and the
    # coefficient of variation of an exponential is 1
    assert abs(gaps.mean() - 0.25) < 4 * 0.25 / math.sqrt(len(gaps))
    assert 0.8 < gaps.std() / gaps.mean() < 1.2


def test_problem_draws_follow_the_recipe(stream):
    dims = np.array([p.dim for p, _ in stream])
    assert 0.15 < (dims == 3).mean() < 0.35
    for p, _ in stream:
        k = round(p.n ** (1.0 / p.dim))
        assert k ** p.dim == p.n and p.x.shape == (p.n, p.dim)
        assert 64 * 0.5 <= p.n <= 1024 * 1.6
        if p.dim == 2:
            assert p.m in (12, 24, 40, 60, 84)
        else:
            assert p.m in (24, 80, 168, 272)
        assert np.isclose(p.w.sum(), 4 * math.pi, rtol=1e-12)
        assert 5 <= p.steps <= 50 and p.dt == 0.01
        # two regions, each sigma_t in [0.1, 100]; one scattering ratio; q = 1 for x_0 < 0.5
        inside = np.all((p.x >= 0.4) & (p.x <= 0.6), axis=1)
        assert np.unique(p.sigma_t[inside]).size <= 1 and np.unique(p.sigma_t[~inside]).size == 1
        assert p.sigma_t.min() >= 0.1 and p.sigma_t.max() <= 100.0
        ratio = p.sigma_s / p.sigma_t
        assert np.allclose(ratio, ratio[0]) and 0.0 <= ratio[0] <= 0.99
        assert np.array_equal(p.q, np.where(p.x[:, 0] < 0.5, 1.0, 0.0))
        assert not p.inflow
    assert any(p.m == 272 for p, _ in stream)          # some 3D requests use the refined set


def test_stream_is_reproducible():
    a = mi.serving_stream(count=5, seed=77, n_range=(64, 256))
    b = mi.serving_stream(count=5, seed=77, n_range=(64, 256))
    for (p, s), (q, t) in zip(a, b):
        assert s == t and np.array_equal(p.x, q.x) and np.array_equal(p.sigma_t, q.sigma_t)
        assert np.array_equal(p.omega, q.omega) and p.steps == q.steps
