"""Pins of the asteroid problem's analytic solution (App. B) and of the oracle's
transport solve against it on a scaled-down asteroid problem (Sec. 5.4).

The analytic side is checked against brute force (optical depth by marching
along the segment, the mu integral by adaptive quadrature); the transport
oracle is then checked against the analytic solution summed over the points of
a smooth source: the error where rays miss the disk is small and falls with
the spacing, the flux deep in the shadow is nearly zero, and the shadow edge
(a discontinuity the discretisation smears) stays bounded."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import mlpg_inputs as mi
from oracle import asteroid as A
from oracle.mlpg_oracle import solve_problem

CENTRE, RADIUS = np.array([0.35, 0.0]), 0.35


def _march(xs, xe, sb, sa, k=200001):
    """Optical depth by the midpoint rule on k pieces of the segment."""
    s = (np.arange(k) + 0.5) / k
    p = xs + s[:, None] * (xe - xs)
    sig = np.where(np.linalg.norm(p - CENTRE, axis=1) < RADIUS, sa, sb)
    return sig.sum() * np.linalg.norm(xe - xs) / k


def test_optical_depth_matches_marching():
    rng = np.random.Generator(np.random.PCG64(11))
    cases = [((-0.55, 0.0), (1.0, 0.0)),      # through the centre, behind the disk
             ((-0.55, 0.0), (0.3, 0.1)),      # ends inside the disk
             ((-0.55, 0.0), (-0.2, 0.3)),     # ends before the disk
             ((-0.55, 0.0), (0.9, 0.9)),      # misses the disk
             ((0.3, 0.05), (0.9, -0.8)),      # starts inside the disk
             ((0.2, 0.0), (0.5, 0.1)),        # wholly inside
             ((-0.55, 0.0), (-0.9, 0.1))]     # points away from the disk
    cases += [(tuple(rng.uniform(-1, 1, 2)), tuple(rng.uniform(-1, 1, 2))) for _ in range(12)]
    for xs, xe in cases:
        xs, xe = np.array(xs), np.array(xe)
        om, r = A.optical_depth(xs, xe[None], CENTRE, RADIUS, 0.5, 10.0)
        assert r[0] == pytest.approx(np.linalg.norm(xe - xs), rel=1e-14)
        assert om[0] == pytest.approx(_march(xs, xe, 0.5, 10.0), rel=2e-4, abs=1e-6), (xs, xe)


def test_chord_of_a_line_through_the_centre_is_the_diameter():
    xs = CENTRE + np.array([-2.0, 0.0])
    for xe, want in [(CENTRE + [2.0, 0.0], 2 * RADIUS), (CENTRE, RADIUS), (CENTRE - [0.5, 0.0], 0.0)]:
        assert A.disk_chord(xs, np.array([xe]), CENTRE, RADIUS)[0] == pytest.approx(want, abs=1e-12)
    # a chord at distance d from the centre is 2 sqrt(R^2 - d^2); at the tangent that is
    # the square root of a discriminant of rounding size, hence the looser bound there
    for d, want, tol in [(RADIUS, 0.0, 1e-6), (0.6 * RADIUS, 1.6 * RADIUS, 1e-12)]:
        ys = CENTRE + np.array([-2.0, d])
        assert A.disk_chord(ys, np.array([ys + [4.0, 0.0]]), CENTRE, RADIUS)[0] == pytest.approx(want, abs=tol)


@pytest.mark.parametrize("omega", [0.0, 1e-3, 0.3, 1.0, 4.0, 15.0])
def test_scalar_flux_is_the_mu_integral_of_the_angular_flux(omega):
    r = 0.7
    want = quad(lambda mu: float(A.angular_flux(omega, r, mu)), 0.0, 1.0, epsabs=1e-15, epsrel=1e-12)[0]
    got = float(A.scalar_flux(omega, r))
    assert got == pytest.approx(want, rel=1e-9, abs=1e-300)
    if omega == 0.0:
        assert got == pytest.approx(1.0 / r, rel=1e-15)


def test_polar_sums_converge_to_the_scalar_flux():
    om = np.array([0.05, 0.5, 2.0, 6.0])
    exact = A.scalar_flux(om, 1.0)
    errs = []
    for K in (2, 4, 8, 16):
        _, _, mu, a = mi.polar_product_quadrature(4, K)
        errs.append(np.abs(A.scalar_flux_polar(om, 1.0, mu, a) - exact).max())
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4


def test_product_set_carries_the_polar_weights():
    om, w, mu, a = mi.polar_product_quadrature(16, 3)
    assert np.allclose(np.linalg.norm(om, axis=1), 1.0, atol=1e-15)
    inplane = np.hypot(om[:, 0], om[:, 1])
    for k in range(3):
        lev = np.isclose(inplane, mu[k], atol=1e-14)
        assert lev.sum() == 16
        assert w[lev].sum() == pytest.approx(2 * math.pi * mu[k] * a[k], rel=1e-14)
        assert np.abs(om[lev, :2].sum(axis=0)).max() < 1e-14     # azimuths balanced


def _segment_distance(xs, X, c):
    """Distance from c to each segment xs -> X[k]."""
    d = X - xs
    t = np.clip((d @ (c - xs)) / np.maximum(np.einsum("ka,ka->k", d, d), 1e-300), 0.0, 1.0)
    return np.linalg.norm(xs + t[:, None] * d - c, axis=1)


def _regions(prob):
    """Points without a source of their own, split by what the rays from the
    source points meet: clear (every ray passes at least 0.1 from the disk),
    deep shadow (at least 5 mean free paths of disk on every ray), and the
    shadow edge in between."""
    src = np.nonzero(prob.q)[0]
    cmin = np.full(prob.n, np.inf)
    dmin = np.full(prob.n, np.inf)
    for j in src:
        cmin = np.minimum(cmin, A.disk_chord(prob.x[j], prob.x, CENTRE, RADIUS))
        dmin = np.minimum(dmin, _segment_distance(prob.x[j], prob.x, CENTRE))
    far = prob.q == 0.0                          # a line source is singular at its own point
    clear = far & (dmin > RADIUS + 0.1)
    deep = far & (10.0 * cmin > 5.0)
    edge = far & ~clear & ~deep
    return src, clear, deep, edge


@pytest.fixture(scope="module")
def solved():
    """Oracle and analytic scalar flux at the points of the 24^2 and 32^2 problems."""
    out = {}
    for n in (24, 32):
        prob = mi.asteroid_2d(n_per_dim=n)
        h = prob.spacing
        src, clear, deep, edge = _regions(prob)
        # polar levels and weights read back from the ordinates
        inplane = np.hypot(prob.omega[:, 0], prob.omega[:, 1])
        mu = np.unique(np.round(inplane, 12))
        a = np.array([prob.w[np.isclose(inplane, m)].sum() / (2 * math.pi * m) for m in mu])
        ana = A.superposed_scalar_flux(prob.x, prob.x[src], prob.q[src] * h * h, CENTRE, RADIUS,
                                       0.5, 10.0, mu, a)
        out[n] = dict(prob=prob, phi=solve_problem(prob), ana=ana, clear=clear, deep=deep, edge=edge)
    return out


def _l1(s, sel):
    return np.abs(s["phi"] - s["ana"])[sel].sum() / s["ana"][sel].sum()


@pytest.mark.parametrize("n", [24, 32])
def test_oracle_matches_the_analytic_solution(n, solved):
    s = solved[n]
    npts = s["prob"].n
    assert s["clear"].sum() > 0.4 * npts and s["deep"].sum() > 20 and s["edge"].sum() > 0.25 * npts
    clear = s["clear"]
    # clear of the disk: L1 within 0.8 % (24^2) and 0.5 % (32^2), measured 0.58 % and 0.34 %;
    # every point within 5 %, measured 2.9 % and 2.8 %
    assert _l1(s, clear) < {24: 8e-3, 32: 5e-3}[n]
    assert (np.abs(s["phi"] - s["ana"])[clear] / s["ana"][clear]).max() < 0.05
    # deep shadow: measured 2e-4 of the peak
    assert np.abs(s["phi"][s["deep"]]).max() < 1e-3 * s["ana"][clear].max()
    # shadow edge: measured 6.3 % and 6.6 %
    assert _l1(s, s["edge"]) < 0.1


def test_oracle_error_falls_with_the_spacing(solved):
    e = [_l1(solved[n], solved[n]["clear"]) for n in (24, 32)]
    assert e[1] < e[0] / 1.4, e          # measured ratio 1.73 (order 1.9)
