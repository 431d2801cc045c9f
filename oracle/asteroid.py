"""Analytic solution of the asteroid problem (Sec. 5.4, App. B) for the oracle.

TEST INFRASTRUCTURE ONLY: used by tests/test_oracle_asteroid.py to pin the
oracle's transport solve; shares no code with the CUDA library.

In 2D the asteroid is an infinite cylinder (a disk of radius ``radius`` centred
at ``centre``) and the point source a line source.  Along the segment from the
source to an evaluation point at distance r the cross section is the disk's
inside it and the background's outside (Eq. optical-depth-asteroid), and with
mu the cosine of the angle between the x-y plane and the direction the
angular flux is exp(-omega / mu) / r (Eq. asteroid-angular).  App. B
integrates it over 0 <= mu <= 1 with unit measure, which gives the scalar flux
(exp(-omega) - omega E1(omega)) / r = E2(omega) / r (Eq. asteroid-scalar);
``scalar_flux_polar`` is the same integral taken with a polar quadrature,
which is what a discrete-ordinates set with those polar levels reaches once its
azimuths are resolved.  The distance travelled inside the disk comes from the
two intercepts of the segment with the circle (Eq. parametric-s,
Eq. s-intercept).  A source spread over several points is the sum of line
sources (the problem is linear and purely absorbing).
"""
from __future__ import annotations

import numpy as np
from scipy.special import exp1


def disk_chord(x_src, x_eval, centre, radius):
    """Length of the segment x_src -> x_eval (x_eval [k, 2]) inside the disk
    (App. B, Eq. parametric-s and Eq. s-intercept).

    With x = x_src + (x_eval - x_src) s and the disk moved to the origin,
    |x|^2 = radius^2 is l2 s^2 + 2 l1 s + l0 = 0 with l0 = |x_src|^2 - radius^2,
    l1 = x_src . (x_eval - x_src), l2 = |x_eval - x_src|^2; a negative
    discriminant means the line misses the disk.  The intercepts are clipped to
    the segment (0 <= s <= 1): the evaluation point may lie before the disk,
    inside it or behind it, and the source may lie inside it."""
    xs = np.asarray(x_src, np.float64) - np.asarray(centre, np.float64)
    xe = np.atleast_2d(np.asarray(x_eval, np.float64)) - np.asarray(centre, np.float64)
    d = xe - xs
    l0 = xs @ xs - radius * radius
    l1 = d @ xs
    l2 = np.einsum("ka,ka->k", d, d)
    disc = l1 * l1 - l0 * l2
    hit = (disc > 0.0) & (l2 > 0.0)
    root = np.sqrt(np.where(hit, disc, 0.0))
    l2s = np.where(hit, l2, 1.0)
    s_in = np.clip((-l1 - root) / l2s, 0.0, 1.0)
    s_out = np.clip((-l1 + root) / l2s, 0.0, 1.0)
    return np.where(hit, (s_out - s_in) * np.sqrt(l2), 0.0)


def optical_depth(x_src, x_eval, centre, radius, sigma_background, sigma_asteroid):
    """omega = integral of sigma_a along the segment (Eq. optical-depth-asteroid);
    returns (omega, r)."""
    xe = np.atleast_2d(np.asarray(x_eval, np.float64))
    r = np.linalg.norm(xe - np.asarray(x_src, np.float64), axis=1)
    inside = disk_chord(x_src, xe, centre, radius)
    return sigma_asteroid * inside + sigma_background * (r - inside), r


def angular_flux(omega, r, mu):
    """Eq. asteroid-angular: exp(-omega / mu) / r for 0 < mu <= 1."""
    return np.exp(-np.asarray(omega) / mu) / np.asarray(r)


def scalar_flux(omega, r):
    """Eq. asteroid-scalar: (exp(-omega) - omega E1(omega)) / r; 1 / r at omega = 0."""
    omega = np.asarray(omega, np.float64)
    pos = omega > 0.0
    tail = np.where(pos, omega * exp1(np.where(pos, omega, 1.0)), 0.0)
    return (np.exp(-omega) - tail) / np.asarray(r, np.float64)


def scalar_flux_polar(omega, r, mu, a):
    """sum_k a_k exp(-omega / mu_k) / r: the mu integral of Eq. asteroid-angular
    with polar nodes mu_k and weights a_k on [0, 1]."""
    omega = np.asarray(omega, np.float64)
    mu = np.asarray(mu, np.float64)
    a = np.asarray(a, np.float64)
    return np.exp(-omega[..., None] / mu) @ a / np.asarray(r, np.float64)


def superposed_scalar_flux(x_eval, sources, strengths, centre, radius, sigma_background,
                           sigma_asteroid, mu=None, a=None):
    """(App. B, by superposition) sum_j S_j phi(x_eval; source j) for line sources at `sources` [J, 2] with
    strengths S_j; the polar integral is exact (E2) unless (mu, a) are given.
    Undefined (inf) at a source point."""
    xe = np.atleast_2d(np.asarray(x_eval, np.float64))
    out = np.zeros(len(xe))
    for xs, s in zip(np.atleast_2d(sources), np.asarray(strengths, np.float64)):
        om, r = optical_depth(xs, xe, centre, radius, sigma_background, sigma_asteroid)
        with np.errstate(divide="ignore", invalid="ignore"):
            phi = scalar_flux(om, r) if mu is None else scalar_flux_polar(om, r, mu, a)
        out += s * np.where(r > 0.0, phi, np.inf)
    return out
