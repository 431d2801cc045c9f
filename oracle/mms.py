"""Manufactured problems of Sec. 5.1 for the oracle (test infrastructure only).

The method of manufactured solutions (Sec. 5.1): pick psi, derive q from the
continuous transport equation (Eq. transport-equation), take psi_b = psi on the
boundary, and compare the discrete point values phi_i with 4 pi psi(x_i).
Both manufactured solutions of the paper are isotropic in angle, so
phi = 4 pi psi and the scattering term reduces to sigma_s psi; the source is
q = d_t psi + Omega . grad psi + sigma_a psi.
"""
from __future__ import annotations

import math

import numpy as np

from .mlpg_oracle import (FOUR_PI, Discretization, Solver, Transport, face_normals,
                          relative_error, rk_at_points)


class Sinusoidal:
    """Sec. 5.1.1: psi = 1 + (1/2pi) prod_a cos(pi (x^a + t)), on [-1, 1]^d,
    sigma_a = 1 + (2/3) prod cos(3 x^a), sigma_s = 1 + (3/4) prod sin(2 x^a)."""
    lo, hi, t_steady = -1.0, 1.0, 0.0

    def psi(self, x, t):
        return 1.0 + np.prod(np.cos(np.pi * (x + t)), axis=1) / (2 * np.pi)

    def grad(self, x, t):
        c = np.cos(np.pi * (x + t))
        s = np.sin(np.pi * (x + t))
        d = x.shape[1]
        g = np.zeros_like(x)
        for a in range(d):
            term = -np.pi * s[:, a]
            for b in range(d):
                if b != a:
                    term = term * c[:, b]
            g[:, a] = term / (2 * np.pi)
        return g

    def dt(self, x, t):
        return self.grad(x, t).sum(axis=1)       # d/dt of cos(pi(x^a + t)) = d/dx^a

    def sigma_a(self, x):
        return 1.0 + (2.0 / 3.0) * np.prod(np.cos(3 * x), axis=1)

    def sigma_s(self, x):
        return 1.0 + 0.75 * np.prod(np.sin(2 * x), axis=1)


class Wave:
    """Sec. 5.1.2: psi = 1 + exp(-10 (|x| - t)^2) / (t^2 + 6) on [-1, 1]^d,
    sigma_a = 0.5, sigma_s = 2; steady case at t = 0.5."""
    lo, hi, t_steady = -1.0, 1.0, 0.5

    def psi(self, x, t):
        r = np.linalg.norm(x, axis=1)
        return 1.0 + np.exp(-10.0 * (r - t) ** 2) / (t * t + 6.0)

    def grad(self, x, t):
        r = np.linalg.norm(x, axis=1)
        e = np.exp(-10.0 * (r - t) ** 2) / (t * t + 6.0)
        dr = -20.0 * (r - t) * e
        with np.errstate(invalid="ignore", divide="ignore"):
            u = np.where(r[:, None] > 0, x / r[:, None], 0.0)
        return dr[:, None] * u

    def dt(self, x, t):
        r = np.linalg.norm(x, axis=1)
        ex = np.exp(-10.0 * (r - t) ** 2)
        return ex * (20.0 * (r - t)) / (t * t + 6.0) - ex * 2 * t / (t * t + 6.0) ** 2

    def sigma_a(self, x):
        return np.full(x.shape[0], 0.5)

    def sigma_s(self, x):
        return np.full(x.shape[0], 2.0)


def mms_run(problem, x, R, omega, w, dt=np.inf, t_end=None, tau_factor=1.0):
    """Solve a manufactured problem on points x; returns eps_rel (Eq. relative-err)
    of phi_i against 4 pi psi(x_i, t_final)."""
    lo = (problem.lo,) * 3
    hi = (problem.hi,) * 3
    disc = Discretization(x, R, lo, hi)
    vq, bq = disc.vq, disc.bq
    sa, ss = problem.sigma_a(vq.x), problem.sigma_s(vq.x)
    F = disc.assemble(sa + ss, ss, np.zeros_like(sa))
    d = disc.dim
    M = omega.shape[0]
    # RK values at volume and boundary quadrature points for the source terms
    vs = rk_at_points(disc.x, disc.R, disc.V, disc.rowptr, disc.col, vq.x, vq.owner)
    bs = rk_at_points(disc.x, disc.R, disc.V, disc.rowptr, disc.col, bq.x, bq.owner)
    vrow = np.repeat(np.arange(len(vq.w)), np.diff(vs[0]))
    brow = np.repeat(np.arange(len(bq.w)), np.diff(bs[0]))
    nf = face_normals(d)
    tau = tau_factor * disc.h

    steady = not np.isfinite(dt)

    def source(t):
        psi_q = problem.psi(vq.x, t)
        q_iso = sa * psi_q + (0.0 if steady else problem.dt(vq.x, t))
        g = problem.grad(vq.x, t)
        psi_b = problem.psi(bq.x, t)
        out = np.zeros((M, disc.n))
        for m in range(M):
            Om = omega[m, :d]
            qm = q_iso + g @ Om                     # q_m at the volume points
            wq = vq.w[vrow] * qm[vrow]
            val = wq * (vs[2] + tau[vs[1]] * (vs[3] @ Om))
            r = np.bincount(vs[1], val, minlength=disc.n)
            on = nf[bq.face, :d] @ Om               # Omega . n at boundary points
            inc = np.where(on < 0.0, -on, 0.0) * psi_b * bq.w
            r += np.bincount(bs[1], inc[brow] * bs[2], minlength=disc.n)
            out[m] = r
        return out

    tr = Transport(disc, F, omega, w, tau_factor=tau_factor)
    sol = Solver(tr, outer_tol=1e-12)
    if np.isfinite(dt):
        steps = int(round(t_end / dt))
        Psi0 = np.tile(problem.psi(disc.x, 0.0), (M, 1))
        _, Phi, _ = sol.run(Psi0, dt, steps, src=lambda k: source(k * dt))
        t_fin = steps * dt
    else:
        t_fin = problem.t_steady
        Psi, Phi, _ = sol.run(np.zeros((M, disc.n)), np.inf, 1, src=lambda k: source(t_fin))
    phi = disc.interpolation_matrix() @ Phi
    return relative_error(phi, FOUR_PI * problem.psi(disc.x, t_fin))
