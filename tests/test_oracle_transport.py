"""Pins of the oracle's transport solve (Sec. 4.1-4.2, Sec. 5).

  * nested scheme (first flight, GMRES on Phi, recovery) == one sparse LU of
    the coupled step system;
  * particle balance of every step (SUPG leaves global balance unchanged,
    Sec. 4.1), exact for uniform tau;
  * infinite-medium backward-Euler recurrence (0D closed form) up to the
    measured divergence-theorem quadrature defect;
  * pure absorber psi = exp(-sigma x) (2D analogue of Sec. 5.2), order ~2;
  * manufactured solutions of Sec. 5.1: second order in space, first in time;
  * planted mistakes in the oracle fail these pins.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import mlpg_inputs as mi
import oracle.mlpg_oracle as O
from oracle import mms


def _tr(n=10, sn=4, seed=1000, **kw):
    p = mi.small_2d(n, sn=sn, seed=seed, **kw)
    d = O.Discretization(p.x, p.R)
    F = d.assemble_per_point(p.sigma_t, p.sigma_s, p.q)
    return p, d, F, O.Transport(d, F, p.omega, p.w, psi_b=p.inflow)


def test_nested_equals_direct():
    p, d, F, tr = _tr(10)
    s = O.Solver(tr, outer_tol=1e-14)
    Psi0 = np.random.default_rng(0).uniform(0, 1, (tr.M, d.n))
    Psi, Phi, st = s.step(Psi0, p.dt)
    Psi2, Phi2 = s.step_direct(Psi0, p.dt)
    assert np.linalg.norm(Phi - Phi2) / np.linalg.norm(Phi2) < 1e-11
    assert np.linalg.norm(Psi - Psi2) / np.linalg.norm(Psi2) < 1e-11
    assert st.outer_iterations > 1


def _balance(tr, Psi, Psi_prev, kappa, psi_b):
    d, F, V = tr.d, tr.F, tr.d.V
    Phi, Phi_prev = tr.D(Psi), tr.D(Psi_prev)
    val = kappa * V @ (d.csr(F["M0"]) @ (Phi - Phi_prev))
    val += V @ (d.csr(F["Mt"]) @ Phi) - V @ (d.csr(F["Ms"]) @ Phi) - 4 * math.pi * V @ F["Q0"]
    for m in range(tr.M):
        for f in range(4):
            on = float(tr.omega[m, :2] @ tr.nf[f, :2])
            if on > 0:
                val += tr.w[m] * on * (V @ (d.csr(F["S"][f]) @ Psi[m]))
            elif on < 0 and f in psi_b:
                val -= tr.w[m] * (-on) * psi_b[f] * (V @ F["B"][f])
    return val


def test_global_balance_every_step():
    p, d, F, tr = _tr(12)
    tr.psi_b = {0: 0.7, 3: 0.2}
    s = O.Solver(tr, outer_tol=1e-14)
    Psi = np.zeros((tr.M, d.n))
    kappa = 1.0 / p.dt
    scale = 4 * math.pi * (d.V @ F["Q0"])
    for _ in range(3):
        new, _, _ = s.step(Psi, p.dt)
        assert abs(_balance(tr, new, Psi, kappa, tr.psi_b)) < 1e-11 * scale
        Psi = new


def test_planted_outflow_sign_breaks_balance():
    p, d, F, tr = _tr(8)
    orig = tr.L_matrix

    def wrong(m, kappa):   # outflow face term with the wrong sign
        A = orig(m, kappa)
        for f in range(4):
            on = float(tr.omega[m, :2] @ tr.nf[f, :2])
            if on > 0:
                A = A - 2 * on * d.csr(F["S"][f])
        return A.tocsr()
    tr.L_matrix = wrong
    s = O.Solver(tr, outer_tol=1e-14)
    Psi = np.zeros((tr.M, d.n))
    new, _, _ = s.step(Psi, p.dt)
    scale = 4 * math.pi * (d.V @ F["Q0"])
    assert abs(_balance(tr, new, Psi, 1.0 / p.dt, {})) > 1e-6 * scale


def test_infinite_medium_recurrence():
    # uniform sigma, q; inflow psi_b = phi^n / 4 pi on every face; uniform start.
    p, d, F, tr = _tr(16, steps=4)
    s = O.Solver(tr, outer_tol=1e-14)
    sa, kap = 0.5, 1.0 / p.dt
    ph = 2.0
    Psi = np.full((tr.M, d.n), ph / (4 * math.pi))
    Phi = tr.D(Psi)
    I = d.interpolation_matrix()
    for _ in range(4):
        ph = (kap * ph + 4 * math.pi * 1.0) / (kap + sa)      # 0D backward Euler
        tr.psi_b = {f: ph / (4 * math.pi) for f in range(4)}
        tr._kappa = None
        Psi, Phi, _ = s.step(Psi, p.dt, Phi_guess=Phi)
        assert np.abs(I @ Phi - ph).max() / ph < 2e-4          # quadrature defect only


def test_steady_equilibrium_value():
    # phi_inf = 4 pi q / sigma_a = 8 pi in the interior of a large medium:
    # uniform inflow at the equilibrium value makes it exact up to quadrature.
    p, d, F, tr = _tr(12)
    tr.psi_b = {f: 2.0 for f in range(4)}
    s = O.Solver(tr, outer_tol=1e-14)
    Psi, Phi, _ = s.step(np.zeros((tr.M, d.n)), np.inf)
    phi = d.interpolation_matrix() @ Phi
    assert np.abs(phi - 8 * math.pi).max() / (8 * math.pi) < 2e-4


def _absorber(n, sigma=5.0):
    x, h = mi.jittered_lattice(n, 2, 0, jitter=0.0)
    d = O.Discretization(x, np.full(len(x), 2 * h))
    F = d.assemble_per_point(np.full(d.n, sigma), np.zeros(d.n), np.zeros(d.n))
    tr = O.Transport(d, F, np.array([[1.0, 0.0, 0.0]]), np.array([4 * math.pi]), psi_b={0: 1.0})
    Psi, Phi, _ = O.Solver(tr).step(np.zeros((1, d.n)), np.inf)
    psi = d.interpolation_matrix() @ Psi[0]
    return np.abs(psi - np.exp(-sigma * x[:, 0])).mean()


def test_pure_absorber_closed_form_order():
    e = [_absorber(n) for n in (8, 16, 32)]
    slopes = np.log2(np.array(e[:-1]) / np.array(e[1:]))
    assert e[-1] < 2e-3
    assert slopes.min() > 1.6          # Sec. 5.2: about second order for linear RK


@pytest.mark.slow
@pytest.mark.parametrize("prob", [mms.Sinusoidal(), mms.Wave()], ids=["sinusoidal", "wave"])
@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_mms_space_second_order(prob, jitter):
    om, w = mi.level_symmetric(4, 2)
    errs = []
    for n in (8, 16, 32):
        x, h = mi.jittered_lattice(n, 2, 5, lo=-1, hi=1, jitter=jitter)
        errs.append(mms.mms_run(prob, x, np.full(len(x), 2 * h), om, w))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 2e-4
    assert slopes.mean() > 1.8


@pytest.mark.slow
def test_mms_time_first_order():
    om, w = mi.level_symmetric(4, 2)
    x, h = mi.jittered_lattice(20, 2, 5, lo=-1, hi=1, jitter=0.0)
    errs = [mms.mms_run(mms.Sinusoidal(), x, np.full(len(x), 2 * h), om, w, dt=dt, t_end=1.0)
            for dt in (0.5, 0.25, 0.125)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 0.6) and np.all(slopes < 1.3)


def test_planted_missing_supg_sigma_term_breaks_mms(monkeypatch):
    # Drop tau Omega <d U_i, sigma_t U_j> from L (a plausible slip): the scheme
    # is no longer consistent and the manufactured error stops converging.
    om, w = mi.level_symmetric(4, 2)
    orig = O.Transport.L_matrix

    def wrong(self, m, kappa):
        A = orig(self, m, kappa)
        T = sp.diags(self.tau)
        return (A - T @ sum(self.omega[m, a] * self.d.csr(self.F["Gt"][a]) for a in range(2))).tocsr()
    monkeypatch.setattr(O.Transport, "L_matrix", wrong)
    errs = []
    for n in (8, 16):
        x, h = mi.jittered_lattice(n, 2, 5, lo=-1, hi=1, jitter=0.0)
        errs.append(mms.mms_run(mms.Sinusoidal(), x, np.full(len(x), 2 * h), om, w))
    assert errs[1] > 2e-3 or np.log2(errs[0] / errs[1]) < 1.5


@pytest.mark.parametrize("ratio", [0.5, 0.9])
def test_source_iteration_converges_to_the_krylov_solution(ratio):
    # the same step by source iteration: the fixed point of Phi <- b_phi + D L^-1 MS Phi;
    # in a nearly infinite medium its error contracts by about the scattering ratio per
    # iteration, so it needs about log(tol)/log(c) iterations where GMRES needs few
    p = mi.small_2d(10, sn=4, seed=1000, sigma_t=4.0, sigma_s=4.0 * ratio)
    d = O.Discretization(p.x, p.R)
    F = d.assemble_per_point(p.sigma_t, p.sigma_s, p.q)
    tr = O.Transport(d, F, p.omega, p.w)
    Psi0 = np.random.default_rng(1).uniform(0, 1, (tr.M, d.n))
    Pg, Fg, sg = O.Solver(tr, outer_tol=1e-13).step(Psi0, p.dt)
    Ps, Fs, ss = O.Solver(tr, outer_tol=1e-13, outer="source-iteration").step(Psi0, p.dt)
    assert np.linalg.norm(Fs - Fg) / np.linalg.norm(Fg) < 1e-11
    assert np.linalg.norm(Ps - Pg) / np.linalg.norm(Pg) < 1e-11
    assert np.abs(tr.D(Ps) - Fs).max() < 1e-13 * np.abs(Fs).max()
    assert ss.outer_iterations <= math.log(1e-13) / math.log(ratio) + 5
    assert ss.outer_iterations > sg.outer_iterations
