"""GPU parity of the DSA-like outer preconditioner (outer_precond = 1).

The library right-preconditions its outer (scattering) GMRES with
I + C^-1 Ms, C the P1-diffusion operator built from the integrated forms
(Sec. 5.3 and Sec. 6 name diffusion acceleration as the remedy for slow outer
solves; the operator is the oracle's Transport.diffusion_matrix).  Its
diffusion solves are FP64 GMRES with block-Jacobi to 1e-10 inside a flexible
outer GMRES.  Checked against the oracle's Solver(precond="dsa"), whose
diffusion solves are exact:
  * the same scalar flux (1e-9 relative L2 in FP64, 1e-8 mixed);
  * outer iterations per step within one of the oracle's;
  * in thick scatterers the outer iterations drop at least threefold against
    the library's own unpreconditioned outer solve;
  * without scattering the preconditioner is the identity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import mlpg_inputs as mi  # noqa: E402
import oracle.mlpg_oracle as O  # noqa: E402
import paper_2008_02205_gb300 as pkg  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _oracle(p, steps, dt, tol, precond):
    d = O.Discretization(p.x, p.R, p.lo, p.hi)
    F = d.assemble_per_point(p.sigma_t, p.sigma_s, p.q)
    tr = O.Transport(d, F, p.omega, p.w, psi_b=p.inflow)
    sol = O.Solver(tr, outer_tol=tol, precond=precond)
    Psi = np.zeros((tr.M, d.n))
    Phi = tr.D(Psi)
    its = []
    for _ in range(steps):
        Psi, Phi, st = sol.step(Psi, dt, Phi_guess=Phi)
        its.append(st.outer_iterations)
    return d.interpolation_matrix() @ Phi, its


def _library(p, steps, dt, tol, **opts):
    with pkg.TransportProblem.from_problem(p, inner_tol=1e-13, outer_tol=tol, **opts) as tp:
        tp.integrate().assemble()
        its, dsa = [], []
        for _ in range(steps):
            tp.step(dt)
            st = tp.stats()
            its.append(st["last_outer_iters"])
            dsa.append(st["last_dsa_iters"])
        return tp.scalar_flux(), its, dsa


@pytest.mark.parametrize("dim", [2, 3])
def test_dsa_matches_the_oracle_flux_and_iterations(dim):
    if dim == 2:
        p = mi.two_region_2d(14, sn=4, steps=2)
    else:
        p = mi.make_problem("3d", 4, 3, 4, 3002, 5.0, 4.9, 1.0, 0.05, 2)
    ref, oits = _oracle(p, p.steps, p.dt, 1e-13, "dsa")
    phi, its, dsa = _library(p, p.steps, p.dt, 1e-13, outer_precond=1)
    print(f"dim {dim}: outer iterations library {its}, oracle {oits}; diffusion iterations {dsa}")
    assert _rel(phi, ref) < 1e-9
    assert all(abs(a - b) <= 1 for a, b in zip(its, oits)), (its, oits)
    assert all(k > 0 for k in dsa)
    plain, pits, _ = _library(p, p.steps, p.dt, 1e-13)
    assert _rel(plain, phi) < 1e-9
    assert sum(its) <= sum(pits)


def test_dsa_cuts_outer_iterations_in_a_thick_scatterer():
    """16^2, S4, sigma_t = 20, scattering ratio 0.99, steady (the oracle's pin
    measured 42 -> 9 outer iterations with its exact diffusion solves)."""
    p = mi.small_2d(16, sn=4, steps=1, sigma_t=20.0, sigma_s=19.8)
    phi_d, its_d, _ = _library(p, 1, np.inf, 1e-10, outer_precond=1)
    phi_p, its_p, _ = _library(p, 1, np.inf, 1e-10)
    ref, oits = _oracle(p, 1, np.inf, 1e-10, "dsa")
    print(f"thick scatterer: outer iterations {its_p[0]} plain, {its_d[0]} with DSA (oracle {oits[0]})")
    assert its_d[0] * 3 <= its_p[0]
    assert abs(its_d[0] - oits[0]) <= 1
    assert _rel(phi_d, phi_p) < 1e-8 and _rel(phi_d, ref) < 1e-8


def test_dsa_is_the_identity_without_scattering():
    p = mi.small_2d(10, sigma_t=2.0, sigma_s=0.0, steps=1)
    a, ia, _ = _library(p, 1, p.dt, 1e-12, outer_precond=1)
    b, ib, _ = _library(p, 1, p.dt, 1e-12)
    assert ia == ib and _rel(a, b) < 1e-13


def test_dsa_in_mixed_precision_matches_the_oracle():
    p = mi.two_region_2d(16, sn=8, steps=3, seed=2216)
    ref, _ = _oracle(p, p.steps, p.dt, 1e-13, None)
    phi, its, dsa = _library(p, p.steps, p.dt, 1e-12, outer_precond=1, precision=pkg.MLPG_MIXED,
                             refine_tol=1e-12)
    assert _rel(phi, ref) < 1e-8
    assert sum(dsa) > 0


def test_dsa_options_are_checked():
    p = mi.small_2d(6, steps=1)
    for bad in (dict(outer_precond=2), dict(outer_precond=1, outer_method=1), dict(outer_precond=1, dsa_tol=0.0),
                dict(outer_precond=1, dsa_max=0)):
        with pytest.raises(pkg.MlpgError):
            pkg.TransportProblem.from_problem(p, **bad)
