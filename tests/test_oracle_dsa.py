"""Pins of the DSA-like preconditioner for the outer (scattering) GMRES.

The paper names diffusion acceleration as the remedy for its slow outer solves
(Sec. 5.3, Sec. 6) without deriving one.  The oracle's low-order operator is a
Galerkin P1-diffusion operator on the same points, built from forms that are
already integrated:
    C = diag(1 / (3 sigma_t_i)) sum_a K_aa + kappa M0 + (Mt - Ms) + 1/2 sum_f S_f.
The outer GMRES is right-preconditioned with I + C^-1 Ms.  Pinned here:
  * C is a diffusion operator: it maps constants to the absorption, time and
    Marshak boundary terms alone (the stiffness annihilates them), and the
    transport flux of a thick, nearly pure scatterer approaches C^-1 (4 pi Q0)
    as the medium thickens (the asymptotic diffusion limit);
  * a preconditioner changes the iterations, not the solution: the same flux
    as the unpreconditioned solve and as the coupled LU of the step;
  * without scattering (Ms = 0) it is the identity, iteration for iteration;
  * in thick scattering media the outer iterations drop several fold."""
import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O


def _setup(p):
    d = O.Discretization(p.x, p.R, p.lo, p.hi)
    F = d.assemble_per_point(p.sigma_t, p.sigma_s, p.q)
    return d, F, O.Transport(d, F, p.omega, p.w, psi_b=p.inflow)


def test_row_sigma_is_exact_for_constant_material():
    p = mi.small_2d(8, sigma_t=3.5, sigma_s=1.0)
    _, _, tr = _setup(p)
    assert np.allclose(tr.sigma_t_rows(), 3.5, rtol=1e-13)


def test_diffusion_operator_on_constants():
    p = mi.two_region_2d(12, sn=4)
    d, F, tr = _setup(p)
    kappa = 37.0
    C = tr.diffusion_matrix(kappa)
    one = np.ones(d.n)
    want = (kappa * d.csr(F["M0"]) + d.csr(F["Mt"]) - d.csr(F["Ms"])) @ one
    want += 0.5 * sum(d.csr(F["S"][f]) @ one for f in range(4))
    assert np.abs(C @ one - want).max() < 1e-11 * np.abs(want).max()
    # the Marshak term holds the boundary moments <U_i, 1> of the test functions;
    # V_i U_i sum to one, so their V-weighted sum is the perimeter of the unit square
    bnd = sum(d.csr(F["S"][f]) @ one for f in range(4))
    assert (d.V * bnd).sum() == pytest.approx(4.0, rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_dsa_changes_iterations_not_the_solution(dim):
    if dim == 2:
        p = mi.two_region_2d(14, sn=4, steps=2)
    else:
        p = mi.make_problem("3d", 4, 3, 4, 3002, 5.0, 4.9, 1.0, 0.05, 2)
    d, F, tr = _setup(p)
    Psi0 = np.zeros((tr.M, d.n))
    _, Pa, sa = O.Solver(tr, outer_tol=1e-13).run(Psi0, p.dt, p.steps)
    _, Pb, sb = O.Solver(tr, outer_tol=1e-13, precond="dsa").run(Psi0, p.dt, p.steps)
    _, Pc, _ = O.Solver(tr).run(Psi0, p.dt, p.steps, direct=True)
    scale = np.abs(Pc).max()
    assert np.abs(Pb - Pa).max() < 1e-10 * scale
    assert np.abs(Pb - Pc).max() < 1e-10 * scale
    assert sum(s.outer_iterations for s in sb) <= sum(s.outer_iterations for s in sa)


def test_dsa_is_the_identity_without_scattering():
    p = mi.small_2d(10, sigma_t=2.0, sigma_s=0.0, steps=1)
    d, F, tr = _setup(p)
    Psi0 = np.zeros((tr.M, d.n))
    _, Pa, sa = O.Solver(tr).run(Psi0, p.dt, 1)
    _, Pb, sb = O.Solver(tr, precond="dsa").run(Psi0, p.dt, 1)
    assert np.array_equal(Pa, Pb)
    assert sa[0].outer_iterations == sb[0].outer_iterations


@pytest.mark.parametrize("sigma_t,plain_min,ratio", [(20.0, 30, 3.0), (100.0, 80, 3.0)])
def test_dsa_cuts_outer_iterations_in_thick_scatterers(sigma_t, plain_min, ratio):
    # 16^2, S4, c = 0.99 / 0.999, steady: measured 42 -> 9 and 120 -> 25
    p = mi.small_2d(16, sn=4, steps=1, sigma_t=sigma_t, sigma_s=sigma_t - (0.2 if sigma_t == 20.0 else 0.1))
    d, F, tr = _setup(p)
    Psi0 = np.zeros((tr.M, d.n))
    _, Pa, sa = O.Solver(tr, outer_tol=1e-10).step(Psi0, np.inf)
    _, Pb, sb = O.Solver(tr, outer_tol=1e-10, precond="dsa").step(Psi0, np.inf)
    assert sa.outer_iterations >= plain_min
    assert sb.outer_iterations * ratio <= sa.outer_iterations, (sa.outer_iterations, sb.outer_iterations)
    assert np.abs(Pb - Pa).max() < 1e-8 * np.abs(Pa).max()


def test_transport_approaches_diffusion_in_thick_scatterers():
    """sigma_a = 0.1 fixed, sigma_t = 10 and 40 on a regular 16^2 lattice, S8,
    steady: the interior point values of the transport flux and of the diffusion
    solution C^-1 (4 pi Q0) differ by 2.5 % and 0.64 % (measured) of the peak."""
    gaps = []
    for st in (10.0, 40.0):
        p = mi.small_2d(16, sn=8, steps=1, sigma_t=st, sigma_s=st - 0.1, jitter=0.0)
        d, F, tr = _setup(p)
        _, Phi, _ = O.Solver(tr, outer_tol=1e-11, precond="dsa").step(np.zeros((tr.M, d.n)), np.inf)
        import scipy.sparse.linalg as spla
        Phid = spla.spsolve(tr.diffusion_matrix(0.0).tocsc(), 4 * np.pi * F["Q0"])
        I = d.interpolation_matrix()
        phi, phid = I @ Phi, I @ Phid
        inner = np.min(np.stack([p.x[:, 0], 1 - p.x[:, 0], p.x[:, 1], 1 - p.x[:, 1]]), 0) > 0.25
        gaps.append(np.abs(phi - phid)[inner].max() / phi.max())
    assert gaps[0] < 0.04 and gaps[1] < 0.012, gaps
    assert gaps[1] < gaps[0] / 2, gaps


def test_dsa_needs_the_gmres_outer():
    p = mi.small_2d(4)
    _, _, tr = _setup(p)
    with pytest.raises(ValueError):
        O.Solver(tr, outer="source-iteration", precond="dsa")
    with pytest.raises(ValueError):
        O.Solver(tr, precond="multigrid")
