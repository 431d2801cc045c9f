"""The oracle's own inner scheme of Sec. 4.2 (restarted GMRES right
preconditioned by an incomplete LU with threshold, per direction) against
its exact sparse-LU inner solves.

Both solve the same linear systems L_m x = b; at inner tolerance 1e-13 the
backward-Euler steps they produce must agree to 1e-10 in the scalar flux, and
the outer scattering GMRES must take the same number of iterations.  The
iteration counts are what the benchmark reports beside the library's."""
import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O


@pytest.mark.parametrize("side", [10, 16])
def test_ilut_gmres_inner_solves_give_the_lu_step(side):
    prob = mi.two_region_2d(n_per_dim=side, steps=2)
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    out = {}
    for inner in ("lu", "ilut-gmres"):
        tr = O.Transport(disc, F, prob.omega, prob.w, psi_b=prob.inflow)
        sol = O.Solver(tr, outer_tol=1e-13, inner=inner, inner_tol=1e-13)
        _, Phi, st = sol.run(np.zeros((tr.M, disc.n)), prob.dt, prob.steps)
        out[inner] = (Phi, [s.outer_iterations for s in st], list(sol.inner_counts))
    (p_lu, o_lu, _), (p_il, o_il, counts) = out["lu"], out["ilut-gmres"]
    assert np.linalg.norm(p_il - p_lu) / np.linalg.norm(p_lu) < 1e-10
    assert o_il == o_lu
    # one count per direction and inner solve: the first flight, the outer
    # GMRES's operator applies (its iterations and its true-residual checks)
    # and the recovery solve of each step
    assert len(counts) % prob.m == 0 and len(counts) >= prob.m * sum(o + 2 for o in o_il)
    assert np.mean(counts) >= 1 and max(counts) < 50   # a zero right-hand side takes 0 iterations
