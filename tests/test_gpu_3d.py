"""GPU parity in 3D: the CUDA path (through the C ABI) against the CPU oracle.

Stages on the same seeded 3D inputs: overlap pattern (bit-exact), polyhedral
cell volumes, integrated forms (volume forms over the fan tetrahedra, surface
forms on the six faces), the batched transport operator in FP64 and FP32,
whole runs in FP64 and mixed precision with inflow on the x = 0 face, and the
lognormal 40^3 S8 configuration at full size through properties that hold at
any size.  Tolerances as in 2D: 1e-9 relative L2 on the scalar flux in FP64,
1e-8 in mixed mode; forms and volumes to rounding.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import mlpg_inputs as mi  # noqa: E402
import oracle.mlpg_oracle as O  # noqa: E402
import paper_2008_02205_gb300 as pkg  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _problem(n=5, sn=4, seed=3001, steps=3, dt=0.02):
    """3D unit cube, jittered n^3 lattice, S_sn (all octants), sigma_t
    lognormal(0, 1) per point, sigma_s = 0.8 sigma_t, inflow 1 on x = 0."""
    return mi.lognormal_3d(n, sn=sn, seed=seed, steps=steps, dt=dt)


@pytest.fixture(scope="module")
def small3():
    prob = _problem()
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tp = pkg.TransportProblem.from_problem(prob, inner_tol=1e-13, outer_tol=1e-13)
    tp.integrate().assemble()
    yield prob, disc, F, tp
    tp.close()


def test_neighbors_bit_exact_3d(small3):
    prob, disc, F, tp = small3
    rowptr, col = tp.neighbors()
    assert np.array_equal(rowptr, disc.rowptr)
    assert np.array_equal(col, disc.col)


def test_volumes_3d(small3):
    prob, disc, F, tp = small3
    V = tp.volumes()
    assert np.abs(V - disc.V).max() <= 1e-13 * disc.V.max()
    assert abs(V.sum() - 1.0) < 1e-13
    st = tp.stats()
    assert st["n_volume_qp"] == len(disc.vq.w) and st["n_boundary_qp"] == len(disc.bq.w)


def test_forms_3d(small3):
    prob, disc, F, tp = small3
    mats, vecs = tp.forms()
    d = 3
    ref_m = np.concatenate([F["M0"][None], F["Mt"][None], F["Ms"][None], F["G"], F["Gt"], F["Gs"],
                            F["K"].reshape(d * d, -1), F["S"]])
    ref_v = np.concatenate([F["Q0"][None], F["Q"], F["B"]])
    assert mats.shape == ref_m.shape and vecs.shape == ref_v.shape
    for k in range(ref_m.shape[0]):
        scale = np.abs(ref_m[k]).max()
        assert np.abs(mats[k] - ref_m[k]).max() <= 1e-12 * scale, k
    for k in range(ref_v.shape[0]):
        scale = max(np.abs(ref_v[k]).max(), 1e-300)
        assert np.abs(vecs[k] - ref_v[k]).max() <= 1e-12 * scale, k


@pytest.mark.parametrize("precision,tol", [(pkg.MLPG_FP64, 1e-13), (pkg.MLPG_MIXED, 3e-6)])
def test_apply_L_3d(small3, precision, tol):
    prob, disc, F, tp = small3
    tr = O.Transport(disc, F, prob.omega, prob.w)
    X = np.random.default_rng(7).uniform(-1, 1, (prob.n, prob.m))
    dtype = torch.float64 if precision == pkg.MLPG_FP64 else torch.float32
    Xd = torch.tensor(X, dtype=dtype, device="cuda")
    Yd = torch.empty_like(Xd)
    pkg.mlpg_apply_L_dev(tp.ctx, prob.dt, precision, Xd.data_ptr(), Yd.data_ptr())
    torch.cuda.synchronize()
    ref = np.stack([tr.L_matrix(m, 1.0 / prob.dt) @ X[:, m] for m in range(prob.m)], axis=1)
    assert _rel(Yd.double().cpu().numpy(), ref) < tol


def _oracle_run(prob):
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tr = O.Transport(disc, F, prob.omega, prob.w, psi_b=prob.inflow)
    Psi, Phi, _ = O.Solver(tr, outer_tol=1e-13).run(np.zeros((tr.M, disc.n)), prob.dt, prob.steps)
    return disc.interpolation_matrix() @ Phi, Phi


@pytest.mark.parametrize("precision,tol", [(pkg.MLPG_FP64, 1e-9), (pkg.MLPG_MIXED, 1e-8)])
def test_run_3d_matches_oracle(precision, tol):
    prob = _problem(6, seed=3002)
    ref, Phi_ref = _oracle_run(prob)
    with pkg.TransportProblem.from_problem(prob, precision=precision, inner_tol=1e-13, outer_tol=1e-13,
                                           refine_tol=1e-12) as tp:
        tp.integrate().assemble()
        phi = tp.run(prob.dt, prob.steps)
        assert _rel(phi, ref) < tol
        assert _rel(tp.scalar_flux(kind=1), Phi_ref) < tol


def test_refined_quadrature_run_matches_oracle():
    """Selectively refined hierarchical quadrature (Alg. 2, levels 0 -> 2,
    refined within 30 degrees of +x, the inflow direction), mixed precision.
    (On coarse lattices with thick cells and small steps some L_m reach
    condition numbers near 1e5 with an indefinite symmetric part, where
    restarted block-Jacobi GMRES stagnates; this lattice keeps them below
    about 1e3.)"""
    prob = mi.lognormal_3d(6, seed=3002, steps=2, dt=0.02, refine=(0, 2, 30.0))
    ref, Phi_ref = _oracle_run(prob)
    with pkg.TransportProblem.from_problem(prob, precision=pkg.MLPG_MIXED, refine_tol=1e-12) as tp:
        tp.integrate().assemble()
        phi = tp.run(prob.dt, prob.steps)
        assert _rel(phi, ref) < 1e-8


@pytest.mark.slow
def test_lognormal_40_cubed_refined_full_size():
    """The 3D configuration at full size (40^3 points, the hierarchical
    quadrature refined within 15 degrees of +x by Alg. 2: 272 directions,
    lognormal sigma_t, sigma_s = 0.8 sigma_t, inflow 1 on x = 0, 10 steps of
    0.01, mixed precision), through properties that hold at any size: volumes
    partition the cube, the integrated forms satisfy the identities of the
    oracle pins, every step's FP64 residual is below the refinement tolerance,
    and every step conserves particles (uniform tau: the balance of Sec. 4.1 is
    exact for the discrete system) when evaluated on the host from the GPU's
    own forms and angular fluxes."""
    import scipy.sparse as sp
    prob = mi.lognormal_3d(refine=(1, 5, 15.0))
    assert (prob.n, prob.m) == (64000, 272)
    with pkg.TransportProblem.from_problem(prob, precision=pkg.MLPG_MIXED) as tp:
        tp.integrate()
        V = tp.volumes()
        assert abs(V.sum() - 1.0) < 1e-12 and np.all(V > 0)
        tp.assemble()
        mats, vecs = tp.forms()
        rowptr, col = tp.neighbors()
        csr = lambda a: sp.csr_matrix((a, col, rowptr), shape=(prob.n, prob.n))
        one = np.ones(prob.n)
        assert abs(V @ csr(mats[0]) @ one - 1.0) < 1e-11
        for a in range(3):
            assert abs(V @ csr(mats[0]) @ prob.x[:, a] - 0.5) < 1e-11
            assert np.abs(V @ csr(mats[3 + a])).max() < 1e-9
        for f in range(6):
            assert abs(V @ csr(mats[21 + f]) @ one - 1.0) < 1e-11
            assert abs(V @ vecs[4 + f] - 1.0) < 1e-11
        # balance rows: V^T M0, V^T Mt, V^T Ms, V^T S_f, V . B_f
        vM0, vMt, vMs = (csr(mats[k]).T @ V for k in range(3))
        vS = [csr(mats[21 + f]).T @ V for f in range(6)]
        nf = O.face_normals(3)
        on = prob.omega @ nf.T                       # [m][6]: Omega . n_f
        kappa = 1.0 / prob.dt
        inflow = sum(prob.w[m] * (-on[m, 0]) * 1.0 * (V @ vecs[4]) for m in range(prob.m) if on[m, 0] < 0)
        Psi_prev = np.zeros((prob.n, prob.m))
        for _ in range(prob.steps):
            tp.step(prob.dt)
            assert tp.stats()["last_residual"] < 1e-11
            Psi = tp.state()                         # [n][m]
            Phi, Phi_prev = Psi @ prob.w, Psi_prev @ prob.w
            val = kappa * vM0 @ (Phi - Phi_prev) + vMt @ Phi - vMs @ Phi - inflow
            for f in range(6):
                wpos = prob.w * np.maximum(on[:, f], 0.0)
                val += vS[f] @ (Psi @ wpos)
            assert abs(val) < 1e-8 * inflow
            Psi_prev = Psi
        phi = tp.scalar_flux(kind=1)
        assert np.all(np.isfinite(phi)) and phi.max() < 4 * math.pi * 1.1


def _functions_per_tet(disc):
    """Largest number of RK functions supported on one tetrahedron (the union
    over its 8 quadrature points, which the oracle lists tetrahedron by
    tetrahedron), from the oracle's own support lists."""
    sptr, sidx, _, _ = O.rk_at_points(disc.x, disc.R, disc.V, disc.rowptr, disc.col, disc.vq.x, disc.vq.owner)
    nq = len(disc.vq.w)
    assert nq % 8 == 0
    return max(len(np.unique(sidx[sptr[q]:sptr[q + 8]])) for q in range(0, nq, 8))


@pytest.fixture(scope="module")
def lattice12():
    """12^3 jittered lattice (1,728 points, 64 of them at least four spacings
    from every face), S4, lognormal sigma_t, inflow on x = 0."""
    prob = _problem(12, seed=3012, steps=2, dt=0.02)
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tr = O.Transport(disc, F, prob.omega, prob.w, psi_b=prob.inflow)
    _, Phi_ref, _ = O.Solver(tr, outer_tol=1e-13).run(np.zeros((tr.M, disc.n)), prob.dt, prob.steps)
    return prob, disc, F, Phi_ref


def test_forms_3d_12_cubed_reach_the_interior_path(lattice12):
    """Every integrated form element by element at 1e-12 of its array's
    magnitude on a lattice whose interior tetrahedra carry the full 3D
    support (the assembly's many-function path)."""
    prob, disc, F, _ = lattice12
    nfun = _functions_per_tet(disc)
    print(f"12^3: largest number of functions on one tetrahedron: {nfun}")
    assert nfun >= 40
    with pkg.TransportProblem.from_problem(prob) as tp:
        tp.integrate().assemble()
        rowptr, col = tp.neighbors()
        assert np.array_equal(rowptr, disc.rowptr) and np.array_equal(col, disc.col)
        V = tp.volumes()
        mats, vecs = tp.forms()
    assert np.abs(V - disc.V).max() <= 1e-13 * disc.V.max()
    d = 3
    ref_m = np.concatenate([F["M0"][None], F["Mt"][None], F["Ms"][None], F["G"], F["Gt"], F["Gs"],
                            F["K"].reshape(d * d, -1), F["S"]])
    ref_v = np.concatenate([F["Q0"][None], F["Q"], F["B"]])
    for k in range(ref_m.shape[0]):
        assert np.abs(mats[k] - ref_m[k]).max() <= 1e-12 * np.abs(ref_m[k]).max(), k
    for k in range(ref_v.shape[0]):
        assert np.abs(vecs[k] - ref_v[k]).max() <= 1e-12 * max(np.abs(ref_v[k]).max(), 1e-300), k


@pytest.mark.parametrize("precision,tol", [(pkg.MLPG_FP64, 1e-9), (pkg.MLPG_MIXED, 1e-8)])
def test_run_3d_12_cubed_matches_oracle(lattice12, precision, tol):
    prob, disc, F, Phi_ref = lattice12
    ref = disc.interpolation_matrix() @ Phi_ref
    with pkg.TransportProblem.from_problem(prob, precision=precision, inner_tol=1e-13, outer_tol=1e-13,
                                           refine_tol=1e-12) as tp:
        tp.integrate().assemble()
        phi = tp.run(prob.dt, prob.steps)
        assert _rel(phi, ref) < tol
        assert _rel(tp.scalar_flux(kind=1), Phi_ref) < tol


def test_refined_run_3d_10_cubed_matches_oracle():
    """Alg. 2 set (levels 0 -> 2 refined within 30 degrees of +x) on a 10^3
    lattice in mixed precision against the oracle."""
    prob = mi.lognormal_3d(10, seed=3010, steps=2, dt=0.02, refine=(0, 2, 30.0))
    ref, _ = _oracle_run(prob)
    with pkg.TransportProblem.from_problem(prob, precision=pkg.MLPG_MIXED, refine_tol=1e-12) as tp:
        tp.integrate().assemble()
        phi = tp.run(prob.dt, prob.steps)
        assert _rel(phi, ref) < 1e-8


def test_rk_order_0_in_3d_forms_and_run():
    """Order-0 RK functions in 3D (Sec. 2.2: the basis P = [1], Shepard
    functions that reproduce constants): every integrated form to 1e-12 of
    its array's magnitude, and a 3-step run in FP64 and mixed precision against
    the oracle at the same order."""
    prob = _problem(6, seed=3006)
    disc = O.Discretization(prob.x, prob.R, prob.lo, prob.hi, rk_order=0)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    d = 3
    ref_m = np.concatenate([F["M0"][None], F["Mt"][None], F["Ms"][None], F["G"], F["Gt"], F["Gs"],
                            F["K"].reshape(d * d, -1), F["S"]])
    ref_v = np.concatenate([F["Q0"][None], F["Q"], F["B"]])
    tr = O.Transport(disc, F, prob.omega, prob.w, psi_b=prob.inflow)
    _, Phi, _ = O.Solver(tr, outer_tol=1e-13).run(np.zeros((tr.M, disc.n)), prob.dt, prob.steps)
    ref = disc.interpolation_matrix() @ Phi
    with pkg.TransportProblem.from_problem(prob, rk_order=0, inner_tol=1e-13, outer_tol=1e-13) as tp:
        tp.integrate().assemble()
        mats, vecs = tp.forms()
        for k in range(ref_m.shape[0]):
            assert np.abs(mats[k] - ref_m[k]).max() <= 1e-12 * np.abs(ref_m[k]).max(), k
        for k in range(ref_v.shape[0]):
            assert np.abs(vecs[k] - ref_v[k]).max() <= 1e-12 * max(np.abs(ref_v[k]).max(), 1e-300), k
        # constants reproduced: sum_j V_j U_j = 1, so V^T M0 1 is the cube's volume
        rowptr, col = tp.neighbors()
        import scipy.sparse as sp
        M0 = sp.csr_matrix((mats[0], col, rowptr), shape=(prob.n, prob.n))
        assert abs(tp.volumes() @ M0 @ np.ones(prob.n) - 1.0) < 1e-12
        assert _rel(tp.run(prob.dt, prob.steps), ref) < 1e-9
    with pkg.TransportProblem.from_problem(prob, rk_order=0, precision=pkg.MLPG_MIXED, refine_tol=1e-12) as tp:
        tp.integrate().assemble()
        assert _rel(tp.run(prob.dt, prob.steps), ref) < 1e-8
