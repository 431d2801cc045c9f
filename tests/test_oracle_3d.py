"""Pins of the oracle's 3D discretisation (Sec. 2-4 with polyhedral cells).

  * conical-product tetrahedron rule: exact to degree 2n - 1, not beyond;
  * polyhedral cells: exact lattice cubes without jitter, a partition of the
    box with jitter, equal to scipy's Voronoi cells in the interior, and every
    random point lies in the cell of its nearest generator;
  * quadrature moments of the box and of its faces;
  * linear reproduction of the 3D RK functions;
  * integrated-form identities (as in 2D) with six faces;
  * transport: nested solve == one sparse LU, particle balance of every step,
    the pure-absorber closed form, the infinite-medium recurrence.
"""
import math

import numpy as np
import pytest
from scipy.spatial import ConvexHull, Voronoi

import mlpg_inputs as mi
import oracle.mlpg_oracle as O


def _disc(n, jitter=0.2, seed=31, **kw):
    x, h = mi.jittered_lattice(n, 3, seed, jitter=jitter)
    return O.Discretization(x, np.full(len(x), 2 * h), **kw), h


@pytest.fixture(scope="module")
def d6():
    return _disc(6)[0]


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_tet_rule_exact_to_degree_2n_minus_1(n):
    xi, w = O.tet_rule(n)
    assert abs(w.sum() - 1.0 / 6.0) < 1e-15
    assert np.all(w > 0) and np.all(xi >= 0) and np.all(xi.sum(1) <= 1 + 1e-15)
    deg = 2 * n - 1
    for a in range(deg + 2):
        for b in range(deg + 2 - a):
            for c in range(deg + 2 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b * xi[:, 2] ** c)
                if a + b + c <= deg:
                    assert abs(got - exact) < 1e-15
    k = deg + 1   # first degree that is not integrated exactly
    assert abs(np.sum(w * xi[:, 0] ** k) - math.factorial(k) / math.factorial(k + 3)) > 1e-12


def test_cells_are_lattice_cubes_without_jitter():
    d, h = _disc(5, jitter=0.0)
    assert np.allclose(d.V, h ** 3, rtol=1e-12, atol=0)
    assert np.all(np.diff(d.fptr) == 6)


def test_cells_partition_the_box(d6):
    assert abs(d6.V.sum() - 1.0) < 1e-13
    assert np.all(d6.V > 0)
    # no kernel-extent face survives (the cells are well inside the 2h boxes)
    assert not np.any(d6.labels == -100)


def test_cells_equal_scipy_voronoi_interior():
    d, h = _disc(7, seed=33)
    vor = Voronoi(d.x)
    interior = np.where(np.all((d.x > 2.5 * h) & (d.x < 1 - 2.5 * h), axis=1))[0]
    assert len(interior) > 0
    for i in interior:
        reg = vor.regions[vor.point_region[i]]
        assert -1 not in reg
        vol = ConvexHull(vor.vertices[reg]).volume
        assert abs(vol - d.V[i]) < 1e-13


def test_random_points_lie_in_the_cell_of_their_nearest_generator(d6):
    rng = np.random.default_rng(5)
    y = rng.uniform(0, 1, (400, 3))
    near = np.argmin(((y[:, None, :] - d6.x[None, :, :]) ** 2).sum(-1), axis=1)
    for p, i in zip(y, near):
        for f in range(d6.fptr[i], d6.fptr[i + 1]):
            P = d6.verts[d6.vptr[f]:d6.vptr[f + 1]]
            nrm = np.zeros(3)   # Newell normal (outward for counter-clockwise faces)
            for k in range(len(P)):
                a, b = P[k], P[(k + 1) % len(P)]
                nrm += np.cross(a, b)
            assert (p - P[0]) @ nrm <= 1e-12 * np.linalg.norm(nrm)


def test_box_and_face_moments(d6):
    x, w = d6.vq.x, d6.vq.w
    assert abs(w.sum() - 1.0) < 1e-13
    assert np.allclose(np.bincount(d6.vq.owner, w, minlength=d6.n), d6.V, rtol=1e-12, atol=0)
    for a in range(3):
        assert abs(w @ x[:, a] - 0.5) < 1e-13
        assert abs(w @ x[:, a] ** 2 - 1.0 / 3.0) < 1e-13
    assert abs(w @ (x[:, 0] * x[:, 1] * x[:, 2]) - 0.125) < 1e-13
    assert abs(w @ (x[:, 0] ** 2 * x[:, 1]) - 1.0 / 6.0) < 1e-13
    for f in range(6):
        on = d6.bq.face == f
        xb, wb = d6.bq.x[on], d6.bq.w[on]
        a = f // 2
        assert np.allclose(xb[:, a], float(f % 2), atol=1e-15)
        assert abs(wb.sum() - 1.0) < 1e-13
        b, c = [e for e in range(3) if e != a]
        assert abs(wb @ xb[:, b] - 0.5) < 1e-13
        assert abs(wb @ (xb[:, b] * xb[:, c]) - 0.25) < 1e-13
        assert abs(wb @ xb[:, c] ** 2 - 1.0 / 3.0) < 1e-13


def test_rk_linear_reproduction_3d(d6):
    pts, owner = d6.vq.x[::7], d6.vq.owner[::7]
    sptr, sidx, U, dU = O.rk_at_points(d6.x, d6.R, d6.V, d6.rowptr, d6.col, pts, owner)
    rows = np.repeat(np.arange(len(pts)), np.diff(sptr))
    N = U * d6.V[sidx]
    dN = dU * d6.V[sidx][:, None]
    assert np.abs(np.bincount(rows, N, minlength=len(pts)) - 1).max() < 1e-12
    hinv = 1.0 / d6.h.min()
    for b in range(3):
        s1 = np.bincount(rows, N * d6.x[sidx, b], minlength=len(pts))
        assert np.abs(s1 - pts[:, b]).max() < 1e-12
        for g in range(3):
            g1 = np.bincount(rows, dN[:, g] * d6.x[sidx, b], minlength=len(pts))
            assert np.abs(g1 - (g == b)).max() < 1e-11 * hinv
        assert np.abs(np.bincount(rows, dN[:, b], minlength=len(pts))).max() < 1e-11 * hinv


@pytest.fixture(scope="module")
def forms3():
    d, _ = _disc(5, seed=35)
    rng = np.random.default_rng(2)
    st = rng.uniform(0.5, 3.0, d.n)
    ss = st * rng.uniform(0.1, 0.9, d.n)
    q = rng.uniform(0.0, 2.0, d.n)
    return d, d.assemble_per_point(st, ss, q), st, ss, q


def test_form_identities_3d(forms3):
    d, F, st, ss, q = forms3
    one = np.ones(d.n)
    M0 = d.csr(F["M0"])
    assert abs(d.V @ M0 @ one - 1.0) < 1e-13
    for a in range(3):
        assert abs(d.V @ M0 @ d.x[:, a] - 0.5) < 1e-13
        assert np.abs(d.V @ d.csr(F["G"][a])).max() < 1e-12
        assert abs(d.V @ d.csr(F["Gt"][a]) @ one) < 1e-11
        assert abs(d.V @ F["Q"][a]) < 1e-11
        for b in range(3):
            K = d.csr(F["K"][a, b])
            assert np.abs(K @ one).max() < 1e-9 * np.abs(F["K"]).max()
            for c in range(3):
                rhs = (c == b) * (d.csr(F["G"][a]) @ one)
                lhs = K @ d.x[:, c]
                assert np.allclose(lhs, rhs, atol=1e-9 * np.abs(lhs).max() + 1e-12)
    A = M0.multiply(d.V[:, None]).toarray()
    assert np.abs(A - A.T).max() < 1e-12
    assert abs(d.V @ d.csr(F["Mt"]) @ one - d.V @ st) < 1e-12
    assert abs(d.V @ d.csr(F["Ms"]) @ one - d.V @ ss) < 1e-12
    assert abs(d.V @ F["Q0"] - d.V @ q) < 1e-12
    for f in range(6):
        assert abs(d.V @ d.csr(F["S"][f]) @ one - 1.0) < 1e-13     # face area
        assert abs(d.V @ F["B"][f] - 1.0) < 1e-13


def _tr3(n=5, sn=4, seed=3100, **kw):
    p = mi.make_problem("3d-test", n, 3, sn, seed, 1.0, 0.6, 1.0, 0.02, 3, **kw)
    d = O.Discretization(p.x, p.R, p.lo, p.hi)
    F = d.assemble_per_point(p.sigma_t, p.sigma_s, p.q)
    return p, d, F, O.Transport(d, F, p.omega, p.w, psi_b=p.inflow)


def test_nested_equals_direct_3d():
    p, d, F, tr = _tr3()
    assert tr.M == 24
    s = O.Solver(tr, outer_tol=1e-14)
    Psi0 = np.random.default_rng(0).uniform(0, 1, (tr.M, d.n))
    Psi, Phi, st = s.step(Psi0, p.dt)
    Psi2, Phi2 = s.step_direct(Psi0, p.dt)
    assert np.linalg.norm(Phi - Phi2) / np.linalg.norm(Phi2) < 1e-11
    assert np.linalg.norm(Psi - Psi2) / np.linalg.norm(Psi2) < 1e-11


def test_particle_balance_every_step_3d():
    p, d, F, tr = _tr3()
    tr.psi_b = {0: 0.7, 5: 0.2}
    s = O.Solver(tr, outer_tol=1e-14)
    V, kappa = d.V, 1.0 / p.dt
    Psi = np.zeros((tr.M, d.n))
    scale = 4 * math.pi * (V @ F["Q0"])
    for _ in range(2):
        new, _, _ = s.step(Psi, p.dt)
        Phi, Phi_prev = tr.D(new), tr.D(Psi)
        val = kappa * V @ (d.csr(F["M0"]) @ (Phi - Phi_prev))
        val += V @ (d.csr(F["Mt"]) @ Phi) - V @ (d.csr(F["Ms"]) @ Phi) - 4 * math.pi * V @ F["Q0"]
        for m in range(tr.M):
            for f in range(6):
                on = float(tr.omega[m] @ tr.nf[f])
                if on > 0:
                    val += tr.w[m] * on * (V @ (d.csr(F["S"][f]) @ new[m]))
                elif on < 0 and f in tr.psi_b:
                    val -= tr.w[m] * (-on) * tr.psi_b[f] * (V @ F["B"][f])
        assert abs(val) < 1e-11 * scale
        Psi = new


def test_pure_absorber_closed_form_3d():
    # psi = exp(-sigma x) for the direction +x with unit inflow on x = 0 (the 3D
    # form of Sec. 5.2); coarse lattices, so a bound rather than an order
    sigma = 3.0
    x, h = mi.jittered_lattice(8, 3, 0, jitter=0.0)
    d = O.Discretization(x, np.full(len(x), 2 * h))
    F = d.assemble_per_point(np.full(d.n, sigma), np.zeros(d.n), np.zeros(d.n))
    tr = O.Transport(d, F, np.array([[1.0, 0.0, 0.0]]), np.array([4 * math.pi]), psi_b={0: 1.0})
    Psi, _, _ = O.Solver(tr).step(np.zeros((1, d.n)), np.inf)
    psi = d.interpolation_matrix() @ Psi[0]
    err = np.abs(psi - np.exp(-sigma * x[:, 0]))
    assert err.mean() < 1e-2 and err.max() < 6e-2


@pytest.mark.parametrize("nref", [2, 3])
def test_infinite_medium_recurrence_3d(nref):
    # uniform material and inflow at the 0D backward-Euler value on all six
    # faces: the flux follows the 0D recurrence up to the divergence-theorem
    # defect of the quadrature, which shrinks with the rule's degree
    p = mi.make_problem("3d-test", 6, 3, 4, 3100, 1.0, 0.6, 1.0, 0.02, 3)
    d = O.Discretization(p.x, p.R, p.lo, p.hi, nref_tet=nref, nref_face=nref)
    F = d.assemble_per_point(p.sigma_t, p.sigma_s, p.q)
    tr = O.Transport(d, F, p.omega, p.w)
    nf = O.face_normals(3)
    defect = max(np.abs(d.csr(F["G"][a]) @ np.ones(d.n) - sum(nf[f, a] * F["B"][f] for f in range(6))).max()
                 / np.abs(d.csr(F["G"][a]) @ np.ones(d.n)).max() for a in range(3))
    s = O.Solver(tr, outer_tol=1e-14)
    sa, kap, ph = 0.4, 1.0 / p.dt, 2.0
    Psi = np.full((tr.M, d.n), ph / (4 * math.pi))
    Phi = tr.D(Psi)
    I = d.interpolation_matrix()
    for _ in range(2):
        ph = (kap * ph + 4 * math.pi * 1.0) / (kap + sa)      # 0D backward Euler
        tr.psi_b = {f: ph / (4 * math.pi) for f in range(6)}
        tr._kappa = None
        Psi, Phi, _ = s.step(Psi, p.dt, Phi_guess=Phi)
        assert np.abs(I @ Phi - ph).max() / ph < defect
    assert defect < (2.5e-2 if nref == 2 else 5e-3)


def test_manufactured_solution_converges_3d():
    # the sinusoidal manufactured solution of Sec. 5.1 in 3D (steady, S4, regular
    # lattices on [-1, 1]^3): at least second order in space (measured about 3)
    from oracle import mms
    om, w = mi.level_symmetric(4, 3)
    errs = []
    for n in (4, 6, 8):
        x, h = mi.jittered_lattice(n, 3, 5, lo=-1, hi=1, jitter=0.0)
        errs.append(mms.mms_run(mms.Sinusoidal(), x, np.full(len(x), 2 * h), om, w))
    errs = np.array(errs)
    hs = 2.0 / np.array([4, 6, 8])
    slopes = np.log(errs[:-1] / errs[1:]) / np.log(hs[:-1] / hs[1:])
    assert slopes.min() > 2.0, slopes
    assert errs[-1] < 5e-3
