"""Pins of the oracle's integrated forms (Alg. 1, forms of Sec. 4.1).

Exact identities that follow from sum_j N_j = 1 (Sec. 2.2) and from the
symmetry of the volume integrals: they catch dropped terms, transposed operands
and wrong weights in the integration loop."""
import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O


@pytest.fixture(scope="module")
def setup():
    x, h = mi.jittered_lattice(14, 2, 21)
    d = O.Discretization(x, np.full(len(x), 2 * h))
    rng = np.random.default_rng(1)
    st = rng.uniform(0.5, 3.0, d.n)
    ss = st * rng.uniform(0.1, 0.9, d.n)
    q = rng.uniform(0.0, 2.0, d.n)
    F = d.assemble_per_point(st, ss, q)
    return d, F, st, ss, q


def test_mass_identities(setup):
    d, F, *_ = setup
    M0 = d.csr(F["M0"])
    one = np.ones(d.n)
    # sum_ij V_i M0_ij = |domain|;  sum_ij V_i M0_ij x_j^a = int x^a
    assert abs(d.V @ M0 @ one - 1.0) < 1e-13
    assert abs(d.V @ M0 @ d.x[:, 0] - 0.5) < 1e-13
    assert abs(d.V @ M0 @ (d.x[:, 0] * 0 + d.x[:, 1]) - 0.5) < 1e-13
    # symmetric with the V_i row weight: V_i M0_ij = V_j M0_ji
    A = (M0.multiply(d.V[:, None])).toarray()
    assert np.abs(A - A.T).max() < 1e-15 * 1e3
    # row sums: sum_j M0_ij = <U_i, 1>;  sum_i V_i <U_i,1> = 1
    assert abs(d.V @ (M0 @ one) - 1.0) < 1e-13


def test_gradient_identities(setup):
    d, F, *_ = setup
    for a in range(2):
        G = d.csr(F["G"][a])
        # sum_i V_i dU_i = d(sum N_i) = 0  ->  V^T G^a = 0
        assert np.abs(d.V @ G).max() < 1e-12
        # sum_j G_ij x_j^b = <d_a U_i, x^b>;  V-weighted: int d_a(sum N_i) x^b = 0
        for b in range(2):
            K = d.csr(F["K"][a, b])
            assert np.abs(K @ np.ones(d.n)).max() < 1e-9 * np.abs(F["K"]).max()  # grad of constant
            # sum_j K^ab_ij x_j^c = <d_a U_i, delta_bc>  -> compare with G^a row sums
            for c in range(2):
                lhs = K @ d.x[:, c]
                rhs = (c == b) * (d.csr(F["G"][a]) @ np.ones(d.n)) / 1.0
                # <d_a U_i, 1> equals row sum of G^a
                assert np.allclose(lhs, rhs, atol=1e-9 * np.abs(lhs).max() + 1e-12)


def test_material_forms(setup):
    d, F, st, ss, q = setup
    # constant over each cell: sum_i V_i Mt_ij 1 = int sigma_t = sum_i V_i sigma_t_i
    one = np.ones(d.n)
    assert abs(d.V @ d.csr(F["Mt"]) @ one - d.V @ st) < 1e-12
    assert abs(d.V @ d.csr(F["Ms"]) @ one - d.V @ ss) < 1e-12
    assert abs(d.V @ F["Q0"] - d.V @ q) < 1e-12
    # V^T Gt^a 1 = int d_a (sum V_i U_i) sigma_t = 0
    for a in range(2):
        assert abs(d.V @ d.csr(F["Gt"][a]) @ one) < 1e-11
        assert abs(d.V @ F["Q"][a]) < 1e-11


def test_surface_forms(setup):
    d, F, *_ = setup
    one = np.ones(d.n)
    for f in range(4):
        S = d.csr(F["S"][f])
        assert abs(d.V @ S @ one - 1.0) < 1e-13        # face length
        assert abs(d.V @ F["B"][f] - 1.0) < 1e-13
        A = (S.multiply(d.V[:, None])).toarray()
        assert np.abs(A - A.T).max() < 1e-12
        # rows touching the face only
        rows = np.unique(np.repeat(np.arange(d.n), np.diff(d.rowptr))[F["S"][f] != 0])
        far = np.abs(d.x[rows, f // 2] - float(f % 2)) < 2 * d.R[rows] + 1e-12
        assert far.all()


def test_divergence_theorem_up_to_quadrature(setup):
    # <d_a U_i, 1> = sum_f (U_i, n_f^a)_f  (integration by parts, Sec. 3.3);
    # U_i is not polynomial, so this holds to the quadrature error only.
    d, F, *_ = setup
    nf = O.face_normals(2)
    for a in range(2):
        lhs = d.csr(F["G"][a]) @ np.ones(d.n)
        rhs = sum(nf[f, a] * F["B"][f] for f in range(4))
        assert np.abs(lhs - rhs).max() < 2e-3 * np.abs(lhs).max()
