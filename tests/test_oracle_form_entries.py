"""Individual entries of the oracle's integrated forms (Alg. 1, Sec. 4.1) against
an independent integration.

The oracle integrates the forms with its C code: RK functions at the points of
degree-9 rules on the fan triangles of the Voronoi cells.  Here the same
entries are recomputed from the definitions alone:
  * the RK functions (Sec. 2.2) in numpy: W_j the cubic B-spline with support
    R_j = 2 h_j, P_j(x) = [1, x - x_j], M(x) = sum_j V_j W_j P_j P_j^T,
    U_j(x) = W_j P_j(x)^T M(x)^-1 e_1, gradients by central differences;
  * the integral over the box that holds both supports (cut to the domain),
    with a composite 6x6-point Gauss-Legendre rule on a 24 x 24 grid of
    squares, independent of the cells.
Entries: M0[i][j] = V_j int U_i U_j, G^a[i][j] = V_j int d_a U_i U_j,
K^ab[i][j] = V_j int d_a U_i d_b U_j.

The composite rule is converged: it agrees with a 64 x 64 grid to 4e-7 of
each form's largest entry.  The differences are the oracle's own quadrature
error on the piecewise-cubic integrand, measured in units of each form's
largest entry:
  * at most 1.7e-5 for the interior pairs;
  * at most 1.5e-3 at the corner, where the moment matrix is worse
    conditioned and the functions steeper.
The bounds, 1e-4 and 5e-3 of each form's largest entry, still fail every
plausible mistake by orders of magnitude: a flipped sign, a dropped V_j, a
pair taken transposed (the G entry of (j, i) has the opposite sign), or the
x and y derivatives swapped.  The test checks the transposed pair against
them too."""
import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O


def _spline(chi):
    w = np.where(chi < 1.0, 1.0 - 1.5 * chi ** 2 + 0.75 * chi ** 3, 0.25 * (2.0 - chi) ** 3)
    return np.where(chi < 2.0, w, 0.0)


def _rk(pts, x, R, V):
    d = pts[:, None, :] - x[None, :, :]
    r = np.sqrt((d ** 2).sum(-1))
    W = np.where(r < R[None, :], _spline(r / (0.5 * R[None, :])), 0.0)
    P = np.concatenate([np.ones(d.shape[:2] + (1,)), d], axis=-1)
    M = np.einsum("qj,qja,qjb->qab", V[None, :] * W, P, P)
    e1 = np.broadcast_to(np.array([1.0, 0.0, 0.0]), (len(pts), 3))[..., None]
    C = np.linalg.solve(M, e1)[..., 0]
    return W * np.einsum("qja,qa->qj", P, C)


def _rk_and_gradient(pts, x, R, V, dl=1e-6):
    U = _rk(pts, x, R, V)
    grad = []
    for a in range(2):
        e = np.zeros(2)
        e[a] = dl
        grad.append((_rk(pts + e, x, R, V) - _rk(pts - e, x, R, V)) / (2.0 * dl))
    return U, grad


def _gauss_box(lo, hi, cells=24, points=6):
    t, w = np.polynomial.legendre.leggauss(points)
    xs, ws = [], []
    for a in range(2):
        edges = np.linspace(lo[a], hi[a], cells + 1)
        c, hw = 0.5 * (edges[:-1] + edges[1:]), 0.5 * (edges[1:] - edges[:-1])
        xs.append((c[:, None] + hw[:, None] * t[None, :]).ravel())
        ws.append((hw[:, None] * w[None, :]).ravel())
    X, Y = np.meshgrid(xs[0], xs[1], indexing="ij")
    WX, WY = np.meshgrid(ws[0], ws[1], indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], 1), (WX * WY).ravel()


def _entries(i, j, x, R, V):
    """(M0, G^x, G^y, K^xx, K^xy, K^yx, K^yy) of entry (i, j), integrated here."""
    lo = np.maximum(np.maximum(x[i] - R[i], x[j] - R[j]), 0.0)
    hi = np.minimum(np.minimum(x[i] + R[i], x[j] + R[j]), 1.0)
    pts, w = _gauss_box(lo, hi)
    acc = np.zeros(7)
    for k in range(0, len(pts), 4096):
        U, (Ux, Uy) = _rk_and_gradient(pts[k:k + 4096], x, R, V)
        wk = w[k:k + 4096]
        ui, uj = U[:, i], U[:, j]
        acc += [np.dot(wk, ui * uj), np.dot(wk, Ux[:, i] * uj), np.dot(wk, Uy[:, i] * uj),
                np.dot(wk, Ux[:, i] * Ux[:, j]), np.dot(wk, Ux[:, i] * Uy[:, j]),
                np.dot(wk, Uy[:, i] * Ux[:, j]), np.dot(wk, Uy[:, i] * Uy[:, j])]
    return V[j] * acc


@pytest.fixture(scope="module")
def lattice():
    x, h = mi.jittered_lattice(8, 2, 91)
    R = np.full(len(x), 2.0 * h)
    disc = O.Discretization(x, R)
    n = len(x)
    F = disc.assemble_per_point(np.ones(n), np.zeros(n), np.ones(n))
    forms = [F["M0"], F["G"][0], F["G"][1], F["K"][0][0], F["K"][0][1], F["K"][1][0], F["K"][1][1]]
    scale = [np.abs(f).max() for f in forms]
    return x, R, disc, forms, scale


def _pos(disc, i, j):
    row = disc.col[disc.rowptr[i]:disc.rowptr[i + 1]]
    return disc.rowptr[i] + int(np.nonzero(row == j)[0][0])


@pytest.mark.parametrize("which", ["interior diagonal", "interior nearest", "interior second ring", "corner"])
def test_form_entries_match_an_independent_integration(lattice, which):
    x, R, disc, forms, scale = lattice
    if which == "corner":
        i = int(np.argmin((x ** 2).sum(1)))
    else:
        i = int(np.argmin(((x - 0.5) ** 2).sum(1)))
    row = disc.col[disc.rowptr[i]:disc.rowptr[i + 1]]
    dist = np.sqrt(((x[row] - x[i]) ** 2).sum(1))
    order = np.argsort(dist)
    if which == "interior diagonal":
        j = i
    elif which == "interior second ring":   # the first neighbour about two spacings away
        j = int(row[order[np.searchsorted(dist[order], 1.9 * 0.5 * R[i])]])
    else:
        j = int(row[order[1]])
    ref = _entries(i, j, x, R, disc.V)
    p = _pos(disc, i, j)
    got = np.array([f[p] for f in forms])
    tol = (5e-3 if which == "corner" else 1e-4) * np.array(scale)
    assert np.all(np.abs(got - ref) <= tol), (which, got, ref, tol)
    if j != i:
        # the transposed pair, taken by mistake, misses the same integrals by far more
        q = _pos(disc, j, i)
        wrong = np.array([f[q] for f in forms])
        g = 1 if abs(ref[1]) >= abs(ref[2]) else 2   # the larger gradient component
        assert abs(wrong[g] - ref[g]) > 10 * tol[g], (which, wrong, ref)
