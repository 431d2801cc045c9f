"""Pins of the RK correction orders 0 and 2 (Sec. 2.2, Sec. 5.2).

An order-k correction reproduces every polynomial of total degree <= k and its
gradient (the reproducing conditions that define the RK functions), and not
degree k + 1 in general.  The pure absorber psi = exp(-sigma x) converges at
about one order above the RK order (Sec. 5.2: order 0 about 2, order 2 with
six neighbours across a kernel radius between 3 and 4)."""
import itertools
import math

import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O


def _monomials(dim, deg):
    return [e for e in itertools.product(range(deg + 1), repeat=dim) if sum(e) == deg]


def _sums(d, order, pts, owner, expo):
    sptr, sidx, U, dU = O.rk_at_points(d.x, d.R, d.V, d.rowptr, d.col, pts, owner, order)
    rows = np.repeat(np.arange(len(pts)), np.diff(sptr))
    N = U * d.V[sidx]
    dN = dU * d.V[sidx][:, None]
    f = np.prod(d.x[sidx] ** np.asarray(expo), axis=1)
    val = np.bincount(rows, N * f, minlength=len(pts))
    grad = np.stack([np.bincount(rows, dN[:, g] * f, minlength=len(pts)) for g in range(d.dim)], 1)
    return val, grad


def _exact(pts, expo):
    expo = np.asarray(expo)
    val = np.prod(pts ** expo, axis=1)
    grad = []
    for g in range(pts.shape[1]):
        e = expo.copy()
        if e[g] == 0:
            grad.append(np.zeros(len(pts)))
            continue
        c = e[g]
        e[g] -= 1
        grad.append(c * np.prod(pts ** e, axis=1))
    return val, np.stack(grad, 1)


@pytest.mark.parametrize("dim,order,rfac,n", [(2, 0, 2.0, 12), (2, 2, 3.0, 12), (3, 2, 3.0, 5), (3, 0, 2.0, 5)])
def test_reproduces_polynomials_up_to_the_order(dim, order, rfac, n):
    x, h = mi.jittered_lattice(n, dim, 17)
    d = O.Discretization(x, np.full(len(x), rfac * h), rk_order=order)
    step = 5 if dim == 2 else 40
    pts, owner = d.vq.x[::step], d.vq.owner[::step]
    hinv = 1.0 / d.h.min()
    for deg in range(order + 1):
        for e in _monomials(dim, deg):
            val, grad = _sums(d, order, pts, owner, e)
            ev, eg = _exact(pts, e)
            assert np.abs(val - ev).max() < 1e-11, (deg, e)
            assert np.abs(grad - eg).max() < 1e-10 * hinv, (deg, e)
    # one degree higher is not reproduced
    e = _monomials(dim, order + 1)[0]
    val, _ = _sums(d, order, pts, owner, e)
    ev, _ = _exact(pts, e)
    assert np.abs(val - ev).max() > 1e-6


def _absorber(n, order, rfac, sigma=5.0):
    x, h = mi.jittered_lattice(n, 2, 0, jitter=0.0)
    d = O.Discretization(x, np.full(len(x), rfac * h), rk_order=order)
    F = d.assemble_per_point(np.full(d.n, sigma), np.zeros(d.n), np.zeros(d.n))
    tr = O.Transport(d, F, np.array([[1.0, 0.0, 0.0]]), np.array([4 * math.pi]), psi_b={0: 1.0})
    Psi, _, _ = O.Solver(tr).step(np.zeros((1, d.n)), np.inf)
    psi = d.interpolation_matrix() @ Psi[0]
    return np.abs(psi - np.exp(-sigma * x[:, 0])).mean()


@pytest.mark.parametrize("order,rfac,min_slope", [(0, 2.0, 1.8), (2, 3.0, 3.2)])
def test_pure_absorber_order_follows_rk_order(order, rfac, min_slope):
    e = np.array([_absorber(n, order, rfac) for n in (8, 16, 32)])
    slopes = np.log2(e[:-1] / e[1:])
    assert slopes.min() > min_slope, slopes
    if order == 2:   # and more accurate than the linear correction on the same kernels
        assert e[-1] < 0.6 * _absorber(32, 1, rfac)
