"""Plain FP64 CPU oracle for the MLPG / RK / Voronoi discrete-ordinates solve.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  It shares no
code with the CUDA library (``paper_2008_02205_gb300``) and never imports it.

Paper: Bassett & Owen, "Meshless discretization of the discrete-ordinates
transport equation with integration based on Voronoi cells", arXiv 2008.02205.

Split of work:
  * ``c/mlpg_oracle.c`` (loaded with ctypes): reference rules, overlap
    connectivity, Voronoi-like cells, quadrature points, RK functions and the
    integration of every bilinear / linear form (Sec. 2-3, Alg. 1, App. A).
  * this file: the transport operators of Sec. 4.2, the first-flight solve,
    the unpreconditioned GMRES on the scalar flux (Eq. krylov-operator), the
    angular recovery solve, backward-Euler time stepping (Sec. 4.1), the
    point-value recovery phi_i = sum_j V_j U_j(x_i) Phi_j (Eq. flux-expansion)
    and the manufactured sources of Sec. 5.1 (``mms.py``).
  * ``asteroid.py``: the analytic line-source solution of App. B.

Inner inverses L_m^{-1} are exact sparse LU solves (a linear solve has a plain
definition; the paper's GMRES + ILUT reaches the same result up to its
tolerance).  ``inner="ilut-gmres"`` runs the paper's own inner scheme instead
(restarted GMRES, right preconditioned by an incomplete LU with threshold) to
report iteration counts.  The outer scattering solve is the paper's
unpreconditioned GMRES; ``precond="dsa"`` right-preconditions it with a
diffusion correction built from the same forms (not in the paper, which names
diffusion acceleration as future work), or source iteration replaces it.
``step_direct`` solves the coupled step system
(L - MS D) Psi = T Psi^{n-1} + r with one sparse LU and pins the nested scheme.

Individual values of the SUPG forms have no closed form.  Besides the
identities and the manufactured-solution convergence orders in
tests/test_oracle_*.py, single 2D entries (mass, gradient and stiffness forms;
interior and corner, diagonal and off-diagonal) are checked against an
independent numpy evaluation of the RK functions, integrated by a converged
composite Gauss rule, to the rules' quadrature error
(tests/test_oracle_form_entries.py).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "mlpg_oracle.c")
_SO = os.path.join(_HERE, "c", "liboracle.so")
FOUR_PI = 4.0 * math.pi

# ---------------------------------------------------------------------------
# C library
# ---------------------------------------------------------------------------
_lib = None


def build(force: bool = False) -> str:
    """Compile the C half of the oracle (gcc, plain -O2, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _SO, _SRC, "-lm"])
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.orc_gauss_jacobi.argtypes = [i32, dbl, dbl, P, P]
        L.orc_triangle_rule.argtypes = [i32, P, P]
        L.orc_line_rule.argtypes = [i32, P, P]
        L.orc_neighbors.argtypes = [i32, i64, P, P, P, P]
        L.orc_neighbors.restype = i64
        L.orc_cells_2d.argtypes = [i64, P, P, P, P, P, P, P, P, P, P]
        L.orc_cells_2d.restype = i64
        L.orc_volume_qps_2d.argtypes = [i64, P, P, P, i32, P, P, P]
        L.orc_volume_qps_2d.restype = i64
        L.orc_boundary_qps_2d.argtypes = [i64, P, P, P, i32, P, P, P, P]
        L.orc_boundary_qps_2d.restype = i64
        L.orc_rk_at_points.argtypes = [i32, i32, i64, P, P, P, P, P, i64, P, P, P, P, P, P]
        L.orc_rk_at_points.restype = i64
        L.orc_n_mats.argtypes = [i32]
        L.orc_n_vecs.argtypes = [i32]
        L.orc_tet_rule.argtypes = [i32, P, P]
        L.orc_cells_3d.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_cells_3d.restype = i64
        L.orc_volume_qps_3d.argtypes = [i64, P, P, P, P, i32, P, P, P]
        L.orc_volume_qps_3d.restype = i64
        L.orc_boundary_qps_3d.argtypes = [i64, P, P, P, P, i32, P, P, P, P]
        L.orc_boundary_qps_3d.restype = i64
        L.orc_assemble.argtypes = [i32, i32, i64, P, P, P, P, P, i64, P, P, P, P, P, P, i64, P, P, P, P, P, P]
        L.orc_assemble.restype = i32
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# reference rules (App. A)
# ---------------------------------------------------------------------------
def gauss_jacobi(n, a, b):
    t = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss_jacobi(n, a, b, _p(t), _p(w)):
        raise ValueError("bad rule size")
    return t, w


def triangle_rule(n):
    xi = np.zeros((n * n, 2))
    w = np.zeros(n * n)
    lib().orc_triangle_rule(n, _p(xi), _p(w))
    return xi, w


def tet_rule(n):
    xi = np.zeros((n ** 3, 3))
    w = np.zeros(n ** 3)
    if lib().orc_tet_rule(n, _p(xi), _p(w)):
        raise ValueError("bad rule size")
    return xi, w


# ---------------------------------------------------------------------------
# geometry, RK, integration (C)
# ---------------------------------------------------------------------------
def neighbors(x, R):
    """Overlap connectivity (Sec. 3.4): CSR rows sorted by column, diagonal kept."""
    x = _c(x, np.float64)
    R = _c(R, np.float64)
    n, dim = x.shape
    rowptr = np.zeros(n + 1, np.int64)
    nnz = lib().orc_neighbors(dim, n, _p(x), _p(R), _p(rowptr), None)
    col = np.zeros(nnz, np.int32)
    lib().orc_neighbors(dim, n, _p(x), _p(R), _p(rowptr), _p(col))
    return rowptr, col


def cells_2d(x, R, lo, hi, rowptr, col):
    """Voronoi-like cells (Sec. 3.1).  Returns cptr, verts[nv,2], labels, V."""
    x = _c(x, np.float64)
    n = x.shape[0]
    lo = _c(lo[:2], np.float64)
    hi = _c(hi[:2], np.float64)
    cptr = np.zeros(n + 1, np.int64)
    vol = np.zeros(n)
    L = lib()
    nv = L.orc_cells_2d(n, _p(x), _p(R), _p(lo), _p(hi), _p(rowptr), _p(col), _p(cptr), None, None, _p(vol))
    verts = np.zeros((nv, 2))
    labels = np.zeros(nv, np.int32)
    L.orc_cells_2d(n, _p(x), _p(R), _p(lo), _p(hi), _p(rowptr), _p(col), _p(cptr), _p(verts), _p(labels), _p(vol))
    return cptr, verts, labels, vol


@dataclass
class QP:
    x: np.ndarray
    w: np.ndarray
    owner: np.ndarray
    face: np.ndarray | None = None


def volume_qps_2d(x, cptr, verts, nref=5):
    n = x.shape[0]
    L = lib()
    c = L.orc_volume_qps_2d(n, _p(x), _p(cptr), _p(verts), nref, None, None, None)
    xq = np.zeros((c, 2))
    wq = np.zeros(c)
    ow = np.zeros(c, np.int32)
    L.orc_volume_qps_2d(n, _p(x), _p(cptr), _p(verts), nref, _p(xq), _p(wq), _p(ow))
    return QP(xq, wq, ow)


def boundary_qps_2d(n, cptr, verts, labels, nref=5):
    L = lib()
    c = L.orc_boundary_qps_2d(n, _p(cptr), _p(verts), _p(labels), nref, None, None, None, None)
    xb = np.zeros((c, 2))
    wb = np.zeros(c)
    fc = np.zeros(c, np.int32)
    ow = np.zeros(c, np.int32)
    L.orc_boundary_qps_2d(n, _p(cptr), _p(verts), _p(labels), nref, _p(xb), _p(wb), _p(fc), _p(ow))
    return QP(xb, wb, ow, fc)


def cells_3d(x, R, lo, hi, rowptr, col):
    """Polyhedral Voronoi-like cells (Sec. 3.1).  Returns fptr (faces of each
    cell), vptr (vertices of each face), verts[nv, 3], labels (per face), V."""
    x = _c(x, np.float64)
    n = x.shape[0]
    lo = _c(lo[:3], np.float64)
    hi = _c(hi[:3], np.float64)
    fptr = np.zeros(n + 1, np.int64)
    vol = np.zeros(n)
    nf = ctypes.c_int64(0)
    L = lib()
    args = (n, _p(x), _p(R), _p(lo), _p(hi), _p(rowptr), _p(col), _p(fptr))
    nv = L.orc_cells_3d(*args, None, None, None, _p(vol), ctypes.byref(nf))
    if nv < 0:
        raise RuntimeError(f"3D cells failed (code {nv})")
    vptr = np.zeros(nf.value + 1, np.int64)
    verts = np.zeros((nv, 3))
    labels = np.zeros(nf.value, np.int32)
    L.orc_cells_3d(*args, _p(vptr), _p(verts), _p(labels), _p(vol), ctypes.byref(nf))
    return fptr, vptr, verts, labels, vol


def volume_qps_3d(x, fptr, vptr, verts, nref=2):
    n = x.shape[0]
    L = lib()
    c = L.orc_volume_qps_3d(n, _p(x), _p(fptr), _p(vptr), _p(verts), nref, None, None, None)
    xq = np.zeros((c, 3))
    wq = np.zeros(c)
    ow = np.zeros(c, np.int32)
    L.orc_volume_qps_3d(n, _p(x), _p(fptr), _p(vptr), _p(verts), nref, _p(xq), _p(wq), _p(ow))
    return QP(xq, wq, ow)


def boundary_qps_3d(n, fptr, vptr, verts, labels, nref=2):
    L = lib()
    c = L.orc_boundary_qps_3d(n, _p(fptr), _p(vptr), _p(verts), _p(labels), nref, None, None, None, None)
    xb = np.zeros((c, 3))
    wb = np.zeros(c)
    fc = np.zeros(c, np.int32)
    ow = np.zeros(c, np.int32)
    L.orc_boundary_qps_3d(n, _p(fptr), _p(vptr), _p(verts), _p(labels), nref, _p(xb), _p(wb), _p(fc), _p(ow))
    return QP(xb, wb, ow, fc)


def rk_at_points(x, R, V, rowptr, col, pts, owner, order=1):
    """RK functions U_j and gradients at arbitrary points (Sec. 2.2).

    Candidates for point p: the overlap row of owner[p].  Returns (sptr, sidx,
    U, dU[:, dim])."""
    x = _c(x, np.float64)
    n, dim = x.shape
    pts = _c(pts, np.float64)
    owner = _c(owner, np.int32)
    npts = pts.shape[0]
    sptr = np.zeros(npts + 1, np.int64)
    L = lib()
    tot = L.orc_rk_at_points(dim, order, n, _p(x), _p(R), _p(V), _p(rowptr), _p(col), npts, _p(pts), _p(owner),
                             _p(sptr), None, None, None)
    if tot < 0:
        raise FloatingPointError(f"RK moment matrix singular (code {tot})")
    sidx = np.zeros(tot, np.int32)
    U = np.zeros(tot)
    dU = np.zeros((tot, dim))
    L.orc_rk_at_points(dim, order, n, _p(x), _p(R), _p(V), _p(rowptr), _p(col), npts, _p(pts), _p(owner),
                       _p(sptr), _p(sidx), _p(U), _p(dU))
    return sptr, sidx, U, dU


def face_normals(dim):
    """Outward normals of the box faces (Sec. 4.1 boundary terms), order -x, +x, -y, +y (, -z, +z)."""
    nf = np.zeros((2 * dim, 3))
    for a in range(dim):
        nf[2 * a, a] = -1.0
        nf[2 * a + 1, a] = 1.0
    return nf


class Discretization:
    """Everything of Sec. 2-3 for one point set: connectivity, cells, volumes,
    quadrature points and the integrated forms of Sec. 4.1."""

    def __init__(self, x, R, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), nref_tri=5, nref_line=5,
                 nref_tet=2, nref_face=2, rk_order=1):
        """2D: 5x5 conical-product triangles (degree 9) and 5-point Gauss-Legendre
        edges.  3D: 2x2x2 conical-product tetrahedra and 2x2 boundary triangles,
        degree 3 like the paper's 8-point third-order rule (Sec. 5)."""
        self.x = _c(x, np.float64)
        self.R = _c(R, np.float64)
        self.n, self.dim = self.x.shape
        if self.dim not in (2, 3):
            raise NotImplementedError("oracle cells are 2D or 3D")
        self.lo = np.asarray(lo, np.float64)
        self.hi = np.asarray(hi, np.float64)
        self.h = 0.5 * self.R                       # smoothing length
        self.rk_order = int(rk_order)               # RK correction order 0, 1 or 2 (Sec. 2.2)
        self.rowptr, self.col = neighbors(self.x, self.R)
        if self.dim == 2:
            self.cptr, self.verts, self.labels, self.V = cells_2d(
                self.x, self.R, self.lo, self.hi, self.rowptr, self.col)
            self.vq = volume_qps_2d(self.x, self.cptr, self.verts, nref_tri)
            self.bq = boundary_qps_2d(self.n, self.cptr, self.verts, self.labels, nref_line)
        else:
            self.fptr, self.vptr, self.verts, self.labels, self.V = cells_3d(
                self.x, self.R, self.lo, self.hi, self.rowptr, self.col)
            self.vq = volume_qps_3d(self.x, self.fptr, self.vptr, self.verts, nref_tet)
            self.bq = boundary_qps_3d(self.n, self.fptr, self.vptr, self.verts, self.labels, nref_face)
        self.nnz = int(self.rowptr[-1])

    # -- integration (Alg. 1) ---------------------------------------------
    def assemble(self, sigma_t_q, sigma_s_q, q_q):
        """Integrate all forms (Alg. 1, Sec. 4.1) with material values given per volume qp."""
        d, n, nnz = self.dim, self.n, self.nnz
        L = lib()
        nm, nv = L.orc_n_mats(d), L.orc_n_vecs(d)
        mats = np.zeros((nm, nnz))
        vecs = np.zeros((nv, n))
        st, ss, qq = (_c(a, np.float64) for a in (sigma_t_q, sigma_s_q, q_q))
        rc = L.orc_assemble(d, self.rk_order, n, _p(self.x), _p(self.R), _p(self.V), _p(self.rowptr), _p(self.col),
                               len(self.vq.w), _p(self.vq.x), _p(self.vq.w), _p(self.vq.owner),
                               _p(st), _p(ss), _p(qq),
                               len(self.bq.w), _p(self.bq.x), _p(self.bq.w), _p(self.bq.face), _p(self.bq.owner),
                               _p(mats), _p(vecs))
        if rc != 0:
            raise FloatingPointError(f"assembly failed (code {rc})")
        k = 0
        F = {}
        F["M0"], F["Mt"], F["Ms"] = mats[0], mats[1], mats[2]
        k = 3
        F["G"] = mats[k:k + d]; k += d
        F["Gt"] = mats[k:k + d]; k += d
        F["Gs"] = mats[k:k + d]; k += d
        F["K"] = mats[k:k + d * d].reshape(d, d, nnz); k += d * d
        F["S"] = mats[k:k + 2 * d]
        F["Q0"] = vecs[0]
        F["Q"] = vecs[1:1 + d]
        F["B"] = vecs[1 + d:1 + 3 * d]
        return F

    def assemble_per_point(self, sigma_t, sigma_s, q):
        """Alg. 1 with materials constant over each point's cell (value of the owner point)."""
        o = self.vq.owner
        return self.assemble(np.asarray(sigma_t)[o], np.asarray(sigma_s)[o], np.asarray(q)[o])

    def csr(self, vals):
        return sp.csr_matrix((vals, self.col, self.rowptr), shape=(self.n, self.n))

    def interpolation_matrix(self):
        """phi_i = sum_j V_j U_j(x_i) Phi_j  (Eq. flux-expansion at the centres)."""
        sptr, sidx, U, _ = rk_at_points(self.x, self.R, self.V, self.rowptr, self.col, self.x,
                                        np.arange(self.n, dtype=np.int32), self.rk_order)
        return sp.csr_matrix((U * self.V[sidx], sidx, sptr), shape=(self.n, self.n))


# ---------------------------------------------------------------------------
# transport operators (Sec. 4.2)
# ---------------------------------------------------------------------------
class Transport:
    """Operators L, T, MS, D and r of Sec. 4.2 for one angular set.

    tau_i = tau_factor * h_i (Sec. 4.1: tau about one point spacing).
    psi_b: dict face -> isotropic incoming angular flux (vacuum if absent), or
    a callable boundary(m) -> vector r_b (n) for direction m.
    """

    def __init__(self, disc: Discretization, forms, omega, w, c=1.0, tau_factor=1.0, psi_b=None):
        self.d = disc
        self.F = forms
        self.omega = np.asarray(omega, np.float64)
        self.w = np.asarray(w, np.float64)
        self.M = self.omega.shape[0]
        self.c = c
        self.tau = tau_factor * disc.h
        self.psi_b = psi_b or {}
        self.nf = face_normals(disc.dim)
        self._lu = None
        self._kappa = None

    # operator pieces ------------------------------------------------------
    def L_matrix(self, m, kappa):
        d, F, Om = self.d.dim, self.F, self.omega[m]
        T = sp.diags(self.tau)
        A = kappa * self.d.csr(F["M0"]) + self.d.csr(F["Mt"])
        adv = sum(Om[a] * self.d.csr(F["G"][a]) for a in range(d))
        A = A - adv
        tg = sum(Om[a] * (kappa * self.d.csr(F["G"][a]) + self.d.csr(F["Gt"][a])) for a in range(d))
        kk = sum(Om[a] * Om[b] * self.d.csr(F["K"][a, b]) for a in range(d) for b in range(d))
        A = A + T @ (tg + kk)
        for f in range(2 * d):
            on = float(Om[:d] @ self.nf[f, :d])
            if on > 0.0:
                A = A + on * self.d.csr(F["S"][f])
        return A.tocsr()

    def T_matrix(self, m, kappa):
        d, F, Om = self.d.dim, self.F, self.omega[m]
        T = sp.diags(self.tau)
        A = self.d.csr(F["M0"]) + T @ sum(Om[a] * self.d.csr(F["G"][a]) for a in range(d))
        return (kappa * A).tocsr()

    def MS_matrix(self, m):
        d, F, Om = self.d.dim, self.F, self.omega[m]
        T = sp.diags(self.tau)
        A = self.d.csr(F["Ms"]) + T @ sum(Om[a] * self.d.csr(F["Gs"][a]) for a in range(d))
        return (A / FOUR_PI).tocsr()

    def r_vector(self, m):
        d, F, Om = self.d.dim, self.F, self.omega[m]
        r = F["Q0"] + self.tau * sum(Om[a] * F["Q"][a] for a in range(d))
        if callable(self.psi_b):
            return r + self.psi_b(m)
        for f, pb in self.psi_b.items():
            on = float(Om[:d] @ self.nf[f, :d])
            if on < 0.0:
                r = r + abs(on) * pb * F["B"][f]
        return r

    # factorisations of L_m, once per dt (Sec. 4.2: factored per step, reused)
    def factor(self, kappa):
        if self._kappa != kappa:
            self._lu = [spla.splu(self.L_matrix(m, kappa).tocsc()) for m in range(self.M)]
            self._L = [self.L_matrix(m, kappa) for m in range(self.M)]
            self._T = [self.T_matrix(m, kappa) for m in range(self.M)]
            self._MS = [self.MS_matrix(m) for m in range(self.M)]
            self._r = [self.r_vector(m) for m in range(self.M)]
            self._kappa = kappa

    def Linv(self, rhs):
        """L^{-1}, block-diagonal in angle (Sec. 4.2); rhs[M, n]."""
        return np.stack([self._lu[m].solve(rhs[m]) for m in range(self.M)])

    def D(self, Psi):
        return self.w @ Psi

    # low-order diffusion operator for the DSA-like preconditioner ----------
    def sigma_t_rows(self):
        """Test-function average of sigma_t per row: (Mt 1)_i / (M0 1)_i =
        int sigma_t v_i / int v_i (the trial functions sum to one)."""
        one = np.ones(self.d.n)
        return (self.d.csr(self.F["Mt"]) @ one) / (self.d.csr(self.F["M0"]) @ one)

    def diffusion_matrix(self, kappa):
        """Galerkin P1-diffusion operator on the same pattern, from the forms
        already integrated (the paper names diffusion acceleration as future
        work, Sec. 6, without deriving one):
            C = diag(1 / (3 sigma_t_i)) sum_a K_aa + kappa M0 + (Mt - Ms) + 1/2 sum_f S_f,
        i.e. -div(D grad phi) + (kappa + sigma_a) phi with D = 1 / (3 sigma_t)
        taken per row, and the Marshak vacuum condition D d_n phi + phi / 2 = 0 on
        every face."""
        d, F = self.d, self.F
        stiff = sum(d.csr(F["K"][a, a]) for a in range(d.dim))
        C = sp.diags(1.0 / (3.0 * self.sigma_t_rows())) @ stiff
        C = C + kappa * d.csr(F["M0"]) + d.csr(F["Mt"]) - d.csr(F["Ms"])
        C = C + 0.5 * sum(d.csr(F["S"][f]) for f in range(2 * d.dim))
        return C.tocsr()

    def MS(self, Phi):
        return np.stack([self._MS[m] @ Phi for m in range(self.M)])


def gmres(apply, b, x0, tol, restart, maxit, precond=None):
    """Restarted GMRES (the Krylov solver of Sec. 4.2; modified Gram-Schmidt Arnoldi, Givens rotations),
    right preconditioned by `precond` when given.  Stops when
    ||b - A x|| <= tol * ||b||.  Returns (x, iterations, relative residual)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return np.zeros_like(b), 0, 0.0
    its = 0
    M = precond if precond is not None else (lambda v: v)
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bn or its >= maxit:
            return x, its, beta / bn
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k = 0
        for k in range(restart):
            wv = apply(M(V[k]))
            for i in range(k + 1):
                H[i, k] = V[i] @ wv
                wv = wv - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(wv)
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            its += 1
            if H[k + 1, k] == 0.0 and den == 0.0:
                break
            if abs(g[k + 1]) <= tol * bn or its >= maxit:
                break
            V.append(wv / np.linalg.norm(wv) if np.linalg.norm(wv) > 0 else wv)
        kk = k + 1
        y = np.linalg.solve(np.triu(H[:kk, :kk]), g[:kk])
        x = x + M(sum(y[i] * V[i] for i in range(kk)))


@dataclass
class StepStats:
    outer_iterations: int = 0
    outer_residual: float = 0.0
    inner_iterations: list | None = None


class Solver:
    """Backward-Euler time stepping with the nested solve of Sec. 4.2."""

    def __init__(self, tr: Transport, outer_tol=1e-13, outer_restart=200, outer_maxit=2000,
                 inner="lu", inner_tol=1e-13, inner_restart=50, outer="gmres", precond=None):
        """outer: "gmres" (the paper's Krylov solve on Phi, Eq. krylov-operator) or
        "source-iteration" (Phi <- b_phi + D L^-1 MS Phi until the update is
        below outer_tol of Phi).  precond="dsa" right-preconditions the outer
        GMRES with P^-1 = I + C^-1 Ms (C: Transport.diffusion_matrix): the
        scattering source of a Krylov direction drives a diffusion correction,
        so the slowly converging smooth modes of thick scattering regions are
        taken out; the solution is the same, the residual tested is the true one."""
        if precond not in (None, "dsa"):
            raise ValueError("precond: None or 'dsa'")
        if precond is not None and outer != "gmres":
            raise ValueError("the DSA-like preconditioner is for the GMRES outer solve")
        self.tr = tr
        self.outer = outer
        self.precond = precond
        self._dsa = None
        self.outer_tol = outer_tol
        self.outer_restart = outer_restart
        self.outer_maxit = outer_maxit
        self.inner = inner
        self.inner_tol = inner_tol
        self.inner_restart = inner_restart
        self.inner_counts = []
        self._ilu = None

    def _Linv(self, rhs):
        tr = self.tr
        if self.inner == "lu":
            return tr.Linv(rhs)
        # the paper's inner scheme: GMRES right-preconditioned by ILUT
        if self._ilu is None or self._ilu[0] != tr._kappa:
            self._ilu = (tr._kappa, [spla.spilu(tr._L[m].tocsc(), drop_tol=1e-4, fill_factor=10)
                                     for m in range(tr.M)])
        out = np.zeros_like(rhs)
        for m in range(tr.M):
            Lm = tr._L[m]
            ilu = self._ilu[1][m]
            out[m], its, _ = gmres(lambda v: Lm @ v, rhs[m], np.zeros(tr.d.n), self.inner_tol,
                                   self.inner_restart, 10000, precond=ilu.solve)
            self.inner_counts.append(its)
        return out

    def step(self, Psi_prev, dt, Phi_guess=None, src=None):
        """One backward-Euler step (Sec. 4.1-4.2).  Psi_prev[M, n] -> (Psi, Phi, stats).
        src[M, n]: extra right-hand side of this step (manufactured sources)."""
        tr = self.tr
        kappa = 0.0 if not np.isfinite(dt) else 1.0 / (tr.c * dt)
        tr.factor(kappa)
        f = np.stack([tr._T[m] @ Psi_prev[m] + tr._r[m] for m in range(tr.M)])
        if src is not None:
            f = f + src
        b_psi = self._Linv(f)                       # first-flight angular flux
        b_phi = tr.D(b_psi)

        def A(Phi):                                 # (I - D L^-1 MS) Phi
            return Phi - tr.D(self._Linv(tr.MS(Phi)))
        x0 = np.zeros(tr.d.n) if Phi_guess is None else Phi_guess
        if self.outer == "source-iteration":
            Phi = np.array(x0, dtype=np.float64, copy=True)
            for its in range(1, self.outer_maxit + 1):
                x = self._Linv(tr.MS(Phi))          # L^-1 MS Phi_k
                new = b_phi + tr.D(x)               # Phi_{k+1}
                res = np.linalg.norm(new - Phi) / max(np.linalg.norm(new), 1e-300)
                Phi = new
                if res <= self.outer_tol:
                    break
            return x + b_psi, Phi, StepStats(its, res)   # D Psi = Phi_{k+1}
        P = None
        if self.precond == "dsa":
            if self._dsa is None or self._dsa[0] != kappa:
                self._dsa = (kappa, spla.splu(tr.diffusion_matrix(kappa).tocsc()), tr.d.csr(tr.F["Ms"]))
            _, C, Ms = self._dsa
            P = lambda v: v + C.solve(Ms @ v)
        Phi, its, res = gmres(A, b_phi, x0, self.outer_tol, self.outer_restart, self.outer_maxit, precond=P)
        Psi = self._Linv(tr.MS(Phi)) + b_psi        # angular recovery
        return Psi, Phi, StepStats(its, res)

    def step_direct(self, Psi_prev, dt):
        """(Sec. 4.2) The same step from one sparse LU of the coupled system
        (L - MS D) Psi = T Psi^{n-1} + r (unknowns ordered direction-major)."""
        tr = self.tr
        kappa = 0.0 if not np.isfinite(dt) else 1.0 / (tr.c * dt)
        tr.factor(kappa)
        n, M = tr.d.n, tr.M
        Lb = sp.block_diag([tr._L[m] for m in range(M)], format="csr")
        MS = sp.vstack([tr._MS[m] for m in range(M)], format="csr")     # [M n, n]
        Dm = sp.hstack([tr.w[m] * sp.identity(n) for m in range(M)], format="csr")  # [n, M n]
        A = (Lb - MS @ Dm).tocsc()
        f = np.concatenate([tr._T[m] @ Psi_prev[m] + tr._r[m] for m in range(M)])
        Psi = spla.spsolve(A, f).reshape(M, n)
        return Psi, tr.D(Psi)

    def run(self, Psi0, dt, steps, direct=False, src=None):
        """Backward-Euler time loop (Sec. 4.1) from Psi0.  src(n) -> [M, n] extra source of step n (1-based)."""
        Psi = np.array(Psi0, dtype=np.float64, copy=True)
        Phi = self.tr.D(Psi)
        stats = []
        for k in range(1, steps + 1):
            if direct:
                Psi, Phi = self.step_direct(Psi, dt)
            else:
                Psi, Phi, st = self.step(Psi, dt, Phi_guess=Phi,
                                         src=None if src is None else src(k))
                stats.append(st)
        return Psi, Phi, stats


# ---------------------------------------------------------------------------
# whole-problem convenience
# ---------------------------------------------------------------------------
def solve_problem(prob, steps=None, direct=False, outer_tol=1e-13, inner="lu", return_all=False):
    """(Sec. 4.1-4.2, Eq. flux-expansion for the output) Run a mlpg_inputs.Problem (per-point materials) for `steps` steps from
    Psi = 0 and return the point values phi_i of the scalar flux."""
    disc = Discretization(prob.x, prob.R, prob.lo, prob.hi)
    F = disc.assemble_per_point(prob.sigma_t, prob.sigma_s, prob.q)
    tr = Transport(disc, F, prob.omega, prob.w, psi_b=prob.inflow)
    sol = Solver(tr, outer_tol=outer_tol, inner=inner)
    Psi0 = np.zeros((tr.M, disc.n))
    Psi, Phi, stats = sol.run(Psi0, prob.dt, prob.steps if steps is None else steps, direct=direct)
    phi = disc.interpolation_matrix() @ Phi
    if return_all:
        return dict(disc=disc, forms=F, transport=tr, solver=sol, Psi=Psi, Phi=Phi, phi=phi, stats=stats)
    return phi


def relative_error(numeric, analytic):
    """Eq. relative-err (Sec. 5): sum |numeric - analytic| / sum analytic."""
    return float(np.sum(np.abs(numeric - analytic)) / np.sum(analytic))
