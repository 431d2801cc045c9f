"""The library's host-side code on the CPU: the 3D cell builder
(csrc/geometry.cpp, which runs on the host cores once per point set) and the
reference rules (csrc/quadrature.cpp, uploaded to the kernels), compiled with
g++ into a small harness and compared with the oracle, which shares no code
with them (Newton vs Golub-Welsch rules, convex-hull vs angle-sorted faces).

Sec. 3.1 (cells), Sec. 3.2 and App. A (rules and their mapping)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import mlpg_inputs as mi
import oracle.mlpg_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2008_02205_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r'''
#include <cstdio>
#include <vector>
#include "internal.h"
// in: n, x[3n], R[n], lo[3], hi[3], nnz, rowptr[n+1] (int32), col[nnz] (int32)
// out: bad, volume[n], ntet, owner[ntet], v[9 ntet], ntri, owner, face, v[9 ntri],
//      then for n1 = 1..4: tet rule (xi[3 n1^3], w), triangle rule (xi[2 n1^2], w),
//      Gauss-Jacobi(a, b) for (0,0), (1,0), (2,0): t[n1], w[n1]
template <class T> static void rd(FILE *f, T *p, size_t k) { if (fread(p, sizeof(T), k, f) != k) throw 1; }
template <class T> static void wr(FILE *f, const T *p, size_t k) { fwrite(p, sizeof(T), k, f); }
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "rb");
    int64_t n, nnz;
    rd(f, &n, 1);
    std::vector<double> x(3 * n), R(n), lo(3), hi(3);
    rd(f, x.data(), 3 * n); rd(f, R.data(), n); rd(f, lo.data(), 3); rd(f, hi.data(), 3);
    rd(f, &nnz, 1);
    std::vector<int32_t> rowptr(n + 1), col(nnz);
    rd(f, rowptr.data(), n + 1); rd(f, col.data(), nnz);
    fclose(f);
    mlpg::HostCells3 c;
    int64_t bad = mlpg::build_cells_3d(n, x.data(), R.data(), lo.data(), hi.data(), rowptr.data(), col.data(), c);
    FILE *o = fopen(argv[2], "wb");
    wr(o, &bad, 1);
    wr(o, c.volume.data(), n);
    int64_t nt = (int64_t)c.tet_owner.size(), nb = (int64_t)c.tri_owner.size();
    wr(o, &nt, 1); wr(o, c.tet_owner.data(), nt); wr(o, c.tet_v.data(), 9 * nt);
    wr(o, &nb, 1); wr(o, c.tri_owner.data(), nb); wr(o, c.tri_face.data(), nb); wr(o, c.tri_v.data(), 9 * nb);
    for (int n1 = 1; n1 <= 4; ++n1) {
        std::vector<double> xi(3 * n1 * n1 * n1), w(n1 * n1 * n1);
        mlpg::tet_rule(n1, xi.data(), w.data());
        wr(o, xi.data(), xi.size()); wr(o, w.data(), w.size());
        std::vector<double> ti(2 * n1 * n1), tw(n1 * n1);
        mlpg::triangle_rule(n1, ti.data(), tw.data());
        wr(o, ti.data(), ti.size()); wr(o, tw.data(), tw.size());
        for (int ab = 0; ab < 3; ++ab) {
            std::vector<double> t(n1), gw(n1);
            mlpg::gauss_jacobi_newton(n1, (double)ab, 0.0, t.data(), gw.data());
            wr(o, t.data(), n1); wr(o, gw.data(), n1);
        }
    }
    fclose(o);
    return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("hostgeo")
    src = d / "main.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    cmd = ["g++", "-O2", "-std=c++17", "-pthread", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
           f"-I{CUDA_INC}", str(src), os.path.join(CSRC, "geometry.cpp"), os.path.join(CSRC, "quadrature.cpp"),
           "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True)
    return d, exe


def _run(harness, x, R, lo, hi):
    d, exe = harness
    rowptr, col = O.neighbors(x, R)
    n = len(x)
    inp, out = d / "in.bin", d / "out.bin"
    with open(inp, "wb") as f:
        np.array([n], np.int64).tofile(f)
        np.ascontiguousarray(x, np.float64).tofile(f)
        np.ascontiguousarray(R, np.float64).tofile(f)
        np.asarray(lo, np.float64).tofile(f)
        np.asarray(hi, np.float64).tofile(f)
        np.array([len(col)], np.int64).tofile(f)
        np.asarray(rowptr, np.int32).tofile(f)
        np.asarray(col, np.int32).tofile(f)
    subprocess.run([str(exe), str(inp), str(out)], check=True, timeout=300)
    b = open(out, "rb").read()
    pos = 0

    def take(dtype, k):
        nonlocal pos
        a = np.frombuffer(b, dtype, k, pos)
        pos += a.nbytes
        return a
    r = {"bad": int(take(np.int64, 1)[0]), "V": take(np.float64, n)}
    nt = int(take(np.int64, 1)[0])
    r["tet_owner"], r["tet_v"] = take(np.int32, nt), take(np.float64, 9 * nt).reshape(nt, 3, 3)
    nb = int(take(np.int64, 1)[0])
    r["tri_owner"], r["tri_face"], r["tri_v"] = take(np.int32, nb), take(np.int32, nb), take(np.float64, 9 * nb).reshape(nb, 3, 3)
    r["rules"] = {}
    for n1 in range(1, 5):
        r["rules"][("tet", n1)] = (take(np.float64, 3 * n1 ** 3).reshape(-1, 3), take(np.float64, n1 ** 3))
        r["rules"][("tri", n1)] = (take(np.float64, 2 * n1 ** 2).reshape(-1, 2), take(np.float64, n1 ** 2))
        for ab in range(3):
            r["rules"][("gj", n1, ab)] = (take(np.float64, n1), take(np.float64, n1))
    return r


def _sorted_rows(a):
    a = np.round(np.asarray(a), 11)
    return a[np.lexsort(a.T[::-1])]


def test_reference_rules_match_the_oracle(harness):
    r = _run(harness, *_lattice(3, 0.0))
    for n1 in range(1, 5):
        for kind, ref in (("tet", O.tet_rule(n1)), ("tri", O.triangle_rule(n1))):
            xi, w = r["rules"][(kind, n1)]
            a = _sorted_rows(np.column_stack([xi, w]))
            b = _sorted_rows(np.column_stack([ref[0], ref[1]]))
            assert np.abs(a - b).max() < 1e-12, (kind, n1)
        for ab in range(3):
            t, w = r["rules"][("gj", n1, ab)]
            rt, rw = O.gauss_jacobi(n1, float(ab), 0.0)
            k, kr = np.argsort(t), np.argsort(rt)
            assert np.abs(t[k] - rt[kr]).max() < 1e-13 and np.abs(w[k] - rw[kr]).max() < 1e-13, (n1, ab)


def _lattice(n, jitter, seed=31):
    x, h = mi.jittered_lattice(n, 3, seed, jitter=jitter)
    return x, np.full(len(x), 2.0 * h), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)


def _match(a_pts, a_w, b_pts, b_w):
    """Every point of a has a point of b at the same place (1e-11) with the same
    weight, one to one."""
    from scipy.spatial import cKDTree
    assert len(a_pts) == len(b_pts)
    d, j = cKDTree(b_pts).query(a_pts)
    assert d.max() < 1e-11
    assert len(np.unique(j)) == len(j)
    assert np.abs(a_w - b_w[j]).max() < 1e-13 * np.abs(b_w).max()


@pytest.mark.parametrize("n,jitter", [(5, 0.0), (5, 0.2), (6, 0.2)])
def test_3d_cells_and_their_quadrature_match_the_oracle(harness, n, jitter):
    x, R, lo, hi = _lattice(n, jitter)
    r = _run(harness, x, R, lo, hi)
    assert r["bad"] == -1
    rowptr, col = O.neighbors(x, R)
    fptr, vptr, verts, labels, V = O.cells_3d(x, R, lo, hi, rowptr, col)
    assert np.abs(r["V"] - V).max() <= 1e-12 * V.max()
    assert abs(r["V"].sum() - 1.0) < 1e-12
    # tetrahedra (x_owner, c_f, v_k, v_k+1): their volumes add up to each cell's
    g = x[r["tet_owner"]]
    e = r["tet_v"] - g[:, None, :]
    tv = np.abs(np.einsum("ta,ta->t", e[:, 0], np.cross(e[:, 1], e[:, 2]))) / 6.0
    assert np.abs(np.bincount(r["tet_owner"], tv, minlength=len(x)) - V).max() <= 1e-12 * V.max()
    # the reference rules mapped onto them (App. A) give the oracle's points
    xi, w = O.tet_rule(2)
    pts = g[:, None, :] + np.einsum("tka,qk->tqa", e, xi)
    wq = tv[:, None] * 6.0 * w[None, :]
    vq = O.volume_qps_3d(x, fptr, vptr, verts, 2)
    own = np.repeat(r["tet_owner"], len(w)).astype(float)
    _match(np.column_stack([pts.reshape(-1, 3), 10.0 * own]), wq.ravel(),
           np.column_stack([vq.x, 10.0 * vq.owner]), vq.w)
    # boundary triangles (c_f, v_k, v_k+1) on the box faces, with their face index
    ti, tw = O.triangle_rule(2)
    tv3 = r["tri_v"]
    e1, e2 = tv3[:, 1] - tv3[:, 0], tv3[:, 2] - tv3[:, 0]
    area2 = np.linalg.norm(np.cross(e1, e2), axis=1)
    bp = tv3[:, None, 0, :] + ti[None, :, 0, None] * e1[:, None, :] + ti[None, :, 1, None] * e2[:, None, :]
    bw = area2[:, None] * tw[None, :]
    bq = O.boundary_qps_3d(len(x), fptr, vptr, verts, labels, 2)
    key = np.repeat(r["tri_owner"] * 6 + r["tri_face"], len(tw)).astype(float)
    _match(np.column_stack([bp.reshape(-1, 3), 10.0 * key]), bw.ravel(),
           np.column_stack([bq.x, 10.0 * (bq.owner * 6 + bq.face)]), bq.w)
