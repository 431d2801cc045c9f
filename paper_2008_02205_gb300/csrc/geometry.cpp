// 3D integration cells on the host (Sec. 3.1), built once per point set on the
// host cores (the 2D cells are built on the device, cells2d.cu).
#include <algorithm>
#include <cmath>
#include <exception>
#include <thread>

#include "internal.h"

// ---------------------------------------------------------------------------
// 3D cells (Sec. 3.1): the kernel-extent cube cut to the domain box, clipped by
// the bisector half-space of every overlap neighbour.  A cell is a list of
// planar faces; a cut keeps the inside part of every face and closes the
// polyhedron with a new face: the convex hull, in the cutting plane, of the
// vertices on the plane and the points where face edges cross it (Andrew's
// monotone chain, counter-clockwise about the outward normal).  Signed
// distances within a small tolerance of the plane count as on it (planes that
// pass through existing edges, as in regular lattices).  Output: one
// tetrahedron (x_i, c_f, v_k, v_k+1) per edge of every face f, c_f the average
// of the face's vertices, and one triangle (c_f, v_k, v_k+1) per edge of every
// face on the domain boundary.
// ---------------------------------------------------------------------------
namespace mlpg {
namespace {
struct P3 {
    double x, y, z;
};
inline P3 sub(const P3 &a, const P3 &b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline double dotp(const P3 &a, const P3 &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline P3 crossp(const P3 &a, const P3 &b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
struct Face3 {
    std::vector<P3> v;
    int32_t lab;
};

// convex hull of points in the plane with unit normal nh, counter-clockwise about
// nh.  Points closer than dist_tol are merged first: the same vertex reached
// from two faces differs by rounding, and two such copies on either side of a
// true corner in the sort order would let the collinearity test drop the corner.
void plane_hull(std::vector<P3> &pts, const P3 &nh, double dist_tol, double area_tol, std::vector<P3> &out) {
    out.clear();
    size_t nu = 0;
    for (size_t k = 0; k < pts.size(); ++k) {
        bool dup = false;
        for (size_t u = 0; u < nu && !dup; ++u) {
            P3 e = sub(pts[k], pts[u]);
            dup = std::sqrt(dotp(e, e)) <= dist_tol;
        }
        if (!dup) pts[nu++] = pts[k];
    }
    pts.resize(nu);
    if (pts.size() < 3) return;
    // in-plane basis (e1, e2) with e1 x e2 = nh
    P3 t = std::fabs(nh.x) < 0.6 ? P3{1, 0, 0} : P3{0, 1, 0};
    P3 e1 = sub(t, {nh.x * dotp(t, nh), nh.y * dotp(t, nh), nh.z * dotp(t, nh)});
    double l = std::sqrt(dotp(e1, e1));
    e1 = {e1.x / l, e1.y / l, e1.z / l};
    P3 e2 = crossp(nh, e1);
    struct Q {
        double u, v;
        int k;
    };
    std::vector<Q> q(pts.size());
    for (size_t k = 0; k < pts.size(); ++k) q[k] = {dotp(pts[k], e1), dotp(pts[k], e2), (int)k};
    std::sort(q.begin(), q.end(), [](const Q &a, const Q &b) { return a.u < b.u || (a.u == b.u && a.v < b.v); });
    auto turn = [](const Q &o, const Q &a, const Q &b) { return (a.u - o.u) * (b.v - o.v) - (a.v - o.v) * (b.u - o.u); };
    std::vector<Q> h(2 * q.size());
    size_t m = 0;
    for (size_t k = 0; k < q.size(); ++k) {   // lower chain
        while (m >= 2 && turn(h[m - 2], h[m - 1], q[k]) <= area_tol) --m;
        h[m++] = q[k];
    }
    for (size_t k = q.size() - 1, lo = m + 1; k-- > 0;) {   // upper chain
        while (m >= lo && turn(h[m - 2], h[m - 1], q[k]) <= area_tol) --m;
        h[m++] = q[k];
    }
    if (m < 4) return;   // fewer than three distinct hull points
    for (size_t k = 0; k + 1 < m; ++k) out.push_back(pts[h[k].k]);
}

// keep {p : nrm.p <= c}; the new face gets label j.  True when the plane cut.
bool clip3(std::vector<Face3> &F, std::vector<Face3> &tmp, std::vector<P3> &onp, std::vector<P3> &hull,
           const P3 &nrm, double c, double eps, double dist_tol, double area_tol, int32_t j) {
    bool any_out = false;
    for (const Face3 &f : F) {
        for (const P3 &p : f.v)
            if (dotp(nrm, p) - c > eps) { any_out = true; break; }
        if (any_out) break;
    }
    if (!any_out) return false;
    tmp.clear();
    onp.clear();
    for (const Face3 &f : F) {
        Face3 g;
        g.lab = f.lab;
        const size_t nv = f.v.size();
        for (size_t k = 0; k < nv; ++k) {
            const P3 &p = f.v[k], &q = f.v[(k + 1) % nv];
            double sp = dotp(nrm, p) - c, sq = dotp(nrm, q) - c;
            if (sp <= eps) {
                g.v.push_back(p);
                if (sp >= -eps) onp.push_back(p);
            }
            if ((sp < -eps && sq > eps) || (sp > eps && sq < -eps)) {
                double t = sp / (sp - sq);
                P3 r{p.x + t * (q.x - p.x), p.y + t * (q.y - p.y), p.z + t * (q.z - p.z)};
                g.v.push_back(r);
                onp.push_back(r);
            }
        }
        if (g.v.size() >= 3) tmp.push_back(std::move(g));
    }
    double ln = std::sqrt(dotp(nrm, nrm));
    plane_hull(onp, {nrm.x / ln, nrm.y / ln, nrm.z / ln}, dist_tol, area_tol, hull);
    if (hull.size() >= 3) tmp.push_back({hull, j});
    F.swap(tmp);
    return true;
}

struct Chunk3 {
    std::vector<int32_t> tet_owner, tri_owner, tri_face;
    std::vector<double> tet_v, tri_v;
    int64_t bad = -1;
};
}  // namespace

int64_t build_cells_3d(int64_t n, const double *x, const double *R, const double *lo, const double *hi,
                       const int32_t *rowptr, const int32_t *col, HostCells3 &out) {
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < 512) nt = 1;
    std::vector<Chunk3> chunks(nt);
    out.volume.assign(n, 0.0);
    auto work = [&](unsigned t) {
        int64_t i0 = n * t / nt, i1 = n * (t + 1) / nt;
        Chunk3 &ch = chunks[t];
        std::vector<Face3> F, tmp;
        std::vector<P3> onp, hull;
        for (int64_t i = i0; i < i1; ++i) {
            const P3 g{x[3 * i], x[3 * i + 1], x[3 * i + 2]};
            const double r = R[i];
            double b0[3] = {g.x - r, g.y - r, g.z - r}, b1[3] = {g.x + r, g.y + r, g.z + r};
            bool dlo[3], dhi[3];
            for (int a = 0; a < 3; ++a) {
                dlo[a] = b0[a] <= lo[a];
                dhi[a] = b1[a] >= hi[a];
                if (dlo[a]) b0[a] = lo[a];
                if (dhi[a]) b1[a] = hi[a];
            }
            auto corner = [&](int k) { return P3{(k & 1) ? b1[0] : b0[0], (k & 2) ? b1[1] : b0[1], (k & 4) ? b1[2] : b0[2]}; };
            // the six faces of the box, counter-clockwise about their outward normals
            // (the orientation fixes the tetrahedra (x_i, c_f, v_k, v_k+1) of each edge)
            static const int quad[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4},
                                           {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
            F.clear();
            for (int f = 0; f < 6; ++f) {
                bool dom = (f & 1) ? dhi[f / 2] : dlo[f / 2];
                Face3 fc;
                fc.lab = dom ? -(f + 1) : kLabelExtent;
                for (int k = 0; k < 4; ++k) fc.v.push_back(corner(quad[f][k]));
                F.push_back(std::move(fc));
            }
            // Two rounds over the neighbours, each in column order: those closer than the kernel
            // extent first, then the rest.  A bisector at distance |d| / 2 cuts nothing while the
            // polyhedron's reach (largest vertex distance from x_i) stays below it; such planes
            // are skipped with a relative margin of 1e-9, far above the rounding of either test,
            // so the cells are those of clipping by every plane in this order.
            auto reach2 = [&]() {
                double r2 = 0.0;
                for (const Face3 &f : F)
                    for (const P3 &v : f.v) r2 = std::max(r2, dotp(sub(v, g), sub(v, g)));
                return r2;
            };
            double r2 = reach2();
            for (int round = 0; round < 2 && !F.empty(); ++round) {
                for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                    int32_t j = col[p];
                    if (j == i) continue;
                    P3 xj{x[3 * (int64_t)j], x[3 * (int64_t)j + 1], x[3 * (int64_t)j + 2]};
                    P3 d = sub(xj, g);
                    const double d2 = dotp(d, d);
                    if ((d2 < r * r) != (round == 0)) continue;
                    if (r2 < 0.25 * d2 * (1.0 - 1e-9)) continue;
                    P3 mid{0.5 * (xj.x + g.x), 0.5 * (xj.y + g.y), 0.5 * (xj.z + g.z)};
                    double dl = std::sqrt(d2);
                    if (clip3(F, tmp, onp, hull, d, dotp(d, mid), 1e-12 * r * dl, 1e-12 * r, 1e-13 * r * r, j))
                        r2 = reach2();
                    if (F.empty()) break;
                }
            }
            double vol = 0.0;
            for (const Face3 &f : F) {
                const size_t nv = f.v.size();
                P3 cf{0, 0, 0};
                for (const P3 &p : f.v) cf = {cf.x + p.x, cf.y + p.y, cf.z + p.z};
                cf = {cf.x / nv, cf.y / nv, cf.z / nv};
                const bool bnd = f.lab < 0 && f.lab != kLabelExtent;
                for (size_t k = 0; k < nv; ++k) {
                    const P3 &a = f.v[k], &b = f.v[(k + 1) % nv];
                    vol += std::fabs(dotp(sub(cf, g), crossp(sub(a, g), sub(b, g)))) / 6.0;
                    ch.tet_owner.push_back((int32_t)i);
                    for (const P3 &p : {cf, a, b}) {
                        ch.tet_v.push_back(p.x);
                        ch.tet_v.push_back(p.y);
                        ch.tet_v.push_back(p.z);
                    }
                    if (bnd) {
                        ch.tri_owner.push_back((int32_t)i);
                        ch.tri_face.push_back(-f.lab - 1);
                        for (const P3 &p : {cf, a, b}) {
                            ch.tri_v.push_back(p.x);
                            ch.tri_v.push_back(p.y);
                            ch.tri_v.push_back(p.z);
                        }
                    }
                }
            }
            out.volume[i] = vol;
            if (!(vol > 0.0) && ch.bad < 0) ch.bad = i;
        }
    };
    // an exception in any share (a failed allocation) is rethrown on this thread once every
    // worker has ended
    std::vector<std::exception_ptr> errs(nt);
    auto guarded = [&](unsigned t) {
        try {
            work(t);
        } catch (...) {
            errs[t] = std::current_exception();
        }
    };
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nt; ++t) th.emplace_back(guarded, t);
    guarded(0);
    for (auto &t : th) t.join();
    for (auto &e : errs)
        if (e) std::rethrow_exception(e);
    out.tet_owner.clear(); out.tet_v.clear();
    out.tri_owner.clear(); out.tri_face.clear(); out.tri_v.clear();
    for (auto &ch : chunks) {
        if (ch.bad >= 0) return ch.bad;
        out.tet_owner.insert(out.tet_owner.end(), ch.tet_owner.begin(), ch.tet_owner.end());
        out.tet_v.insert(out.tet_v.end(), ch.tet_v.begin(), ch.tet_v.end());
        out.tri_owner.insert(out.tri_owner.end(), ch.tri_owner.begin(), ch.tri_owner.end());
        out.tri_face.insert(out.tri_face.end(), ch.tri_face.begin(), ch.tri_face.end());
        out.tri_v.insert(out.tri_v.end(), ch.tri_v.begin(), ch.tri_v.end());
    }
    return -1;
}

}  // namespace mlpg
