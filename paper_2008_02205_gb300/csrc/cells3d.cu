// 3D integration cells on the device (Sec. 3.1): one thread per point starts
// from the kernel-extent cube cut to the domain box and clips it by the
// bisector half-space of every overlap neighbour, then splits the polyhedron
// into tetrahedra (x_i, c_f, v_k, v_k+1) per face edge and boundary triangles
// (c_f, v_k, v_k+1) per edge of a face on the box (c_f: the face's vertex
// average).  A cut keeps the inside part of every face and closes the
// polyhedron with a new face: the convex hull, in the cutting plane, of the
// vertices on the plane and the points where face edges cross it (monotone
// chain).  Distances within 1e-12 R |x_j - x_i| of a plane count as on it.
//
// The same steps, in the same order and the same arithmetic, as the host
// builder (geometry.cpp); this file is compiled without floating-point
// contraction, so both give the same cells.  Two passes around a scan: the
// first counts each cell's tetrahedra and boundary triangles and records its
// volume, the second writes the elements at the cell's offsets, in cell
// order.  With the cells on the device the whole integration stage of a 3D
// point set runs on the GPU and can be repeated when the points move.
#include "internal.h"

namespace mlpg {
namespace {

constexpr int kMaxF = 64;    // faces of a cell during clipping
constexpr int kMaxV = 384;   // vertices over all faces
constexpr int kMaxOn = 96;   // points on a cutting plane

struct P3 {
    double x, y, z;
};
__device__ __forceinline__ P3 sub(const P3 &a, const P3 &b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dotp(const P3 &a, const P3 &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ P3 crossp(const P3 &a, const P3 &b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// faces as vertex runs: face f has vertices v[f0[f] .. f0[f] + nv[f]) and label lab[f]
struct Poly {
    int nf, nvt;
    int f0[kMaxF], nv[kMaxF];
    int32_t lab[kMaxF];
    P3 v[kMaxV];
};

struct Q2 {
    double u, v;
    int k;
};

// convex hull of the points (merged within dist_tol) in the plane of unit
// normal nh, counter-clockwise about nh; fewer than three points: empty
__device__ int plane_hull(P3 *pts, int np, const P3 &nh, double dist_tol, double area_tol, P3 *out, Q2 *q,
                          Q2 *h) {
    int nu = 0;
    for (int k = 0; k < np; ++k) {
        bool dup = false;
        for (int u = 0; u < nu && !dup; ++u) {
            const P3 e = sub(pts[k], pts[u]);
            dup = sqrt(dotp(e, e)) <= dist_tol;
        }
        if (!dup) pts[nu++] = pts[k];
    }
    if (nu < 3) return 0;
    const P3 t = fabs(nh.x) < 0.6 ? P3{1, 0, 0} : P3{0, 1, 0};
    P3 e1 = sub(t, {nh.x * dotp(t, nh), nh.y * dotp(t, nh), nh.z * dotp(t, nh)});
    const double l = sqrt(dotp(e1, e1));
    e1 = {e1.x / l, e1.y / l, e1.z / l};
    const P3 e2 = crossp(nh, e1);
    for (int k = 0; k < nu; ++k) q[k] = {dotp(pts[k], e1), dotp(pts[k], e2), k};
    for (int a = 1; a < nu; ++a) {   // insertion sort by (u, v)
        const Q2 key = q[a];
        int b = a - 1;
        while (b >= 0 && (key.u < q[b].u || (key.u == q[b].u && key.v < q[b].v))) {
            q[b + 1] = q[b];
            --b;
        }
        q[b + 1] = key;
    }
    auto turn = [](const Q2 &o, const Q2 &a, const Q2 &b) {
        return (a.u - o.u) * (b.v - o.v) - (a.v - o.v) * (b.u - o.u);
    };
    int m = 0;
    for (int k = 0; k < nu; ++k) {   // lower chain
        while (m >= 2 && turn(h[m - 2], h[m - 1], q[k]) <= area_tol) --m;
        h[m++] = q[k];
    }
    for (int k = nu - 1, lo = m + 1; k-- > 0;) {   // upper chain
        while (m >= lo && turn(h[m - 2], h[m - 1], q[k]) <= area_tol) --m;
        h[m++] = q[k];
    }
    if (m < 4) return 0;
    for (int k = 0; k + 1 < m; ++k) out[k] = pts[h[k].k];
    return m - 1;
}

// keep {p : nrm . p <= c}; the new face gets label j.  *cut: the result is in
// T (F is unchanged otherwise).  False on overflow.
__device__ bool clip3(const Poly &F, Poly &T, bool *cut, P3 *onp, P3 *hull, Q2 *q, Q2 *h, const P3 &nrm, double c,
                      double eps, double dist_tol, double area_tol, int32_t j) {
    bool any_out = false;
    for (int k = 0; k < F.nvt && !any_out; ++k) any_out = dotp(nrm, F.v[k]) - c > eps;
    *cut = any_out;
    if (!any_out) return true;
    T.nf = 0;
    T.nvt = 0;
    int non = 0;
    for (int f = 0; f < F.nf; ++f) {
        const int start = T.nvt, nv = F.nv[f];
        const P3 *fv = F.v + F.f0[f];
        for (int k = 0; k < nv; ++k) {
            const P3 &p = fv[k], &qq = fv[(k + 1) % nv];
            const double sp = dotp(nrm, p) - c, sq = dotp(nrm, qq) - c;
            if (sp <= eps) {
                if (T.nvt >= kMaxV) return false;
                T.v[T.nvt++] = p;
                if (sp >= -eps) {
                    if (non >= kMaxOn) return false;
                    onp[non++] = p;
                }
            }
            if ((sp < -eps && sq > eps) || (sp > eps && sq < -eps)) {
                const double t = sp / (sp - sq);
                const P3 r{p.x + t * (qq.x - p.x), p.y + t * (qq.y - p.y), p.z + t * (qq.z - p.z)};
                if (T.nvt >= kMaxV || non >= kMaxOn) return false;
                T.v[T.nvt++] = r;
                onp[non++] = r;
            }
        }
        if (T.nvt - start >= 3) {
            if (T.nf >= kMaxF) return false;
            T.f0[T.nf] = start;
            T.nv[T.nf] = T.nvt - start;
            T.lab[T.nf] = F.lab[f];
            ++T.nf;
        } else {
            T.nvt = start;   // a face with fewer than three vertices left is dropped
        }
    }
    const double ln = sqrt(dotp(nrm, nrm));
    const int nh = plane_hull(onp, non, {nrm.x / ln, nrm.y / ln, nrm.z / ln}, dist_tol, area_tol, hull, q, h);
    if (nh >= 3) {
        if (T.nf >= kMaxF || T.nvt + nh > kMaxV) return false;
        T.f0[T.nf] = T.nvt;
        T.nv[T.nf] = nh;
        T.lab[T.nf] = j;
        ++T.nf;
        for (int k = 0; k < nh; ++k) T.v[T.nvt++] = hull[k];
    }
    return true;
}

// largest squared distance of a vertex from g
__device__ double reach2(const Poly &F, const P3 &g) {
    double r2 = 0.0;
    for (int k = 0; k < F.nvt; ++k) {
        const P3 e = sub(F.v[k], g);
        r2 = fmax(r2, dotp(e, e));
    }
    return r2;
}

struct Cell3Args {
    int64_t n, i0;                 // points of this slab: i0 .. i0 + n - 1
    const double *x, *R;
    const int32_t *rowptr, *col;
    double lo[3], hi[3];
    int32_t *ntet, *ntri;          // [n] counts (first pass)
    double *vol;                   // [n]
    const int32_t *tptr, *bptr;    // [n + 1] offsets (second pass)
    int32_t *tet_owner, *tri_owner, *tri_face;
    double *tet_v, *tri_v;
    int *flag;                     // bit 128: a cell overflowed its buffers or is empty
    int32_t *bad;                  // smallest failing point
};

template <bool WRITE>
__global__ void __launch_bounds__(64) k_cells_3d(Cell3Args A, Poly *work, P3 *onbuf, Q2 *qbuf) {
    const int64_t li = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (li >= A.n) return;
    const int64_t i = A.i0 + li;
    // per-thread work buffers in global memory (one slot per thread of the slab): the
    // current polyhedron and the next, swapped after every cut
    Poly *pf = work + 2 * li, *pt = pf + 1;
    Poly &F0 = *pf;   // the starting polyhedron
    P3 *onp = onbuf + 2 * kMaxOn * li, *hull = onp + kMaxOn;
    Q2 *q = qbuf + 3 * kMaxOn * li, *h = q + kMaxOn;   // h: room for the two chains, 2 kMaxOn
    const P3 g{A.x[3 * i], A.x[3 * i + 1], A.x[3 * i + 2]};
    const double r = A.R[i];
    double b0[3] = {g.x - r, g.y - r, g.z - r}, b1[3] = {g.x + r, g.y + r, g.z + r};
    bool dlo[3], dhi[3];
    for (int a = 0; a < 3; ++a) {
        dlo[a] = b0[a] <= A.lo[a];
        dhi[a] = b1[a] >= A.hi[a];
        if (dlo[a]) b0[a] = A.lo[a];
        if (dhi[a]) b1[a] = A.hi[a];
    }
    // the six faces of the box, counter-clockwise about their outward normals
    const int quad[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
    F0.nf = 6;
    F0.nvt = 24;
    for (int f = 0; f < 6; ++f) {
        const bool dom = (f & 1) ? dhi[f / 2] : dlo[f / 2];
        F0.f0[f] = 4 * f;
        F0.nv[f] = 4;
        F0.lab[f] = dom ? -(f + 1) : kLabelExtent;
        for (int k = 0; k < 4; ++k) {
            const int c = quad[f][k];
            F0.v[4 * f + k] = {(c & 1) ? b1[0] : b0[0], (c & 2) ? b1[1] : b0[1], (c & 4) ? b1[2] : b0[2]};
        }
    }
    bool okc = true;
    // A bisector at distance |d| / 2 from g cuts nothing while every vertex lies closer to g:
    // then d . v - c <= |d| (|v - g| - |d| / 2) < 0, so the vertex scan of clip3 would find no
    // vertex beyond the plane.  Such planes are skipped on the polyhedron's reach (its largest
    // vertex distance from g), with a relative margin of 1e-9 far above the rounding of either
    // test: the cells stay those of the scan, bit for bit.
    // Two rounds over the neighbours, each in column order: those closer than the kernel
    // extent first (they carve the cell to about its final size), then the rest, most of
    // which the reach test skips.  The host builder takes the same order.
    double r2 = reach2(*pf, g);
    bool empty = false;
    for (int round = 0; round < 2 && okc && !empty; ++round) {
        for (int32_t p = A.rowptr[i]; p < A.rowptr[i + 1] && okc; ++p) {
            const int32_t j = A.col[p];
            if (j == i) continue;
            const P3 xj{A.x[3 * (int64_t)j], A.x[3 * (int64_t)j + 1], A.x[3 * (int64_t)j + 2]};
            const P3 d = sub(xj, g);
            const double d2 = dotp(d, d);
            if ((d2 < r * r) != (round == 0)) continue;
            if (r2 < 0.25 * d2 * (1.0 - 1e-9)) continue;
            const P3 mid{0.5 * (xj.x + g.x), 0.5 * (xj.y + g.y), 0.5 * (xj.z + g.z)};
            const double dl = sqrt(d2);
            bool cut = false;
            okc = clip3(*pf, *pt, &cut, onp, hull, q, h, d, dotp(d, mid), 1e-12 * r * dl, 1e-12 * r, 1e-13 * r * r, j);
            if (cut) {
                Poly *tmp = pf;
                pf = pt;
                pt = tmp;
                r2 = reach2(*pf, g);
            }
            if (pf->nf == 0) {
                empty = true;
                break;
            }
        }
    }
    const Poly &F = *pf;
    double vol = 0.0;
    int nt = 0, nb = 0;
    const int32_t to = WRITE ? A.tptr[i] : 0, bo = WRITE ? A.bptr[i] : 0;
    for (int f = 0; f < F.nf && okc; ++f) {
        const int nv = F.nv[f];
        const P3 *fv = F.v + F.f0[f];
        P3 cf{0, 0, 0};
        for (int k = 0; k < nv; ++k) cf = {cf.x + fv[k].x, cf.y + fv[k].y, cf.z + fv[k].z};
        cf = {cf.x / nv, cf.y / nv, cf.z / nv};
        const bool bnd = F.lab[f] < 0 && F.lab[f] != kLabelExtent;
        for (int k = 0; k < nv; ++k) {
            const P3 &a = fv[k], &b = fv[(k + 1) % nv];
            vol += fabs(dotp(sub(cf, g), crossp(sub(a, g), sub(b, g)))) / 6.0;
            if (WRITE) {
                const int64_t e = to + nt;
                A.tet_owner[e] = (int32_t)i;
                const P3 pts[3] = {cf, a, b};
                for (int c = 0; c < 3; ++c) {
                    A.tet_v[9 * e + 3 * c] = pts[c].x;
                    A.tet_v[9 * e + 3 * c + 1] = pts[c].y;
                    A.tet_v[9 * e + 3 * c + 2] = pts[c].z;
                }
                if (bnd) {
                    const int64_t eb = bo + nb;
                    A.tri_owner[eb] = (int32_t)i;
                    A.tri_face[eb] = -F.lab[f] - 1;
                    for (int c = 0; c < 3; ++c) {
                        A.tri_v[9 * eb + 3 * c] = pts[c].x;
                        A.tri_v[9 * eb + 3 * c + 1] = pts[c].y;
                        A.tri_v[9 * eb + 3 * c + 2] = pts[c].z;
                    }
                }
            }
            ++nt;
            nb += bnd;
        }
    }
    if (!WRITE) {
        const bool bad = !okc || !(vol > 0.0);
        if (bad) {
            atomicOr(A.flag, 128);
            atomicMin(A.bad, (int32_t)i);
        }
        A.ntet[i] = bad ? 0 : nt;
        A.ntri[i] = bad ? 0 : nb;
        A.vol[i] = vol;
    }
}

// exclusive scans of two count arrays into out[n + 1], out2[n + 1] (one block)
__global__ void k_scan_two(int64_t n, const int32_t *__restrict__ c1, const int32_t *__restrict__ c2,
                           int32_t *__restrict__ o1, int32_t *__restrict__ o2) {
    __shared__ long long p1[1024], p2[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int64_t chunk = (n + T - 1) / T, a = t * chunk, b = min(n, a + chunk);
    long long s1 = 0, s2 = 0;
    for (int64_t k = a; k < b; ++k) {
        s1 += c1[k];
        s2 += c2[k];
    }
    p1[t] = s1;
    p2[t] = s2;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        const long long v1 = t >= off ? p1[t - off] : 0, v2 = t >= off ? p2[t - off] : 0;
        __syncthreads();
        p1[t] += v1;
        p2[t] += v2;
        __syncthreads();
    }
    long long r1 = p1[t] - s1, r2 = p2[t] - s2;
    for (int64_t k = a; k < b; ++k) {
        o1[k] = (int32_t)r1;
        o2[k] = (int32_t)r2;
        r1 += c1[k];
        r2 += c2[k];
    }
    if (t == T - 1) {
        o1[n] = (int32_t)p1[T - 1];
        o2[n] = (int32_t)p2[T - 1];
    }
}

}  // namespace

// The cells of all points, the tetrahedra and boundary triangles into the
// context's element arrays (tet_owner, tet_v, tri_owner, tri_face, tri_v), the
// volumes into V.  Cells are built in slabs of kSlab points, whose per-thread
// work buffers (about 11 KB a point) exist only during this call.
mlpg_status run_cells_3d(mlpg_ctx *ctx) {
    constexpr int64_t kSlab = 8192;
    const int64_t n = ctx->n;
    cudaStream_t s = ctx->stream;
    const int64_t slab = std::min<int64_t>(n, kSlab);
    struct Scratch {   // transient buffers, released on every return
        void *p[3] = {nullptr, nullptr, nullptr};
        ~Scratch() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } tmp;
    CU(ctx, cudaMalloc(&tmp.p[0], sizeof(Poly) * 2 * slab));
    CU(ctx, cudaMalloc(&tmp.p[1], sizeof(P3) * 2 * kMaxOn * slab));
    CU(ctx, cudaMalloc(&tmp.p[2], sizeof(Q2) * 3 * kMaxOn * slab));
    Poly *work = static_cast<Poly *>(tmp.p[0]);
    P3 *onbuf = static_cast<P3 *>(tmp.p[1]);
    Q2 *qbuf = static_cast<Q2 *>(tmp.p[2]);
    int32_t *ntet, *ntri, *bad, *tptr, *bptr;
    MLPG_TRY(dalloc(ctx, &ntet, n));
    MLPG_TRY(dalloc(ctx, &ntri, n));
    MLPG_TRY(dalloc(ctx, &tptr, n + 1));
    MLPG_TRY(dalloc(ctx, &bptr, n + 1));
    MLPG_TRY(dalloc(ctx, &bad, 1));
    if (!ctx->d_flag) MLPG_TRY(dalloc(ctx, &ctx->d_flag, 1));
    CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
    const int32_t big = 0x7fffffff;
    CU(ctx, cudaMemcpyAsync(bad, &big, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    Cell3Args a{};
    a.x = ctx->x; a.R = ctx->R; a.rowptr = ctx->rowptr; a.col = ctx->col;
    for (int d = 0; d < 3; ++d) { a.lo[d] = ctx->opt.lo[d]; a.hi[d] = ctx->opt.hi[d]; }
    a.ntet = ntet; a.ntri = ntri; a.vol = ctx->V; a.tptr = tptr; a.bptr = bptr;
    a.flag = ctx->d_flag; a.bad = bad;
    auto pass = [&](bool write) -> mlpg_status {
        a.tet_owner = ctx->tet_owner; a.tri_owner = ctx->tri_owner; a.tri_face = ctx->tri_face;
        a.tet_v = ctx->tet_v; a.tri_v = ctx->tri_v;
        for (int64_t i0 = 0; i0 < n; i0 += slab) {
            Cell3Args b = a;
            b.i0 = i0;
            b.n = std::min(slab, n - i0);
            const unsigned G = (unsigned)((b.n + 63) / 64);
            if (write) k_cells_3d<true><<<G, 64, 0, s>>>(b, work, onbuf, qbuf);
            else k_cells_3d<false><<<G, 64, 0, s>>>(b, work, onbuf, qbuf);
            CU_LAUNCH(ctx);
        }
        return MLPG_OK;
    };
    MLPG_TRY(pass(false));
    k_scan_two<<<1, 1024, 0, s>>>(n, ntet, ntri, tptr, bptr);
    CU_LAUNCH(ctx);
    int32_t tot[2] = {0, 0}, badi = big;
    int flag = 0;
    CU(ctx, cudaMemcpyAsync(&tot[0], tptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaMemcpyAsync(&tot[1], bptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaMemcpyAsync(&badi, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    if (flag & 128) return set_err(ctx, MLPG_ERR_GEOMETRY, "empty or oversized cell at point " + std::to_string(badi));
    ctx->ntet = tot[0];
    ctx->nbtri = tot[1];
    ctx->nvq = 8 * ctx->ntet;
    ctx->nbq = 4 * ctx->nbtri;
    MLPG_TRY(dalloc(ctx, &ctx->tet_owner, ctx->ntet));
    MLPG_TRY(dalloc(ctx, &ctx->tet_v, 9 * ctx->ntet));
    MLPG_TRY(dalloc(ctx, &ctx->tri_owner, ctx->nbtri + 1));
    MLPG_TRY(dalloc(ctx, &ctx->tri_face, ctx->nbtri + 1));
    MLPG_TRY(dalloc(ctx, &ctx->tri_v, 9 * ctx->nbtri + 9));
    MLPG_TRY(pass(true));
    CU(ctx, cudaStreamSynchronize(s));   // before the work buffers are released
    return MLPG_OK;
}

}  // namespace mlpg
