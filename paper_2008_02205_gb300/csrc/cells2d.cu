// 2D integration cells on the device (Sec. 3.1): one thread per point clips
// the kernel-extent square, cut to the domain box, by the perpendicular
// bisector of every overlap neighbour.  Two passes over the cells: the first
// counts vertices and boundary edges and records the area, the second (after a
// scan of the counts) writes every cell's vertices and edge labels at its
// offset.  The cells depend only on the points and extents, so the whole
// integration stage can rerun on the device when the points move.
#include "internal.h"

namespace mlpg {
namespace {

constexpr int kMaxPoly = 32;   // polygon vertices during clipping

struct CellArgs {
    int64_t n;
    const double *x, *R;
    const int32_t *rowptr, *col;
    double lo0, lo1, hi0, hi1;
    int32_t *nvert;        // [n]
    int32_t *nbedge;       // [n]
    double *vol;           // [n]
    const int32_t *cptr;   // [n + 1] (second pass)
    double *verts;         // [2 * total] (second pass)
    int32_t *labels;       // [total] (second pass)
    int *flag;             // bit 64: a cell needs more than kMaxPoly vertices or is empty
    int32_t *bad;          // smallest failing point
};

// keep {p : a p.x + b p.y <= c}; edges created by the cut get label j
__device__ int clip_poly(int nv, double *px, double *py, int32_t *lab, double *tx, double *ty, int32_t *tl,
                         double a, double b, double c, int32_t j, bool *overflow) {
    bool any_out = false;
    for (int k = 0; k < nv; ++k)
        if (a * px[k] + b * py[k] - c > 0.0) { any_out = true; break; }
    if (!any_out) return nv;
    int out = 0;
    for (int k = 0; k < nv; ++k) {
        const int k1 = k + 1 == nv ? 0 : k + 1;
        const double sp = a * px[k] + b * py[k] - c, sq = a * px[k1] + b * py[k1] - c;
        const bool pin = sp <= 0.0, qin = sq <= 0.0;
        if (pin) {
            if (out >= kMaxPoly) { *overflow = true; return 0; }
            tx[out] = px[k]; ty[out] = py[k]; tl[out] = lab[k]; ++out;
        }
        if (pin != qin) {
            if (out >= kMaxPoly) { *overflow = true; return 0; }
            const double t = sp / (sp - sq);
            tx[out] = px[k] + t * (px[k1] - px[k]);
            ty[out] = py[k] + t * (py[k1] - py[k]);
            tl[out] = pin ? j : lab[k];
            ++out;
        }
    }
    for (int k = 0; k < out; ++k) { px[k] = tx[k]; py[k] = ty[k]; lab[k] = tl[k]; }
    return out;
}

template <bool WRITE>
__global__ void k_cells_2d(CellArgs A) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    double px[kMaxPoly], py[kMaxPoly], tx[kMaxPoly], ty[kMaxPoly];
    int32_t lab[kMaxPoly], tl[kMaxPoly];
    const double xi = A.x[2 * i], yi = A.x[2 * i + 1], r = A.R[i];
    double x0 = xi - r, x1 = xi + r, y0 = yi - r, y1 = yi + r;
    const bool bx0 = x0 <= A.lo0, bx1 = x1 >= A.hi0, by0 = y0 <= A.lo1, by1 = y1 >= A.hi1;
    x0 = bx0 ? A.lo0 : x0;
    x1 = bx1 ? A.hi0 : x1;
    y0 = by0 ? A.lo1 : y0;
    y1 = by1 ? A.hi1 : y1;
    // counter-clockwise from the lower-left corner; the label is that of the edge starting there
    px[0] = x0; py[0] = y0; lab[0] = by0 ? -3 : kLabelExtent;   // face 2 (-y)
    px[1] = x1; py[1] = y0; lab[1] = bx1 ? -2 : kLabelExtent;   // face 1 (+x)
    px[2] = x1; py[2] = y1; lab[2] = by1 ? -4 : kLabelExtent;   // face 3 (+y)
    px[3] = x0; py[3] = y1; lab[3] = bx0 ? -1 : kLabelExtent;   // face 0 (-x)
    int nv = 4;
    bool overflow = false;
    for (int32_t p = A.rowptr[i]; p < A.rowptr[i + 1] && nv > 0; ++p) {
        const int32_t j = A.col[p];
        if (j == i) continue;
        const double xj = A.x[2 * (int64_t)j], yj = A.x[2 * (int64_t)j + 1];
        const double ax = xj - xi, ay = yj - yi;
        const double c = ax * 0.5 * (xj + xi) + ay * 0.5 * (yj + yi);
        nv = clip_poly(nv, px, py, lab, tx, ty, tl, ax, ay, c, j, &overflow);
    }
    double area2 = 0.0;
    int nb = 0;
    for (int k = 0; k < nv; ++k) {
        const int k1 = k + 1 == nv ? 0 : k + 1;
        area2 += px[k] * py[k1] - px[k1] * py[k];
        nb += lab[k] < 0 && lab[k] != kLabelExtent;
    }
    if (!WRITE) {
        const bool bad = overflow || nv < 3 || !(area2 > 0.0);
        if (bad) {
            atomicOr(A.flag, 64);
            atomicMin(A.bad, (int32_t)i);
        }
        A.nvert[i] = bad ? 0 : nv;
        A.nbedge[i] = bad ? 0 : nb;
        A.vol[i] = 0.5 * area2;
        return;
    }
    const int32_t o = A.cptr[i];
    if (A.cptr[i + 1] - o != nv) return;   // unchanged between passes (same arithmetic)
    for (int k = 0; k < nv; ++k) {
        A.verts[2 * (o + k)] = px[k];
        A.verts[2 * (o + k) + 1] = py[k];
        A.labels[o + k] = lab[k];
    }
}

// exclusive scan of n counts into out[n + 1] and the two totals (one block)
__global__ void k_scan_counts(int64_t n, const int32_t *__restrict__ cnt, const int32_t *__restrict__ cnt2,
                              int32_t *__restrict__ out, long long *__restrict__ totals) {
    __shared__ long long part[1024];
    __shared__ long long part2[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int64_t chunk = (n + T - 1) / T, a = t * chunk, b = min(n, a + chunk);
    long long s = 0, s2 = 0;
    for (int64_t k = a; k < b; ++k) {
        s += cnt[k];
        s2 += cnt2[k];
    }
    part[t] = s;
    part2[t] = s2;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        long long v = t >= off ? part[t - off] : 0, v2 = t >= off ? part2[t - off] : 0;
        __syncthreads();
        part[t] += v;
        part2[t] += v2;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (int64_t k = a; k < b; ++k) {
        out[k] = (int32_t)run;
        run += cnt[k];
    }
    if (t == T - 1) {
        out[n] = (int32_t)part[T - 1];
        totals[0] = part[T - 1];
        totals[1] = part2[T - 1];
    }
}

}  // namespace

mlpg_status run_cells_2d(mlpg_ctx *ctx, int tri_points, int line_points) {
    const int64_t n = ctx->n;
    cudaStream_t s = ctx->stream;
    int32_t *nvert, *nbedge, *bad;
    long long *totals;
    MLPG_TRY(dalloc(ctx, &nvert, n));
    MLPG_TRY(dalloc(ctx, &nbedge, n));
    MLPG_TRY(dalloc(ctx, &bad, 1));
    MLPG_TRY(dalloc(ctx, &totals, 2));
    MLPG_TRY(dalloc(ctx, &ctx->cptr, n + 1));
    if (!ctx->d_flag) MLPG_TRY(dalloc(ctx, &ctx->d_flag, 1));
    CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
    const int32_t big = 0x7fffffff;
    CU(ctx, cudaMemcpyAsync(bad, &big, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CellArgs a{};
    a.n = n; a.x = ctx->x; a.R = ctx->R; a.rowptr = ctx->rowptr; a.col = ctx->col;
    a.lo0 = ctx->opt.lo[0]; a.lo1 = ctx->opt.lo[1]; a.hi0 = ctx->opt.hi[0]; a.hi1 = ctx->opt.hi[1];
    a.nvert = nvert; a.nbedge = nbedge; a.vol = ctx->V; a.cptr = ctx->cptr; a.flag = ctx->d_flag; a.bad = bad;
    const unsigned G = (unsigned)((n + 127) / 128);
    k_cells_2d<false><<<G, 128, 0, s>>>(a);
    CU_LAUNCH(ctx);
    k_scan_counts<<<1, 1024, 0, s>>>(n, nvert, nbedge, ctx->cptr, totals);
    CU_LAUNCH(ctx);
    long long tot[2] = {0, 0};
    int flag = 0;
    int32_t badi = big;
    CU(ctx, cudaMemcpyAsync(tot, totals, sizeof(tot), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaMemcpyAsync(&badi, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    if (flag & 64) return set_err(ctx, MLPG_ERR_GEOMETRY, "empty or oversized cell at point " + std::to_string(badi));
    ctx->nverts = tot[0];
    ctx->nvq = tot[0] * tri_points;
    ctx->nbq = tot[1] * line_points;
    MLPG_TRY(dalloc(ctx, &ctx->verts, 2 * ctx->nverts));
    MLPG_TRY(dalloc(ctx, &ctx->labels, ctx->nverts));
    a.verts = ctx->verts;
    a.labels = ctx->labels;
    k_cells_2d<true><<<G, 128, 0, s>>>(a);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

}  // namespace mlpg
