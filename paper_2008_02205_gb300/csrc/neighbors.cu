// Overlap connectivity on the device (Sec. 3.4).
//
// Points i and j interact in the MLPG forms when their kernel supports overlap,
// |x_i - x_j| < R_i + R_j.  Points are binned into a uniform grid of cell size
// 2 max(R); every overlap partner of i then lies in the 3^d grid cells around
// it.  Two passes (count, fill) build the CSR pattern; each row is then sorted
// by column so that the pattern is canonical.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace mlpg {

namespace {

__device__ __forceinline__ int grid_coord(double v, double lo, double inv, int gd) {
    int c = (int)floor((v - lo) * inv);
    return c < 0 ? 0 : (c >= gd ? gd - 1 : c);
}

__global__ void k_bin(int64_t n, int dim, const double *__restrict__ x, double3 lo, double inv,
                      int3 gd, int *__restrict__ cell_of, int *__restrict__ cell_count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = grid_coord(x[i * dim], lo.x, inv, gd.x);
    int cy = grid_coord(x[i * dim + 1], lo.y, inv, gd.y);
    int cz = dim > 2 ? grid_coord(x[i * dim + 2], lo.z, inv, gd.z) : 0;
    int c = (cz * gd.y + cy) * gd.x + cx;
    cell_of[i] = c;
    atomicAdd(&cell_count[c], 1);
}

__global__ void k_bin_fill(int64_t n, const int *__restrict__ cell_of, const int *__restrict__ start,
                           int *__restrict__ cursor, int *__restrict__ pts) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell_of[i];
    int slot = atomicAdd(&cursor[c], 1);
    pts[start[c] + slot] = (int)i;
}

// mode 0: count overlap partners of i; mode 1: write them (unsorted).
template <int MODE>
__global__ void k_pairs(int64_t n, int dim, const double *__restrict__ x, const double *__restrict__ R,
                        double3 lo, double inv, int3 gd, const int *__restrict__ start,
                        const int *__restrict__ count, const int *__restrict__ pts,
                        int *__restrict__ rowcnt, const int32_t *__restrict__ rowptr,
                        int32_t *__restrict__ col) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi = x[i * dim], yi = x[i * dim + 1], zi = dim > 2 ? x[i * dim + 2] : 0.0;
    double ri = R[i];
    int cx = grid_coord(xi, lo.x, inv, gd.x), cy = grid_coord(yi, lo.y, inv, gd.y);
    int cz = dim > 2 ? grid_coord(zi, lo.z, inv, gd.z) : 0;
    int zlo = dim > 2 ? max(cz - 1, 0) : 0, zhi = dim > 2 ? min(cz + 1, gd.z - 1) : 0;
    int c = 0;
    int32_t base = MODE ? rowptr[i] : 0;
    for (int z = zlo; z <= zhi; ++z)
        for (int y = max(cy - 1, 0); y <= min(cy + 1, gd.y - 1); ++y)
            for (int xx = max(cx - 1, 0); xx <= min(cx + 1, gd.x - 1); ++xx) {
                int cell = (z * gd.y + y) * gd.x + xx;
                int s = start[cell], e = s + count[cell];
                for (int p = s; p < e; ++p) {
                    int j = pts[p];
                    double dx = x[(int64_t)j * dim] - xi, dy = x[(int64_t)j * dim + 1] - yi;
                    double d2 = dx * dx + dy * dy;
                    if (dim > 2) {
                        double dz = x[(int64_t)j * dim + 2] - zi;
                        d2 += dz * dz;
                    }
                    if (sqrt(d2) < ri + R[j]) {
                        if (MODE) col[base + c] = j;
                        ++c;
                    }
                }
            }
    if (!MODE) rowcnt[i] = c;
}

__global__ void k_sort_rows(int64_t n, const int32_t *__restrict__ rowptr, int32_t *__restrict__ col,
                            int32_t *__restrict__ diag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t s = rowptr[i], e = rowptr[i + 1];
    for (int32_t a = s + 1; a < e; ++a) {
        int32_t v = col[a], b = a - 1;
        while (b >= s && col[b] > v) {
            col[b + 1] = col[b];
            --b;
        }
        col[b + 1] = v;
    }
    int32_t d = -1;
    for (int32_t a = s; a < e; ++a)
        if (col[a] == (int32_t)i) d = a;
    diag[i] = d;
}

// Exclusive scan of n ints in one block; out has n + 1 entries; total also in *tot.
__global__ void k_scan(int64_t n, const int *__restrict__ in, int32_t *__restrict__ out,
                       long long *__restrict__ tot) {
    __shared__ long long part[1024];
    int t = threadIdx.x, T = blockDim.x;
    int64_t chunk = (n + T - 1) / T;
    int64_t a = t * chunk, b = min(n, a + chunk);
    long long s = 0;
    for (int64_t k = a; k < b; ++k) s += in[k];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {  // inclusive Hillis-Steele over the block
        long long v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = part[t] - s;
    for (int64_t k = a; k < b; ++k) {
        out[k] = (int32_t)run;
        run += in[k];
    }
    if (t == T - 1) {
        out[n] = (int32_t)part[T - 1];
        *tot = part[T - 1];
    }
}

}  // namespace

mlpg_status run_neighbors(mlpg_ctx *ctx) {
    const int64_t n = ctx->n;
    const int dim = ctx->dim;
    double rmax = 0.0;
    for (double r : ctx->h_R) rmax = std::max(rmax, r);
    double g = 2.0 * rmax;
    int gd[3] = {1, 1, 1};
    int64_t ncell = 1;
    for (int a = 0; a < dim; ++a) {
        double span = ctx->opt.hi[a] - ctx->opt.lo[a];
        gd[a] = std::max(1, (int)std::ceil(span / g));
        ncell *= gd[a];
    }
    while (ncell > (1 << 22)) {  // keep the bin table small for tiny supports
        g *= 2.0;
        ncell = 1;
        for (int a = 0; a < dim; ++a) {
            gd[a] = std::max(1, (int)std::ceil((ctx->opt.hi[a] - ctx->opt.lo[a]) / g));
            ncell *= gd[a];
        }
    }
    cudaStream_t s = ctx->stream;
    int *cell_of, *cell_count, *cell_start, *cursor, *pts, *rowcnt;
    long long *dtot;
    MLPG_TRY(dalloc(ctx, &cell_of, n));
    MLPG_TRY(dalloc(ctx, &cell_count, ncell));
    MLPG_TRY(dalloc(ctx, &cell_start, ncell + 1));
    MLPG_TRY(dalloc(ctx, &cursor, ncell));
    MLPG_TRY(dalloc(ctx, &pts, n));
    MLPG_TRY(dalloc(ctx, &rowcnt, n));
    MLPG_TRY(dalloc(ctx, &dtot, 2));
    CU(ctx, cudaMemsetAsync(cell_count, 0, ncell * sizeof(int), s));
    CU(ctx, cudaMemsetAsync(cursor, 0, ncell * sizeof(int), s));
    double3 lo = make_double3(ctx->opt.lo[0], ctx->opt.lo[1], ctx->opt.lo[2]);
    int3 g3 = make_int3(gd[0], gd[1], gd[2]);
    double inv = 1.0 / g;
    int B = 256;
    int64_t G = (n + B - 1) / B;
    k_bin<<<G, B, 0, s>>>(n, dim, ctx->x, lo, inv, g3, cell_of, cell_count);
    CU_LAUNCH(ctx);
    k_scan<<<1, 1024, 0, s>>>(ncell, cell_count, (int32_t *)cell_start, dtot);
    CU_LAUNCH(ctx);
    k_bin_fill<<<G, B, 0, s>>>(n, cell_of, cell_start, cursor, pts);
    CU_LAUNCH(ctx);
    k_pairs<0><<<G, B, 0, s>>>(n, dim, ctx->x, ctx->R, lo, inv, g3, cell_start, cell_count, pts, rowcnt,
                               nullptr, nullptr);
    CU_LAUNCH(ctx);
    MLPG_TRY(dalloc(ctx, &ctx->rowptr, n + 1));
    k_scan<<<1, 1024, 0, s>>>(n, rowcnt, ctx->rowptr, dtot + 1);
    CU_LAUNCH(ctx);
    long long tot = 0;
    CU(ctx, cudaMemcpyAsync(&tot, dtot + 1, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    if (tot >= (1LL << 31) - 1) return set_err(ctx, MLPG_ERR_ARG, "overlap pattern exceeds 2^31 entries");
    ctx->nnz = tot;
    MLPG_TRY(dalloc(ctx, &ctx->col, tot));
    MLPG_TRY(dalloc(ctx, &ctx->diag, n));
    k_pairs<1><<<G, B, 0, s>>>(n, dim, ctx->x, ctx->R, lo, inv, g3, cell_start, cell_count, pts, nullptr,
                               ctx->rowptr, ctx->col);
    CU_LAUNCH(ctx);
    k_sort_rows<<<G, B, 0, s>>>(n, ctx->rowptr, ctx->col, ctx->diag);
    CU_LAUNCH(ctx);
    ctx->h_rowptr.resize(n + 1);
    ctx->h_col.resize(tot);
    CU(ctx, cudaMemcpyAsync(ctx->h_rowptr.data(), ctx->rowptr, (n + 1) * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaMemcpyAsync(ctx->h_col.data(), ctx->col, tot * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    return MLPG_OK;
}

}  // namespace mlpg
