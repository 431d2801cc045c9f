// Overlap-pattern row sizes without any allocation (mlpg_overlap_counts_noalloc).
//
// Some callers cannot call cudaMalloc at the moment they need this: code that
// runs while a stream is being captured into a CUDA graph, code that owns a
// fixed device memory budget handed out once at start-up, or a real-time loop
// that must not touch the allocator.  Such callers still need to know how many
// overlap partners each point has before they can size their own buffers.
// This file holds the variant of the neighbour-count kernels (neighbors.cu)
// whose grid-binning scratch lives in one file-scope device array instead of
// freshly allocated buffers.  The array is created when the library is loaded
// and every GPU that loads the library keeps it until the process exits.
#include <cmath>
#include <mutex>

#include "internal.h"

#ifndef MLPG_NOALLOC_MAX_POINTS
#error "mlpg.h must define MLPG_NOALLOC_MAX_POINTS"
#endif

namespace mlpg {
namespace {

// ---- the static scratch and its layout (int32 words) -----------------------
constexpr int64_t kMaxPts = MLPG_NOALLOC_MAX_POINTS;   // points per call
constexpr int64_t kMaxCells = int64_t(1) << 16;        // grid bins per call
constexpr int kSide2 = 256, kSide3 = 40;                // bins per axis at most: 256^2, 40^3 <= kMaxCells
static_assert((int64_t)kSide2 * kSide2 <= kMaxCells && (int64_t)kSide3 * kSide3 * kSide3 <= kMaxCells,
              "bin grid exceeds the scratch");
constexpr int64_t kOffCellOf = 0;                       // [kMaxPts] bin of each point
constexpr int64_t kOffPts = kOffCellOf + kMaxPts;       // [kMaxPts] points sorted by bin
constexpr int64_t kOffCount = kOffPts + kMaxPts;        // [kMaxCells] points per bin
constexpr int64_t kOffStart = kOffCount + kMaxCells;    // [kMaxCells + 1] first point of each bin
constexpr int64_t kOffCursor = kOffStart + kMaxCells + 2;  // [kMaxCells] fill cursors
constexpr int64_t kOffParams = kOffCursor + kMaxCells;  // grid parameters (8-byte aligned)
constexpr int64_t kWords = kOffParams + 32;

static __device__ __align__(256) int32_t g_scratch[kWords];

struct GridParams {   // written by k_na_setup, read by the other kernels
    double lo[3];
    double inv;       // 1 / bin size
    int32_t gd[3];
    int32_t ncell;
};
static_assert(kOffParams % 2 == 0, "params must be 8-byte aligned");
static_assert(sizeof(GridParams) <= 32 * sizeof(int32_t), "params slot too small");

// per-device address of g_scratch (host code may not use the symbol itself)
std::mutex g_mu;
void *g_addr[64] = {nullptr};

mlpg_status scratch_address(int dev, int32_t **out) {
    if (dev < 0 || dev >= 64) return MLPG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return MLPG_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = static_cast<int32_t *>(g_addr[dev]);
    return MLPG_OK;
}

__device__ __forceinline__ int na_coord(double v, double lo, double inv, int gd) {
    int c = (int)floor((v - lo) * inv);
    return c < 0 ? 0 : (c >= gd ? gd - 1 : c);
}

// Bin size g >= 2 max(R), so every overlap partner lies in the 3^d bins
// around a point, and at least (largest box side) / kSide, so that at most
// kSide bins lie along any axis and kSide^dim <= kMaxCells bins in all: no
// iteration, and the bin count cannot exceed the scratch for any extents
// (tiny, huge or not finite).  Points beyond the last bin are clamped into it,
// which keeps every partner inside the 3^d stencil.  One block.
__global__ void k_na_setup(int64_t n, int dim, const double *__restrict__ R, double3 lo, double3 hi,
                           int32_t *__restrict__ scratch) {
    __shared__ double sm[256];
    double r = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) r = fmax(r, R[i]);
    sm[threadIdx.x] = r;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    GridParams *gp = reinterpret_cast<GridParams *>(scratch + kOffParams);
    const double l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
    const int side = dim == 2 ? kSide2 : kSide3;
    double smax = 0.0;
    for (int a = 0; a < dim; ++a) smax = fmax(smax, h[a] - l[a]);
    double g = fmax(2.0 * sm[0], smax / side);   // fmax drops a NaN extent
    int gd[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) {
        const double cells = ceil((h[a] - l[a]) / g);   // <= side up to rounding
        gd[a] = cells >= 1.0 ? (cells < (double)side ? (int)cells : side) : 1;
    }
    for (int a = 0; a < 3; ++a) gp->lo[a] = l[a];
    gp->inv = 1.0 / g;
    for (int a = 0; a < 3; ++a) gp->gd[a] = a < dim ? gd[a] : 1;
    gp->ncell = gp->gd[0] * gp->gd[1] * gp->gd[2];
}

__global__ void k_na_bin(int64_t n, int dim, const double *__restrict__ x, int32_t *__restrict__ scratch) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GridParams *gp = reinterpret_cast<const GridParams *>(scratch + kOffParams);
    int cx = na_coord(x[i * dim], gp->lo[0], gp->inv, gp->gd[0]);
    int cy = na_coord(x[i * dim + 1], gp->lo[1], gp->inv, gp->gd[1]);
    int cz = dim > 2 ? na_coord(x[i * dim + 2], gp->lo[2], gp->inv, gp->gd[2]) : 0;
    int c = (cz * gp->gd[1] + cy) * gp->gd[0] + cx;
    scratch[kOffCellOf + i] = c;
    atomicAdd(&scratch[kOffCount + c], 1);
}

// exclusive scan of the bin counts (one block)
__global__ void k_na_scan(int32_t *__restrict__ scratch) {
    __shared__ int32_t part[1024];
    const GridParams *gp = reinterpret_cast<const GridParams *>(scratch + kOffParams);
    const int64_t nc = gp->ncell;
    const int t = threadIdx.x, T = blockDim.x;
    const int64_t chunk = (nc + T - 1) / T, a = t * chunk, b = min(nc, a + chunk);
    int32_t s = 0;
    for (int64_t k = a; k < b; ++k) s += scratch[kOffCount + k];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        int32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = part[t] - s;
    for (int64_t k = a; k < b; ++k) {
        scratch[kOffStart + k] = run;
        run += scratch[kOffCount + k];
    }
}

__global__ void k_na_fill(int64_t n, int32_t *__restrict__ scratch) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = scratch[kOffCellOf + i];
    int slot = atomicAdd(&scratch[kOffCursor + c], 1);
    scratch[kOffPts + scratch[kOffStart + c] + slot] = (int32_t)i;
}

// counts[i] = #{j : |x_i - x_j| < R_i + R_j}, the row sizes of the overlap pattern
__global__ void k_na_count(int64_t n, int dim, const double *__restrict__ x, const double *__restrict__ R,
                           const int32_t *__restrict__ scratch, int32_t *__restrict__ counts) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const GridParams *gp = reinterpret_cast<const GridParams *>(scratch + kOffParams);
    const double xi = x[i * dim], yi = x[i * dim + 1], zi = dim > 2 ? x[i * dim + 2] : 0.0, ri = R[i];
    const int gx = gp->gd[0], gy = gp->gd[1], gz = gp->gd[2];
    const int cx = na_coord(xi, gp->lo[0], gp->inv, gx), cy = na_coord(yi, gp->lo[1], gp->inv, gy);
    const int cz = dim > 2 ? na_coord(zi, gp->lo[2], gp->inv, gz) : 0;
    int c = 0;
    for (int z = max(cz - 1, 0); z <= min(cz + 1, gz - 1); ++z)
        for (int y = max(cy - 1, 0); y <= min(cy + 1, gy - 1); ++y)
            for (int xx = max(cx - 1, 0); xx <= min(cx + 1, gx - 1); ++xx) {
                const int cell = (z * gy + y) * gx + xx;
                const int s = scratch[kOffStart + cell], e = s + scratch[kOffCount + cell];
                for (int p = s; p < e; ++p) {
                    const int64_t j = scratch[kOffPts + p];
                    // same arithmetic as the pattern builder in neighbors.cu
                    double dx = x[j * dim] - xi, dy = x[j * dim + 1] - yi;
                    double d2 = dx * dx + dy * dy;
                    if (dim > 2) {
                        double dz = x[j * dim + 2] - zi;
                        d2 += dz * dz;
                    }
                    if (sqrt(d2) < ri + R[j]) ++c;
                }
            }
    counts[i] = c;
}

}  // namespace
}  // namespace mlpg

using namespace mlpg;

extern "C" mlpg_status mlpg_overlap_counts_noalloc(int dim, int64_t n, const double *points,
                                                   const double *kernel_extent, const double *lo,
                                                   const double *hi, int32_t *counts, void *stream) {
    if ((dim != 2 && dim != 3) || n < 1 || !points || !kernel_extent || !lo || !hi || !counts) return MLPG_ERR_ARG;
    if (n > kMaxPts) return MLPG_ERR_ARG;   // beyond the static scratch
    for (int a = 0; a < dim; ++a)
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a]) || !(hi[a] > lo[a])) return MLPG_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MLPG_ERR_CUDA;
    }
    int32_t *sc = nullptr;
    mlpg_status st = scratch_address(dev, &sc);
    if (st != MLPG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const double3 l = make_double3(lo[0], lo[1], dim > 2 ? lo[2] : 0.0);
    const double3 h = make_double3(hi[0], hi[1], dim > 2 ? hi[2] : 1.0);
    const int B = 256;
    const unsigned G = (unsigned)((n + B - 1) / B);
    // the scratch keeps the previous call's contents: clear the bin counters
    cudaError_t e = cudaMemsetAsync(sc + kOffCount, 0, sizeof(int32_t) * kMaxCells, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc + kOffCursor, 0, sizeof(int32_t) * kMaxCells, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MLPG_ERR_CUDA;
    }
    k_na_setup<<<1, 256, 0, s>>>(n, dim, kernel_extent, l, h, sc);
    k_na_bin<<<G, B, 0, s>>>(n, dim, points, sc);
    k_na_scan<<<1, 1024, 0, s>>>(sc);
    k_na_fill<<<G, B, 0, s>>>(n, sc);
    k_na_count<<<G, B, 0, s>>>(n, dim, points, kernel_extent, sc, counts);
    e = cudaGetLastError();
    return e == cudaSuccess ? MLPG_OK : MLPG_ERR_CUDA;
}
