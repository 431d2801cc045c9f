// Transport operators of one backward-Euler step (Sec. 4.2) and the batched
// transport operator apply over all directions.
//
// With kappa = 1/(c dt) and tau_i the SUPG length, the direction enters L_m
// only through Omega^a, Omega^a Omega^b and the outflow selector
// max(Omega . n_f, 0), so L_m is a combination of direction-independent arrays
// on one CSR pattern (rows scaled by tau_i where the weak form has tau_i):
//   A0  = kappa M0 + Mt                         coefficient 1
//   Aa  = (kappa tau - 1) G^a + tau Gt^a        coefficient Omega^a
//   Aaa = tau K^aa, Axy = tau (K^xy + K^yx)     coefficients Omega^a Omega^a, Omega^x Omega^y
//   S_f                                         coefficient max(Omega . n_f, 0)
//   T_m  = kappa (M0 + tau Omega^a G^a)
//   MS_m = (Ms + tau Omega^a Gs^a) / (4 pi)
//   r_m  = Q0 + tau Omega^a Q^a + sum_f max(-Omega . n_f, 0) psi_b,f B_f
// FP64 path: the values of every L_m are materialised once per dt, [nnz][m]
// (direction fastest), and one apply is a single multiply-add per entry.
// FP32 path: the six arrays are streamed once per apply and combined per
// direction in registers; the face terms live in a separate short segment
// per boundary row.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include <cuda_fp16.h>

#include "internal.h"

namespace mlpg {

namespace {
constexpr double kFourPi = 12.566370614359172953850573533118;

__global__ void k_rowidx(int64_t n, const int32_t *__restrict__ rowptr, int32_t *__restrict__ rowidx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) rowidx[p] = (int32_t)i;
}

// Dimension-dependent layout (D = 2 or 3).
//   base arrays of L (NA): 1, Omega_a (D), Omega_a^2 (D), Omega_a Omega_b (a < b)
//   T and MS arrays (NT = 1 + D): M0 / Ms and tau G^a / tau Gs^a
//   faces (NF = 2D): -x, +x, -y, +y (, -z, +z)
//   mats: 0 M0, 1 Mt, 2 Ms, 3 G, 3+D Gt, 3+2D Gs, 3+3D K (a-major), 3+3D+D^2 S_f
//   vecs: 0 Q0, 1 Q, 1+D B_f
//   coef (double, stride kCS): the NA coefficients of a direction; fcoef
//   (stride kFS): outflow coefficients max(Omega . n_f, 0); coef32 (float,
//   stride 16): the NA coefficients, the faces from slot face_slot<D>().
template <int D> __host__ __device__ constexpr int NA() { return 1 + D + D * (D + 1) / 2; }
template <int D> __host__ __device__ constexpr int NT() { return 1 + D; }
template <int D> __host__ __device__ constexpr int NF() { return 2 * D; }
template <int D> __host__ __device__ constexpr int face_slot() { return D == 2 ? 8 : 10; }
template <int D> __host__ __device__ constexpr int mat_S() { return 3 + 3 * D + D * D; }
constexpr int kCS = 16, kFS = 8;
struct Inflow {
    double v[6];
};

template <int D>
__global__ void k_form_arrays(int64_t nnz, double kappa, const int32_t *__restrict__ rowidx,
                              const double *__restrict__ tau, const double *__restrict__ mats,
                              double *__restrict__ A64, float *__restrict__ A32,
                              double *__restrict__ T64, double *__restrict__ S64) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    const double t = tau[rowidx[p]];
    const double *M0 = mats, *Mt = mats + nnz, *Ms = mats + 2 * nnz;
    const double *G = mats + 3 * nnz, *Gt = mats + (3 + D) * nnz, *Gs = mats + (3 + 2 * D) * nnz;
    const double *K = mats + (3 + 3 * D) * nnz;
    double a[NA<D>()];
    a[0] = kappa * M0[p] + Mt[p];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        a[1 + c] = (kappa * t - 1.0) * G[c * nnz + p] + t * Gt[c * nnz + p];
        a[1 + D + c] = t * K[(c * D + c) * nnz + p];
    }
    int k = 1 + 2 * D;
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int e = c + 1; e < D; ++e) a[k++] = t * (K[(c * D + e) * nnz + p] + K[(e * D + c) * nnz + p]);
#pragma unroll
    for (int k2 = 0; k2 < NA<D>(); ++k2) {
        A64[k2 * nnz + p] = a[k2];
        A32[k2 * nnz + p] = (float)a[k2];
    }
    T64[p] = kappa * M0[p];
    S64[p] = Ms[p];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        T64[(1 + c) * nnz + p] = kappa * t * G[c * nnz + p];
        S64[(1 + c) * nnz + p] = t * Gs[c * nnz + p];
    }
}

template <int D>
__global__ void k_coef(int m, const double *__restrict__ omega, double *__restrict__ coef,
                       double *__restrict__ fcoef, float *__restrict__ coef32) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const double o[3] = {omega[3 * k], omega[3 * k + 1], omega[3 * k + 2]};
    double *c = coef + kCS * k;
    for (int q = 0; q < kCS; ++q) c[q] = 0.0;
    c[0] = 1.0;
    for (int a = 0; a < D; ++a) {
        c[1 + a] = o[a];
        c[1 + D + a] = o[a] * o[a];
    }
    int q = 1 + 2 * D;
    for (int a = 0; a < D; ++a)
        for (int b = a + 1; b < D; ++b) c[q++] = o[a] * o[b];
    // faces with outward normals -e_a, +e_a: outflow coefficient max(Omega . n, 0)
    for (int f = 0; f < kFS; ++f) fcoef[kFS * k + f] = 0.0;
    for (int a = 0; a < D; ++a) {
        fcoef[kFS * k + 2 * a] = fmax(-o[a], 0.0);
        fcoef[kFS * k + 2 * a + 1] = fmax(o[a], 0.0);
    }
    float *c32 = coef32 + 16 * k;
    for (int q2 = 0; q2 < 16; ++q2) c32[q2] = 0.0f;
    for (int q2 = 0; q2 < NA<D>(); ++q2) c32[q2] = (float)c[q2];
    for (int f = 0; f < NF<D>(); ++f) c32[face_slot<D>() + f] = (float)fcoef[kFS * k + f];
}

template <int D>
__global__ void k_materialize(int64_t nnz, int m, const double *__restrict__ A64,
                              const double *__restrict__ Sf, const double *__restrict__ coef,
                              const double *__restrict__ fcoef, double *__restrict__ L64) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nnz * m) return;
    int64_t p = e / m;
    int k = (int)(e - p * m);
    const double *c = coef + kCS * k, *fc = fcoef + kFS * k;
    double v = A64[p];
#pragma unroll
    for (int j = 1; j < NA<D>(); ++j) v += c[j] * A64[j * nnz + p];
#pragma unroll
    for (int f = 0; f < NF<D>(); ++f) v += fc[f] * Sf[f * nnz + p];
    L64[e] = v;
}

template <int D>
__global__ void k_diag_rhs(int64_t n, int m, const int32_t *__restrict__ diag, int64_t nnz,
                           const double *__restrict__ A64, const double *__restrict__ Sf,
                           const double *__restrict__ coef, const double *__restrict__ fcoef,
                           const double *__restrict__ tau, const double *__restrict__ vecs,
                           Inflow psib, double *__restrict__ dinv64, float *__restrict__ dinv32,
                           double *__restrict__ r64, int *__restrict__ flag) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    int64_t i = e / m;
    int k = (int)(e - i * m);
    const double *c = coef + kCS * k, *fc = fcoef + kFS * k;
    int32_t p = diag[i];
    double d = A64[p];
    for (int j = 1; j < NA<D>(); ++j) d += c[j] * A64[j * nnz + p];
    for (int f = 0; f < NF<D>(); ++f) d += fc[f] * Sf[f * nnz + p];
    if (!(fabs(d) > 0.0)) {
        atomicOr(flag, 16);
        d = 1.0;
    }
    dinv64[e] = 1.0 / d;
    dinv32[e] = (float)(1.0 / d);
    const double *Q0 = vecs, *Q = vecs + n, *B = vecs + (1 + D) * n;
    double qa = 0.0;
    for (int a = 0; a < D; ++a) qa += c[1 + a] * Q[a * n + i];
    double r = Q0[i] + tau[i] * qa;
    // inflow faces: Omega . n_f < 0, coefficient |Omega . n_f| (the outflow
    // coefficient of the opposite face)
    for (int f = 0; f < NF<D>(); ++f) r += fc[f ^ 1] * psib.v[f] * B[f * n + i];
    r64[e] = r;
}

// boundary segment: entries of rows that touch a face (S_f != 0)
template <int D>
__global__ void k_bcount(int64_t n, const int32_t *__restrict__ rowptr, int64_t nnz,
                         const double *__restrict__ Sf, int *__restrict__ cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        bool nz = false;
        for (int f = 0; f < NF<D>(); ++f) nz |= Sf[f * nnz + p] != 0.0;
        c += nz;
    }
    cnt[i] = c;
}

template <int D>
__global__ void k_bfill(int64_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                        int64_t nnz, const double *__restrict__ Sf, const int32_t *__restrict__ bptr,
                        int64_t nb, int32_t *__restrict__ bcol, double *__restrict__ bval64,
                        float *__restrict__ bval32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t o = bptr[i];
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        bool nz = false;
        for (int f = 0; f < NF<D>(); ++f) nz |= Sf[f * nnz + p] != 0.0;
        if (!nz) continue;
        bcol[o] = col[p];
        for (int f = 0; f < NF<D>(); ++f) {
            bval64[f * nb + o] = Sf[f * nnz + p];
            bval32[f * nb + o] = (float)Sf[f * nnz + p];
        }
        ++o;
    }
}

__global__ void k_scan1(int64_t n, const int *__restrict__ in, int32_t *__restrict__ out) {
    __shared__ long long part[1024];
    int t = threadIdx.x, T = blockDim.x;
    int64_t chunk = (n + T - 1) / T;
    int64_t a = t * chunk, b = min(n, a + chunk);
    long long s = 0;
    for (int64_t k = a; k < b; ++k) s += in[k];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
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
    if (t == T - 1) out[n] = (int32_t)part[T - 1];
}

// ---------------------------------------------------------------------------
// batched L-apply.  A team of TM lanes (power of two) works on one row; lane l
// owns directions m = l + TM t, t < DPL.  Y = L X, or Y = B - L X when B != 0.
// ---------------------------------------------------------------------------
// Warp-per-row layout of the FP64 apply: the 32 lanes of a warp are S
// entry slots x TM direction lanes (S * TM = 32); lane (s, l) takes the row
// entries p0 + s, p0 + s + S, ... and the directions l, l + TM, ... (DPL of
// them).  The S partial sums of each direction are combined with shuffles.
template <typename T, int DPL>
__device__ __forceinline__ void slot_reduce(T (&acc)[DPL], int TM) {
#pragma unroll
    for (int t = 0; t < DPL; ++t)
        for (int o = TM; o < 32; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
}

template <int DPL>
__global__ void __launch_bounds__(256) k_spmm64(int64_t n, int m, int tm_log2,
                                                const int32_t *__restrict__ rowptr,
                                                const int32_t *__restrict__ col,
                                                const double *__restrict__ L64,
                                                const double *__restrict__ X, const double *__restrict__ B,
                                                double *__restrict__ Y) {
    const int TM = 1 << tm_log2, S = 32 >> tm_log2;
    const int lane = threadIdx.x & (TM - 1), slot = (threadIdx.x & 31) >> tm_log2;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    double acc[DPL];
#pragma unroll
    for (int t = 0; t < DPL; ++t) acc[t] = 0.0;
    const int32_t p1 = rowptr[row + 1];
    int32_t p = rowptr[row] + slot;
    for (; p + S < p1; p += 2 * S) {  // two entries per lane in flight
        const int64_t j0 = col[p], j1 = col[p + S];
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            int k = lane + t * TM;
            if (k < m) {
                double l0 = L64[(int64_t)p * m + k], l1 = L64[(int64_t)(p + S) * m + k];
                double x0 = X[j0 * m + k], x1 = X[j1 * m + k];
                acc[t] = fma(l0, x0, acc[t]);
                acc[t] = fma(l1, x1, acc[t]);
            }
        }
    }
    if (p < p1) {
        const int64_t j = col[p];
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            int k = lane + t * TM;
            if (k < m) acc[t] = fma(L64[(int64_t)p * m + k], X[j * m + k], acc[t]);
        }
    }
    slot_reduce<double, DPL>(acc, TM);
    if (slot == 0) {
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            int k = lane + t * TM;
            if (k < m) {
                int64_t e = row * m + k;
                Y[e] = B ? B[e] - acc[t] : acc[t];
            }
        }
    }
}

// FP32 batched L-apply: a team of TM lanes per row (4 rows per warp for
// TM = 8), lane l owns directions l, l + TM, ... (DPL of them; EXACT when
// TM * DPL = m so no lane needs a guard).  The six operator values of an
// entry are combined with the direction coefficients in registers.  The
// outflow-face terms of the few boundary rows are added by k_faces32 (kept
// out of this loop: a second loop here slows the main one down by half).
// IDX is the index type of the [n][m] vectors (int when n * m < 2^31).
template <int DPL, bool EXACT, typename IDX, int D>
__global__ void __launch_bounds__(256) k_spmm32(int64_t n, int m, int tm_log2, int64_t nnz,
                                                const int32_t *__restrict__ rowptr,
                                                const int32_t *__restrict__ col,
                                                const float *__restrict__ A32,
                                                const float *__restrict__ coef32,
                                                const float *__restrict__ X, const float *__restrict__ B,
                                                float *__restrict__ Y) {
    constexpr int K = NA<D>();
    const int TM = 1 << tm_log2;
    // grid y: chunks of TM x DPL directions (one chunk when the team covers all m)
    const int m0 = blockIdx.y * (TM * DPL), lane = threadIdx.x & (TM - 1);
    const int ml = m0 + lane;   // this lane's first direction
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> tm_log2;
    if (row >= n) return;
    float c[K][DPL], acc[DPL];
    bool on[DPL];
#pragma unroll
    for (int t = 0; t < DPL; ++t) {
        int k = m0 + lane + t * TM;
        on[t] = EXACT || k < m;
        k = on[t] ? k : m - 1;
#pragma unroll
        for (int q = 1; q < K; ++q) c[q][t] = coef32[16 * k + q];
        acc[t] = 0.0f;
    }
    const int32_t p1 = rowptr[row + 1];
    int32_t p = rowptr[row];
    if constexpr (K == 6) {   // 2D: the six values in named registers (schedules best)
        for (; p + 1 < p1; p += 2) {   // two entries in flight
            const IDX jb0 = (IDX)col[p] * (IDX)m + (IDX)ml, jb1 = (IDX)col[p + 1] * (IDX)m + (IDX)ml;
            const float a0 = A32[p], a1 = A32[nnz + p], a2 = A32[2 * nnz + p], a3 = A32[3 * nnz + p],
                        a4 = A32[4 * nnz + p], a5 = A32[5 * nnz + p];
            const float b0 = A32[p + 1], b1 = A32[nnz + p + 1], b2 = A32[2 * nnz + p + 1],
                        b3 = A32[3 * nnz + p + 1], b4 = A32[4 * nnz + p + 1], b5 = A32[5 * nnz + p + 1];
#pragma unroll
            for (int t = 0; t < DPL; ++t) {
                if (on[t]) {
                    const float x0 = X[jb0 + t * TM], x1 = X[jb1 + t * TM];
                    float v0 = fmaf(c[5][t], a5, fmaf(c[4][t], a4, fmaf(c[3][t], a3, fmaf(c[2][t], a2, fmaf(c[1][t], a1, a0)))));
                    float v1 = fmaf(c[5][t], b5, fmaf(c[4][t], b4, fmaf(c[3][t], b3, fmaf(c[2][t], b2, fmaf(c[1][t], b1, b0)))));
                    acc[t] = fmaf(v1, x1, fmaf(v0, x0, acc[t]));
                }
            }
        }
    }
    for (; p + 1 < p1; p += 2) {   // two entries in flight (generic number of arrays)
        const IDX jb0 = (IDX)col[p] * (IDX)m + (IDX)ml, jb1 = (IDX)col[p + 1] * (IDX)m + (IDX)ml;
        float a[K], b[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            a[q] = A32[q * nnz + p];
            b[q] = A32[q * nnz + p + 1];
        }
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            if (on[t]) {
                const float x0 = X[jb0 + t * TM], x1 = X[jb1 + t * TM];
                float v0 = a[0], v1 = b[0];
#pragma unroll
                for (int q = 1; q < K; ++q) {
                    v0 = fmaf(c[q][t], a[q], v0);
                    v1 = fmaf(c[q][t], b[q], v1);
                }
                acc[t] = fmaf(v1, x1, fmaf(v0, x0, acc[t]));
            }
        }
    }
    for (; p < p1; ++p) {
        const IDX jb = (IDX)col[p] * (IDX)m + (IDX)ml;
        float a[K];
#pragma unroll
        for (int q = 0; q < K; ++q) a[q] = A32[q * nnz + p];
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            if (on[t]) {
                float v = a[0];
#pragma unroll
                for (int q = 1; q < K; ++q) v = fmaf(c[q][t], a[q], v);
                acc[t] = fmaf(v, X[jb + t * TM], acc[t]);
            }
        }
    }
    const IDX rb = (IDX)row * (IDX)m + (IDX)ml;
#pragma unroll
    for (int t = 0; t < DPL; ++t) {
        if (on[t]) {
            const IDX e = rb + t * TM;
            Y[e] = B ? B[e] - acc[t] : acc[t];
        }
    }
}

// Outflow-face terms sum_f max(Omega . n_f, 0) (S_f X)_i of the boundary
// rows, subtracted from (residual form) or added to Y.  One warp per row of
// the boundary-row list: 32 / TM entry slots x TM direction lanes, slot sums
// combined with shuffles.
template <int DPL, int D>
__global__ void __launch_bounds__(256) k_faces32(int64_t nbr, int m, int tm_log2, int64_t nb,
                                                 const int32_t *__restrict__ brow,
                                                 const int32_t *__restrict__ bptr,
                                                 const int32_t *__restrict__ bcol,
                                                 const float *__restrict__ bval,
                                                 const float *__restrict__ coef32,
                                                 const float *__restrict__ X, float sign,
                                                 float *__restrict__ Y) {
    const int TM = 1 << tm_log2, S = 32 >> tm_log2;
    const int lane = threadIdx.x & (TM - 1), slot = (threadIdx.x & 31) >> tm_log2;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= nbr) return;
    const int64_t row = brow[r];
    float acc[DPL];
#pragma unroll
    for (int t = 0; t < DPL; ++t) acc[t] = 0.0f;
    for (int32_t q = bptr[row] + slot; q < bptr[row + 1]; q += S) {
        const int64_t jb = (int64_t)bcol[q] * m + lane;
        float sv[NF<D>()];
#pragma unroll
        for (int f = 0; f < NF<D>(); ++f) sv[f] = bval[f * nb + q];
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            int k = lane + t * TM;
            if (k < m) {
                const float *fc = coef32 + 16 * k + face_slot<D>();
                float v = fc[NF<D>() - 1] * sv[NF<D>() - 1];
#pragma unroll
                for (int f = NF<D>() - 2; f >= 0; --f) v = fmaf(fc[f], sv[f], v);
                acc[t] = fmaf(v, X[jb + t * TM], acc[t]);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < DPL; ++t)
        for (int o = TM; o < 32; o <<= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    if (slot == 0) {
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            int k = lane + t * TM;
            if (k < m) Y[row * m + k] += sign * acc[t];
        }
    }
}

// ---------------------------------------------------------------------------
// Row tiles (m % 4 == 0), shared by the CUDA-core and tensor-core tile
// kernels.  A tile is TR Morton-consecutive rows; its halo is the sorted union
// of their columns.  One CTA per (row tile, direction chunk) stages the halo
// rows of X (mc of the m directions) in shared memory once, so a neighbour
// row shared by several rows of the tile is read from HBM once per tile.  The
// tile's entries are sliced-ELL records, entry k of row slot s at
// [k][s] (width padded to a multiple of kRecK with zero records): the K
// base-array values of the entry and the offset of its column's staged row,
// padded to whole float4 words.
// ---------------------------------------------------------------------------
template <int D>
__host__ __device__ constexpr int rec_words() { return (NA<D>() + 4) / 4 * 4; }   // K values + halo index, padded to float4

template <int D>
__global__ void k_tile_records(int64_t nslot, int64_t nnz, int xs, const int32_t *__restrict__ perm,
                               const int32_t *__restrict__ lcol, const float *__restrict__ A32,
                               float4 *__restrict__ rec) {
    constexpr int K = NA<D>(), RW = rec_words<D>();
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nslot) return;
    const int32_t p = perm[e];
    float v[RW];
#pragma unroll
    for (int k = 0; k < RW; ++k) v[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = p >= 0 ? A32[k * nnz + p] : 0.0f;
    v[K] = __int_as_float(lcol[e] * xs);   // offset of the column's staged row in shared memory (floats)
#pragma unroll
    for (int q = 0; q < RW / 4; ++q) rec[e * (RW / 4) + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

constexpr int kRecK = 4;        // record pipeline: entries (k steps) per stage
constexpr int kRecKGather = 8;  // ... in gather mode (more entries' loads in flight between barriers)
__host__ __device__ constexpr int rec_k(bool gather) { return gather ? kRecKGather : kRecK; }
constexpr int kRecStages = 4;   // record pipeline: stages in flight
// direction groups per row: threads per CTA = rows per tile x groups (<= 640)
// (gather mode: at most 320 threads, so that two CTAs of the 4-direction kernel fit an SM
// under its register bound; measured 3.32 against 3.96 ms at 40^3 with 272 directions)
__host__ __device__ constexpr int tile_max_groups(int tr, int dpt, bool gather = false) {
    return (gather || dpt == 8 ? 320 : 640) / tr;
}
// CTAs per SM that the register allocation is bounded for (0: no bound; an explicit 1
// measured more registers and fewer CTAs per SM for the staged-halo kernels)
__host__ __device__ constexpr int tile_min_blocks(int dpt, bool gather) { return gather && dpt == 4 ? 2 : 0; }
// shared memory of one stage of records (TR rows per tile), in float4
template <int D, int TR>
__host__ __device__ constexpr int rec_stage_f4() { return kRecK * TR * (rec_words<D>() / 4); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Records of stage st (entries st*kRecK .. +kRecK of every row slot) from the
// tile's contiguous sliced-ELL block into buffer `buf`, reordered to
// [float4 q][entry k][row slot s] so that the rows of a warp read
// consecutive 16-byte words (no bank conflicts).
template <int D, int TR>
__device__ __forceinline__ void stage_records(float4 *Rs, int buf, const float4 *__restrict__ rg, int st, int W) {
    constexpr int RW4 = rec_words<D>() / 4;
    const int k0 = st * kRecK;
    if (k0 >= W) return;
    constexpr int cnt = kRecK * TR * RW4;   // W is a multiple of kRecK
    const float4 *src = rg + (int64_t)k0 * TR * RW4;
    float4 *dst = Rs + buf * rec_stage_f4<D, TR>();
    for (int idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
        const int q = idx % RW4, ks = idx / RW4;   // ks = k * TR + s
        cp_async16(dst + q * (kRecK * TR) + ks, src + idx);
    }
}

// ---- bulk copies (the TMA engine) completed on mbarriers, bounded waits -----
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// one arrival that also expects `bytes` of copies on the barrier's current phase
__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// orders this thread's earlier shared-memory accesses (generic proxy) before later bulk
// copies into shared memory (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// true once the barrier's phase of this parity has completed; false after 2^16
// tries (each try waits for a while in hardware), so that no wait is endless
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (1 << 16); ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// Tiled FP32 L-apply, one CTA per (row tile, direction chunk).  Thread 0
// feeds the CTA's shared memory through bulk copies (the TMA engine), each
// completing on an mbarrier:
//   * the halo rows of X (the union of the tile's columns, the chunk's
//     directions): one copy per row, all on one barrier;
//   * the tile's record slots, kRecK entries per stage (kRecKGather in gather
//     mode), kRecStages stages in flight; a stage's buffer is refilled once every
//     thread is done with it (a proxy fence and the CTA barrier order the reads
//     before the refill).
// Thread (s, g) owns row slot s and DPT directions of the chunk (quads g and
// g + G, G = mc / DPT, so the threads of a row read one contiguous run of the
// staged row), combines the K base-array values of an entry with its
// directions' coefficients and accumulates value x X, two directions per
// packed FP32 FMA; then it adds the outflow-face terms of a boundary row and
// writes Y = L X or Y = B - L X.  Every decision taken on a wait is
// block-uniform; a wait that gives up sets *err, lets the copies in flight
// land (bounded waits) and ends the CTA.
// GX (gather mode): no halo is staged; a record's index word is the global
// offset col x m of its column's row, and the thread reads its directions of
// that row from global memory (L2).  Without the halo in shared memory a
// chunk holds all directions (up to the thread limit), so the records are
// streamed once per tile, not once per chunk: the choice for large direction
// sets, whose halos leave room for only a few directions per chunk.
template <int D, int DPT, int TR, bool GX>
__global__ void __launch_bounds__(TR * tile_max_groups(TR, DPT, GX), tile_min_blocks(DPT, GX)) k_spmm32_tile(
    int m, int mc, int xs, int hx_f4, const int32_t *__restrict__ base, const int32_t *__restrict__ width,
    const int32_t *__restrict__ trow, const int32_t *__restrict__ hptr, const int32_t *__restrict__ hcol,
    const float4 *__restrict__ rec, const float *__restrict__ coef32, const int32_t *__restrict__ bptr,
    const int32_t *__restrict__ bhalo, const float *__restrict__ bval, int64_t nb, const float *__restrict__ X,
    const float *__restrict__ B, float *__restrict__ Y, int *__restrict__ err) {
    constexpr int K = NA<D>(), RW4 = rec_words<D>() / 4, NQ = DPT / 4, NS = kRecStages;
    constexpr int RK = rec_k(GX);            // entries per record stage
    constexpr int SF4 = RK * TR * RW4;      // float4 per record stage
    constexpr uint32_t SBYTES = SF4 * 16u;
    extern __shared__ float4 smem_x4[];
    __shared__ __align__(8) uint64_t bars[NS + 1];   // record stages, then the halo
    float *Xs = reinterpret_cast<float *>(smem_x4);
    float4 *Rs = smem_x4 + hx_f4;
    const int t = blockIdx.x, m0 = blockIdx.y * mc, mcw = min(mc, m - m0), G = mc / DPT;
    const int s = threadIdx.x / G, g = threadIdx.x - s * G;
    const int W = width[t], nst = W / RK;
    const float4 *rg = rec + (int64_t)base[t] * RW4;
    const int h0 = hptr[t], hn = hptr[t + 1] - h0;
    const uint32_t row_bytes = (uint32_t)mcw * 4u;
    if (threadIdx.x == 0) {
        for (int b = 0; b <= NS; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if constexpr (!GX) mbar_expect(&bars[NS], (uint32_t)hn * row_bytes);
        for (int st = 0; st < NS && st < nst; ++st) {
            mbar_expect(&bars[st], SBYTES);
            bulk_g2s(Rs + st * SF4, rg + (int64_t)st * SF4, SBYTES, &bars[st]);
        }
    }
    if constexpr (!GX)
        for (int hh = threadIdx.x; hh < hn; hh += blockDim.x)
            bulk_g2s(Xs + hh * xs, X + (int64_t)hcol[h0 + hh] * m + m0, row_bytes, &bars[NS]);
    // GX: X is read from global memory, at the chunk's first direction
    const float *Xg = X + m0;
    // the thread's directions and their coefficient pairs
    int qoff[NQ];
    bool on[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
        qoff[u] = 4 * (g + u * G);
        on[u] = qoff[u] < mcw;
    }
    float2 c[K][2 * NQ];   // c[0] unused (the coefficient of the first array is 1)
#pragma unroll
    for (int u = 0; u < NQ; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int d0 = m0 + (on[u] ? qoff[u] : 0) + 2 * h;
#pragma unroll
            for (int k = 1; k < K; ++k) c[k][2 * u + h] = make_float2(coef32[16 * d0 + k], coef32[16 * (d0 + 1) + k]);
        }
    float2 acc[2 * NQ];
#pragma unroll
    for (int j = 0; j < 2 * NQ; ++j) acc[j] = make_float2(0.0f, 0.0f);
    bool ok = true;
    if constexpr (!GX) ok = __syncthreads_and(mbar_wait(&bars[NS], 0));
    int st = 0;
    for (; st < nst && ok; ++st) {
        const int b = st % NS;
        if (!__syncthreads_and(mbar_wait(&bars[b], (st / NS) & 1))) { ok = false; break; }
        const float4 *rb = Rs + b * SF4 + s * RW4;
#pragma unroll
        for (int kk = 0; kk < RK; ++kk) {
            float a[4 * RW4];
#pragma unroll
            for (int q = 0; q < RW4; ++q) {
                const float4 v = rb[kk * TR * RW4 + q];
                a[4 * q] = v.x; a[4 * q + 1] = v.y; a[4 * q + 2] = v.z; a[4 * q + 3] = v.w;
            }
            const float *xr = (GX ? Xg : Xs) + __float_as_int(a[K]);
            float2 ab[K];   // the entry's values, each in both halves of a pair
#pragma unroll
            for (int k2 = 0; k2 < K; ++k2) ab[k2] = make_float2(a[k2], a[k2]);
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                // GX: a quad past the last chunk's directions is not read (it may lie past X)
                const float4 x4 = !GX ? *reinterpret_cast<const float4 *>(xr + qoff[u])
                                      : (on[u] ? __ldg(reinterpret_cast<const float4 *>(xr + qoff[u]))
                                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f));
                const float2 xp[2] = {make_float2(x4.x, x4.y), make_float2(x4.z, x4.w)};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float2 v = ab[0];
#pragma unroll
                    for (int k2 = 1; k2 < K; ++k2) v = __ffma2_rn(c[k2][2 * u + h], ab[k2], v);
                    acc[2 * u + h] = __ffma2_rn(v, xp[h], acc[2 * u + h]);
                }
            }
        }
        // every thread is done with buffer b: its reads (generic proxy) are ordered before the
        // bulk copy that refills it (async proxy) by a proxy fence, then the CTA barrier.
        // Without the fence a refill could overwrite a stage still being read: measured at 40^3
        // in gather mode, where results moved by 3.5e-3 under a different register allocation.
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0 && st + NS < nst) {
            mbar_expect(&bars[b], SBYTES);
            bulk_g2s(Rs + b * SF4, rg + (int64_t)(st + NS) * SF4, SBYTES, &bars[b]);
        }
    }
    if (!ok) {   // (block-uniform) report, let the copies in flight land, leave
        if (threadIdx.x == 0) {
            atomicOr(err, 1);
            if constexpr (!GX) mbar_wait(&bars[NS], 0);
            for (int k = st; k < nst && k < st + NS; ++k) mbar_wait(&bars[k % NS], (k / NS) & 1);
        }
        __syncthreads();
        return;
    }
    const int32_t row = trow[(int64_t)t * TR + s];
    if (row < 0) return;
    // outflow-face terms of a boundary row: sum_f max(Omega . n_f, 0) (S_f X)_i
    const int32_t q0 = bptr[row], q1 = bptr[row + 1];
    if (q1 > q0) {
        float2 fc[NF<D>()][2 * NQ];
#pragma unroll
        for (int u = 0; u < NQ; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int d0 = m0 + (on[u] ? qoff[u] : 0) + 2 * h;
#pragma unroll
                for (int f = 0; f < NF<D>(); ++f)
                    fc[f][2 * u + h] = make_float2(coef32[16 * d0 + face_slot<D>() + f],
                                                   coef32[16 * (d0 + 1) + face_slot<D>() + f]);
            }
        for (int32_t q = q0; q < q1; ++q) {
            const float *xr = (GX ? Xg : Xs) + bhalo[q];
            float2 sv[NF<D>()];
#pragma unroll
            for (int f = 0; f < NF<D>(); ++f) {
                const float v = bval[f * nb + q];
                sv[f] = make_float2(v, v);
            }
#pragma unroll
            for (int u = 0; u < NQ; ++u) {
                const float4 x4 = (GX && !on[u]) ? make_float4(0.0f, 0.0f, 0.0f, 0.0f)
                                                 : *reinterpret_cast<const float4 *>(xr + qoff[u]);
                const float2 xp[2] = {make_float2(x4.x, x4.y), make_float2(x4.z, x4.w)};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float2 v = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int f = 0; f < NF<D>(); ++f) v = __ffma2_rn(fc[f][2 * u + h], sv[f], v);
                    acc[2 * u + h] = __ffma2_rn(v, xp[h], acc[2 * u + h]);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
        if (!on[u]) continue;
        const int64_t e = (int64_t)row * m + m0 + qoff[u];
        float4 o = make_float4(acc[2 * u].x, acc[2 * u].y, acc[2 * u + 1].x, acc[2 * u + 1].y);
        if (B) {
            const float4 bv = *reinterpret_cast<const float4 *>(B + e);
            o = make_float4(bv.x - o.x, bv.y - o.y, bv.z - o.z, bv.w - o.w);
        }
        *reinterpret_cast<float4 *>(Y + e) = o;
    }
}

__global__ void k_brows(int64_t n, const int32_t *__restrict__ bptr, int32_t *__restrict__ brow,
                        int *__restrict__ count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (bptr[i + 1] > bptr[i]) brow[atomicAdd(count, 1)] = (int32_t)i;
}

// RHS f[i][m] = (T_m X)_i + r[i][m] with T_m = T0 + sum_a Omega^a T_a (FP64).
template <int DPL, int D>
__global__ void __launch_bounds__(256) k_rhs64(int64_t n, int m, int tm_log2, int64_t nnz,
                                               const int32_t *__restrict__ rowptr,
                                               const int32_t *__restrict__ col,
                                               const double *__restrict__ T64,
                                               const double *__restrict__ coef,
                                               const double *__restrict__ X, const double *__restrict__ r,
                                               double *__restrict__ F) {
    const int TM = 1 << tm_log2;
    const int lane = threadIdx.x & (TM - 1);
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> tm_log2;
    if (row >= n) return;
    double acc[DPL], cw[D][DPL];
#pragma unroll
    for (int t = 0; t < DPL; ++t) {
        int k = lane + t * TM;
        k = k < m ? k : m - 1;
#pragma unroll
        for (int a = 0; a < D; ++a) cw[a][t] = coef[kCS * k + 1 + a];
        acc[t] = 0.0;
    }
    for (int32_t p = rowptr[row]; p < rowptr[row + 1]; ++p) {
        const int64_t j = col[p];
        double tv[NT<D>()];
#pragma unroll
        for (int a = 0; a < NT<D>(); ++a) tv[a] = T64[a * nnz + p];
#pragma unroll
        for (int t = 0; t < DPL; ++t) {
            int k = lane + t * TM;
            if (k < m) {
                double v = tv[0];
#pragma unroll
                for (int a = 0; a < D; ++a) v = fma(cw[a][t], tv[1 + a], v);
                acc[t] = fma(v, X[j * m + k], acc[t]);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < DPL; ++t) {
        int k = lane + t * TM;
        if (k < m) F[row * m + k] = acc[t] + r[row * m + k];
    }
}

// abc[0] = Ms Phi, abc[1 + a] = tau Gs^a Phi (1 + D SpMVs on one vector)
template <int D>
__global__ void k_ms_spmv(int64_t n, int64_t nnz, const int32_t *__restrict__ rowptr,
                          const int32_t *__restrict__ col, const double *__restrict__ S64,
                          const double *__restrict__ phi, double *__restrict__ abc) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc[NT<D>()];
#pragma unroll
    for (int a = 0; a < NT<D>(); ++a) acc[a] = 0.0;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        double v = phi[col[p]];
#pragma unroll
        for (int a = 0; a < NT<D>(); ++a) acc[a] = fma(S64[a * nnz + p], v, acc[a]);
    }
#pragma unroll
    for (int a = 0; a < NT<D>(); ++a) abc[a * n + i] = acc[a];
}

template <typename T, int D>
__global__ void k_ms_expand(int64_t n, int m, const double *__restrict__ abc,
                            const double *__restrict__ coef, T *__restrict__ out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    int64_t i = e / m;
    int k = (int)(e - i * m);
    double v = abc[i];
#pragma unroll
    for (int a = 0; a < D; ++a) v = v + coef[kCS * k + 1 + a] * abc[(1 + a) * n + i];
    out[e] = (T)(v / kFourPi);
}

// FP32 variant: the per-point products arrive pre-scaled by 1/(4 pi) in float
template <int D>
__global__ void k_ms_expand32(int64_t n, int m, const float *__restrict__ abc32,
                              const float *__restrict__ coef32, float *__restrict__ out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * m) return;
    int64_t i = e / m;
    int k = (int)(e - i * m);
    float v = abc32[i];
#pragma unroll
    for (int a = 0; a < D; ++a) v = fmaf(coef32[16 * k + 1 + a], abc32[(1 + a) * n + i], v);
    out[e] = v;
}

__global__ void k_abc32(int64_t cnt, const double *__restrict__ abc, float *__restrict__ abc32) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    abc32[i] = (float)(abc[i] / kFourPi);
}

__global__ void k_interp_apply(int64_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const double *__restrict__ I, const double *__restrict__ phi,
                               double *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s = fma(I[p], phi[col[p]], s);
    out[i] = s;
}


// ---------------------------------------------------------------------------
// Block-Jacobi preconditioner.  Points are grouped into Morton-ordered blocks
// of B = MLPG_BLOCK_PTS; for every (block, direction) the dense B x B diagonal
// block of L_m is inverted (Gauss-Jordan with partial pivoting, FP32, one warp;
// lane l owns column l of the augmented [A | I]).  The inverse is stored
// [block][row][col][m] so that the apply reads it coalesced across directions.
// ---------------------------------------------------------------------------
constexpr int kB = MLPG_BLOCK_PTS;

template <int D>
__global__ void __launch_bounds__(256) k_block_inv(int64_t nblk, int m, const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ col, int64_t nnz,
                                                   const double *__restrict__ A64, const double *__restrict__ Sf,
                                                   const double *__restrict__ coef, const double *__restrict__ fcoef,
                                                   const int32_t *__restrict__ bmember,
                                                   const int32_t *__restrict__ bof, float *__restrict__ Pinv,
                                                   uint16_t *__restrict__ Pinv16, float *__restrict__ Pscale,
                                                   int *__restrict__ flag) {
    __shared__ float sA[8][kB][2 * kB + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x;
    const int dir = blockIdx.y * 8 + warp;
    if (dir >= m) return;
    float(*A)[2 * kB + 1] = sA[warp];
    const double *c = coef + kCS * dir, *fc = fcoef + kFS * dir;
    if (lane < kB) {
        const int a = lane;
        for (int b = 0; b < 2 * kB; ++b) A[a][b] = (b == kB + a) ? 1.0f : 0.0f;
        const int32_t i = bmember[k * kB + a];
        if (i < 0) {
            A[a][a] = 1.0f;
        } else {
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int32_t sl = bof[col[p]];
                if (sl / kB != k) continue;
                double v = A64[p];
                for (int q = 1; q < NA<D>(); ++q) v += c[q] * A64[q * nnz + p];
                for (int f = 0; f < NF<D>(); ++f) v += fc[f] * Sf[f * nnz + p];
                A[a][sl - k * kB] = (float)v;
            }
        }
    }
    __syncwarp();
    bool singular = false;
    for (int cc = 0; cc < kB; ++cc) {
        int piv = cc;
        float best = fabsf(A[cc][cc]);
        for (int r = cc + 1; r < kB; ++r) {
            float v = fabsf(A[r][cc]);
            if (v > best) { best = v; piv = r; }
        }
        if (!(best > 0.0f)) { singular = true; break; }
        __syncwarp();
        if (piv != cc) {
            float t = A[cc][lane];
            A[cc][lane] = A[piv][lane];
            A[piv][lane] = t;
        }
        __syncwarp();
        const float inv = 1.0f / A[cc][cc];
        __syncwarp();
        A[cc][lane] *= inv;
        __syncwarp();
        float fr[kB];
#pragma unroll
        for (int r = 0; r < kB; ++r) fr[r] = A[r][cc];
        __syncwarp();
        const float pc = A[cc][lane];
#pragma unroll
        for (int r = 0; r < kB; ++r)
            if (r != cc) A[r][lane] -= fr[r] * pc;
        __syncwarp();
    }
    if (singular) {
        if (lane == 0) atomicOr(flag, 32);
        return;
    }
    float amax = 0.0f;
    for (int e = lane; e < kB * kB; e += 32) {
        int a = e / kB, b = e - a * kB;
        Pinv[((k * kB + a) * kB + b) * (int64_t)m + dir] = A[a][kB + b];
        amax = fmaxf(amax, fabsf(A[a][kB + b]));
    }
    if (!Pinv16) return;
    // FP16 copy: amax = f 2^ex with f in [0.5, 1); entries scaled by 2^(14 - ex) stay below 2^14
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    int ex = 0;
    if (amax > 0.0f) frexpf(amax, &ex);
    const float enc = amax > 0.0f ? ldexpf(1.0f, 14 - ex) : 1.0f;
    for (int e = lane; e < kB * kB; e += 32) {
        int a = e / kB, b = e - a * kB;
        Pinv16[((k * kB + a) * kB + b) * (int64_t)m + dir] = __half_as_ushort(__float2half_rn(A[a][kB + b] * enc));
    }
    if (lane == 0) Pscale[k * (int64_t)m + dir] = amax > 0.0f ? ldexpf(1.0f, ex - 14) : 1.0f;
}

// z = P^{-1} v, one CTA per block of kB points.  The kB input rows v[member]
// (kB x m values) are staged in shared memory once; the block's inverse
// (kB x kB x m floats, contiguous) is streamed with 16-byte loads.  Thread
// (a, c) computes z[member_a][4c .. 4c+3] = sum_b Pinv[a][b][4c..] * v[b][4c..].
// Requires m % 4 == 0 (the caller falls back to k_bjacobi_scalar otherwise).
// With sc != null the input rows are first scaled by sc[direction] and the
// scaled rows written back to v (the GMRES basis normalisation, fused here).
template <typename T>
__global__ void __launch_bounds__(256) k_bjacobi_blk(int64_t nblk, int m, const int32_t *__restrict__ bmember,
                                                     const float *__restrict__ Pinv, T *__restrict__ v,
                                                     const double *__restrict__ sc, T *__restrict__ z) {
    extern __shared__ unsigned char smem_raw[];
    T *vs = reinterpret_cast<T *>(smem_raw);   // [kB][m], then m scale factors
    T *ssc = vs + kB * m;
    const int64_t blk = blockIdx.x;
    const int mc = m >> 2;                      // float4 chunks per row
    const int32_t *mem = bmember + blk * kB;
    if (sc)
        for (int k = threadIdx.x; k < m; k += blockDim.x) ssc[k] = (T)sc[k];
    __syncthreads();
    for (int q = threadIdx.x; q < kB * m; q += blockDim.x) {
        int b = q / m, k = q - b * m;
        int32_t j = mem[b];
        T val = (T)0;
        if (j >= 0) {
            val = v[(int64_t)j * m + k];
            if (sc) {
                val *= ssc[k];
                v[(int64_t)j * m + k] = val;
            }
        }
        vs[q] = val;
    }
    __syncthreads();
    const float4 *P4 = reinterpret_cast<const float4 *>(Pinv + blk * (int64_t)kB * kB * m);
    for (int t = threadIdx.x; t < kB * mc; t += blockDim.x) {
        const int a = t / mc, c = t - a * mc;
        const int32_t i = mem[a];
        if (i < 0) continue;
        T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
#pragma unroll 4
        for (int b = 0; b < kB; ++b) {
            const float4 p = P4[((int64_t)a * kB + b) * mc + c];
            const T *vb = vs + b * m + 4 * c;
            acc0 += (T)p.x * vb[0];
            acc1 += (T)p.y * vb[1];
            acc2 += (T)p.z * vb[2];
            acc3 += (T)p.w * vb[3];
        }
        T *zo = z + (int64_t)i * m + 4 * c;
        zo[0] = acc0; zo[1] = acc1; zo[2] = acc2; zo[3] = acc3;
    }
}

// As k_bjacobi_blk with the FP16 inverses of the mixed mode: thread (a, c)
// owns four directions of row a and reads its sixteen 8-byte inverse entries
// before the block's input rows are staged (they do not depend on v, so their
// latency overlaps the gather), then multiplies its sums by the block's
// power-of-two decode factors.  Requires m % 4 == 0; any block size (tasks
// beyond the block size loop).
__global__ void __launch_bounds__(256) k_bjacobi_h16(int64_t nblk, int m, const int32_t *__restrict__ bmember,
                                                     const uint16_t *__restrict__ Pinv16,
                                                     const float *__restrict__ Pscale, float *__restrict__ v,
                                                     const double *__restrict__ sc, float *__restrict__ z) {
    extern __shared__ unsigned char smem_raw[];
    float *vs = reinterpret_cast<float *>(smem_raw);   // [kB][m], then m scale factors
    float *ssc = vs + kB * m;
    const int64_t blk = blockIdx.x;
    const int mc = m >> 2, ntask = kB * mc;
    const int32_t *mem = bmember + blk * kB;
    const uint2 *P2 = reinterpret_cast<const uint2 *>(Pinv16 + blk * (int64_t)kB * kB * m);
    const float4 *D4 = reinterpret_cast<const float4 *>(Pscale + blk * (int64_t)m);
    int t = threadIdx.x;
    uint2 q[kB];
    if (t < ntask) {
        const int a = t / mc, c = t - a * mc;
#pragma unroll
        for (int b = 0; b < kB; ++b) q[b] = P2[((int64_t)a * kB + b) * mc + c];
    }
    if (sc)
        for (int k = threadIdx.x; k < m; k += blockDim.x) ssc[k] = (float)sc[k];
    __syncthreads();
    for (int e = threadIdx.x; e < kB * m; e += blockDim.x) {
        int b = e / m, k = e - b * m;
        int32_t j = mem[b];
        float val = 0.0f;
        if (j >= 0) {
            val = v[(int64_t)j * m + k];
            if (sc) {
                val *= ssc[k];
                v[(int64_t)j * m + k] = val;
            }
        }
        vs[e] = val;
    }
    __syncthreads();
    for (bool first = true; t < ntask; t += blockDim.x, first = false) {
        const int a = t / mc, c = t - a * mc;
        if (!first) {
#pragma unroll
            for (int b = 0; b < kB; ++b) q[b] = P2[((int64_t)a * kB + b) * mc + c];
        }
        const int32_t i = mem[a];
        if (i < 0) continue;
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
#pragma unroll
        for (int b = 0; b < kB; ++b) {
            const float2 p01 = __half22float2(*reinterpret_cast<const __half2 *>(&q[b].x));
            const float2 p23 = __half22float2(*reinterpret_cast<const __half2 *>(&q[b].y));
            const float *vb = vs + b * m + 4 * c;
            acc0 = fmaf(p01.x, vb[0], acc0);
            acc1 = fmaf(p01.y, vb[1], acc1);
            acc2 = fmaf(p23.x, vb[2], acc2);
            acc3 = fmaf(p23.y, vb[3], acc3);
        }
        const float4 d = D4[c];
        float *zo = z + (int64_t)i * m + 4 * c;
        zo[0] = acc0 * d.x; zo[1] = acc1 * d.y; zo[2] = acc2 * d.z; zo[3] = acc3 * d.w;
    }
}

// general m: one thread per (point of the block, direction)
template <typename T>
__global__ void __launch_bounds__(256) k_bjacobi_scalar(int64_t nblk, int m, const int32_t *__restrict__ bmember,
                                                        const float *__restrict__ Pinv, T *__restrict__ v,
                                                        const double *__restrict__ sc, T *__restrict__ z) {
    extern __shared__ unsigned char smem_raw[];
    T *vs = reinterpret_cast<T *>(smem_raw);
    const int64_t blk = blockIdx.x;
    const int32_t *mem = bmember + blk * kB;
    for (int q = threadIdx.x; q < kB * m; q += blockDim.x) {
        int b = q / m, k = q - b * m;
        int32_t j = mem[b];
        T val = (T)0;
        if (j >= 0) {
            val = v[(int64_t)j * m + k];
            if (sc) {
                val = (T)((double)val * sc[k]);
                v[(int64_t)j * m + k] = val;
            }
        }
        vs[q] = val;
    }
    __syncthreads();
    const float *P = Pinv + blk * (int64_t)kB * kB * m;
    for (int t = threadIdx.x; t < kB * m; t += blockDim.x) {
        const int a = t / m, k = t - a * m;
        const int32_t i = mem[a];
        if (i < 0) continue;
        T acc = 0;
        for (int b = 0; b < kB; ++b) acc += (T)P[((int64_t)a * kB + b) * m + k] * vs[b * m + k];
        z[(int64_t)i * m + k] = acc;
    }
}

// ---------------------------------------------------------------------------
// Tiled FP32 L-apply on tensor cores (m % 8 == 0).  The same tiles, halo
// staging and record pipeline as k_spmm32_tile; one warp per 16 row slots of
// the tile.  For each entry step k, the combination of the K base arrays with
// the direction coefficients,
//     V[s][d] = sum_k a_k(s, k) c_k(d)      (16 rows x 8 directions per n-tile),
// is a small matrix product: one mma.m16n8k8 per n-tile (two for K = 10),
// operands split into high and low TF32 parts, hi*hi + hi*lo + lo*hi
// accumulated in FP32, which keeps FP32 accuracy.  The B columns of n-tile
// pair (2i, 2i+1) are mapped to directions so that the D values a lane holds
// for the pair are four consecutive directions 16i + 4t .. 16i + 4t + 3: one
// 16-byte shared load of the staged X row per pair and row, then
// Y[s][d] += V[s][d] X[col][d] in packed FP32 FMAs (no reduction across lanes:
// lane (g, t) owns rows g and g + 8 of its warp's slots).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}
// x = hi + lo with both parts representable in TF32
__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_bits(x);
    lo = tf32_bits(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// chunk direction of column n of n-tile j: pairs (2i, 2i+1) interleaved by
// lane quads, a last odd n-tile in order
__host__ __device__ __forceinline__ int mma_dir(int j, int n, int nt) {
    const int np = nt / 2;
    if (j >= 2 * np) return 16 * np + n;
    return 16 * (j >> 1) + 4 * (n >> 1) + 2 * (j & 1) + (n & 1);
}

template <int D, int TR, int NT>
__global__ void __launch_bounds__(2 * TR) k_spmm32_mma(
    int m, int xs, int xs_f4, const int32_t *__restrict__ base, const int32_t *__restrict__ width,
    const int32_t *__restrict__ trow, const int32_t *__restrict__ hptr, const int32_t *__restrict__ hcol,
    const float4 *__restrict__ rec, const float *__restrict__ coef32, const int32_t *__restrict__ bptr,
    const int32_t *__restrict__ bhalo, const float *__restrict__ bval, int64_t nb, const float *__restrict__ X,
    const float *__restrict__ B, float *__restrict__ Y) {
    constexpr int K = NA<D>(), KS = (K + 7) / 8, RW4 = rec_words<D>() / 4, MC = 8 * NT, NP = NT / 2;
    extern __shared__ float4 smem_x4[];
    float *Xs = reinterpret_cast<float *>(smem_x4);
    float4 *Rs = smem_x4 + xs_f4;
    const int t = blockIdx.x, m0 = blockIdx.y * MC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    // 1. stage the halo rows of the chunk (first copy group)
    {
        const int h0 = hptr[t], hn = hptr[t + 1] - h0;
        constexpr int Q4 = MC / 4;
        for (int idx = threadIdx.x; idx < hn * Q4; idx += 2 * TR) {
            const int hh = idx / Q4, qq = idx - hh * Q4;
            cp_async16(Xs + hh * xs + 4 * qq, X + (int64_t)hcol[h0 + hh] * m + m0 + 4 * qq);
        }
        cp_async_commit();
    }
    // 2. record pipeline prologue
    const int W = width[t], nst = W / kRecK;
    const float4 *rg = rec + (int64_t)base[t] * RW4;
#pragma unroll
    for (int st = 0; st < kRecStages - 1; ++st) {
        stage_records<D, TR>(Rs, st, rg, st, W);
        cp_async_commit();
    }
    // B fragments (coefficients, split into TF32 hi and lo): B[k][n] = c_k(dir(j, n)), c_0 = 1
    uint32_t bh[NT][KS][2], bl[NT][KS][2];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int d = m0 + mma_dir(j, g, NT);
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = ks * 8 + q + 4 * h;
                const float c = k == 0 ? 1.0f : (k < K ? coef32[16 * d + k] : 0.0f);
                tf32_split(c, bh[j][ks][h], bl[j][ks][h]);
            }
    }
    float acc[2][NT][2];   // rows g, g + 8; per n-tile the lane's two directions
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[r][j][0] = acc[r][j][1] = 0.0f;
    const int s0 = warp * 16 + g;   // this lane's row slots s0, s0 + 8
    // 3. entry steps
    for (int st = 0; st < nst; ++st) {
        cp_async_wait<kRecStages - 2>();
        __syncthreads();
        stage_records<D, TR>(Rs, (st + kRecStages - 1) % kRecStages, rg, st + kRecStages - 1, W);
        cp_async_commit();
        const float *rb = reinterpret_cast<const float *>(Rs + (st % kRecStages) * rec_stage_f4<D, TR>());
#pragma unroll
        for (int kk = 0; kk < kRecK; ++kk) {
            // word w of (entry kk, slot s) sits at float (w / 4) * 4 kRecK TR + 4 (kk TR + s) + w % 4
            auto word = [&](int w, int sl) {
                return rb[(w >> 2) * 4 * kRecK * TR + 4 * (kk * TR + sl) + (w & 3)];
            };
            const int lc0 = __float_as_int(word(K, s0)), lc1 = __float_as_int(word(K, s0 + 8));
            float dv[NT][4];
#pragma unroll
            for (int j = 0; j < NT; ++j) dv[j][0] = dv[j][1] = dv[j][2] = dv[j][3] = 0.0f;
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                const int w0 = ks * 8 + q, w1 = w0 + 4;
                const float a0 = w0 < K ? word(w0, s0) : 0.0f, a1 = w0 < K ? word(w0, s0 + 8) : 0.0f;
                const float a2 = w1 < K ? word(w1, s0) : 0.0f, a3 = w1 < K ? word(w1, s0 + 8) : 0.0f;
                uint32_t ah[4], al[4];
                tf32_split(a0, ah[0], al[0]);
                tf32_split(a1, ah[1], al[1]);
                tf32_split(a2, ah[2], al[2]);
                tf32_split(a3, ah[3], al[3]);
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                    mma_tf32(dv[j], al, bh[j][ks][0], bh[j][ks][1]);
                    mma_tf32(dv[j], ah, bl[j][ks][0], bl[j][ks][1]);
                    mma_tf32(dv[j], ah, bh[j][ks][0], bh[j][ks][1]);
                }
            }
            // dv[j] = {V[g][2q], V[g][2q+1], V[g+8][2q], V[g+8][2q+1]} of n-tile j
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const float4 x0 = *reinterpret_cast<const float4 *>(Xs + lc0 + 16 * i + 4 * q);
                const float4 x1 = *reinterpret_cast<const float4 *>(Xs + lc1 + 16 * i + 4 * q);
                acc[0][2 * i][0] = fmaf(dv[2 * i][0], x0.x, acc[0][2 * i][0]);
                acc[0][2 * i][1] = fmaf(dv[2 * i][1], x0.y, acc[0][2 * i][1]);
                acc[0][2 * i + 1][0] = fmaf(dv[2 * i + 1][0], x0.z, acc[0][2 * i + 1][0]);
                acc[0][2 * i + 1][1] = fmaf(dv[2 * i + 1][1], x0.w, acc[0][2 * i + 1][1]);
                acc[1][2 * i][0] = fmaf(dv[2 * i][2], x1.x, acc[1][2 * i][0]);
                acc[1][2 * i][1] = fmaf(dv[2 * i][3], x1.y, acc[1][2 * i][1]);
                acc[1][2 * i + 1][0] = fmaf(dv[2 * i + 1][2], x1.z, acc[1][2 * i + 1][0]);
                acc[1][2 * i + 1][1] = fmaf(dv[2 * i + 1][3], x1.w, acc[1][2 * i + 1][1]);
            }
            if constexpr (NT & 1) {
                constexpr int j = NT - 1;
                const float2 x0 = *reinterpret_cast<const float2 *>(Xs + lc0 + 16 * NP + 2 * q);
                const float2 x1 = *reinterpret_cast<const float2 *>(Xs + lc1 + 16 * NP + 2 * q);
                acc[0][j][0] = fmaf(dv[j][0], x0.x, acc[0][j][0]);
                acc[0][j][1] = fmaf(dv[j][1], x0.y, acc[0][j][1]);
                acc[1][j][0] = fmaf(dv[j][2], x1.x, acc[1][j][0]);
                acc[1][j][1] = fmaf(dv[j][3], x1.y, acc[1][j][1]);
            }
        }
    }
    cp_async_wait<0>();
    // 4. face terms and the write, for the lane's two rows
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int32_t row = trow[(int64_t)t * TR + s0 + 8 * r];
        if (row < 0) continue;
        for (int32_t bq = bptr[row]; bq < bptr[row + 1]; ++bq) {
            const float *xr = Xs + bhalo[bq];
            float sv[NF<D>()];
#pragma unroll
            for (int f = 0; f < NF<D>(); ++f) sv[f] = bval[f * nb + bq];
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int d = mma_dir(j, 2 * q + e, NT);
                    const float *fc = coef32 + 16 * (m0 + d) + face_slot<D>();
                    float v = 0.0f;
#pragma unroll
                    for (int f = 0; f < NF<D>(); ++f) v = fmaf(fc[f], sv[f], v);
                    acc[r][j][e] = fmaf(v, xr[d], acc[r][j][e]);
                }
        }
        const int64_t rb0 = (int64_t)row * m + m0;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const int64_t e = rb0 + 16 * i + 4 * q;
            float4 o = make_float4(acc[r][2 * i][0], acc[r][2 * i][1], acc[r][2 * i + 1][0], acc[r][2 * i + 1][1]);
            if (B) {
                const float4 b = *reinterpret_cast<const float4 *>(B + e);
                o = make_float4(b.x - o.x, b.y - o.y, b.z - o.z, b.w - o.w);
            }
            *reinterpret_cast<float4 *>(Y + e) = o;
        }
        if constexpr (NT & 1) {
            constexpr int j = NT - 1;
            const int64_t e = rb0 + 16 * NP + 2 * q;
            float2 o = make_float2(acc[r][j][0], acc[r][j][1]);
            if (B) {
                const float2 b = *reinterpret_cast<const float2 *>(B + e);
                o = make_float2(b.x - o.x, b.y - o.y);
            }
            *reinterpret_cast<float2 *>(Y + e) = o;
        }
    }
}

// ---------------------------------------------------------------------------
// Diffusion operator of the DSA-like outer preconditioner (FP64, on the
// overlap pattern), built from the forms already integrated:
//   C = diag(1 / (3 sigma_t,i)) sum_a K_aa + kappa M0 + (Mt - Ms) + 1/2 sum_f S_f,
// sigma_t,i = (Mt 1)_i / (M0 1)_i, the test-function average of sigma_t: a
// Galerkin P1-diffusion operator with the Marshak vacuum condition on every
// face.  The paper names diffusion acceleration as the remedy for slow outer
// solves (Sec. 5.3, Sec. 6) without deriving one.
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_diff_values(int64_t n, int64_t nnz, double kappa, const int32_t *__restrict__ rowptr,
                              const double *__restrict__ mats, double *__restrict__ C) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *M0 = mats, *Mt = mats + nnz, *Ms = mats + 2 * nnz;
    const double *K = mats + (3 + 3 * D) * nnz, *S = mats + mat_S<D>() * nnz;
    double st = 0.0, m0 = 0.0;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        st += Mt[p];
        m0 += M0[p];
    }
    const double dco = m0 / (3.0 * st);   // 1 / (3 sigma_t,i)
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        double kk = 0.0, sf = 0.0;
#pragma unroll
        for (int a = 0; a < D; ++a) kk += K[(a * D + a) * nnz + p];
#pragma unroll
        for (int f = 0; f < NF<D>(); ++f) sf += S[f * nnz + p];
        C[p] = dco * kk + kappa * M0[p] + (Mt[p] - Ms[p]) + 0.5 * sf;
    }
}

// Inverse of the diagonal block (MLPG_BLOCK_PTS Morton points) of one FP64
// operator on the pattern: one warp per block, Gauss-Jordan with partial
// pivoting on [A | I] in shared memory, lane l owning column l.
__global__ void __launch_bounds__(256) k_block_inv64(int64_t nblk, const int32_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ col, const double *__restrict__ A,
                                                     const int32_t *__restrict__ bmember,
                                                     const int32_t *__restrict__ bof, double *__restrict__ Pinv,
                                                     int *__restrict__ flag) {
    __shared__ double sA[8][kB][2 * kB + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * 8 + warp;
    if (k >= nblk) return;
    double(*W)[2 * kB + 1] = sA[warp];
    if (lane < kB) {
        const int a = lane;
        for (int b = 0; b < 2 * kB; ++b) W[a][b] = (b == kB + a) ? 1.0 : 0.0;
        const int32_t i = bmember[k * kB + a];
        if (i < 0) {
            W[a][a] = 1.0;
        } else {
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                const int32_t sl = bof[col[p]];
                if (sl / kB == k) W[a][sl - k * kB] = A[p];
            }
        }
    }
    __syncwarp();
    for (int cc = 0; cc < kB; ++cc) {
        int piv = cc;
        double best = fabs(W[cc][cc]);
        for (int r = cc + 1; r < kB; ++r) {
            const double v = fabs(W[r][cc]);
            if (v > best) { best = v; piv = r; }
        }
        if (!(best > 0.0)) {
            if (lane == 0) atomicOr(flag, 64);
            return;
        }
        __syncwarp();
        if (piv != cc) {
            const double t = W[cc][lane];
            W[cc][lane] = W[piv][lane];
            W[piv][lane] = t;
        }
        __syncwarp();
        const double inv = 1.0 / W[cc][cc];
        __syncwarp();
        W[cc][lane] *= inv;
        __syncwarp();
        double fr[kB];
#pragma unroll
        for (int r = 0; r < kB; ++r) fr[r] = W[r][cc];
        __syncwarp();
        const double pc = W[cc][lane];
#pragma unroll
        for (int r = 0; r < kB; ++r)
            if (r != cc) W[r][lane] -= fr[r] * pc;
        __syncwarp();
    }
    for (int e = lane; e < kB * kB; e += 32) {
        const int a = e / kB, b = e - a * kB;
        Pinv[(k * kB + a) * kB + b] = W[a][kB + b];
    }
}

// z = P^{-1} v for one vector (block-Jacobi with FP64 block inverses); with
// sc != null, v is first scaled in place by sc[0].  One CTA of kB threads per
// block.
__global__ void __launch_bounds__(kB) k_bjacobi64_vec(int64_t nblk, const int32_t *__restrict__ bmember,
                                                      const double *__restrict__ Pinv, double *__restrict__ v,
                                                      const double *__restrict__ sc, double *__restrict__ z) {
    __shared__ double vs[kB];
    const int64_t blk = blockIdx.x;
    const int a = threadIdx.x;
    const int32_t i = bmember[blk * kB + a];
    double val = 0.0;
    if (i >= 0) {
        val = v[i];
        if (sc) {
            val *= sc[0];
            v[i] = val;
        }
    }
    vs[a] = val;
    __syncthreads();
    if (i < 0) return;
    const double *P = Pinv + (blk * kB + a) * kB;
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < kB; ++b) acc = fma(P[b], vs[b], acc);
    z[i] = acc;
}

// y = A x (B == null) or y = B - A x: FP64 CSR times one vector
__global__ void k_csr_spmv64(int64_t n, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                             const double *__restrict__ A, const double *__restrict__ x,
                             const double *__restrict__ B, double *__restrict__ y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s = fma(A[p], x[col[p]], s);
    y[i] = B ? B[i] - s : s;
}

struct Team {
    int tm_log2, dpl;
};
// direction lanes per row: the power of two TM <= 32 that wastes the fewest
// lanes (TM * DPL >= m, DPL <= 16)
Team pick_team(int m) {
    Team best{5, (m + 31) / 32};
    double beff = -1.0;
    for (int lg = 5; lg >= 2; --lg) {
        int tm = 1 << lg;
        int dpl = (m + tm - 1) / tm;
        if (dpl > 16) continue;
        double eff = double(m) / double(tm * dpl);
        if (eff > beff + 0.05) { beff = eff; best = {lg, dpl}; }
    }
    return best;
}

}  // namespace

#define DISPATCH_DPL(dpl, KERNEL, ...)                                   \
    switch (dpl) {                                                       \
        case 1: KERNEL<1><<<grid, 256, 0, s>>>(__VA_ARGS__); break;      \
        case 2: KERNEL<2><<<grid, 256, 0, s>>>(__VA_ARGS__); break;      \
        case 3: KERNEL<3><<<grid, 256, 0, s>>>(__VA_ARGS__); break;      \
        case 4: KERNEL<4><<<grid, 256, 0, s>>>(__VA_ARGS__); break;      \
        case 5: case 6: KERNEL<6><<<grid, 256, 0, s>>>(__VA_ARGS__); break; \
        case 7: case 8: KERNEL<8><<<grid, 256, 0, s>>>(__VA_ARGS__); break; \
        default: KERNEL<16><<<grid, 256, 0, s>>>(__VA_ARGS__); break;    \
    }

// one warp per row (slot layout) / one team of TM lanes per row
static int64_t team_grid(int64_t n, const Team &) { return (n * 32 + 255) / 256; }
static int64_t rowteam_grid(int64_t n, const Team &tm) { return ((n << tm.tm_log2) + 255) / 256; }

// Row tiles of the FP32 L-apply: built once per point set when m % 4 == 0.
// Tile shape: TR rows per tile and DPT directions per thread, from the options
// or by default 64 rows and 8 directions (4 when m % 8 != 0) with a staged
// halo, 4 directions and at most 320 threads per CTA in gather mode; G = chunk
// / DPT thread groups per row.  The directions are split into chunks (one CTA
// each) until a tile's staged halo, halo x (chunk + 4) floats, and the record
// stages fit kTileSmem (staged halo), or until G fits the thread limit
// (gather).  The automatic choice stages the halo while that takes at most
// two chunks, and gathers otherwise.
constexpr size_t kTileSmem = 100 * 1024;

template <int D, int DPT, int TR, bool GX>
static mlpg_status launch_tile(mlpg_ctx *ctx, const float *X, const float *B, float *Y) {
    const dim3 tg((unsigned)ctx->ntile, (unsigned)((ctx->m + ctx->tile_chunk - 1) / ctx->tile_chunk));
    const int threads = TR * (ctx->tile_chunk / DPT);
    k_spmm32_tile<D, DPT, TR, GX><<<tg, threads, ctx->tile_smem, ctx->stream>>>(
        ctx->m, ctx->tile_chunk, ctx->tile_xs, ctx->tile_xs_f4, ctx->t_base, ctx->t_width, ctx->t_row, ctx->t_hptr,
        ctx->t_hcol, reinterpret_cast<const float4 *>(ctx->t_rec), ctx->coef32, ctx->bptr, ctx->t_bhalo, ctx->bval32,
        ctx->nb, X, B, Y, ctx->d_tile_err);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}
template <int D, int TR, int NT>
static mlpg_status launch_mma(mlpg_ctx *ctx, const float *X, const float *B, float *Y) {
    const dim3 tg((unsigned)ctx->ntile, (unsigned)(ctx->m / (8 * NT)));
    k_spmm32_mma<D, TR, NT><<<tg, 2 * TR, ctx->tile_smem, ctx->stream>>>(
        ctx->m, ctx->tile_xs, ctx->tile_xs_f4, ctx->t_base, ctx->t_width, ctx->t_row, ctx->t_hptr, ctx->t_hcol,
        reinterpret_cast<const float4 *>(ctx->t_rec), ctx->coef32, ctx->bptr, ctx->t_bhalo, ctx->bval32, ctx->nb, X,
        B, Y);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}
#define MMA_NT_SWITCH(D, TR, FN, ...)                   \
    switch (ctx->tile_chunk / 8) {                      \
        case 2: return FN<D, TR, 2>(__VA_ARGS__);       \
        case 3: return FN<D, TR, 3>(__VA_ARGS__);       \
        case 4: return FN<D, TR, 4>(__VA_ARGS__);       \
        case 5: return FN<D, TR, 5>(__VA_ARGS__);       \
        default: return FN<D, TR, 6>(__VA_ARGS__);      \
    }
template <int D, int TR, int NT>
static mlpg_status mma_attr(mlpg_ctx *ctx) {
    CU(ctx, cudaFuncSetAttribute(k_spmm32_mma<D, TR, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kTileSmem));
    return MLPG_OK;
}

template <int D>
static mlpg_status run_tile(mlpg_ctx *ctx, const float *X, const float *B, float *Y) {
    if (ctx->tile_mma) {
        if (ctx->tile_rows == 32) { MMA_NT_SWITCH(D, 32, launch_mma, ctx, X, B, Y) }
        MMA_NT_SWITCH(D, 64, launch_mma, ctx, X, B, Y)
    }
    const int key = ctx->tile_dpt * 100 + ctx->tile_rows;
    if (ctx->tile_gather) switch (key) {
            case 804: return launch_tile<D, 8, 4, true>(ctx, X, B, Y);
            case 404: return launch_tile<D, 4, 4, true>(ctx, X, B, Y);
            case 808: return launch_tile<D, 8, 8, true>(ctx, X, B, Y);
            case 816: return launch_tile<D, 8, 16, true>(ctx, X, B, Y);
            case 832: return launch_tile<D, 8, 32, true>(ctx, X, B, Y);
            case 408: return launch_tile<D, 4, 8, true>(ctx, X, B, Y);
            case 416: return launch_tile<D, 4, 16, true>(ctx, X, B, Y);
            default: return launch_tile<D, 4, 32, true>(ctx, X, B, Y);
        }
    switch (key) {
        case 832: return launch_tile<D, 8, 32, false>(ctx, X, B, Y);
        case 864: return launch_tile<D, 8, 64, false>(ctx, X, B, Y);
        case 432: return launch_tile<D, 4, 32, false>(ctx, X, B, Y);
        default: return launch_tile<D, 4, 64, false>(ctx, X, B, Y);
    }
}
template <int D, int DPT, int TR, bool GX>
static mlpg_status tile_attr(mlpg_ctx *ctx) {
    // the kernel's attribute is shared by every context: set to the fixed budget, never lowered
    // (the record stages of 32-row gather tiles alone reach the 48 KB default)
    CU(ctx, cudaFuncSetAttribute(k_spmm32_tile<D, DPT, TR, GX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kTileSmem));
    return MLPG_OK;
}

// One tile layout: rows per tile, directions per thread and per CTA (chunk),
// staged halo or gather mode, the host-side tiles.  chunk == 0: no layout.
struct TilePlan {
    int tr = 0, dpt = 0, chunk = 0;
    bool gather = false, mma = false;
    size_t rec_smem = 0;
    TileLayout tl;
    int64_t nslot = 0;
};

// Plans the tiles of one mode; an explicit request that cannot be met is an
// error, the automatic choice only finds no layout (chunk 0).
template <int D>
static mlpg_status plan_tiles(mlpg_ctx *ctx, bool gather, bool mma, TilePlan &P) {
    const int m = ctx->m;
    const bool ask = ctx->opt.apply_kernel != 0;
    P = TilePlan();
    P.gather = gather;
    P.mma = mma;
    // gather: four directions per thread measured fastest (more CTAs per SM)
    const int dpt = ctx->opt.tile_dpt ? ctx->opt.tile_dpt : ((m & 7) == 0 && !gather ? 8 : 4);
    if (m % dpt != 0) return set_err(ctx, MLPG_ERR_ARG, "tile_dpt must divide the number of directions");
    int tr = ctx->opt.tile_rows;
    if (gather && tr == 0) {   // the most rows per tile with at most 320 threads per CTA
        const int G = (m + dpt - 1) / dpt;
        tr = 4;
        for (int c : {32, 16, 8})
            if (c * G <= 320) {
                tr = c;
                break;
            }
    }
    if (tr == 0) tr = 64;
    if (gather && tr == 64)
        return ask ? set_err(ctx, MLPG_ERR_ARG, "apply_kernel 4 takes 4, 8, 16 or 32 rows per tile") : MLPG_OK;
    if (gather && (int64_t)ctx->n * m >= (int64_t(1) << 31))
        return ask ? set_err(ctx, MLPG_ERR_ARG, "apply_kernel 4 needs n x m < 2^31 (32-bit record offsets)") : MLPG_OK;
    const int rk = rec_k(gather);
    P.nslot = build_tiles(ctx->n, ctx->h_rowptr.data(), ctx->h_col.data(), ctx->h_order.data(), tr, rk, P.tl);
    const TileLayout &tl = P.tl;
    if (P.nslot * (int64_t)(rec_words<D>() / 4) >= (int64_t(1) << 31) || tl.hptr.back() >= (int64_t(1) << 31))
        return MLPG_OK;   // beyond 32-bit slot indices: the row-team kernel serves
    P.rec_smem = (size_t)kRecStages * rk * tr * (rec_words<D>() / 4) * sizeof(float4);
    int chunk = 0;
    if (mma) {
        // tensor-core tiles: chunks of 8 NT directions (NT <= 6) dividing m; shared-memory row stride
        // 16 mod 32 words (two rows read by one 8-lane phase then fall on disjoint banks half the time)
        if ((m & 7) != 0) return set_err(ctx, MLPG_ERR_ARG, "apply_kernel 3 needs a multiple of 8 directions");
        for (int nt = 6; nt >= 2 && !chunk; --nt) {
            const int mc = 8 * nt, xs = mc + (16 - mc % 32 + 32) % 32;
            if (m % mc == 0 && (size_t)tl.max_halo * xs * sizeof(float) + P.rec_smem <= kTileSmem) chunk = mc;
        }
        if (!chunk) return set_err(ctx, MLPG_ERR_ARG, "apply_kernel 3: no direction chunk fits shared memory");
    }
    for (int nchunk = 1; nchunk <= m / 4 && !mma; ++nchunk) {
        const int G = (m + dpt * nchunk - 1) / (dpt * nchunk);
        if (G > tile_max_groups(tr, dpt, gather)) continue;
        if (gather || (size_t)tl.max_halo * (G * dpt + 4) * sizeof(float) + P.rec_smem <= kTileSmem) {
            chunk = G * dpt;
            break;
        }
    }
    P.tr = tr;
    P.dpt = dpt;
    P.chunk = chunk;
    return MLPG_OK;
}

template <int D>
static mlpg_status init_tiles(mlpg_ctx *ctx) {
    const int m = ctx->m, kind = ctx->opt.apply_kernel;
    if ((m & 3) != 0 || kind == 1) return MLPG_OK;
    TilePlan P;
    if (kind != 4) {
        MLPG_TRY(plan_tiles<D>(ctx, false, kind == 3, P));
        // automatic choice: staged halos pay while the records are read by few chunks;
        // past two chunks the gather mode reads them once
        if (kind == 0 && P.chunk && (m + P.chunk - 1) / P.chunk > 2) P.chunk = 0;
    }
    if (kind == 4 || (kind == 0 && P.chunk == 0)) MLPG_TRY(plan_tiles<D>(ctx, true, false, P));
    if (P.chunk == 0) return MLPG_OK;
    const int tr = P.tr, dpt = P.dpt, chunk = P.chunk;
    const bool gather = P.gather, mma = P.mma;
    const size_t rec_smem = P.rec_smem;
    const int64_t nslot = P.nslot;
    TileLayout &tl = P.tl;
    ctx->tile_rows = tr;
    ctx->tile_dpt = dpt;
    ctx->tile_chunk = chunk;
    ctx->tile_mma = mma;
    ctx->tile_gather = gather;
    // gather: the record index is the column's global offset col x m; otherwise the column's
    // staged row in shared memory, a padded row that spreads halo rows over the banks
    ctx->tile_xs = gather ? m : (mma ? chunk + (16 - chunk % 32 + 32) % 32 : chunk + 4);
    if (gather) {   // global columns of the slots (zero for padding: a zero record)
        for (int64_t e = 0; e < nslot; ++e) tl.lcol[e] = tl.perm[e] >= 0 ? ctx->h_col[tl.perm[e]] : 0;
    }
    ctx->ntile = tl.ntile;
    ctx->nslot = nslot;
    cudaStream_t s = ctx->stream;
    std::vector<int32_t> base32(tl.ntile + 1), hptr32(tl.ntile + 1);
    for (int64_t t = 0; t <= tl.ntile; ++t) {
        base32[t] = (int32_t)tl.base[t];
        hptr32[t] = (int32_t)tl.hptr[t];
    }
    MLPG_TRY(dalloc(ctx, &ctx->t_base, tl.ntile + 1));
    MLPG_TRY(dalloc(ctx, &ctx->t_width, tl.ntile));
    MLPG_TRY(dalloc(ctx, &ctx->t_row, tl.ntile * tr));
    MLPG_TRY(dalloc(ctx, &ctx->t_hptr, tl.ntile + 1));
    MLPG_TRY(dalloc(ctx, &ctx->t_hcol, tl.hcol.size()));
    MLPG_TRY(dalloc(ctx, &ctx->t_perm, nslot));
    MLPG_TRY(dalloc(ctx, &ctx->t_lcol, nslot));
    MLPG_TRY(dalloc(ctx, &ctx->t_rec, nslot * rec_words<D>()));
    CU(ctx, cudaMemcpyAsync(ctx->t_base, base32.data(), base32.size() * 4, cudaMemcpyHostToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->t_width, tl.width.data(), tl.width.size() * 4, cudaMemcpyHostToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->t_row, tl.row.data(), tl.row.size() * 4, cudaMemcpyHostToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->t_hptr, hptr32.data(), hptr32.size() * 4, cudaMemcpyHostToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->t_hcol, tl.hcol.data(), tl.hcol.size() * 4, cudaMemcpyHostToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->t_perm, tl.perm.data(), nslot * 4, cudaMemcpyHostToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->t_lcol, tl.lcol.data(), nslot * 4, cudaMemcpyHostToDevice, s));
    // halo offset (index x shared-memory row stride) of every boundary-segment entry's column
    {
        std::vector<int32_t> bptr(ctx->n + 1), bcol(std::max<int64_t>(ctx->nb, 1)), bhalo(std::max<int64_t>(ctx->nb, 1), 0);
        CU(ctx, cudaMemcpyAsync(bptr.data(), ctx->bptr, (ctx->n + 1) * 4, cudaMemcpyDeviceToHost, s));
        if (ctx->nb > 0) CU(ctx, cudaMemcpyAsync(bcol.data(), ctx->bcol, ctx->nb * 4, cudaMemcpyDeviceToHost, s));
        CU(ctx, cudaStreamSynchronize(s));
        for (int64_t r = 0; r < tl.ntile * tr; ++r) {
            const int32_t i = tl.row[r];
            if (i < 0) continue;
            if (gather) {
                for (int32_t q = bptr[i]; q < bptr[i + 1]; ++q) bhalo[q] = bcol[q] * m;
                continue;
            }
            const int64_t t = r / tr;
            const int32_t *hb = tl.hcol.data() + tl.hptr[t], *he = tl.hcol.data() + tl.hptr[t + 1];
            for (int32_t q = bptr[i]; q < bptr[i + 1]; ++q) {
                const int32_t *hit = std::lower_bound(hb, he, bcol[q]);
                if (hit == he || *hit != bcol[q]) return set_err(ctx, MLPG_ERR_ARG, "boundary entry outside its tile's halo");
                bhalo[q] = (int32_t)(hit - hb) * ctx->tile_xs;
            }
        }
        MLPG_TRY(dalloc(ctx, &ctx->t_bhalo, bhalo.size()));
        CU(ctx, cudaMemcpyAsync(ctx->t_bhalo, bhalo.data(), bhalo.size() * 4, cudaMemcpyHostToDevice, s));
        CU(ctx, cudaStreamSynchronize(s));
    }
    CU(ctx, cudaStreamSynchronize(s));   // the host vectors go out of scope
    if (mma) {
        mlpg_status st = MLPG_OK;
        auto set = [&]() -> mlpg_status {
            if (tr == 32) { MMA_NT_SWITCH(D, 32, mma_attr, ctx) }
            MMA_NT_SWITCH(D, 64, mma_attr, ctx)
        };
        st = set();
        if (st != MLPG_OK) return st;
    } else if (gather) switch (dpt * 100 + tr) {
            case 804: MLPG_TRY((tile_attr<D, 8, 4, true>(ctx))); break;
            case 808: MLPG_TRY((tile_attr<D, 8, 8, true>(ctx))); break;
            case 816: MLPG_TRY((tile_attr<D, 8, 16, true>(ctx))); break;
            case 832: MLPG_TRY((tile_attr<D, 8, 32, true>(ctx))); break;
            case 404: MLPG_TRY((tile_attr<D, 4, 4, true>(ctx))); break;
            case 408: MLPG_TRY((tile_attr<D, 4, 8, true>(ctx))); break;
            case 416: MLPG_TRY((tile_attr<D, 4, 16, true>(ctx))); break;
            default: MLPG_TRY((tile_attr<D, 4, 32, true>(ctx))); break;
        }
    else switch (dpt * 100 + tr) {
            case 832: MLPG_TRY((tile_attr<D, 8, 32, false>(ctx))); break;
            case 864: MLPG_TRY((tile_attr<D, 8, 64, false>(ctx))); break;
            case 432: MLPG_TRY((tile_attr<D, 4, 32, false>(ctx))); break;
            default: MLPG_TRY((tile_attr<D, 4, 64, false>(ctx))); break;
        }
    ctx->tile_xs_f4 = gather ? 0 : (int)(tl.max_halo * ctx->tile_xs / 4);
    ctx->tile_smem = (size_t)ctx->tile_xs_f4 * sizeof(float4) + rec_smem;
    ctx->tile_max_halo = tl.max_halo;
    if (!ctx->d_tile_err) {
        MLPG_TRY(dalloc(ctx, &ctx->d_tile_err, 1));
        CU(ctx, cudaMemsetAsync(ctx->d_tile_err, 0, sizeof(int), s));
    }
    return MLPG_OK;
}

template <int D>
static mlpg_status init_operator_storage_d(mlpg_ctx *ctx) {
    const int64_t n = ctx->n, nnz = ctx->nnz;
    const int m = ctx->m;
    cudaStream_t s = ctx->stream;
    MLPG_TRY(dalloc(ctx, &ctx->rowidx, nnz));
    k_rowidx<<<(n + 255) / 256, 256, 0, s>>>(n, ctx->rowptr, ctx->rowidx);
    CU_LAUNCH(ctx);
    MLPG_TRY(dalloc(ctx, &ctx->A64, NA<D>() * nnz));
    MLPG_TRY(dalloc(ctx, &ctx->A32, NA<D>() * nnz));
    MLPG_TRY(dalloc(ctx, &ctx->T64, NT<D>() * nnz));
    MLPG_TRY(dalloc(ctx, &ctx->S64, NT<D>() * nnz));
    MLPG_TRY(dalloc(ctx, &ctx->L64, (size_t)nnz * m));
    MLPG_TRY(dalloc(ctx, &ctx->coef, kCS * m));
    MLPG_TRY(dalloc(ctx, &ctx->fcoef, kFS * m));
    MLPG_TRY(dalloc(ctx, &ctx->coef32, 16 * m));
    MLPG_TRY(dalloc(ctx, &ctx->dinv64, (size_t)n * m));
    MLPG_TRY(dalloc(ctx, &ctx->dinv32, (size_t)n * m));
    MLPG_TRY(dalloc(ctx, &ctx->r64, (size_t)n * m));
    // [NT][n] FP64 products + [NT][n] float copy
    MLPG_TRY(dalloc(ctx, &ctx->abc, (NT<D>() + (NT<D>() + 1) / 2) * n));
    MLPG_TRY(dalloc(ctx, &ctx->Pinv, (size_t)ctx->nblk * kB * kB * m));
    if (ctx->opt.precision == MLPG_MIXED && ctx->opt.mixed_half_prec && (m & 3) == 0) {
        MLPG_TRY(dalloc(ctx, &ctx->Pinv16, (size_t)ctx->nblk * kB * kB * m));
        MLPG_TRY(dalloc(ctx, &ctx->Pscale, (size_t)ctx->nblk * m));
    }
    // boundary segment (the face arrays do not depend on dt)
    int *cnt;
    MLPG_TRY(dalloc(ctx, &cnt, n));
    MLPG_TRY(dalloc(ctx, &ctx->bptr, n + 1));
    const double *Sf = ctx->mats + mat_S<D>() * nnz;
    k_bcount<D><<<(n + 255) / 256, 256, 0, s>>>(n, ctx->rowptr, nnz, Sf, cnt);
    CU_LAUNCH(ctx);
    k_scan1<<<1, 1024, 0, s>>>(n, cnt, ctx->bptr);
    CU_LAUNCH(ctx);
    int32_t nb32 = 0;
    CU(ctx, cudaMemcpyAsync(&nb32, ctx->bptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    ctx->nb = nb32;
    MLPG_TRY(dalloc(ctx, &ctx->bcol, ctx->nb));
    MLPG_TRY(dalloc(ctx, &ctx->bval64, NF<D>() * ctx->nb));
    MLPG_TRY(dalloc(ctx, &ctx->bval32, NF<D>() * ctx->nb));
    k_bfill<D><<<(n + 255) / 256, 256, 0, s>>>(n, ctx->rowptr, ctx->col, nnz, Sf, ctx->bptr, ctx->nb,
                                            ctx->bcol, ctx->bval64, ctx->bval32);
    CU_LAUNCH(ctx);
    // list of the rows that have face terms
    MLPG_TRY(dalloc(ctx, &ctx->brow, n));
    int *bcount;
    MLPG_TRY(dalloc(ctx, &bcount, 1));
    CU(ctx, cudaMemsetAsync(bcount, 0, sizeof(int), s));
    k_brows<<<(n + 255) / 256, 256, 0, s>>>(n, ctx->bptr, ctx->brow, bcount);
    CU_LAUNCH(ctx);
    int nbr = 0;
    CU(ctx, cudaMemcpyAsync(&nbr, bcount, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    ctx->nbrow = nbr;
    k_coef<D><<<(m + 127) / 128, 128, 0, s>>>(m, ctx->omega, ctx->coef, ctx->fcoef, ctx->coef32);
    CU_LAUNCH(ctx);
    if (ctx->opt.precision == MLPG_MIXED) MLPG_TRY(init_tiles<D>(ctx));
    return MLPG_OK;
}

static mlpg_status init_operator_storage(mlpg_ctx *ctx) {
    return ctx->dim == 3 ? init_operator_storage_d<3>(ctx) : init_operator_storage_d<2>(ctx);
}

template <int D>
static mlpg_status form_operators_d(mlpg_ctx *ctx, double kappa) {
    const int64_t n = ctx->n, nnz = ctx->nnz;
    const int m = ctx->m;
    cudaStream_t s = ctx->stream;
    if (!ctx->A64) MLPG_TRY(init_operator_storage(ctx));
    const double *Sf = ctx->mats + mat_S<D>() * nnz;
    k_form_arrays<D><<<(nnz + 255) / 256, 256, 0, s>>>(nnz, kappa, ctx->rowidx, ctx->tau, ctx->mats,
                                                    ctx->A64, ctx->A32, ctx->T64, ctx->S64);
    CU_LAUNCH(ctx);
    if (ctx->t_rec) {
        k_tile_records<D><<<(ctx->nslot + 255) / 256, 256, 0, s>>>(ctx->nslot, nnz, ctx->tile_xs, ctx->t_perm, ctx->t_lcol,
                                                                   ctx->A32, reinterpret_cast<float4 *>(ctx->t_rec));
        CU_LAUNCH(ctx);
    }
    int64_t tot = nnz * m;
    k_materialize<D><<<(tot + 255) / 256, 256, 0, s>>>(nnz, m, ctx->A64, Sf, ctx->coef, ctx->fcoef, ctx->L64);
    CU_LAUNCH(ctx);
    CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
    Inflow pb;
    for (int f = 0; f < 6; ++f) pb.v[f] = ctx->psi_b[f];
    int64_t nm = n * m;
    k_diag_rhs<D><<<(nm + 255) / 256, 256, 0, s>>>(n, m, ctx->diag, nnz, ctx->A64, Sf, ctx->coef, ctx->fcoef,
                                                ctx->tau, ctx->vecs, pb, ctx->dinv64, ctx->dinv32, ctx->r64,
                                                ctx->d_flag);
    CU_LAUNCH(ctx);
    int flag = 0;
    CU(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    if (flag & 16) return set_err(ctx, MLPG_ERR_ARG, "transport operator has a zero diagonal entry");
    // block-Jacobi inverses of every direction
    {
        dim3 grid((unsigned)ctx->nblk, (unsigned)((m + 7) / 8));
        k_block_inv<D><<<grid, 256, 0, s>>>(ctx->nblk, m, ctx->rowptr, ctx->col, nnz, ctx->A64, Sf, ctx->coef,
                                         ctx->fcoef, ctx->bmember, ctx->bof, ctx->Pinv, ctx->Pinv16, ctx->Pscale,
                                         ctx->d_flag);
        CU_LAUNCH(ctx);
        CU(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(ctx, cudaStreamSynchronize(s));
        if (flag & 32) return set_err(ctx, MLPG_ERR_ARG, "singular diagonal block in the transport operator");
    }
    ctx->kappa = kappa;
    for (int f = 0; f < 6; ++f) ctx->ops_psib[f] = ctx->psi_b[f];
    ctx->st.spmm_bytes = 0;
    return MLPG_OK;
}

mlpg_status form_operators(mlpg_ctx *ctx, double kappa) {
    MLPG_TRY(ctx->dim == 3 ? form_operators_d<3>(ctx, kappa) : form_operators_d<2>(ctx, kappa));
    if (ctx->opt.outer_precond == 1) MLPG_TRY(form_diffusion(ctx, kappa));
    return MLPG_OK;
}

mlpg_status form_diffusion(mlpg_ctx *ctx, double kappa) {
    const int64_t n = ctx->n;
    cudaStream_t s = ctx->stream;
    if (!ctx->Cdiff) {
        MLPG_TRY(dalloc(ctx, &ctx->Cdiff, ctx->nnz));
        MLPG_TRY(dalloc(ctx, &ctx->Cinv, (size_t)ctx->nblk * kB * kB));
        MLPG_TRY(dalloc(ctx, &ctx->dsa_buf, 2 * n));
    }
    if (ctx->dim == 3)
        k_diff_values<3><<<(n + 255) / 256, 256, 0, s>>>(n, ctx->nnz, kappa, ctx->rowptr, ctx->mats, ctx->Cdiff);
    else
        k_diff_values<2><<<(n + 255) / 256, 256, 0, s>>>(n, ctx->nnz, kappa, ctx->rowptr, ctx->mats, ctx->Cdiff);
    CU_LAUNCH(ctx);
    CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
    k_block_inv64<<<(unsigned)((ctx->nblk + 7) / 8), 256, 0, s>>>(ctx->nblk, ctx->rowptr, ctx->col, ctx->Cdiff,
                                                                 ctx->bmember, ctx->bof, ctx->Cinv, ctx->d_flag);
    CU_LAUNCH(ctx);
    int flag = 0;
    CU(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(ctx, cudaStreamSynchronize(s));
    if (flag & 64) return set_err(ctx, MLPG_ERR_ARG, "singular diagonal block in the diffusion operator");
    return MLPG_OK;
}

mlpg_status apply_C(mlpg_ctx *ctx, const double *X, const double *B, double *Y) {
    k_csr_spmv64<<<(ctx->n + 255) / 256, 256, 0, ctx->stream>>>(ctx->n, ctx->rowptr, ctx->col, ctx->Cdiff, X, B, Y);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

mlpg_status apply_Ms_scalar(mlpg_ctx *ctx, const double *X, double *Y) {
    k_csr_spmv64<<<(ctx->n + 255) / 256, 256, 0, ctx->stream>>>(ctx->n, ctx->rowptr, ctx->col,
                                                                 ctx->mats + 2 * ctx->nnz, X, nullptr, Y);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

mlpg_status apply_Cprec(mlpg_ctx *ctx, double *v, double *z, const double *sc) {
    k_bjacobi64_vec<<<(unsigned)ctx->nblk, kB, 0, ctx->stream>>>(ctx->nblk, ctx->bmember, ctx->Cinv, v, sc, z);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

// Device time of each batched L-apply: event pairs from a pool, harvested
// (elapsed time summed) when the pool is full and whenever stats are read.
static void timing_begin(mlpg_ctx *ctx) {
    if (!ctx->timing) return;
    if (ctx->ev_used == (int)ctx->ev_pool.size()) harvest_timing(ctx);
    cudaEventRecord(ctx->ev_pool[ctx->ev_used].first, ctx->stream);
}
static void timing_end(mlpg_ctx *ctx) {
    ctx->st.spmm_launches++;
    if (!ctx->timing) return;
    cudaEventRecord(ctx->ev_pool[ctx->ev_used].second, ctx->stream);
    ctx->ev_used++;
}

mlpg_status apply_L64_res(mlpg_ctx *ctx, const double *X, const double *B, double *Y) {
    Team tm = pick_team(ctx->m);
    int64_t grid = team_grid(ctx->n, tm);
    cudaStream_t s = ctx->stream;
    timing_begin(ctx);
    DISPATCH_DPL(tm.dpl, k_spmm64, ctx->n, ctx->m, tm.tm_log2, ctx->rowptr, ctx->col, ctx->L64, X, B, Y);
    timing_end(ctx);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

template <int DIM>
static mlpg_status apply_faces32(mlpg_ctx *ctx, const Team &tm, const float *X, const float *B, float *Y);

template <int DIM>
static mlpg_status apply_L32_res_d(mlpg_ctx *ctx, const float *X, const float *B, float *Y) {
    Team tm = pick_team(ctx->m);
    int64_t grid = team_grid(ctx->n, tm);
    cudaStream_t s = ctx->stream;
    timing_begin(ctx);
    if (ctx->t_rec) {   // the face terms are added inside the tile kernel
        MLPG_TRY(run_tile<DIM>(ctx, X, B, Y));
        timing_end(ctx);
        return MLPG_OK;
    }
    // ten base arrays (3D): at most four directions per lane, the rest in direction chunks
    // (grid y), so that the coefficient registers leave room for enough warps per SM
    Team tt = tm;
    int nchunk = 1;
    if (DIM == 3 && tm.dpl > 4) {
        nchunk = (ctx->m + 127) / 128;
        tt.tm_log2 = 5;
        tt.dpl = (ctx->m + 32 * nchunk - 1) / (32 * nchunk);
    }
    const dim3 tgrid((unsigned)rowteam_grid(ctx->n, tt), (unsigned)nchunk);
    const bool small = ctx->n * (int64_t)ctx->m < (int64_t(1) << 31);
    const bool exact = nchunk == 1 && (tt.dpl << tt.tm_log2) == ctx->m;
#define SPMM32_ARGS ctx->n, ctx->m, tt.tm_log2, ctx->nnz, ctx->rowptr, ctx->col, ctx->A32, ctx->coef32, X, B, Y
#define SPMM32_CASE(D)                                                                          \
    case D:                                                                                     \
        if (exact && small) k_spmm32<D, true, int32_t, DIM><<<tgrid, 256, 0, s>>>(SPMM32_ARGS); \
        else if (small) k_spmm32<D, false, int32_t, DIM><<<tgrid, 256, 0, s>>>(SPMM32_ARGS);    \
        else k_spmm32<D, false, int64_t, DIM><<<tgrid, 256, 0, s>>>(SPMM32_ARGS);               \
        break;
    switch (tt.dpl) {
        SPMM32_CASE(1) SPMM32_CASE(2) SPMM32_CASE(3) SPMM32_CASE(4) SPMM32_CASE(5) SPMM32_CASE(6)
        SPMM32_CASE(7) SPMM32_CASE(8) SPMM32_CASE(9) SPMM32_CASE(10) SPMM32_CASE(11) SPMM32_CASE(12)
        default:
            if (small) k_spmm32<16, false, int32_t, DIM><<<tgrid, 256, 0, s>>>(SPMM32_ARGS);
            else k_spmm32<16, false, int64_t, DIM><<<tgrid, 256, 0, s>>>(SPMM32_ARGS);
            break;
    }
    CU_LAUNCH(ctx);
#undef SPMM32_CASE
#undef SPMM32_ARGS
    return apply_faces32<DIM>(ctx, tm, X, B, Y);
}

// the outflow-face pass after either FP32 apply kernel, then the timing event
template <int DIM>
static mlpg_status apply_faces32(mlpg_ctx *ctx, const Team &tm, const float *X, const float *B, float *Y) {
    cudaStream_t s = ctx->stream;
    if (ctx->nbrow > 0) {
        int64_t gb = team_grid(ctx->nbrow, tm);
        float sign = B ? -1.0f : 1.0f;
#define FACE_CASE(D) \
    case D: k_faces32<D, DIM><<<gb, 256, 0, s>>>(ctx->nbrow, ctx->m, tm.tm_log2, ctx->nb, ctx->brow, ctx->bptr, ctx->bcol, \
                                          ctx->bval32, ctx->coef32, X, sign, Y); break;
        switch (tm.dpl) {
            FACE_CASE(1) FACE_CASE(2) FACE_CASE(3) FACE_CASE(4) FACE_CASE(5) FACE_CASE(6) FACE_CASE(8)
            case 7: k_faces32<8, DIM><<<gb, 256, 0, s>>>(ctx->nbrow, ctx->m, tm.tm_log2, ctx->nb, ctx->brow, ctx->bptr,
                                                    ctx->bcol, ctx->bval32, ctx->coef32, X, sign, Y); break;
            default: k_faces32<16, DIM><<<gb, 256, 0, s>>>(ctx->nbrow, ctx->m, tm.tm_log2, ctx->nb, ctx->brow, ctx->bptr,
                                                       ctx->bcol, ctx->bval32, ctx->coef32, X, sign, Y); break;
        }
#undef FACE_CASE
        CU_LAUNCH(ctx);
    }
    timing_end(ctx);
    return MLPG_OK;
}

mlpg_status apply_L32_res(mlpg_ctx *ctx, const float *X, const float *B, float *Y) {
    return ctx->dim == 3 ? apply_L32_res_d<3>(ctx, X, B, Y) : apply_L32_res_d<2>(ctx, X, B, Y);
}

mlpg_status apply_L64(mlpg_ctx *ctx, const double *X, double *Y) { return apply_L64_res(ctx, X, nullptr, Y); }
mlpg_status apply_L32(mlpg_ctx *ctx, const float *X, float *Y) { return apply_L32_res(ctx, X, nullptr, Y); }

template <int DIM>
static mlpg_status rhs_T_d(mlpg_ctx *ctx, const double *Psi_prev, double *F) {
    Team tm = pick_team(ctx->m);
    cudaStream_t s = ctx->stream;
    const int64_t grid = rowteam_grid(ctx->n, tm);
#define RHS_ARGS ctx->n, ctx->m, tm.tm_log2, ctx->nnz, ctx->rowptr, ctx->col, ctx->T64, ctx->coef, Psi_prev, ctx->r64, F
    switch (tm.dpl) {
        case 1: k_rhs64<1, DIM><<<grid, 256, 0, s>>>(RHS_ARGS); break;
        case 2: k_rhs64<2, DIM><<<grid, 256, 0, s>>>(RHS_ARGS); break;
        case 3: k_rhs64<3, DIM><<<grid, 256, 0, s>>>(RHS_ARGS); break;
        case 4: k_rhs64<4, DIM><<<grid, 256, 0, s>>>(RHS_ARGS); break;
        case 5: case 6: k_rhs64<6, DIM><<<grid, 256, 0, s>>>(RHS_ARGS); break;
        case 7: case 8: k_rhs64<8, DIM><<<grid, 256, 0, s>>>(RHS_ARGS); break;
        default: k_rhs64<16, DIM><<<grid, 256, 0, s>>>(RHS_ARGS); break;
    }
#undef RHS_ARGS
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

mlpg_status rhs_T(mlpg_ctx *ctx, const double *Psi_prev, double *F) {
    return ctx->dim == 3 ? rhs_T_d<3>(ctx, Psi_prev, F) : rhs_T_d<2>(ctx, Psi_prev, F);
}

template <typename T, int D>
static mlpg_status apply_MS_d(mlpg_ctx *ctx, const double *phi, T *out) {
    const int64_t n = ctx->n;
    cudaStream_t s = ctx->stream;
    k_ms_spmv<D><<<(n + 255) / 256, 256, 0, s>>>(n, ctx->nnz, ctx->rowptr, ctx->col, ctx->S64, phi, ctx->abc);
    CU_LAUNCH(ctx);
    int64_t nm = n * ctx->m;
    if constexpr (sizeof(T) == 4) {
        float *abc32 = (float *)(ctx->abc + NT<D>() * n);
        k_abc32<<<(NT<D>() * n + 255) / 256, 256, 0, s>>>(NT<D>() * n, ctx->abc, abc32);
        CU_LAUNCH(ctx);
        k_ms_expand32<D><<<(nm + 255) / 256, 256, 0, s>>>(n, ctx->m, abc32, ctx->coef32, (float *)out);
    } else {
        k_ms_expand<T, D><<<(nm + 255) / 256, 256, 0, s>>>(n, ctx->m, ctx->abc, ctx->coef, out);
    }
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

template <typename T>
mlpg_status apply_MS(mlpg_ctx *ctx, const double *phi, T *out) {
    return ctx->dim == 3 ? apply_MS_d<T, 3>(ctx, phi, out) : apply_MS_d<T, 2>(ctx, phi, out);
}
template mlpg_status apply_MS<double>(mlpg_ctx *, const double *, double *);
template mlpg_status apply_MS<float>(mlpg_ctx *, const double *, float *);

template <typename T>
mlpg_status apply_prec(mlpg_ctx *ctx, T *v, T *z, const double *sc) {
    const size_t smem = sizeof(T) * (kB + 1) * ctx->m;
    if (smem > 200 * 1024) return set_err(ctx, MLPG_ERR_ARG, "too many directions for the block preconditioner");
    if (smem > 48 * 1024) {
        CU(ctx, cudaFuncSetAttribute(k_bjacobi_blk<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CU(ctx, cudaFuncSetAttribute(k_bjacobi_scalar<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CU(ctx, cudaFuncSetAttribute(k_bjacobi_h16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if constexpr (std::is_same<T, float>::value) {
        if (ctx->Pinv16) {   // one thread per (row, four directions) task, up to 256
            const int ntask = kB * (ctx->m >> 2);
            const int bs = ntask >= 256 ? 256 : (ntask + 31) / 32 * 32;
            k_bjacobi_h16<<<(unsigned)ctx->nblk, bs, smem, ctx->stream>>>(ctx->nblk, ctx->m, ctx->bmember,
                                                                          ctx->Pinv16, ctx->Pscale, v, sc, z);
            CU_LAUNCH(ctx);
            return MLPG_OK;
        }
    }
    if ((ctx->m & 3) == 0)
        k_bjacobi_blk<T><<<(unsigned)ctx->nblk, 256, smem, ctx->stream>>>(ctx->nblk, ctx->m, ctx->bmember, ctx->Pinv, v,
                                                                           sc, z);
    else
        k_bjacobi_scalar<T><<<(unsigned)ctx->nblk, 256, smem, ctx->stream>>>(ctx->nblk, ctx->m, ctx->bmember, ctx->Pinv,
                                                                              v, sc, z);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}
template mlpg_status apply_prec<double>(mlpg_ctx *, double *, double *, const double *);
template mlpg_status apply_prec<float>(mlpg_ctx *, float *, float *, const double *);

// Morton order of the points (host, once per point set) cut into blocks of
// MLPG_BLOCK_PTS consecutive points.
mlpg_status build_blocks(mlpg_ctx *ctx) {
    const int64_t n = ctx->n;
    const int d = ctx->dim;
    std::vector<std::pair<uint64_t, int32_t>> key(n);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t code = 0;
        uint32_t qv[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
            double t = (ctx->h_x[i * d + a] - ctx->opt.lo[a]) / (ctx->opt.hi[a] - ctx->opt.lo[a]);
            t = t < 0 ? 0 : (t > 1 ? 1 : t);
            qv[a] = (uint32_t)(t * 1048575.0);
        }
        for (int b = 19; b >= 0; --b)
            for (int a = d - 1; a >= 0; --a) code = (code << 1) | ((qv[a] >> b) & 1u);
        key[i] = {code, (int32_t)i};
    }
    std::sort(key.begin(), key.end());
    ctx->nblk = (n + kB - 1) / kB;
    std::vector<int32_t> member(ctx->nblk * kB, -1), bof(n);
    ctx->h_order.resize(n);
    for (int64_t r = 0; r < n; ++r) {
        member[r] = key[r].second;
        bof[key[r].second] = (int32_t)r;
        ctx->h_order[r] = key[r].second;
    }
    MLPG_TRY(dalloc(ctx, &ctx->bmember, ctx->nblk * kB));
    MLPG_TRY(dalloc(ctx, &ctx->bof, n));
    CU(ctx, cudaMemcpyAsync(ctx->bmember, member.data(), member.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                            ctx->stream));
    CU(ctx, cudaMemcpyAsync(ctx->bof, bof.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return MLPG_OK;
}

mlpg_status interp_flux(mlpg_ctx *ctx, double *out_dev, int kind) {
    const int64_t n = ctx->n;
    if (kind == 1) {
        CU(ctx, cudaMemcpyAsync(out_dev, ctx->Phi, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        return MLPG_OK;
    }
    k_interp_apply<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, ctx->rowptr, ctx->col, ctx->interp, ctx->Phi,
                                                              out_dev);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

}  // namespace mlpg
