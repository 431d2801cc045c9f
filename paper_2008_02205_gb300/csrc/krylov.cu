// Krylov solves of one backward-Euler step (Sec. 4.2).
//
// Batched GMRES: M independent systems advance together.  Vectors use the
// layout v[i][m] (system index fastest).  Each system has its own Hessenberg
// matrix, Givens rotations, residual estimate and convergence mask, all kept
// on the device; the host only polls the number of systems still iterating
// every few Arnoldi steps.  Orthogonalisation is classical Gram-Schmidt
// applied twice (CGS2) in FP64, or once in the FP32 correction solves (16-byte
// vectorised passes); block sums are formed in FP64 whatever the vector type.
// Right preconditioning by the block-Jacobi inverses (16-point Morton blocks)
// of each L_m.
//
// The same engine with M = 1 runs the scattering iteration on the
// scalar-flux coefficients, Eq. krylov-operator:
//   (I - D L^{-1} MS) Phi = D L^{-1} (T Psi^{n-1} + r),
// whose operator apply is one batched transport solve (all directions); it is
// unpreconditioned (the paper's) or right-preconditioned by the DSA-like
// diffusion correction (flexible GMRES), and with M = 1 it also solves the
// diffusion systems of that correction.
#include <algorithm>
#include <cmath>
#include <functional>
#include <type_traits>

#include "internal.h"

namespace mlpg {

namespace {

constexpr int kBlock = 256;
constexpr int kChunkRows = 8;   // FP32 partial sums over this many rows before the FP64 accumulator

// arithmetic type of the element-wise work: FP32 vectors are combined in FP32
template <typename T>
struct Arith { using type = double; };
template <>
struct Arith<float> { using type = float; };

struct Map2 {       // (direction, row) mapping of a 256-thread block
    int MB, RB, mchunks;
};
Map2 map2(int M) {
    Map2 r;
    r.MB = M <= kBlock ? M : kBlock;
    r.RB = kBlock / r.MB;
    r.mchunks = (M + r.MB - 1) / r.MB;
    return r;
}
// multiprocessors of the current device (queried once per device)
int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;
    }
    if (!cache[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        cache[dev] = v;
    }
    return cache[dev];
}
// row blocks of the streaming passes (about 8 per SM)
int row_blocks() { return 8 * sm_count(); }
int grid_rows(int64_t n, const Map2 &mp, int nl) {
    int64_t maxg = (n + mp.RB - 1) / mp.RB;
    int64_t g = (row_blocks() + mp.mchunks * nl - 1) / (mp.mchunks * nl);
    if (g > maxg) g = maxg;
    if (g < 1) g = 1;
    return (int)g;
}

// partial[(l * M + m) * G + block] = sum over this block's rows of V_l[i][m] * w[i][m]
template <typename T>
__global__ void __launch_bounds__(kBlock) k_dots(int64_t n, int M, int MB, int RB, const T *__restrict__ V,
                                                 int64_t vstride, const T *__restrict__ w,
                                                 double *__restrict__ partial) {
    using A = typename Arith<T>::type;
    __shared__ double sh[kBlock];
    const int t = threadIdx.x, ml = t % MB, r = t / MB;
    const int m = blockIdx.y * MB + ml, l = blockIdx.z, G = gridDim.x;
    double acc = 0.0;
    if (r < RB && m < M) {
        const T *v = V + l * vstride;
        const int64_t stride = (int64_t)G * RB;
        int64_t i = blockIdx.x * (int64_t)RB + r;
        while (i < n) {
            A part = 0;
#pragma unroll
            for (int c = 0; c < kChunkRows; ++c, i += stride)
                if (i < n) part += (A)v[i * M + m] * (A)w[i * M + m];
            acc += (double)part;
        }
    }
    sh[t] = acc;
    __syncthreads();
    if (r == 0 && m < M) {
        double s = 0.0;
        for (int k = 0; k < RB; ++k) s += sh[k * MB + ml];
        partial[((int64_t)l * M + m) * G + blockIdx.x] = s;
    }
}

// out[l * M + m] = sum_g partial[(l * M + m) * G + g]; one warp per output
// (contiguous partials), fixed lane order and shuffle tree: deterministic.
__device__ __forceinline__ double warp_sum_partials(const double *__restrict__ part, int G, int lane) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int g = lane;
    for (; g + 96 < G; g += 128) {
        s0 += part[g];
        s1 += part[g + 32];
        s2 += part[g + 64];
        s3 += part[g + 96];
    }
    for (; g < G; g += 32) s0 += part[g];
    double s = (s0 + s1) + (s2 + s3);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

__global__ void k_reduce(int M, int nl, int G, const double *__restrict__ partial, double *__restrict__ out) {
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)M * nl) return;
    const double s = warp_sum_partials(partial + wid * G, G, lane);
    if (lane == 0) out[wid] = s;
}

// w[i][m] -= sum_{l < nl} h[l][m] V_l[i][m]
template <typename T>
__global__ void k_update(int64_t n, int M, int nl, const T *__restrict__ V, int64_t vstride,
                         const double *__restrict__ h, T *__restrict__ w) {
    using A = typename Arith<T>::type;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * M) return;
    int m = (int)(e % M);
    A s = (A)w[e];
    for (int l = 0; l < nl; ++l) s -= (A)h[l * M + m] * (A)V[l * vstride + e];
    w[e] = (T)s;
}

// as k_update, and partial sums of the squared result (norm)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_update_norm(int64_t n, int M, int MB, int RB, int nl,
                                                        const T *__restrict__ V, int64_t vstride,
                                                        const double *__restrict__ h, T *__restrict__ w,
                                                        double *__restrict__ partial) {
    using A = typename Arith<T>::type;
    __shared__ double sh[kBlock];
    const int t = threadIdx.x, ml = t % MB, r = t / MB;
    const int m = blockIdx.y * MB + ml, G = gridDim.x;
    double acc = 0.0;
    if (r < RB && m < M) {
        const int64_t stride = (int64_t)G * RB;
        int64_t i = blockIdx.x * (int64_t)RB + r;
        while (i < n) {
            A part = 0;
#pragma unroll 1
            for (int c = 0; c < kChunkRows; ++c, i += stride) {
                if (i >= n) break;
                int64_t e = i * M + m;
                A s = (A)w[e];
                for (int l = 0; l < nl; ++l) s -= (A)h[l * M + m] * (A)V[l * vstride + e];
                T st = (T)s;
                w[e] = st;
                part += (A)st * (A)st;
            }
            acc += (double)part;
        }
    }
    sh[t] = acc;
    __syncthreads();
    if (r == 0 && m < M) {
        double s = 0.0;
        for (int k = 0; k < RB; ++k) s += sh[k * MB + ml];
        partial[(int64_t)m * G + blockIdx.x] = s;
    }
}

// One fused pass of classical Gram-Schmidt over the basis V_0..V_{nl-1}
// (all in registers for nl <= MAXL; each thread owns one system m and a
// strided set of rows):
//   MODE 0:  h_l = V_l . w
//   MODE 1:  w <- w - sum_l hin_l V_l, then h_l = V_l . w
//   MODE 2:  w <- w - sum_l hin_l V_l, then ||w||^2
// Block sums go to partial[(l * M + m) * G + block].
template <typename T, int MAXL, int MODE>
__global__ void __launch_bounds__(kBlock) k_cgs(int64_t n, int M, int MB, int RB, int nl,
                                                const T *__restrict__ V, int64_t vs,
                                                const double *__restrict__ hin, T *__restrict__ w,
                                                double *__restrict__ partial) {
    using A = typename Arith<T>::type;
    constexpr int NACC = MODE == 2 ? 1 : MAXL;
    constexpr int GRP = NACC < 8 ? NACC : 8;     // block sums staged per barrier pair
    __shared__ double sh[GRP][kBlock];
    const int t = threadIdx.x, ml = t % MB, r = t / MB;
    const int m = blockIdx.y * MB + ml, G = gridDim.x;
    const bool act = r < RB && m < M;
    A acc[NACC], hl[MAXL];
#pragma unroll
    for (int l = 0; l < NACC; ++l) acc[l] = 0;
#pragma unroll
    for (int l = 0; l < MAXL; ++l) hl[l] = (MODE >= 1 && act && l < nl) ? (A)hin[l * M + m] : (A)0;
    if (act) {
        const int64_t stride = (int64_t)G * RB;
        for (int64_t i = blockIdx.x * (int64_t)RB + r; i < n; i += stride) {
            const int64_t e = i * M + m;
            A wv = (A)w[e];
            if (MODE >= 1) {
#pragma unroll
                for (int l = 0; l < MAXL; ++l)
                    if (l < nl) wv -= hl[l] * (A)V[l * vs + e];
                w[e] = (T)wv;
                wv = (A)(T)wv;
            }
            if (MODE <= 1) {
#pragma unroll
                for (int l = 0; l < MAXL; ++l)
                    if (l < nl) acc[l] += (A)V[l * vs + e] * wv;
            } else {
                acc[0] += wv * wv;
            }
        }
    }
    if constexpr (NACC == 1) {   // one output (the norm pass)
        sh[0][t] = act ? (double)acc[0] : 0.0;
        __syncthreads();
        if (r == 0 && m < M) {
            double s = 0.0;
            for (int k = 0; k < RB; ++k) s += sh[0][k * MB + ml];
            partial[(int64_t)m * G + blockIdx.x] = s;
        }
        return;
    }
    // block sums of GRP outputs at a time: stage, one barrier, all threads reduce over RB
    const int nout = nl;
#pragma unroll
    for (int l0 = 0; l0 < NACC; l0 += GRP) {
        if (l0 < nout) {
#pragma unroll
            for (int g = 0; g < GRP; ++g) sh[g][t] = act ? (double)acc[l0 + g] : 0.0;
            __syncthreads();
            const int ng = min(GRP, nout - l0);
            for (int q = t; q < ng * MB; q += kBlock) {
                const int g = q / MB, mq = q - g * MB, mm = blockIdx.y * MB + mq;
                if (mm < M) {
                    double s = 0.0;
                    for (int k = 0; k < RB; ++k) s += sh[g][k * MB + mq];
                    partial[((int64_t)(l0 + g) * M + mm) * G + blockIdx.x] = s;
                }
            }
            __syncthreads();
        }
    }
}

template <typename T, int MODE>
static void launch_cgs(dim3 grid, cudaStream_t s, int64_t n, int M, int MB, int RB, int nl, const T *V,
                       int64_t vs, const double *hin, T *w, double *partial) {
    if (nl <= 4) k_cgs<T, 4, MODE><<<grid, kBlock, 0, s>>>(n, M, MB, RB, nl, V, vs, hin, w, partial);
    else if (nl <= 8) k_cgs<T, 8, MODE><<<grid, kBlock, 0, s>>>(n, M, MB, RB, nl, V, vs, hin, w, partial);
    else if (nl <= 16) k_cgs<T, 16, MODE><<<grid, kBlock, 0, s>>>(n, M, MB, RB, nl, V, vs, hin, w, partial);
    else k_cgs<T, 32, MODE><<<grid, kBlock, 0, s>>>(n, M, MB, RB, nl, V, vs, hin, w, partial);
}

// Vectorised Gram-Schmidt passes (M a multiple of VEC = 16 / sizeof(T)):
// thread (r, q) owns directions q*VEC .. q*VEC + VEC - 1 of the rows
// r, r + RB, ... of its block's row stride and moves them with 16-byte loads.
//   k_cgsv_dots:  h_l = V_l . w for l in group blockIdx.y (kDotGroup vectors
//                 per group, so that the accumulators stay in registers; w is
//                 re-read by each group, mostly from L2)
//   k_cgsv_upd:   w <- w - sum_{l < nl} hin_l V_l, then ||w||^2 (hin staged
//                 in shared memory)
// Block sums go to partial[(l * M + m) * G + block], G = gridDim.x.
constexpr int kDotGroup = 8;
constexpr int kGsBlocksPerSm = 4;   // grid of the vectorised passes (measured: 2 -> 4 saves 2.7 % of a step, 8 loses)
constexpr int kDsaRestart = 30;   // restart length of the diffusion solves
constexpr size_t kUpdSmem = 96 * 1024;   // largest staged Hessenberg column block of k_cgsv_upd
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };
__device__ __forceinline__ void unpack(const float4 &v, float *o) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
__device__ __forceinline__ void unpack(const double2 &v, double *o) { o[0] = v.x; o[1] = v.y; }
__device__ __forceinline__ float4 pack4(const float *o) { return make_float4(o[0], o[1], o[2], o[3]); }
__device__ __forceinline__ double2 pack2(const double *o) { return make_double2(o[0], o[1]); }
template <typename T> __device__ __forceinline__ typename Vec16<T>::type pack(const T *o);
template <> __device__ __forceinline__ float4 pack<float>(const float *o) { return pack4(o); }
template <> __device__ __forceinline__ double2 pack<double>(const double *o) { return pack2(o); }

// Block sums of `nacc` accumulators per thread (VEC components each) over the
// RB row slots, staged through shared memory kDotGroup accumulators at a time.
template <typename T, int VEC>
__device__ __forceinline__ void block_sums(const T (*acc)[VEC], int nacc, int l0, int M, int MQ, int RB, bool act,
                                           double *__restrict__ partial, int G) {
    __shared__ T sh[kDotGroup * kBlock * VEC];
    const int t = threadIdx.x, q = t % MQ, r = t / MQ;
    const int RM = RB * M;   // staged values per accumulator
    for (int a0 = 0; a0 < nacc; a0 += kDotGroup) {
        const int na = min(kDotGroup, nacc - a0);
        if (act)
            for (int a = 0; a < na; ++a)
#pragma unroll
                for (int c = 0; c < VEC; ++c) sh[a * RM + r * M + q * VEC + c] = acc[a0 + a][c];
        __syncthreads();
        for (int o = t; o < na * M; o += kBlock) {
            const int a = o / M, m = o - a * M;
            double sum = 0.0;
            for (int k = 0; k < RB; ++k) sum += (double)sh[a * RM + k * M + m];
            partial[((int64_t)(l0 + a0 + a) * M + m) * G + blockIdx.x] = sum;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_cgsv_dots(int64_t n, int M, int nl, const T *__restrict__ V, int64_t vs,
                                                      const T *__restrict__ w, double *__restrict__ partial) {
    using A = typename Arith<T>::type;
    using V16 = typename Vec16<T>::type;
    constexpr int VEC = Vec16<T>::n;
    const int MQ = M / VEC, RB = kBlock / MQ, G = gridDim.x;
    const int t = threadIdx.x, q = t % MQ, r = t / MQ;
    const bool act = r < RB;
    const int l0 = blockIdx.y * kDotGroup, nlg = min(kDotGroup, nl - l0);
    A acc[kDotGroup][VEC];
#pragma unroll
    for (int a = 0; a < kDotGroup; ++a)
#pragma unroll
        for (int c = 0; c < VEC; ++c) acc[a][c] = 0;
    if (act) {
        const int64_t stride = (int64_t)G * RB;
        for (int64_t i = blockIdx.x * (int64_t)RB + r; i < n; i += stride) {
            const int64_t e = i * M + q * VEC;
            T wv[VEC];
            unpack(__ldg(reinterpret_cast<const V16 *>(w + e)), wv);
#pragma unroll
            for (int a = 0; a < kDotGroup; ++a) {
                if (a < nlg) {
                    T v[VEC];
                    unpack(__ldg(reinterpret_cast<const V16 *>(V + (l0 + a) * vs + e)), v);
#pragma unroll
                    for (int c = 0; c < VEC; ++c) acc[a][c] += (A)v[c] * (A)wv[c];
                }
            }
        }
    }
    block_sums<A, VEC>(acc, nlg, l0, M, MQ, RB, act, partial, G);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_cgsv_upd(int64_t n, int M, int nl, const T *__restrict__ V, int64_t vs,
                                                     const double *__restrict__ hin, T *__restrict__ w,
                                                     double *__restrict__ partial) {
    using A = typename Arith<T>::type;
    using V16 = typename Vec16<T>::type;
    constexpr int VEC = Vec16<T>::n;
    extern __shared__ unsigned char smem_h[];
    A *hs = reinterpret_cast<A *>(smem_h);   // [nl][M]
    const int MQ = M / VEC, RB = kBlock / MQ, G = gridDim.x;
    const int t = threadIdx.x, q = t % MQ, r = t / MQ;
    const bool act = r < RB;
    for (int k = t; k < nl * M; k += kBlock) hs[k] = (A)hin[k];
    __syncthreads();
    A acc[1][VEC];
#pragma unroll
    for (int c = 0; c < VEC; ++c) acc[0][c] = 0;
    if (act) {
        const int64_t stride = (int64_t)G * RB;
        for (int64_t i = blockIdx.x * (int64_t)RB + r; i < n; i += stride) {
            const int64_t e = i * M + q * VEC;
            T wt[VEC];
            unpack(*reinterpret_cast<const V16 *>(w + e), wt);
            A wv[VEC];
#pragma unroll
            for (int c = 0; c < VEC; ++c) wv[c] = (A)wt[c];
#pragma unroll 4
            for (int l = 0; l < nl; ++l) {
                T v[VEC];
                unpack(__ldg(reinterpret_cast<const V16 *>(V + l * vs + e)), v);
                const A *hl = hs + l * M + q * VEC;
#pragma unroll
                for (int c = 0; c < VEC; ++c) wv[c] -= hl[c] * (A)v[c];
            }
#pragma unroll
            for (int c = 0; c < VEC; ++c) {
                wt[c] = (T)wv[c];
                acc[0][c] += (A)wt[c] * (A)wt[c];
            }
            *reinterpret_cast<V16 *>(w + e) = pack<T>(wt);
        }
    }
    block_sums<A, VEC>(acc, 1, 0, M, MQ, RB, act, partial, G);
}

// Start of a cycle: beta = ||r|| (nrm2 = ||r||^2); decide which systems iterate.
__global__ void k_start(int M, int R, const double *__restrict__ nrm2, double *__restrict__ bnorm,
                        double *__restrict__ g, double *__restrict__ sc, int *__restrict__ active,
                        int *__restrict__ kcol, double *__restrict__ resid, double tol, int set_bnorm,
                        int *__restrict__ count) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double beta = sqrt(nrm2[m]);
    if (set_bnorm) bnorm[m] = beta;
    resid[m] = beta;
    kcol[m] = 0;
    bool act = beta > tol * bnorm[m] && beta > 0.0;
    active[m] = act;
    g[m * (R + 1)] = beta;
    for (int k = 1; k <= R; ++k) g[m * (R + 1) + k] = 0.0;
    sc[m] = act ? 1.0 / beta : 0.0;
    if (act) atomicAdd(count, 1);
}

// Column j of the Hessenberg matrix, Givens rotations, residual estimate.
// One warp per system: the warp first sums the G norm partials of ||w||^2.
__global__ void k_givens(int M, int R, int j, int G, const double *__restrict__ partial,
                         const double *__restrict__ h1, const double *__restrict__ h2, double *__restrict__ H,
                         double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
                         double *__restrict__ sc, int *__restrict__ active, int *__restrict__ kcol,
                         int *__restrict__ its, double *__restrict__ resid, const double *__restrict__ bnorm,
                         double tol, int *__restrict__ count) {
    const int m = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= M) return;
    if (!active[m]) {
        if (lane == 0) sc[m] = 0.0;
        return;
    }
    const double nrm2 = warp_sum_partials(partial + (int64_t)m * G, G, lane);
    const double hn = sqrt(nrm2);
    double *Hm = H + (int64_t)m * (R + 1) * R;  // Hm[row * R + col]
    // lane l holds entry l of the new column (l <= j < R <= 32) and the earlier rotation l (l < j);
    // every lane runs the same rotation chain down the column in registers and keeps its own entry
    double hl = 0.0, cl = 1.0, sl = 0.0;
    if (lane <= j) hl = h1[lane * M + m] + (h2 ? h2[lane * M + m] : 0.0);
    if (lane < j) {
        cl = cs[m * R + lane];
        sl = sn[m * R + lane];
    }
    double carry = __shfl_sync(0xffffffffu, hl, 0), mine = 0.0;
    for (int l = 0; l < j; ++l) {
        const double c = __shfl_sync(0xffffffffu, cl, l), sv = __shfl_sync(0xffffffffu, sl, l);
        const double b = __shfl_sync(0xffffffffu, hl, l + 1);
        const double a = carry;
        const double r = c * a + sv * b;
        carry = -sv * a + c * b;
        if (lane == l) mine = r;
    }
    if (lane < j) Hm[lane * R + j] = mine;
    if (lane != 0) return;
    // the new rotation zeroes the subdiagonal entry hn
    double a = carry, b = hn;
    double den = hypot(a, b);
    double c = den > 0.0 ? a / den : 1.0, sv = den > 0.0 ? b / den : 0.0;
    cs[m * R + j] = c;
    sn[m * R + j] = sv;
    Hm[j * R + j] = den;
    Hm[(j + 1) * R + j] = 0.0;
    double gj = g[m * (R + 1) + j];
    g[m * (R + 1) + j] = c * gj;
    g[m * (R + 1) + j + 1] = -sv * gj;
    its[m] += 1;
    kcol[m] = j + 1;
    double res = fabs(sv * gj);
    resid[m] = res;
    bool done = res <= tol * bnorm[m] || !(hn > 0.0) || j + 1 == R;
    if (done) {
        active[m] = 0;
        sc[m] = 0.0;
    } else {
        sc[m] = 1.0 / hn;
        atomicAdd(count, 1);
    }
}

// w = w * sc[m]  (in the vector's own precision)
template <typename T>
__global__ void k_scale(int64_t n, int M, T *__restrict__ w, const double *__restrict__ sc) {
    using A = typename Arith<T>::type;
    __shared__ A ssc[MLPG_MAX_DIR];
    for (int k = threadIdx.x; k < M; k += blockDim.x) ssc[k] = (A)sc[k];
    __syncthreads();
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * M) return;
    int m = (int)(e % M);
    w[e] = (T)((A)w[e] * ssc[m]);
}

// y = R^{-1} g per system (upper triangular part of the rotated Hessenberg);
// also a float copy for FP32 vectors
__global__ void k_backsolve(int M, int R, const double *__restrict__ H, const double *__restrict__ g,
                            const int *__restrict__ kcol, double *__restrict__ y, float *__restrict__ y32) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int k = kcol[m];
    const double *Hm = H + (int64_t)m * (R + 1) * R;
    for (int r = k - 1; r >= 0; --r) {
        double s = g[m * (R + 1) + r];
        for (int c = r + 1; c < k; ++c) s -= Hm[r * R + c] * y[c * M + m];
        y[r * M + m] = Hm[r * R + r] != 0.0 ? s / Hm[r * R + r] : 0.0;
        y32[r * M + m] = (float)y[r * M + m];
    }
}

template <typename T>
static const typename Arith<T>::type *y_of(const Gmres<T> &G);
template <>
const double *y_of<double>(const Gmres<double> &G) { return G.y; }
template <>
const float *y_of<float>(const Gmres<float> &G) { return G.y32; }

// u = sum_{l < kcol[m]} y_l V_l, with y already in the vector's arithmetic type
template <typename T>
__global__ void k_combine(int64_t n, int M, int kmax, const T *__restrict__ V, int64_t vstride,
                          const typename Arith<T>::type *__restrict__ y, const int *__restrict__ kcol,
                          T *__restrict__ u) {
    using A = typename Arith<T>::type;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * M) return;
    int m = (int)(e % M);
    int k = min(kcol[m], kmax);
    A s = 0;
    for (int l = 0; l < k; ++l) s += y[l * M + m] * (A)V[l * vstride + e];
    u[e] = (T)s;
}

// acc += sum_{l < kcol[0]} y_l bank_l   (single system: the outer solve)
template <typename T>
__global__ void k_bank_combine(int64_t N, int kmax, const T *__restrict__ bank,
                               const typename Arith<T>::type *__restrict__ y, const int *__restrict__ kcol,
                               T *__restrict__ acc) {
    using A = typename Arith<T>::type;
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    const int k = min(kcol[0], kmax);
    A s = (A)acc[e];
    for (int l = 0; l < k; ++l) s += y[l] * (A)bank[(int64_t)l * N + e];
    acc[e] = (T)s;
}

// total += sum_m its[m]  (one warp)
__global__ void k_bump(long long *__restrict__ c) { *c += 1; }

// source-iteration update: d <- b_phi + d (the new Phi), e <- d - phi, phi <- d
__global__ void k_si_update(int64_t n, const double *__restrict__ bphi, double *__restrict__ d,
                            double *__restrict__ phi, double *__restrict__ e) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = bphi[i] + d[i];
    e[i] = v - phi[i];
    phi[i] = v;
    d[i] = v;
}

__global__ void k_add_its(int M, const int *__restrict__ its, long long *__restrict__ total) {
    long long s = 0;
    for (int m = threadIdx.x; m < M; m += 32) s += its[m];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *total += s;
}

template <typename T>
__global__ void k_axpy1(int64_t N, const T *__restrict__ u, T *__restrict__ x) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < N) x[e] += u[e];
}

// out[i] = sum_m w[m] x[i][m]  (angular reduction D, Sec. 4.2)
template <typename T>
__global__ void k_Dreduce(int64_t n, int M, const double *__restrict__ w, const T *__restrict__ x,
                          double *__restrict__ out) {
    using A = typename Arith<T>::type;
    int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (i >= n) return;
    A sl = 0;
    for (int m = lane; m < M; m += 32) sl += (A)w[m] * (A)x[i * M + m];
    double s = (double)sl;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
}

template <typename Ti, typename To>
__global__ void k_convert(int64_t N, const Ti *__restrict__ a, To *__restrict__ b) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < N) b[e] = (To)a[e];
}

// Initial guess of a step from the last states, in place:
//   psi <- a psi + b h1 + c h2   (psi = Psi^{n-1}, h1 = Psi^{n-2}, h2 = Psi^{n-3})
// and h2 <- Psi^{n-1} (h2 becomes the newest history entry).
__global__ void k_extrap(int64_t N, double a, double b, double c, double *__restrict__ psi,
                         const double *__restrict__ h1, double *__restrict__ h2) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N) return;
    const double p = psi[e];
    // a history entry with a zero weight is not read: it may not hold a state yet
    double v = a * p;
    if (b != 0.0) v += b * h1[e];
    if (c != 0.0) v += c * h2[e];
    psi[e] = v;
    h2[e] = p;
}

// c = a + b (mixed types; c may alias a)
template <typename Ta, typename Tb>
__global__ void k_add(int64_t N, const Ta *a, const Tb *__restrict__ b, double *c) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < N) c[e] = (double)a[e] + (double)b[e];
}

// y = B - (X - d)   or   y = X - d       (outer operator I - D L^{-1} MS)
__global__ void k_outer_combine(int64_t n, const double *__restrict__ X, const double *__restrict__ d,
                                const double *__restrict__ B, double *__restrict__ Y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = X[i] - d[i];
    Y[i] = B ? B[i] - v : v;
}

// partial sums of squares over N elements (for global norms)
__global__ void k_sumsq(int64_t N, const double *__restrict__ a, double *__restrict__ partial) {
    __shared__ double sh[kBlock];
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        s += a[e] * a[e];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kBlock / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

inline int64_t nblk(int64_t N) { return (N + kBlock - 1) / kBlock; }

}  // namespace

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
template <typename T>
static mlpg_status gmres_alloc(mlpg_ctx *ctx, Gmres<T> &G, int64_t n, int M, int R, bool flexible = false) {
    if (G.n == n && G.M == M && G.R == R && (!flexible || G.Zf)) return MLPG_OK;
    if (G.n == n && G.M == M && G.R == R) {   // the same shape: only the flexible buffer is new
        MLPG_TRY(dalloc(ctx, &G.Zf, (size_t)R * n * M));
        return MLPG_OK;
    }
    if (R > MLPG_MAX_RESTART || R < 1) return set_err(ctx, MLPG_ERR_ARG, "restart length out of range");
    G.n = n; G.M = M; G.R = R;
    MLPG_TRY(dalloc(ctx, &G.V, (size_t)(R + 1) * n * M));
    MLPG_TRY(dalloc(ctx, &G.Z, (size_t)n * M));
    MLPG_TRY(dalloc(ctx, &G.W, (size_t)n * M));
    MLPG_TRY(dalloc(ctx, &G.H, (size_t)M * (R + 1) * R));
    MLPG_TRY(dalloc(ctx, &G.cs, (size_t)M * R));
    MLPG_TRY(dalloc(ctx, &G.sn, (size_t)M * R));
    MLPG_TRY(dalloc(ctx, &G.g, (size_t)M * (R + 1)));
    MLPG_TRY(dalloc(ctx, &G.h, (size_t)(R + 1) * M));
    MLPG_TRY(dalloc(ctx, &G.h2, (size_t)(R + 1) * M));
    MLPG_TRY(dalloc(ctx, &G.y, (size_t)R * M));
    MLPG_TRY(dalloc(ctx, &G.y32, (size_t)R * M));
    MLPG_TRY(dalloc(ctx, &G.bnorm, M));
    MLPG_TRY(dalloc(ctx, &G.nrm2, M));
    MLPG_TRY(dalloc(ctx, &G.beta, M));   // scale factors 1/||w||
    MLPG_TRY(dalloc(ctx, &G.resid, M));
    MLPG_TRY(dalloc(ctx, &G.active, M));
    MLPG_TRY(dalloc(ctx, &G.kcol, M));
    MLPG_TRY(dalloc(ctx, &G.its, M));
    // the fused Gram-Schmidt passes write G * nl * M partials with G <= row_blocks(), nl <= R + 1
    G.partial_cap = (int64_t)row_blocks() * (R + 1) * M;
    MLPG_TRY(dalloc(ctx, &G.partial, G.partial_cap));
    MLPG_TRY(dalloc(ctx, &G.d_active_count, 1));
    if (flexible) MLPG_TRY(dalloc(ctx, &G.Zf, (size_t)R * n * M));
    CU(ctx, cudaFuncSetAttribute(k_cgsv_upd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUpdSmem));
    void *hp = nullptr;
    CU(ctx, cudaHostAlloc(&hp, sizeof(int) * 4, cudaHostAllocDefault));
    ctx->host_allocs.push_back(hp);
    G.h_active = (int *)hp;
    return MLPG_OK;
}

template <typename T>
using ApplyFn = std::function<mlpg_status(const T *X, const T *B, T *Y)>;
template <typename T>
using PrecFn = std::function<mlpg_status(T *v, T *z, const double *sc)>;  // z = P^{-1} (v *= sc)
// called after each cycle's least-squares solve: y (FP64 and FP32 copies), kcol
using CycleFn = std::function<mlpg_status(const double *y, const float *y32, const int *kcol, int kmax)>;

// Solve A x = b for all M systems, right preconditioned by P (identity when
// empty); x holds the initial guess.  Returns the summed iteration count in
// *iters and MLPG_ERR_NOT_CONVERGED on the cap; with cap_ok the iterate
// reached at the cap is kept instead (an approximate solve).
template <typename T>
static mlpg_status gmres_solve(mlpg_ctx *ctx, Gmres<T> &G, const ApplyFn<T> &A, const PrecFn<T> &P, const T *b,
                               T *x, double tol, int max_its, int check_every, int64_t *iters,
                               const CycleFn &on_cycle = CycleFn(), int *slot = nullptr, bool x_zero = false,
                               bool cap_ok = false) {
    const int64_t n = G.n, N = n * G.M;
    const int M = G.M, R = G.R;
    const int64_t vs = N;
    cudaStream_t s = ctx->stream;
    const Map2 mp = map2(M);
    const int wblk = (int)((M * 32 + kBlock - 1) / kBlock);
    using Ar = typename Arith<T>::type;
    constexpr int VEC = Vec16<T>::n;
    const bool vec_ok = M % VEC == 0 && M / VEC <= kBlock;
    const int64_t vrows = vec_ok ? (n + kBlock / (M / VEC) - 1) / (kBlock / (M / VEC)) : 1;   // row iterations
    CU(ctx, cudaMemsetAsync(G.its, 0, sizeof(int) * M, s));
    auto norm2 = [&](const T *v) -> mlpg_status {   // G.nrm2[m] = ||v_m||^2
        int g1 = grid_rows(n, mp, 1);
        k_dots<T><<<dim3(g1, mp.mchunks, 1), kBlock, 0, s>>>(n, M, mp.MB, mp.RB, v, 0, v, G.partial);
        CU_LAUNCH(ctx);
        k_reduce<<<wblk, kBlock, 0, s>>>(M, 1, g1, G.partial, G.nrm2);
        CU_LAUNCH(ctx);
        return MLPG_OK;
    };
    // normalise v by sc (when given) and precondition: returns the vector to apply A to
    auto precond = [&](T *v, T *z, const double *sc) -> const T * {
        if (!P) {
            if (sc) k_scale<T><<<nblk(N), kBlock, 0, s>>>(n, M, v, sc);
            return cudaGetLastError() == cudaSuccess ? v : nullptr;
        }
        return P(v, z, sc) == MLPG_OK ? z : nullptr;
    };
    int64_t total = 0;
    for (int cycle = 0;; ++cycle) {
        // an approximate solve (cap_ok) keeps its iterate at the cap, without a final residual
        if (cap_ok && cycle > 0 && (int64_t)cycle * R >= max_its) break;
        const bool first_zero = cycle == 0 && x_zero;   // r = b: no operator apply needed
        if (cycle == 0 && !x_zero) {
            MLPG_TRY(norm2(b));
            CU(ctx, cudaMemsetAsync(G.d_active_count, 0, sizeof(int), s));
            k_start<<<(M + 127) / 128, 128, 0, s>>>(M, R, G.nrm2, G.bnorm, G.g, G.beta, G.active, G.kcol, G.resid,
                                                    0.0, 1, G.d_active_count);
            CU_LAUNCH(ctx);
        }
        if (first_zero) {
            CU(ctx, cudaMemcpyAsync(G.V, b, sizeof(T) * N, cudaMemcpyDeviceToDevice, s));
        } else {
            if (slot) *slot = cycle == 0 ? -1 : -2;   // -1: first residual, -2: later residuals
            MLPG_TRY(A(x, b, G.V));  // r = b - A x -> V_0
        }
        MLPG_TRY(norm2(G.V));
        CU(ctx, cudaMemsetAsync(G.d_active_count, 0, sizeof(int), s));
        k_start<<<(M + 127) / 128, 128, 0, s>>>(M, R, G.nrm2, G.bnorm, G.g, G.beta, G.active, G.kcol, G.resid, tol,
                                                first_zero ? 1 : 0, G.d_active_count);
        CU_LAUNCH(ctx);
        if (!first_zero) {
            // later cycles: stop when every system has converged.  (A first cycle
            // from x = 0 always iterates; systems with b = 0 are masked.)
            CU(ctx, cudaMemcpyAsync(G.h_active, G.d_active_count, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(ctx, cudaStreamSynchronize(s));
            if (*G.h_active == 0) break;
        }
        if ((int64_t)cycle * R >= max_its) {
            k_add_its<<<1, 32, 0, s>>>(M, G.its, ctx->d_its + G.its_slot);
            return set_err(ctx, MLPG_ERR_NOT_CONVERGED, "GMRES reached its iteration cap");
        }
        // flexible GMRES keeps every preconditioned basis vector (the preconditioner may change between applies)
        const T *z = precond(G.V, G.Zf ? G.Zf : G.Z, G.beta);
        if (!z) return MLPG_ERR_CUDA;
        int jlast = 0;
        for (int j = 0; j < R; ++j) {
            T *w = G.V + (j + 1) * vs;
            if (slot) *slot = j;                      // operator applied to basis vector j
            MLPG_TRY(A(z, nullptr, w));
            int gnorm = 0;
            const int nl = j + 1;
            if (vec_ok && !G.reorth && (size_t)nl * M * sizeof(Ar) <= kUpdSmem) {
                // single classical pass, 16-byte vectors: dots (groups of kDotGroup
                // basis vectors per grid row), reduce, update + norm partials
                const int ng = (nl + kDotGroup - 1) / kDotGroup;
                // kGsBlocksPerSm blocks per SM: enough loads in flight, few partial sums for k_reduce / k_givens
                const int gd = (int)std::max<int64_t>(
                    1, std::min<int64_t>(vrows, (kGsBlocksPerSm * sm_count() + ng - 1) / ng));
                if ((int64_t)gd * nl * M > G.partial_cap || (int64_t)kGsBlocksPerSm * sm_count() * M > G.partial_cap)
                    return set_err(ctx, MLPG_ERR_ARG, "reduction buffer too small");
                k_cgsv_dots<T><<<dim3(gd, ng), kBlock, 0, s>>>(n, M, nl, G.V, vs, w, G.partial);
                CU_LAUNCH(ctx);
                k_reduce<<<(int)(((int64_t)nl * M * 32 + kBlock - 1) / kBlock), kBlock, 0, s>>>(M, nl, gd, G.partial,
                                                                                              G.h);
                CU_LAUNCH(ctx);
                const int gu = (int)std::max<int64_t>(1, std::min<int64_t>(vrows, kGsBlocksPerSm * sm_count()));
                k_cgsv_upd<T><<<gu, kBlock, (size_t)nl * M * sizeof(Ar), s>>>(n, M, nl, G.V, vs, G.h, w, G.partial);
                CU_LAUNCH(ctx);
                gnorm = gu;
            } else {
                // CGS2 in three fused passes over V_0..V_j (CGS1: two passes, h2 unused)
                // fewer, longer-running blocks as the basis grows (bounded partial sums)
                const int g1 = grid_rows(n, mp, (nl + 3) / 4);
                const dim3 grid(g1, mp.mchunks);
                if ((int64_t)g1 * nl * mp.mchunks * mp.MB > G.partial_cap)
                    return set_err(ctx, MLPG_ERR_ARG, "reduction buffer too small");
                const int rblk = (int)(((int64_t)nl * M * 32 + kBlock - 1) / kBlock);
                launch_cgs<T, 0>(grid, s, n, M, mp.MB, mp.RB, nl, G.V, vs, nullptr, w, G.partial);
                CU_LAUNCH(ctx);
                k_reduce<<<rblk, kBlock, 0, s>>>(M, nl, g1, G.partial, G.h);
                CU_LAUNCH(ctx);
                if (G.reorth) {
                    launch_cgs<T, 1>(grid, s, n, M, mp.MB, mp.RB, nl, G.V, vs, G.h, w, G.partial);
                    CU_LAUNCH(ctx);
                    k_reduce<<<rblk, kBlock, 0, s>>>(M, nl, g1, G.partial, G.h2);
                    CU_LAUNCH(ctx);
                }
                launch_cgs<T, 2>(grid, s, n, M, mp.MB, mp.RB, nl, G.V, vs, G.reorth ? G.h2 : G.h, w, G.partial);
                CU_LAUNCH(ctx);
                gnorm = g1;   // the norm partials are reduced inside k_givens
            }
            CU(ctx, cudaMemsetAsync(G.d_active_count, 0, sizeof(int), s));
            k_givens<<<wblk, kBlock, 0, s>>>(M, R, j, gnorm, G.partial, G.h, G.reorth ? G.h2 : nullptr, G.H, G.cs, G.sn, G.g, G.beta,
                                             G.active, G.kcol, G.its, G.resid, G.bnorm, tol, G.d_active_count);
            CU_LAUNCH(ctx);
            jlast = j;
            bool check = (j + 1) % check_every == 0 || j + 1 == R;
            if (check) {
                CU(ctx, cudaMemcpyAsync(G.h_active, G.d_active_count, sizeof(int), cudaMemcpyDeviceToHost, s));
                CU(ctx, cudaStreamSynchronize(s));
                if (*G.h_active == 0) break;
            }
            if (j + 1 == R) break;   // no next basis vector in this cycle
            z = precond(w, G.Zf ? G.Zf + (int64_t)(j + 1) * N : G.Z, G.beta);
            if (!z) return MLPG_ERR_CUDA;
        }
        k_backsolve<<<(M + 127) / 128, 128, 0, s>>>(M, R, G.H, G.g, G.kcol, G.y, G.y32);
        CU_LAUNCH(ctx);
        if (on_cycle) MLPG_TRY(on_cycle(G.y, G.y32, G.kcol, jlast + 1));
        const T *u = G.W;
        if (G.Zf) {   // x += sum_l y_l z_l
            k_combine<T><<<nblk(N), kBlock, 0, s>>>(n, M, jlast + 1, G.Zf, vs, y_of<T>(G), G.kcol, G.W);
            CU_LAUNCH(ctx);
        } else {      // x += P^{-1} sum_l y_l v_l
            k_combine<T><<<nblk(N), kBlock, 0, s>>>(n, M, jlast + 1, G.V, vs, y_of<T>(G), G.kcol, G.W);
            CU_LAUNCH(ctx);
            u = precond(G.W, G.Z, nullptr);
            if (!u) return MLPG_ERR_CUDA;
        }
        k_axpy1<T><<<nblk(N), kBlock, 0, s>>>(N, u, x);
        CU_LAUNCH(ctx);
    }
    // iteration counts stay on the device (summed into ctx->d_its, read once per step)
    k_add_its<<<1, 32, 0, s>>>(M, G.its, ctx->d_its + G.its_slot);
    CU_LAUNCH(ctx);
    *iters = total;
    return MLPG_OK;
}

// ---------------------------------------------------------------------------
// one batched transport solve L_m x_m = b_m, all directions (x0 = 0)
// ---------------------------------------------------------------------------
template <typename T>
static mlpg_status inner_solve(mlpg_ctx *ctx, const T *b, T *x, double tol);

template <>
mlpg_status inner_solve<double>(mlpg_ctx *ctx, const double *b, double *x, double tol) {
    MLPG_TRY(gmres_alloc(ctx, ctx->g64, ctx->n, ctx->m, ctx->opt.inner_restart));
    CU(ctx, cudaMemsetAsync(x, 0, sizeof(double) * ctx->n * ctx->m, ctx->stream));
    ApplyFn<double> A = [ctx](const double *X, const double *B, double *Y) { return apply_L64_res(ctx, X, B, Y); };
    PrecFn<double> P = [ctx](double *v, double *z, const double *sc) { return apply_prec<double>(ctx, v, z, sc); };
    int64_t its = 0;
    mlpg_status st = gmres_solve<double>(ctx, ctx->g64, A, P, b, x, tol, ctx->opt.max_inner,
                                         ctx->opt.check_every, &its, CycleFn(), nullptr, true);
    (void)its;
    ctx->st.last_inner_solves += 1;
    return st;
}

template <>
mlpg_status inner_solve<float>(mlpg_ctx *ctx, const float *b, float *x, double tol) {
    MLPG_TRY(gmres_alloc(ctx, ctx->g32, ctx->n, ctx->m, ctx->opt.mixed_restart));
    ctx->g32.reorth = ctx->opt.mixed_reorth != 0;
    CU(ctx, cudaMemsetAsync(x, 0, sizeof(float) * ctx->n * ctx->m, ctx->stream));
    ApplyFn<float> A = [ctx](const float *X, const float *B, float *Y) { return apply_L32_res(ctx, X, B, Y); };
    PrecFn<float> P = [ctx](float *v, float *z, const double *sc) { return apply_prec<float>(ctx, v, z, sc); };
    int64_t its = 0;
    mlpg_status st = gmres_solve<float>(ctx, ctx->g32, A, P, b, x, tol, ctx->opt.max_inner,
                                        ctx->opt.check_every, &its, CycleFn(), nullptr, true, true);
    (void)its;
    ctx->st.last_inner_solves += 1;
    return st;
}

static mlpg_status ensure_step_buffers(mlpg_ctx *ctx) {
    if (ctx->f64) return MLPG_OK;
    const size_t N = (size_t)ctx->n * ctx->m;
    MLPG_TRY(dalloc(ctx, &ctx->f64, N));
    MLPG_TRY(dalloc(ctx, &ctx->res64, N));
    MLPG_TRY(dalloc(ctx, &ctx->tmp64, N));
    MLPG_TRY(dalloc(ctx, &ctx->bpsi64, N));
    MLPG_TRY(dalloc(ctx, &ctx->rhs64b, N));
    MLPG_TRY(dalloc(ctx, &ctx->sol64, N));
    MLPG_TRY(dalloc(ctx, &ctx->rhs32, N));
    MLPG_TRY(dalloc(ctx, &ctx->sol32, N));
    MLPG_TRY(dalloc(ctx, &ctx->bpsi32, N));
    if (!ctx->nvec) MLPG_TRY(dalloc(ctx, &ctx->nvec, 8 * ctx->n));   // mlpg_scalar_flux may have made it
    ctx->red_cap = 4096;
    MLPG_TRY(dalloc(ctx, &ctx->red, ctx->red_cap));
    void *hp = nullptr;
    CU(ctx, cudaHostAlloc(&hp, sizeof(double) * 16, cudaHostAllocDefault));
    ctx->host_allocs.push_back(hp);
    ctx->h_red = (double *)hp;
    return MLPG_OK;
}

template <typename T>
static mlpg_status outer_bank(mlpg_ctx *ctx, int R, T **bank, T **xacc) {
    const size_t N = (size_t)ctx->n * ctx->m;
    void **slotp = sizeof(T) == 8 ? &ctx->bank64 : &ctx->bank32;
    if (!*slotp) {
        T *p = nullptr;
        MLPG_TRY(dalloc(ctx, &p, (size_t)(R + 1) * N));
        *slotp = p;
    }
    T *base = static_cast<T *>(*slotp);
    *bank = base;
    *xacc = base + (size_t)R * N;
    return MLPG_OK;
}

// DSA-like right preconditioner of the outer solve: z = v + C^{-1} Ms v, the
// scattering source of the Krylov direction v driving a diffusion correction
// (C: form_diffusion).  The diffusion system is solved by FP64 GMRES with
// block-Jacobi (the blocks of C), to dsa_tol; the outer GMRES is flexible, so
// an inexact diffusion solve changes iterations, not the solution.
static mlpg_status dsa_precond(mlpg_ctx *ctx, double *v, double *z, const double *sc) {
    const int64_t n = ctx->n;
    cudaStream_t s = ctx->stream;
    if (sc) {
        k_scale<double><<<nblk(n), kBlock, 0, s>>>(n, 1, v, sc);
        CU_LAUNCH(ctx);
    }
    double *rhs = ctx->dsa_buf, *y = ctx->dsa_buf + n;
    MLPG_TRY(apply_Ms_scalar(ctx, v, rhs));
    MLPG_TRY(gmres_alloc(ctx, ctx->gdsa, n, 1, kDsaRestart));
    ctx->gdsa.its_slot = 2;
    CU(ctx, cudaMemsetAsync(y, 0, sizeof(double) * n, s));
    ApplyFn<double> A = [ctx](const double *X, const double *B, double *Y) { return apply_C(ctx, X, B, Y); };
    PrecFn<double> P = [ctx](double *vv, double *zz, const double *ss) { return apply_Cprec(ctx, vv, zz, ss); };
    int64_t its = 0;
    MLPG_TRY(gmres_solve<double>(ctx, ctx->gdsa, A, P, rhs, y, ctx->opt.dsa_tol, ctx->opt.dsa_max, 5, &its,
                                 CycleFn(), nullptr, true, true));
    k_add<double, double><<<nblk(n), kBlock, 0, s>>>(n, v, y, z);
    CU_LAUNCH(ctx);
    return MLPG_OK;
}

// Nested solve of (L - MS D) Psi = f (Sec. 4.2): first flight, GMRES on Phi,
// recovery.  f and Psi are FP64 [n][m]; inner solves run in T.  Phi_io holds
// the initial guess of Phi on entry (may be null) and the result on exit.
static mlpg_status global_norm(mlpg_ctx *ctx, const double *a, int64_t N, double *out_host_slot);

template <typename T>
static mlpg_status nested_solve(mlpg_ctx *ctx, const double *f, double *Psi_out, double *Phi_io,
                                double inner_tol, double outer_tol) {
    const int64_t n = ctx->n, N = n * ctx->m;
    cudaStream_t s = ctx->stream;
    T *rhs, *bpsi, *x;
    if constexpr (sizeof(T) == 8) {
        rhs = (T *)ctx->rhs64b;
        bpsi = (T *)ctx->bpsi64;
        x = (T *)ctx->sol64;
    } else {
        rhs = (T *)ctx->rhs32;
        bpsi = (T *)ctx->bpsi32;
        x = (T *)ctx->sol32;
    }
    double *bphi = ctx->nvec, *d = ctx->nvec + n, *phi = ctx->nvec + 2 * ctx->n;
    k_convert<double, T><<<nblk(N), kBlock, 0, s>>>(N, f, rhs);
    CU_LAUNCH(ctx);
    // first flight b_psi = L^{-1} f, b_phi = D b_psi
    MLPG_TRY(inner_solve<T>(ctx, rhs, bpsi, inner_tol));
    k_Dreduce<T><<<nblk(n * 32), kBlock, 0, s>>>(n, ctx->m, ctx->w, bpsi, bphi);
    CU_LAUNCH(ctx);
    MLPG_TRY(shard_sum_dev(ctx, bphi, n));
    // scattering GMRES: (I - D L^{-1} MS) Phi = b_phi
    const bool dsa = ctx->opt.outer_precond == 1;
    MLPG_TRY(gmres_alloc(ctx, ctx->gout, n, 1, ctx->opt.outer_restart, dsa));
    ctx->gout.its_slot = 1;
    if (Phi_io) CU(ctx, cudaMemcpyAsync(phi, Phi_io, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    else CU(ctx, cudaMemsetAsync(phi, 0, sizeof(double) * n, s));
    if (ctx->opt.outer_method == 1) {
        // source iteration: Phi <- b_phi + D L^-1 MS Phi, one transport solve per
        // iteration.  Psi = L^-1 MS Phi_k + b_psi satisfies D Psi = Phi_{k+1}.
        // In a mixed-precision correction (T = float) the iterate reached after
        // outer_restart iterations is kept, as for the GMRES outer solve.
        double *e = ctx->nvec + 4 * n;
        const bool correction = sizeof(T) == 4;
        const int cap = correction ? ctx->opt.outer_restart : ctx->opt.max_outer;
        for (int k = 0;; ++k) {
            MLPG_TRY(apply_MS<T>(ctx, phi, rhs));
            MLPG_TRY(inner_solve<T>(ctx, rhs, x, inner_tol));
            k_Dreduce<T><<<nblk(n * 32), kBlock, 0, s>>>(n, ctx->m, ctx->w, x, d);
            CU_LAUNCH(ctx);
            MLPG_TRY(shard_sum_dev(ctx, d, n));
            k_si_update<<<nblk(n), kBlock, 0, s>>>(n, bphi, d, phi, e);
            CU_LAUNCH(ctx);
            k_bump<<<1, 1, 0, s>>>(ctx->d_its + 1);
            CU_LAUNCH(ctx);
            MLPG_TRY(global_norm(ctx, e, n, ctx->h_red + 4));
            MLPG_TRY(global_norm(ctx, phi, n, ctx->h_red + 5));
            CU(ctx, cudaStreamSynchronize(s));
            if (std::sqrt(ctx->h_red[4]) <= outer_tol * std::sqrt(ctx->h_red[5])) break;
            if (k + 1 >= cap) {
                if (correction) break;
                return set_err(ctx, MLPG_ERR_NOT_CONVERGED, "source iteration reached its iteration cap");
            }
        }
        k_add<T, T><<<nblk(N), kBlock, 0, s>>>(N, x, bpsi, Psi_out);
        CU_LAUNCH(ctx);
        if (Phi_io) CU(ctx, cudaMemcpyAsync(Phi_io, phi, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        return MLPG_OK;
    }
    // Each operator apply solves x = L^{-1} MS v for one outer basis vector v.
    // Those solutions are kept (bank) so that L^{-1} MS Phi, needed for the
    // angular recovery Psi = L^{-1} MS Phi + b_psi, is the same combination of
    // them as Phi is of the basis: no separate recovery solve.
    const int Rout = ctx->opt.outer_restart;
    T *bank, *xacc;
    MLPG_TRY(outer_bank<T>(ctx, Rout, &bank, &xacc));
    int slot = -1;
    ApplyFn<double> A = [ctx, rhs, x, d, n, N, s, bank, xacc, &slot](const double *X, const double *B,
                                                                    double *Y) -> mlpg_status {
        T *xt = slot >= 0 ? bank + (int64_t)slot * N : (slot == -1 ? xacc : x);
        MLPG_TRY(apply_MS<T>(ctx, X, rhs));
        MLPG_TRY(inner_solve<T>(ctx, rhs, xt, ctx->cur_inner_tol));
        k_Dreduce<T><<<nblk(n * 32), kBlock, 0, s>>>(n, ctx->m, ctx->w, xt, d);
        CU_LAUNCH(ctx);
        MLPG_TRY(shard_sum_dev(ctx, d, n));
        k_outer_combine<<<nblk(n), kBlock, 0, s>>>(n, X, d, B, Y);
        CU_LAUNCH(ctx);
        return MLPG_OK;
    };
    CycleFn on_cycle = [ctx, N, s, bank, xacc](const double *y, const float *y32, const int *kcol,
                                                int kmax) -> mlpg_status {
        const typename Arith<T>::type *yy;
        if constexpr (sizeof(T) == 8) yy = y; else yy = y32;
        k_bank_combine<T><<<nblk(N), kBlock, 0, s>>>(N, kmax, bank, yy, kcol, xacc);
        CU_LAUNCH(ctx);
        return MLPG_OK;
    };
    ctx->cur_inner_tol = inner_tol;
    int64_t oits = 0;
    const bool phi_zero = Phi_io == nullptr;   // then L^{-1} MS Phi_0 = 0
    if (phi_zero) CU(ctx, cudaMemsetAsync(xacc, 0, sizeof(T) * N, s));
    // In a mixed-precision correction (T = float) the outer solve is one
    // restart cycle at most and its iterate is kept: the FP64 step residual
    // decides convergence, and the inexact inner solves inside the operator
    // can hold the outer residual near its own tolerance.
    const bool correction = sizeof(T) == 4;
    PrecFn<double> Pout;
    if (dsa) Pout = [ctx](double *v, double *z, const double *sc) { return dsa_precond(ctx, v, z, sc); };
    MLPG_TRY(gmres_solve<double>(ctx, ctx->gout, A, Pout, bphi, phi, outer_tol,
                                 correction ? Rout : ctx->opt.max_outer, 1, &oits, on_cycle, &slot, phi_zero,
                                 correction));
    (void)oits;
    // Psi = L^{-1} MS Phi + b_psi
    k_add<T, T><<<nblk(N), kBlock, 0, s>>>(N, xacc, bpsi, Psi_out);
    CU_LAUNCH(ctx);
    if (Phi_io) CU(ctx, cudaMemcpyAsync(Phi_io, phi, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    return MLPG_OK;
}

static mlpg_status global_norm(mlpg_ctx *ctx, const double *a, int64_t N, double *out_host_slot) {
    int64_t G = std::min<int64_t>(1024, nblk(N));
    k_sumsq<<<G, kBlock, 0, ctx->stream>>>(N, a, ctx->red);
    CU_LAUNCH(ctx);
    k_reduce<<<1, 32, 0, ctx->stream>>>(1, 1, (int)G, ctx->red, ctx->red + 2048);
    CU_LAUNCH(ctx);
    CU(ctx, cudaMemcpyAsync(out_host_slot, ctx->red + 2048, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return MLPG_OK;
}

static mlpg_status ensure_history(mlpg_ctx *ctx) {
    if (!ctx->hist[0]) {
        const size_t N = (size_t)ctx->n * ctx->m;
        MLPG_TRY(dalloc(ctx, &ctx->hist[0], N));
        MLPG_TRY(dalloc(ctx, &ctx->hist[1], N));
        CU(ctx, cudaMemsetAsync(ctx->hist[0], 0, sizeof(double) * N, ctx->stream));
        CU(ctx, cudaMemsetAsync(ctx->hist[1], 0, sizeof(double) * N, ctx->stream));
        ctx->nhist = 0;
    }
    return MLPG_OK;
}

static mlpg_status reset_step_stats(mlpg_ctx *ctx) {
    ctx->st.last_outer_iters = 0;
    ctx->st.last_inner_iters = 0;
    ctx->st.last_inner_solves = 0;
    ctx->st.last_refinements = 0;
    ctx->st.last_dsa_iters = 0;
    if (!ctx->d_its) MLPG_TRY(dalloc(ctx, &ctx->d_its, 3));
    CU(ctx, cudaMemsetAsync(ctx->d_its, 0, 3 * sizeof(long long), ctx->stream));
    return MLPG_OK;
}

static mlpg_status prepare_step(mlpg_ctx *ctx, double dt) {
    double kappa = std::isfinite(dt) ? 1.0 / (ctx->opt.c * dt) : 0.0;
    bool same_inflow = true;
    for (int f = 0; f < 6; ++f) same_inflow &= ctx->ops_psib[f] == ctx->psi_b[f];
    if (kappa != ctx->kappa || !same_inflow) MLPG_TRY(form_operators(ctx, kappa));
    MLPG_TRY(ensure_step_buffers(ctx));
    MLPG_TRY(reset_step_stats(ctx));
    return MLPG_OK;
}

static mlpg_status finish_step_stats(mlpg_ctx *ctx) {
    if (ctx->d_tile_err) {   // a bounded wait of the tile kernel gave up during this step
        int terr = 0;
        CU(ctx, cudaMemcpyAsync(&terr, ctx->d_tile_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        if (terr) return set_err(ctx, MLPG_ERR_CUDA, "a copy into the tile kernel's shared memory timed out");
    }
    long long its[3] = {0, 0, 0};
    if (cudaMemcpyAsync(its, ctx->d_its, sizeof(its), cudaMemcpyDeviceToHost, ctx->stream) == cudaSuccess &&
        cudaStreamSynchronize(ctx->stream) == cudaSuccess) {
        ctx->st.last_inner_iters = its[0];
        ctx->st.last_outer_iters = (int32_t)its[1];
        ctx->st.last_dsa_iters = its[2];
    }
    cudaGetLastError();
    ctx->st.steps += 1;
    ctx->st.total_outer_iters += ctx->st.last_outer_iters;
    ctx->st.total_inner_iters += ctx->st.last_inner_iters;
    ctx->st.total_dsa_iters += ctx->st.last_dsa_iters;
    return MLPG_OK;
}

mlpg_status step_fp64(mlpg_ctx *ctx, double dt) {
    MLPG_TRY(prepare_step(ctx, dt));
    const int64_t n = ctx->n, N = n * ctx->m;
    cudaStream_t s = ctx->stream;
    MLPG_TRY(rhs_T(ctx, ctx->Psi, ctx->f64));
    MLPG_TRY(nested_solve<double>(ctx, ctx->f64, ctx->tmp64, ctx->Phi, ctx->opt.inner_tol, ctx->opt.outer_tol));
    CU(ctx, cudaMemcpyAsync(ctx->Psi, ctx->tmp64, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    k_Dreduce<double><<<nblk(n * 32), kBlock, 0, s>>>(n, ctx->m, ctx->w, ctx->Psi, ctx->Phi);
    CU_LAUNCH(ctx);
    MLPG_TRY(shard_sum_dev(ctx, ctx->Phi, n));
    // report the FP64 step residual
    MLPG_TRY(apply_L64_res(ctx, ctx->Psi, ctx->f64, ctx->res64));
    MLPG_TRY(apply_MS<double>(ctx, ctx->Phi, ctx->tmp64));
    k_add<double, double><<<nblk(N), kBlock, 0, s>>>(N, ctx->res64, ctx->tmp64, ctx->res64);
    CU_LAUNCH(ctx);
    MLPG_TRY(global_norm(ctx, ctx->res64, N, ctx->h_red));
    MLPG_TRY(global_norm(ctx, ctx->f64, N, ctx->h_red + 1));
    CU(ctx, cudaStreamSynchronize(s));
    MLPG_TRY(shard_sum_host(ctx, ctx->h_red, 2));
    ctx->st.last_residual = ctx->h_red[1] > 0 ? std::sqrt(ctx->h_red[0] / ctx->h_red[1]) : 0.0;
    return finish_step_stats(ctx);
}

mlpg_status step_mixed(mlpg_ctx *ctx, double dt) {
    MLPG_TRY(prepare_step(ctx, dt));
    const int64_t n = ctx->n, N = n * ctx->m;
    cudaStream_t s = ctx->stream;
    MLPG_TRY(rhs_T(ctx, ctx->Psi, ctx->f64));
    MLPG_TRY(global_norm(ctx, ctx->f64, N, ctx->h_red + 1));
    // Initial guess: polynomial extrapolation of the last states (the
    // converged result does not depend on it; a close guess saves sweeps).
    MLPG_TRY(ensure_history(ctx));
    {
        double *h1 = ctx->hist[0], *h2 = ctx->hist[1];   // Psi^{n-2}, Psi^{n-3} (when valid)
        const int nh = ctx->nhist;
        if (nh == 0) {
            CU(ctx, cudaMemcpyAsync(h2, ctx->Psi, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        } else {
            // linear (one history state) or quadratic (two) extrapolation
            const double a = nh >= 2 ? 3.0 : 2.0, b = nh >= 2 ? -3.0 : -1.0, c = nh >= 2 ? 1.0 : 0.0;
            k_extrap<<<nblk(N), kBlock, 0, s>>>(N, a, b, c, ctx->Psi, h1, h2);
            CU_LAUNCH(ctx);
        }
        ctx->hist[0] = h2;   // Psi^{n-1}
        ctx->hist[1] = h1;   // Psi^{n-2}
        ctx->nhist = nh < 2 ? nh + 1 : 2;
    }
    // refine Psi += (L - MS D)^{-1}_{FP32} R
    double *phi_c = ctx->nvec + 3 * n;
    int k = 0;
    double rel = 0.0;
    for (;; ++k) {
        k_Dreduce<double><<<nblk(n * 32), kBlock, 0, s>>>(n, ctx->m, ctx->w, ctx->Psi, phi_c);
        CU_LAUNCH(ctx);
        MLPG_TRY(shard_sum_dev(ctx, phi_c, n));
        MLPG_TRY(apply_L64_res(ctx, ctx->Psi, ctx->f64, ctx->res64));
        MLPG_TRY(apply_MS<double>(ctx, phi_c, ctx->tmp64));
        k_add<double, double><<<nblk(N), kBlock, 0, s>>>(N, ctx->res64, ctx->tmp64, ctx->res64);
        CU_LAUNCH(ctx);
        MLPG_TRY(global_norm(ctx, ctx->res64, N, ctx->h_red));
        CU(ctx, cudaStreamSynchronize(s));
        if (k == 0) MLPG_TRY(shard_sum_host(ctx, ctx->h_red + 1, 1));   // ||f||^2, once per step
        MLPG_TRY(shard_sum_host(ctx, ctx->h_red, 1));
        rel = ctx->h_red[1] > 0 ? std::sqrt(ctx->h_red[0] / ctx->h_red[1]) : 0.0;
        if (rel <= ctx->opt.refine_tol) break;
        if (k >= ctx->opt.max_refine) {
            ctx->st.last_residual = rel;
            return set_err(ctx, MLPG_ERR_NOT_CONVERGED, "mixed-precision refinement did not converge");
        }
        double tol = ctx->opt.mixed_inner_tol;
        MLPG_TRY(nested_solve<float>(ctx, ctx->res64, ctx->tmp64, nullptr, tol, tol));
        k_add<double, double><<<nblk(N), kBlock, 0, s>>>(N, ctx->Psi, ctx->tmp64, ctx->Psi);
        CU_LAUNCH(ctx);
    }
    k_Dreduce<double><<<nblk(n * 32), kBlock, 0, s>>>(n, ctx->m, ctx->w, ctx->Psi, ctx->Phi);
    CU_LAUNCH(ctx);
    MLPG_TRY(shard_sum_dev(ctx, ctx->Phi, n));
    ctx->st.last_refinements = k;
    ctx->st.last_residual = rel;
    return finish_step_stats(ctx);
}

}  // namespace mlpg
