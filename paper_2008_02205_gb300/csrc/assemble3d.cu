// 3D integration (Sec. 3.2, Alg. 1) over the elements of the polyhedral cells:
// one CTA per tetrahedron (volume forms) or per boundary triangle (surface
// forms).  Each element's quadrature points are mapped from the reference rule
// (App. A); the functions supported at any of its points are taken from the
// overlap row of the cell's generator; the RK functions and gradients are
// evaluated warp-cooperatively per point (Sec. 2.2, basis P = [1, (x - x_j)/s]
// for the linear correction or P = [1] for order 0, s = h of the generator);
// every pair's forms are summed over the element's
// points in registers and added to the shared pattern with FP64 atomics.
//
// mats layout in 3D: 0 M0, 1 Mt, 2 Ms, 3-5 G, 6-8 Gt, 9-11 Gs, 12-20 K (a-major),
// 21-26 S_f; vecs: 0 Q0, 1-3 Q, 4-9 B_f.
#include <cmath>

#include "internal.h"

namespace mlpg {

namespace {
constexpr int kMaxS3 = 96;        // functions supported on one element
constexpr int kMaxQ3 = 27;        // points per element (tetrahedron rule up to 3x3x3)
constexpr int kThreads3 = 256;
constexpr int kMaxCand = 1024;    // overlap row length

__constant__ double c3_tet_xi[3 * kMaxQ3];
__constant__ double c3_tet_w[kMaxQ3];
__constant__ double c3_tri_xi[2 * kMaxQ3];
__constant__ double c3_tri_w[kMaxQ3];

__device__ __forceinline__ double w3(double chi) {   // cubic spline, support chi < 2
    if (chi < 1.0) return 1.0 - chi * chi * (1.5 - 0.75 * chi);
    if (chi < 2.0) { double t = 2.0 - chi; return 0.25 * t * t * t; }
    return 0.0;
}
__device__ __forceinline__ double dw3(double chi) {
    if (chi < 1.0) return chi * (2.25 * chi - 3.0);
    if (chi < 2.0) { double t = 2.0 - chi; return -0.75 * t * t; }
    return 0.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// index of the symmetric NP x NP entry (i, j) in a packed array of NP (NP + 1) / 2
template <int NP>
__device__ __forceinline__ int symn(int i, int j) {
    return i <= j ? i * NP - i * (i - 1) / 2 + (j - i) : j * NP - j * (j - 1) / 2 + (i - j);
}

// RK functions of the S staged functions at p (one warp; lane owns a = lane +
// 32 k), basis P_j = [1] (order 0, NP = 1) or [1, (p - x_j)/s] (order 1,
// NP = 4).  Writes U, dU (3 components) at tab[c * cs + a], c = 0..3, and the
// support mask bits into mk[2].  Returns false when the moment matrix is not
// positive definite.
template <int NP>
__device__ bool rk3_warp(const double p[3], double s, int S, const double *fx, const double *fR2,
                         const double *finvh, const double *fV, double *tab, int cs, uint64_t *mk) {
    static_assert(NP == 1 || NP == 4, "order 0 or 1");
    constexpr int NE = NP * (NP + 1) / 2;
    const int lane = threadIdx.x & 31;
    const double is = 1.0 / s;
    double M[NE], D[3][NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) { M[e] = 0.0; D[0][e] = D[1][e] = D[2][e] = 0.0; }
    double Wl[3], Gl[3][3];
    bool on[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = lane + 32 * k;
        on[k] = false;
        Wl[k] = 0.0;
        Gl[k][0] = Gl[k][1] = Gl[k][2] = 0.0;
        if (a >= S) continue;
        const double d0 = p[0] - fx[3 * a], d1 = p[1] - fx[3 * a + 1], d2 = p[2] - fx[3 * a + 2];
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (!(r2 < fR2[a])) continue;
        on[k] = true;
        const double ir = r2 > 0.0 ? rsqrt(r2) : 0.0;
        const double chi = r2 * ir * finvh[a];
        const double W = w3(chi), g = dw3(chi) * finvh[a] * ir;
        const double Wg[3] = {g * d0, g * d1, g * d2}, v = fV[a];
        Wl[k] = W;
        Gl[k][0] = Wg[0]; Gl[k][1] = Wg[1]; Gl[k][2] = Wg[2];
        const double Pall[4] = {1.0, d0 * is, d1 * is, d2 * is};
#pragma unroll
        for (int i = 0; i < NP; ++i)
#pragma unroll
            for (int j = i; j < NP; ++j) {
                const int e = symn<NP>(i, j);
                const double pp = Pall[i] * Pall[j];
                M[e] += v * W * pp;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double dp = ((i == c + 1) * Pall[j] + (j == c + 1) * Pall[i]) * is;
                    D[c][e] += v * (dp * W + pp * Wg[c]);
                }
            }
    }
#pragma unroll
    for (int e = 0; e < NE; ++e) {
        M[e] = warp_sum(M[e]);
        D[0][e] = warp_sum(D[0][e]);
        D[1][e] = warp_sum(D[1][e]);
        D[2][e] = warp_sum(D[2][e]);
    }
    // support mask of this point
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        unsigned b = __ballot_sync(0xffffffffu, on[k]);
        if (lane == 0) {
            if (k == 0) mk[0] = b;
            else if (k == 1) mk[0] |= uint64_t(b) << 32;
            else mk[1] = b;
        }
    }
    // Cholesky of M (every lane, same values)
    double L[NP][NP];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int j = 0; j < NP; ++j) L[i][j] = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        double dsum = M[symn<NP>(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) dsum -= L[j][k] * L[j][k];
        if (!(dsum > 1e-14 * M[symn<NP>(j, j)])) return false;
        L[j][j] = sqrt(dsum);
#pragma unroll
        for (int i = j + 1; i < NP; ++i) {
            double t = M[symn<NP>(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    auto solve = [&](const double b[NP], double o[NP]) {
        double y[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            double t = b[i];
#pragma unroll
            for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
            y[i] = t / L[i][i];
        }
#pragma unroll
        for (int i = NP - 1; i >= 0; --i) {
            double t = y[i];
#pragma unroll
            for (int k = i + 1; k < NP; ++k) t -= L[k][i] * o[k];
            o[i] = t / L[i][i];
        }
    };
    // C = M^-1 e1, and its derivatives Cd[c] = -M^-1 (dM/dx_c) C
    double C[NP], Cd[3][NP];
    double e1[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) e1[i] = i == 0 ? 1.0 : 0.0;
    solve(e1, C);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double b[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            double t = 0.0;
#pragma unroll
            for (int j = 0; j < NP; ++j) t += D[c][symn<NP>(i, j)] * C[j];
            b[i] = -t;
        }
        solve(b, Cd[c]);
    }
    // U_a = W_a P_a . C;  d_c U_a = W_a (dP_a/dx_c . C + P_a . Cd[c]) + (P_a . C) dW_a/dx_c
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = lane + 32 * k;
        if (a >= S) continue;
        double u = 0.0, ud[3] = {0.0, 0.0, 0.0};
        if (on[k]) {
            const double Pall[4] = {1.0, (p[0] - fx[3 * a]) * is, (p[1] - fx[3 * a + 1]) * is,
                                    (p[2] - fx[3 * a + 2]) * is};
            double PC = 0.0;
#pragma unroll
            for (int i = 0; i < NP; ++i) PC += Pall[i] * C[i];
            const double W = Wl[k];
            u = W * PC;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double t = NP > 1 ? C[NP > 1 ? c + 1 : 0] * is : 0.0;
#pragma unroll
                for (int i = 0; i < NP; ++i) t += Pall[i] * Cd[c][i];
                ud[c] = W * t + PC * Gl[k][c];
            }
        }
        tab[a] = u;
        tab[cs + a] = ud[0];
        tab[2 * cs + a] = ud[1];
        tab[3 * cs + a] = ud[2];
    }
    return true;
}

__device__ int find_col3(const int32_t *__restrict__ col, int32_t lo, int32_t hi, int32_t key) {
    hi -= 1;
    while (lo <= hi) {
        int32_t mid = (lo + hi) >> 1;
        int32_t c = col[mid];
        if (c == key) return mid;
        if (c < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

struct Asm3Args {
    int64_t n, nnz, nelem;
    const double *x, *R, *V, *sig_t, *sig_s, *q;
    const int32_t *rowptr, *col;
    const int32_t *owner, *face;   // face: boundary triangles only
    const double *ev;              // 9 per element: three vertices
    int nq;
    double *mats, *vecs;
    int *flag;
};

// BND = false: tetrahedra (generator, v0, v1, v2) -> M0, Mt, Ms, G, Gt, Gs, K, Q0, Q.
// BND = true: boundary triangles (v0, v1, v2) on face f -> S_f, B_f.
template <bool BND, int NP>
__global__ void __launch_bounds__(kThreads3) k_assemble_3d(Asm3Args A) {
    __shared__ double fx[3 * kMaxS3], fR2[kMaxS3], finvh[kMaxS3], fV[kMaxS3];
    __shared__ int32_t fidx[kMaxS3];
    __shared__ double qx[3 * kMaxQ3], qw[kMaxQ3];
    __shared__ uint64_t qmk[kMaxQ3][2];
    __shared__ int wcnt[kThreads3 / 32];
    __shared__ int S_sh, bad;
    extern __shared__ double tab[];   // [nq][4][kMaxS3]
    const int64_t e = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t o = A.owner[e];
    const int nq = A.nq;
    if (tid == 0) { S_sh = 0; bad = 0; }
    // quadrature points of the element (App. A maps)
    if (tid < nq) {
        const double *v = A.ev + 9 * e;
        double p0[3], e1[3], e2[3], e3[3], wq;
        if (!BND) {
            const double *g = A.x + 3 * (int64_t)o;
            for (int c = 0; c < 3; ++c) {
                p0[c] = g[c];
                e1[c] = v[c] - g[c];
                e2[c] = v[3 + c] - g[c];
                e3[c] = v[6 + c] - g[c];
            }
            const double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
                               e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
            const double a = c3_tet_xi[3 * tid], b = c3_tet_xi[3 * tid + 1], c = c3_tet_xi[3 * tid + 2];
            for (int k = 0; k < 3; ++k) qx[3 * tid + k] = p0[k] + e1[k] * a + e2[k] * b + e3[k] * c;
            wq = c3_tet_w[tid] * fabs(det);
        } else {
            for (int c = 0; c < 3; ++c) {
                p0[c] = v[c];
                e1[c] = v[3 + c] - v[c];
                e2[c] = v[6 + c] - v[c];
            }
            const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                         cz = e1[0] * e2[1] - e1[1] * e2[0];
            const double a = c3_tri_xi[2 * tid], b = c3_tri_xi[2 * tid + 1];
            for (int k = 0; k < 3; ++k) qx[3 * tid + k] = p0[k] + e1[k] * a + e2[k] * b;
            wq = c3_tri_w[tid] * sqrt(cx * cx + cy * cy + cz * cz);
        }
        qw[tid] = wq;
    }
    __syncthreads();
    // functions supported at some point of the element, in overlap-row order
    const int32_t r0 = A.rowptr[o], rl = A.rowptr[o + 1] - r0;
    if (rl > kMaxCand) {
        if (tid == 0) atomicOr(A.flag, 2);
        return;
    }
    for (int base = 0; base < rl; base += kThreads3) {
        const int c = base + tid;
        bool sup = false;
        int32_t j = -1;
        if (c < rl) {
            j = A.col[r0 + c];
            const double xj = A.x[3 * (int64_t)j], yj = A.x[3 * (int64_t)j + 1], zj = A.x[3 * (int64_t)j + 2];
            const double R2 = A.R[j] * A.R[j];
            for (int q = 0; q < nq && !sup; ++q) {
                const double dx = qx[3 * q] - xj, dy = qx[3 * q + 1] - yj, dz = qx[3 * q + 2] - zj;
                sup = dx * dx + dy * dy + dz * dz < R2;
            }
        }
        const unsigned b = __ballot_sync(0xffffffffu, sup);
        if (lane == 0) wcnt[warp] = __popc(b);
        __syncthreads();
        int off = S_sh;
        for (int w = 0; w < warp; ++w) off += wcnt[w];
        const int slot = off + __popc(b & ((1u << lane) - 1u));
        if (sup) {
            if (slot < kMaxS3) {
                fidx[slot] = j;
                fx[3 * slot] = A.x[3 * (int64_t)j];
                fx[3 * slot + 1] = A.x[3 * (int64_t)j + 1];
                fx[3 * slot + 2] = A.x[3 * (int64_t)j + 2];
                fR2[slot] = A.R[j] * A.R[j];
                finvh[slot] = 2.0 / A.R[j];
                fV[slot] = A.V[j];
            } else {
                bad = 1;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int w = 0; w < kThreads3 / 32; ++w) t += wcnt[w];
            S_sh += t;
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) atomicOr(A.flag, 2);
        return;
    }
    const int S = S_sh;
    // RK at every point: one warp per point
    const double s = 0.5 * A.R[o];
    for (int q = warp; q < nq; q += kThreads3 / 32) {
        const double p[3] = {qx[3 * q], qx[3 * q + 1], qx[3 * q + 2]};
        if (!rk3_warp<NP>(p, s, S, fx, fR2, finvh, fV, tab + (int64_t)q * 4 * kMaxS3, kMaxS3, qmk[q])) {
            if (lane == 0) atomicOr(A.flag, 1);
        }
    }
    __syncthreads();
    const int64_t nnz = A.nnz, n = A.n;
    const double st = A.sig_t[o], ss = A.sig_s[o], qv = A.q[o];
    // pairs (a, b): forms summed over the element's points, then added to the pattern
    for (int pidx = tid; pidx < S * S; pidx += kThreads3) {
        const int a = pidx / S, b = pidx - a * S;
        const uint64_t ba = a < 64 ? (uint64_t(1) << a) : 0, bb = b < 64 ? (uint64_t(1) << b) : 0;
        const uint64_t ha = a >= 64 ? (uint64_t(1) << (a - 64)) : 0, hb = b >= 64 ? (uint64_t(1) << (b - 64)) : 0;
        if (BND) {
            double uu = 0.0;
            for (int q = 0; q < nq; ++q) {
                const bool sa = (qmk[q][0] & ba) || (qmk[q][1] & ha), sb = (qmk[q][0] & bb) || (qmk[q][1] & hb);
                if (!(sa && sb)) continue;
                const double *t = tab + (int64_t)q * 4 * kMaxS3;
                uu += qw[q] * t[a] * t[b];
            }
            if (uu == 0.0) continue;
            const int pos = find_col3(A.col, A.rowptr[fidx[a]], A.rowptr[fidx[a] + 1], fidx[b]);
            if (pos < 0) { atomicOr(A.flag, 8); continue; }
            atomicAdd(&A.mats[(21 + A.face[e]) * nnz + pos], uu * fV[b]);
        } else {
            double uu = 0.0, g[3] = {0, 0, 0}, k[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int q = 0; q < nq; ++q) {
                const bool sa = (qmk[q][0] & ba) || (qmk[q][1] & ha), sb = (qmk[q][0] & bb) || (qmk[q][1] & hb);
                if (!(sa && sb)) continue;
                const double *t = tab + (int64_t)q * 4 * kMaxS3;
                const double w = qw[q], ub = t[b];
                const double da[3] = {w * t[kMaxS3 + a], w * t[2 * kMaxS3 + a], w * t[3 * kMaxS3 + a]};
                const double db[3] = {t[kMaxS3 + b], t[2 * kMaxS3 + b], t[3 * kMaxS3 + b]};
                uu += w * t[a] * ub;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    g[c] += da[c] * ub;
#pragma unroll
                    for (int d = 0; d < 3; ++d) k[3 * c + d] += da[c] * db[d];
                }
            }
            if (uu == 0.0 && g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
            const int pos = find_col3(A.col, A.rowptr[fidx[a]], A.rowptr[fidx[a] + 1], fidx[b]);
            if (pos < 0) { atomicOr(A.flag, 8); continue; }
            const double vb = fV[b], m0 = uu * vb;
            atomicAdd(&A.mats[pos], m0);
            atomicAdd(&A.mats[nnz + pos], st * m0);
            atomicAdd(&A.mats[2 * nnz + pos], ss * m0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double gc = g[c] * vb;
                atomicAdd(&A.mats[(3 + c) * nnz + pos], gc);
                atomicAdd(&A.mats[(6 + c) * nnz + pos], st * gc);
                atomicAdd(&A.mats[(9 + c) * nnz + pos], ss * gc);
            }
#pragma unroll
            for (int c = 0; c < 9; ++c) atomicAdd(&A.mats[(12 + c) * nnz + pos], k[c] * vb);
        }
    }
    // vectors: Q0, Q (volume), B_f (boundary)
    if (tid < S) {
        const int a = tid;
        const uint64_t ba = a < 64 ? (uint64_t(1) << a) : 0, ha = a >= 64 ? (uint64_t(1) << (a - 64)) : 0;
        double v0 = 0.0, vg[3] = {0, 0, 0};
        for (int q = 0; q < nq; ++q) {
            if (!((qmk[q][0] & ba) || (qmk[q][1] & ha))) continue;
            const double *t = tab + (int64_t)q * 4 * kMaxS3;
            v0 += qw[q] * t[a];
            if (!BND)
                for (int c = 0; c < 3; ++c) vg[c] += qw[q] * t[(c + 1) * kMaxS3 + a];
        }
        const int32_t i = fidx[a];
        if (BND) {
            if (v0 != 0.0) atomicAdd(&A.vecs[(4 + A.face[e]) * n + i], v0);
        } else {
            if (v0 != 0.0) atomicAdd(&A.vecs[i], qv * v0);
            for (int c = 0; c < 3; ++c)
                if (vg[c] != 0.0) atomicAdd(&A.vecs[(1 + c) * n + i], qv * vg[c]);
        }
    }
}

// interp[pos(i, j)] = V_j U_j(x_i): one warp per point, candidates from row i
template <int NP>
__global__ void __launch_bounds__(128) k_interp_3d(int64_t n, const double *__restrict__ x,
                                                   const double *__restrict__ R, const double *__restrict__ V,
                                                   const int32_t *__restrict__ rowptr,
                                                   const int32_t *__restrict__ col, double *__restrict__ interp,
                                                   int *__restrict__ flag) {
    constexpr int W = 4;   // warps per block
    __shared__ double fx[W][3 * kMaxS3], fR2[W][kMaxS3], finvh[W][kMaxS3], fV[W][kMaxS3];
    __shared__ int32_t fp[W][kMaxS3];
    __shared__ double tab[W][4 * kMaxS3];
    __shared__ uint64_t mk[W][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = blockIdx.x * (int64_t)W + w;
    if (i >= n) return;
    const double p[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    const int32_t r0 = rowptr[i], rl = rowptr[i + 1] - r0;
    int S = 0;
    for (int base = 0; base < rl; base += 32) {
        const int c = base + lane;
        bool sup = false;
        int32_t j = -1;
        if (c < rl) {
            j = col[r0 + c];
            const double dx = p[0] - x[3 * (int64_t)j], dy = p[1] - x[3 * (int64_t)j + 1], dz = p[2] - x[3 * (int64_t)j + 2];
            sup = dx * dx + dy * dy + dz * dz < R[j] * R[j];
        }
        const unsigned b = __ballot_sync(0xffffffffu, sup);
        const int slot = S + __popc(b & ((1u << lane) - 1u));
        if (sup && slot < kMaxS3) {
            fp[w][slot] = r0 + c;
            fx[w][3 * slot] = x[3 * (int64_t)j];
            fx[w][3 * slot + 1] = x[3 * (int64_t)j + 1];
            fx[w][3 * slot + 2] = x[3 * (int64_t)j + 2];
            fR2[w][slot] = R[j] * R[j];
            finvh[w][slot] = 2.0 / R[j];
            fV[w][slot] = V[j];
        }
        S += __popc(b);
    }
    if (S > kMaxS3) {
        if (lane == 0) atomicOr(flag, 2);
        return;
    }
    __syncwarp();
    if (!rk3_warp<NP>(p, 0.5 * R[i], S, fx[w], fR2[w], finvh[w], fV[w], tab[w], kMaxS3, mk[w])) {
        if (lane == 0) atomicOr(flag, 1);
        return;
    }
    __syncwarp();
    for (int a = lane; a < S; a += 32) interp[fp[w][a]] = fV[w][a] * tab[w][a];
}

}  // namespace

static mlpg_status check_flag3(mlpg_ctx *ctx, const char *stage) {
    int flag = 0;
    CU(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag & 1) return set_err(ctx, MLPG_ERR_RK_SINGULAR, std::string(stage) + ": RK moment matrix singular");
    if (flag & 2) return set_err(ctx, MLPG_ERR_ARG, std::string(stage) + ": too many functions reach one element");
    if (flag & 8) return set_err(ctx, MLPG_ERR_GEOMETRY, std::string(stage) + ": support pair outside the overlap pattern");
    return MLPG_OK;
}

mlpg_status run_interp_3d(mlpg_ctx *ctx) {
    MLPG_TRY(dalloc(ctx, &ctx->interp, ctx->nnz));
    if (!ctx->d_flag) MLPG_TRY(dalloc(ctx, &ctx->d_flag, 1));
    CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    CU(ctx, cudaMemsetAsync(ctx->interp, 0, ctx->nnz * sizeof(double), ctx->stream));
    const int64_t blocks = (ctx->n + 3) / 4;
    if (ctx->opt.rk_order == 0)
        k_interp_3d<1><<<(unsigned)blocks, 128, 0, ctx->stream>>>(ctx->n, ctx->x, ctx->R, ctx->V, ctx->rowptr,
                                                                  ctx->col, ctx->interp, ctx->d_flag);
    else
        k_interp_3d<4><<<(unsigned)blocks, 128, 0, ctx->stream>>>(ctx->n, ctx->x, ctx->R, ctx->V, ctx->rowptr,
                                                                  ctx->col, ctx->interp, ctx->d_flag);
    CU_LAUNCH(ctx);
    return check_flag3(ctx, "interpolation");
}

mlpg_status run_assemble_3d(mlpg_ctx *ctx) {
    const int n1 = 2;   // 2x2x2 tetrahedron rule, 2x2 triangle rule (degree 3)
    {
        double xi[3 * kMaxQ3], w[kMaxQ3], ti[2 * kMaxQ3], tw[kMaxQ3];
        tet_rule(n1, xi, w);
        triangle_rule(n1, ti, tw);
        CU(ctx, cudaMemcpyToSymbolAsync(c3_tet_xi, xi, sizeof(double) * 3 * n1 * n1 * n1, 0,
                                        cudaMemcpyHostToDevice, ctx->stream));
        CU(ctx, cudaMemcpyToSymbolAsync(c3_tet_w, w, sizeof(double) * n1 * n1 * n1, 0, cudaMemcpyHostToDevice,
                                        ctx->stream));
        CU(ctx, cudaMemcpyToSymbolAsync(c3_tri_xi, ti, sizeof(double) * 2 * n1 * n1, 0, cudaMemcpyHostToDevice,
                                        ctx->stream));
        CU(ctx, cudaMemcpyToSymbolAsync(c3_tri_w, tw, sizeof(double) * n1 * n1, 0, cudaMemcpyHostToDevice,
                                        ctx->stream));
    }
    ctx->nmats = mlpg_n_matrices(3);
    ctx->nvecs = mlpg_n_vectors(3);
    if (!ctx->mats) MLPG_TRY(dalloc(ctx, &ctx->mats, (size_t)ctx->nmats * ctx->nnz));
    if (!ctx->vecs) MLPG_TRY(dalloc(ctx, &ctx->vecs, (size_t)ctx->nvecs * ctx->n));
    CU(ctx, cudaMemsetAsync(ctx->mats, 0, sizeof(double) * ctx->nmats * ctx->nnz, ctx->stream));
    CU(ctx, cudaMemsetAsync(ctx->vecs, 0, sizeof(double) * ctx->nvecs * ctx->n, ctx->stream));
    CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    Asm3Args a;
    a.n = ctx->n; a.nnz = ctx->nnz;
    a.x = ctx->x; a.R = ctx->R; a.V = ctx->V; a.sig_t = ctx->sig_t; a.sig_s = ctx->sig_s; a.q = ctx->q;
    a.rowptr = ctx->rowptr; a.col = ctx->col;
    a.mats = ctx->mats; a.vecs = ctx->vecs; a.flag = ctx->d_flag;
    // volume elements
    a.nelem = ctx->ntet; a.owner = ctx->tet_owner; a.face = nullptr; a.ev = ctx->tet_v; a.nq = n1 * n1 * n1;
    size_t smem = sizeof(double) * (size_t)a.nq * 4 * kMaxS3;
    if (a.nelem > 0) {
        if (ctx->opt.rk_order == 0) k_assemble_3d<false, 1><<<(unsigned)a.nelem, kThreads3, smem, ctx->stream>>>(a);
        else k_assemble_3d<false, 4><<<(unsigned)a.nelem, kThreads3, smem, ctx->stream>>>(a);
        CU_LAUNCH(ctx);
    }
    // boundary elements
    a.nelem = ctx->nbtri; a.owner = ctx->tri_owner; a.face = ctx->tri_face; a.ev = ctx->tri_v; a.nq = n1 * n1;
    smem = sizeof(double) * (size_t)a.nq * 4 * kMaxS3;
    if (a.nelem > 0) {
        if (ctx->opt.rk_order == 0) k_assemble_3d<true, 1><<<(unsigned)a.nelem, kThreads3, smem, ctx->stream>>>(a);
        else k_assemble_3d<true, 4><<<(unsigned)a.nelem, kThreads3, smem, ctx->stream>>>(a);
        CU_LAUNCH(ctx);
    }
    return check_flag3(ctx, "assembly");
}

}  // namespace mlpg
