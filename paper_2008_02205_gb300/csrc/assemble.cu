// Reproducing-kernel functions at quadrature points and the quadrature-
// outermost integration of the SUPG transport forms (Sec. 2.2, Sec. 3.2,
// Alg. 1, Eq. weak-transport), 2D.
//
// One CTA integrates one cell i.  The functions that can reach the cell (at
// most MLPG_MAX_CELL_FUNCS, drawn from the overlap row of i) are staged in
// shared memory.  Quadrature points are generated in the kernel from the cell
// polygon: fan triangles (x_i, v_k, v_{k+1}) with the conical-product rule
// mapped by x = p0 + (p1 - p0) xi1 + (p2 - p0) xi2 (App. A), and Gauss-Legendre
// points on edges that lie on the domain boundary.  Chunks of points are
// evaluated one point per thread (RK moment matrix, Cholesky, corrections and
// derivatives, FP64), their values written to a shared table, and every thread
// then accumulates its own unordered function pairs a <= b over the chunk (the
// sums of both entries (a, b) and (b, a): the mass, diagonal stiffness and
// face forms are symmetric, the mixed stiffness forms are each other's
// transposes, and both gradient forms use the same point values).  The
// per-cell sums are added into the CSR pattern at the end.
// Materials are constant over the cell, so sigma-weighted forms are the cell
// sums times sigma_t(i), sigma_s(i).
#include <cmath>

#include "internal.h"

namespace mlpg {

namespace {

constexpr int kMaxS = MLPG_MAX_CELL_FUNCS;
constexpr int kThreads = 512;
constexpr int kChunk = 64;                                       // points per RK chunk
constexpr int kMaxTri = 64;   // reference triangle rule size cap
constexpr int kMaxLine = 16;

__constant__ double c_tri_xi[2 * kMaxTri];
__constant__ double c_tri_w[kMaxTri];
__constant__ double c_line_t[kMaxLine];
__constant__ double c_line_w[kMaxLine];

__device__ __forceinline__ double spline_w(double chi) {
    if (chi < 1.0) return 1.0 - chi * chi * (1.5 - 0.75 * chi);
    if (chi < 2.0) { double t = 2.0 - chi; return 0.25 * t * t * t; }
    return 0.0;
}
__device__ __forceinline__ double spline_dw(double chi) {
    if (chi < 1.0) return chi * (2.25 * chi - 3.0);
    if (chi < 2.0) { double t = 2.0 - chi; return -0.75 * t * t; }
    return 0.0;
}

// RK functions at (px, py) for the S staged functions; basis P = [1, d/s].
// Writes U, Ux, Uy (zero outside the support); returns false when the moment
// matrix is not positive definite.
__device__ bool rk_point(double px, double py, double s, int S, const double *fx, const double *fy,
                         const double *fR, const double *fV, double *U, double *Ux, double *Uy,
                         int stride) {
    double M[3][3] = {{0}}, Dx[3][3] = {{0}}, Dy[3][3] = {{0}};
    const double is = 1.0 / s;
    for (int a = 0; a < S; ++a) {
        double dx = px - fx[a], dy = py - fy[a];
        double r = sqrt(dx * dx + dy * dy);
        if (!(r < fR[a])) continue;
        double h = 0.5 * fR[a], chi = r / h;
        double W = spline_w(chi);
        double g = r > 0.0 ? spline_dw(chi) / (r * h) : 0.0;
        double Wx = g * dx, Wy = g * dy, v = fV[a];
        double P[3] = {1.0, dx * is, dy * is};
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                double pp = P[i] * P[j];
                M[i][j] += v * W * pp;
                double ex = ((i == 1) * P[j] + (j == 1) * P[i]) * is;
                double ey = ((i == 2) * P[j] + (j == 2) * P[i]) * is;
                Dx[i][j] += v * (ex * W + pp * Wx);
                Dy[i][j] += v * (ey * W + pp * Wy);
            }
    }
    // Cholesky M = L L^T
    double L00 = M[0][0];
    if (!(L00 > 0.0)) return false;
    L00 = sqrt(L00);
    double L10 = M[1][0] / L00, L20 = M[2][0] / L00;
    double d1 = M[1][1] - L10 * L10;
    if (!(d1 > 1e-14 * M[1][1])) return false;
    double L11 = sqrt(d1);
    double L21 = (M[2][1] - L20 * L10) / L11;
    double d2 = M[2][2] - L20 * L20 - L21 * L21;
    if (!(d2 > 1e-14 * M[2][2])) return false;
    double L22 = sqrt(d2);
    auto solve = [&](double b0, double b1, double b2, double *o) {
        double y0 = b0 / L00, y1 = (b1 - L10 * y0) / L11, y2 = (b2 - L20 * y0 - L21 * y1) / L22;
        o[2] = y2 / L22;
        o[1] = (y1 - L21 * o[2]) / L11;
        o[0] = (y0 - L10 * o[1] - L20 * o[2]) / L00;
    };
    double C[3], Cx[3], Cy[3];
    solve(1.0, 0.0, 0.0, C);
    solve(-(Dx[0][0] * C[0] + Dx[0][1] * C[1] + Dx[0][2] * C[2]),
          -(Dx[1][0] * C[0] + Dx[1][1] * C[1] + Dx[1][2] * C[2]),
          -(Dx[2][0] * C[0] + Dx[2][1] * C[1] + Dx[2][2] * C[2]), Cx);
    solve(-(Dy[0][0] * C[0] + Dy[0][1] * C[1] + Dy[0][2] * C[2]),
          -(Dy[1][0] * C[0] + Dy[1][1] * C[1] + Dy[1][2] * C[2]),
          -(Dy[2][0] * C[0] + Dy[2][1] * C[1] + Dy[2][2] * C[2]), Cy);
    for (int a = 0; a < S; ++a) {
        double dx = px - fx[a], dy = py - fy[a];
        double r = sqrt(dx * dx + dy * dy);
        double u = 0.0, ux = 0.0, uy = 0.0;
        if (r < fR[a]) {
            double h = 0.5 * fR[a], chi = r / h;
            double W = spline_w(chi);
            double g = r > 0.0 ? spline_dw(chi) / (r * h) : 0.0;
            double P1 = dx * is, P2 = dy * is;
            double PC = C[0] + P1 * C[1] + P2 * C[2];
            u = W * PC;
            ux = W * (C[1] * is + Cx[0] + P1 * Cx[1] + P2 * Cx[2]) + PC * g * dx;
            uy = W * (C[2] * is + Cy[0] + P1 * Cy[1] + P2 * Cy[2]) + PC * g * dy;
        }
        U[a * stride] = u;
        Ux[a * stride] = ux;
        Uy[a * stride] = uy;
    }
    return true;
}

// RK functions at (px, py) for the assembly kernel, writing into the shared
// table (U, Ux, Uy at [a * stride]).  The first pass stores W and its
// gradient in the table slots so that the second pass does not repeat the
// square roots; support tests compare squared distances.  Returns the
// support mask (bit a set when function a is supported), or 0 when the
// moment matrix is not positive definite.
__device__ uint64_t rk_point_tab(double px, double py, double s, int S, const double *fx, const double *fy,
                                 const double *fR2, const double *finvh, const double *fV, double *U, double *Ux,
                                 double *Uy, int stride) {
    // M, Dx, Dy are symmetric: their six distinct entries (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
    constexpr int EI[6] = {0, 0, 0, 1, 1, 2}, EJ[6] = {0, 1, 2, 1, 2, 2};
    double m[6] = {0}, mx[6] = {0}, my[6] = {0};
    const double is = 1.0 / s;
    uint64_t mask = 0;
    for (int a = 0; a < S; ++a) {
        const double dx = px - fx[a], dy = py - fy[a];
        const double r2 = dx * dx + dy * dy;
        if (!(r2 < fR2[a])) {
            U[a * stride] = 0.0;
            Ux[a * stride] = 0.0;
            Uy[a * stride] = 0.0;
            continue;
        }
        mask |= uint64_t(1) << a;
        const double ir = r2 > 0.0 ? rsqrt(r2) : 0.0;
        const double chi = r2 * ir * finvh[a];
        const double W = spline_w(chi);
        const double g = spline_dw(chi) * finvh[a] * ir;
        const double Wx = g * dx, Wy = g * dy, v = fV[a];
        U[a * stride] = W;
        Ux[a * stride] = Wx;
        Uy[a * stride] = Wy;
        const double P[3] = {1.0, dx * is, dy * is};
        const double vW = v * W, vWx = v * Wx, vWy = v * Wy;
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const int i = EI[e], j = EJ[e];
            const double pp = P[i] * P[j];
            const double ex = ((i == 1) * P[j] + (j == 1) * P[i]) * is;
            const double ey = ((i == 2) * P[j] + (j == 2) * P[i]) * is;
            m[e] += vW * pp;
            mx[e] += ex * vW + pp * vWx;
            my[e] += ey * vW + pp * vWy;
        }
    }
    // M = L L^T; the triangular solves multiply by the reciprocal pivots
    double L00 = m[0];
    if (!(L00 > 0.0)) return 0;
    L00 = sqrt(L00);
    const double r00 = 1.0 / L00;
    const double L10 = m[1] * r00, L20 = m[2] * r00;
    const double d1 = m[3] - L10 * L10;
    if (!(d1 > 1e-14 * m[3])) return 0;
    const double L11 = sqrt(d1), r11 = 1.0 / L11;
    const double L21 = (m[4] - L20 * L10) * r11;
    const double d2 = m[5] - L20 * L20 - L21 * L21;
    if (!(d2 > 1e-14 * m[5])) return 0;
    const double r22 = 1.0 / sqrt(d2);
    auto solve = [&](double b0, double b1, double b2, double *o) {
        double y0 = b0 * r00, y1 = (b1 - L10 * y0) * r11, y2 = (b2 - L20 * y0 - L21 * y1) * r22;
        o[2] = y2 * r22;
        o[1] = (y1 - L21 * o[2]) * r11;
        o[0] = (y0 - L10 * o[1] - L20 * o[2]) * r00;
    };
    double C[3], Cx[3], Cy[3];
    solve(1.0, 0.0, 0.0, C);
    solve(-(mx[0] * C[0] + mx[1] * C[1] + mx[2] * C[2]), -(mx[1] * C[0] + mx[3] * C[1] + mx[4] * C[2]),
          -(mx[2] * C[0] + mx[4] * C[1] + mx[5] * C[2]), Cx);
    solve(-(my[0] * C[0] + my[1] * C[1] + my[2] * C[2]), -(my[1] * C[0] + my[3] * C[1] + my[4] * C[2]),
          -(my[2] * C[0] + my[4] * C[1] + my[5] * C[2]), Cy);
    for (uint64_t bits = mask; bits; bits &= bits - 1) {
        const int a = __ffsll((long long)bits) - 1;
        const double W = U[a * stride], Wx = Ux[a * stride], Wy = Uy[a * stride];
        const double P1 = (px - fx[a]) * is, P2 = (py - fy[a]) * is;
        const double PC = C[0] + P1 * C[1] + P2 * C[2];
        U[a * stride] = W * PC;
        Ux[a * stride] = W * (C[1] * is + Cx[0] + P1 * Cx[1] + P2 * Cx[2]) + PC * Wx;
        Uy[a * stride] = W * (C[2] * is + Cy[0] + P1 * Cy[1] + P2 * Cy[2]) + PC * Wy;
    }
    return mask;
}

// RK functions of order ORD (0 or 2; order 1 is rk_point_tab) at (px, py):
// the basis is every monomial of xi = (p - x_j)/s up to degree ORD, ordered
// 1, xi_x, xi_y, xi_x^2, xi_x xi_y, xi_y^2.  Same table layout, first-pass use
// of the table and return value (support mask, 0 when the moment matrix is
// not positive definite) as rk_point_tab.
template <int ORD>
__device__ uint64_t rk_point_gen(double px, double py, double s, int S, const double *fx, const double *fy,
                                 const double *fR2, const double *finvh, const double *fV, double *U, double *Ux,
                                 double *Uy, int stride) {
    constexpr int NP = ORD == 0 ? 1 : (ORD == 1 ? 3 : 6);
    double M[NP][NP], Dx[NP][NP], Dy[NP][NP];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int j = 0; j < NP; ++j) M[i][j] = Dx[i][j] = Dy[i][j] = 0.0;
    const double is = 1.0 / s;
    // basis and its x, y derivatives at offset (dx, dy)
    auto basis = [&](double dx, double dy, double *P, double *Px, double *Py) {
        const double ex = dx * is, ey = dy * is;
        P[0] = 1.0; Px[0] = 0.0; Py[0] = 0.0;
        if (ORD >= 1) {
            P[1] = ex; Px[1] = is; Py[1] = 0.0;
            P[2] = ey; Px[2] = 0.0; Py[2] = is;
        }
        if (ORD >= 2) {
            P[3] = ex * ex; Px[3] = 2.0 * ex * is; Py[3] = 0.0;
            P[4] = ex * ey; Px[4] = ey * is; Py[4] = ex * is;
            P[5] = ey * ey; Px[5] = 0.0; Py[5] = 2.0 * ey * is;
        }
    };
    uint64_t mask = 0;
    for (int a = 0; a < S; ++a) {
        const double dx = px - fx[a], dy = py - fy[a];
        const double r2 = dx * dx + dy * dy;
        if (!(r2 < fR2[a])) {
            U[a * stride] = 0.0;
            Ux[a * stride] = 0.0;
            Uy[a * stride] = 0.0;
            continue;
        }
        mask |= uint64_t(1) << a;
        const double ir = r2 > 0.0 ? rsqrt(r2) : 0.0;
        const double chi = r2 * ir * finvh[a];
        const double W = spline_w(chi), g = spline_dw(chi) * finvh[a] * ir;
        const double Wx = g * dx, Wy = g * dy, v = fV[a];
        U[a * stride] = W;
        Ux[a * stride] = Wx;
        Uy[a * stride] = Wy;
        double P[NP], Px[NP], Py[NP];
        basis(dx, dy, P, Px, Py);
#pragma unroll
        for (int i = 0; i < NP; ++i)
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const double pp = P[i] * P[j];
                M[i][j] += v * W * pp;
                Dx[i][j] += v * ((Px[i] * P[j] + P[i] * Px[j]) * W + pp * Wx);
                Dy[i][j] += v * ((Py[i] * P[j] + P[i] * Py[j]) * W + pp * Wy);
            }
    }
    // Cholesky M = L L^T
    double L[NP][NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        double d = M[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 1e-14 * M[j][j])) return 0;
        L[j][j] = sqrt(d);
#pragma unroll
        for (int i = j + 1; i < NP; ++i) {
            double t = M[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    auto solve = [&](double *b) {   // in place: b <- M^{-1} b
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            double t = b[i];
#pragma unroll
            for (int k = 0; k < i; ++k) t -= L[i][k] * b[k];
            b[i] = t / L[i][i];
        }
#pragma unroll
        for (int i = NP - 1; i >= 0; --i) {
            double t = b[i];
#pragma unroll
            for (int k = i + 1; k < NP; ++k) t -= L[k][i] * b[k];
            b[i] = t / L[i][i];
        }
    };
    double C[NP], Cx[NP], Cy[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) C[i] = i == 0 ? 1.0 : 0.0;
    solve(C);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        double tx = 0.0, ty = 0.0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            tx += Dx[i][j] * C[j];
            ty += Dy[i][j] * C[j];
        }
        Cx[i] = -tx;
        Cy[i] = -ty;
    }
    solve(Cx);
    solve(Cy);
    for (uint64_t bits = mask; bits; bits &= bits - 1) {
        const int a = __ffsll((long long)bits) - 1;
        const double W = U[a * stride], Wx = Ux[a * stride], Wy = Uy[a * stride];
        double P[NP], Px[NP], Py[NP];
        basis(px - fx[a], py - fy[a], P, Px, Py);
        double PC = 0.0, dxC = 0.0, dyC = 0.0, PCx = 0.0, PCy = 0.0;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            PC += P[i] * C[i];
            dxC += Px[i] * C[i];
            dyC += Py[i] * C[i];
            PCx += P[i] * Cx[i];
            PCy += P[i] * Cy[i];
        }
        U[a * stride] = W * PC;
        Ux[a * stride] = W * (dxC + PCx) + PC * Wx;
        Uy[a * stride] = W * (dyC + PCy) + PC * Wy;
    }
    return mask;
}

__device__ int find_col(const int32_t *__restrict__ col, int32_t lo, int32_t hi, int32_t key) {
    hi -= 1;
    while (lo <= hi) {
        int32_t mid = (lo + hi) >> 1;
        int32_t c = col[mid];
        if (c == key) return mid;
        if (c < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

struct AsmArgs {
    int64_t n, nnz;
    const double *x, *R, *V, *sig_t, *sig_s, *q;
    const int32_t *rowptr, *col, *cptr, *labels;
    const double *verts;
    int ntri, nline;
    double *mats, *vecs;
    int *flag;
};

// mats layout: 0 M0, 1 Mt, 2 Ms, 3-4 G, 5-6 Gt, 7-8 Gs, 9-12 K (xx, xy, yx, yy), 13-16 S_f
// ORD: RK order; MAXS: functions reaching one cell (<= 64, one mask word);
// CHUNK: quadrature points per RK pass.  The linear path is <1, 40, 64>.
template <int ORD, int MAXS, int CHUNK>
__global__ void __launch_bounds__(kThreads, 1) k_assemble_2d(AsmArgs A) {
    // unordered pairs a <= b of the staged functions: M0, K^xx, K^yy and the face forms are
    // symmetric, K^yx(a, b) = K^xy(b, a), and both G(a, b) and G(b, a) come from the same
    // point values, so one pass over a <= b fills both entries (a, b) and (b, a)
    constexpr int kMaxS = MAXS, kChunk = CHUNK, kPairs = MAXS * (MAXS + 1) / 2;
    constexpr int kPPT = (kPairs + kThreads - 1) / kThreads;
    constexpr int kAcc = 11;   // running sums per unordered pair
    static_assert(MAXS <= 64 && CHUNK <= kThreads, "one 64-bit support mask per point");
    const int64_t i = blockIdx.x;
    __shared__ double fx[kMaxS], fy[kMaxS], fR[kMaxS], fV[kMaxS], fR2[kMaxS], finvh[kMaxS];
    __shared__ uint64_t tMask[kChunk];
    __shared__ int32_t fidx[kMaxS];
    __shared__ uint8_t pairA[kPairs], pairB[kPairs];
    __shared__ int S;
    __shared__ int face_slot[2];
    extern __shared__ double tab[];  // [6][kChunk][kMaxS] + [kChunk] weights + [kChunk] face
    double *tU = tab, *tUx = tU + kChunk * kMaxS, *tUy = tUx + kChunk * kMaxS;
    double *tW = tUy + kChunk * kMaxS;                 // weight per point
    int *tF = (int *)(tW + kChunk);                    // face slot (-1 volume)

    const int tid = threadIdx.x;
    const double xi = A.x[2 * i], yi = A.x[2 * i + 1];
    const int32_t c0 = A.cptr[i], nv = A.cptr[i + 1] - c0;
    if (tid == 0) {
        // radius of the cell around its generator and the boundary faces it touches
        double rc = 0.0;
        int nf = 0;
        face_slot[0] = face_slot[1] = -1;
        for (int k = 0; k < nv; ++k) {
            double dx = A.verts[2 * (c0 + k)] - xi, dy = A.verts[2 * (c0 + k) + 1] - yi;
            rc = fmax(rc, sqrt(dx * dx + dy * dy));
            int32_t L = A.labels[c0 + k];
            if (L < 0 && L != kLabelExtent) {
                int f = -L - 1;
                if (face_slot[0] != f && face_slot[1] != f) {
                    if (nf < 2) face_slot[nf] = f;
                    ++nf;
                }
            }
        }
        if (nf > 2) atomicOr(A.flag, 4);
        int s = 0;
        for (int32_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
            int32_t j = A.col[p];
            double dx = A.x[2 * j] - xi, dy = A.x[2 * j + 1] - yi;
            if (sqrt(dx * dx + dy * dy) < A.R[j] + rc * (1.0 + 1e-12)) {
                if (s < kMaxS) {
                    fidx[s] = j;
                    fx[s] = A.x[2 * j];
                    fy[s] = A.x[2 * j + 1];
                    fR[s] = A.R[j];
                    fR2[s] = A.R[j] * A.R[j];
                    finvh[s] = 2.0 / A.R[j];
                    fV[s] = A.V[j];
                }
                ++s;
            }
        }
        if (s > kMaxS) atomicOr(A.flag, 2);
        S = s > kMaxS ? kMaxS : s;
    }
    __syncthreads();
    const int nS = S, nP = nS * (nS + 1) / 2;
    const double scale = 0.5 * A.R[i];
    // unordered pair p = (a, b), a <= b, row by row of the upper triangle
    if (tid < nS) {
        const int a = tid, p0 = a * nS - a * (a - 1) / 2;
        for (int b = a; b < nS; ++b) {
            pairA[p0 + b - a] = (uint8_t)a;
            pairB[p0 + b - a] = (uint8_t)b;
        }
    }
    // pairs owned by this thread: p = tid + k * kThreads.  Their running sums live in
    // shared memory, sacc[f][p] (one owner per p):
    //   0 M0, 1-2 G(a, b), 3-4 G(b, a), 5 K^xx, 6 K^xy(a, b), 7 K^yx(a, b), 8 K^yy, 9-10 faces
    double *sacc = tab + 3 * kChunk * kMaxS + kChunk + kChunk / 2 + 1;
    for (int p = tid; p < kPairs; p += kThreads)
#pragma unroll
        for (int f = 0; f < kAcc; ++f) sacc[f * kPairs + p] = 0.0;
    double vq0 = 0.0, vqx = 0.0, vqy = 0.0, vb0 = 0.0, vb1 = 0.0;  // vectors for a = tid

    // count boundary points of this cell
    int nbe = 0;
    for (int k = 0; k < nv; ++k) {
        int32_t L = A.labels[c0 + k];
        nbe += (L < 0 && L != kLabelExtent);
    }
    const int nvol = nv * A.ntri, ntot = nvol + nbe * A.nline;
    for (int base = 0; base < ntot; base += kChunk) {
        const int cnt = min(kChunk, ntot - base);
        if (tid < cnt) {
            int k = base + tid;
            double px, py, wq;
            int fslot = -1;
            if (k < nvol) {
                int e = k / A.ntri, r = k - e * A.ntri;
                int e1 = (e + 1 == nv) ? 0 : e + 1;
                double ax = A.verts[2 * (c0 + e)] - xi, ay = A.verts[2 * (c0 + e) + 1] - yi;
                double bx = A.verts[2 * (c0 + e1)] - xi, by = A.verts[2 * (c0 + e1) + 1] - yi;
                double det = fabs(ax * by - ay * bx);
                px = xi + ax * c_tri_xi[2 * r] + bx * c_tri_xi[2 * r + 1];
                py = yi + ay * c_tri_xi[2 * r] + by * c_tri_xi[2 * r + 1];
                wq = c_tri_w[r] * det;
            } else {
                int kb = k - nvol, eb = kb / A.nline, r = kb - eb * A.nline;
                // eb-th boundary edge of the cell
                int e = -1, c = -1;
                for (int t = 0; t < nv; ++t) {
                    int32_t L = A.labels[c0 + t];
                    if (L < 0 && L != kLabelExtent && ++c == eb) { e = t; break; }
                }
                int e1 = (e + 1 == nv) ? 0 : e + 1;
                double p0x = A.verts[2 * (c0 + e)], p0y = A.verts[2 * (c0 + e) + 1];
                double dx = A.verts[2 * (c0 + e1)] - p0x, dy = A.verts[2 * (c0 + e1) + 1] - p0y;
                double s01 = 0.5 * (c_line_t[r] + 1.0);
                px = p0x + dx * s01;
                py = p0y + dy * s01;
                wq = c_line_w[r] * 0.5 * sqrt(dx * dx + dy * dy);
                int f = -A.labels[c0 + e] - 1;
                fslot = (f == face_slot[0]) ? 0 : 1;
            }
            uint64_t mk;
            if constexpr (ORD == 1)
                mk = rk_point_tab(px, py, scale, nS, fx, fy, fR2, finvh, fV, tU + tid, tUx + tid, tUy + tid, kChunk);
            else
                mk = rk_point_gen<ORD>(px, py, scale, nS, fx, fy, fR2, finvh, fV, tU + tid, tUx + tid, tUy + tid,
                                       kChunk);
            if (!mk) atomicOr(A.flag, 1);
            tMask[tid] = mk;
            tW[tid] = wq;
            tF[tid] = fslot;
        }
        __syncthreads();
        for (int qk = 0; qk < cnt; ++qk) {
            const double wq = tW[qk];
            const int fs = tF[qk];
            const uint64_t mk = tMask[qk];
#pragma unroll
            for (int k = 0; k < kPPT; ++k) {
                int p = tid + k * kThreads;
                if (p >= nP) break;
                const int a = pairA[p], b = pairB[p];
                if (!((mk >> a) & (mk >> b) & 1)) continue;   // both functions must be supported here
                double ua = tU[a * kChunk + qk];
                double uax = tUx[a * kChunk + qk], uay = tUy[a * kChunk + qk];
                double ub = tU[b * kChunk + qk];
                double ubx = tUx[b * kChunk + qk], uby = tUy[b * kChunk + qk];
                if (fs < 0) {
                    double wa = wq * ua, wax = wq * uax, way = wq * uay;
                    sacc[0 * kPairs + p] += wa * ub;
                    sacc[1 * kPairs + p] += wax * ub;
                    sacc[2 * kPairs + p] += way * ub;
                    sacc[3 * kPairs + p] += wa * ubx;
                    sacc[4 * kPairs + p] += wa * uby;
                    sacc[5 * kPairs + p] += wax * ubx;
                    sacc[6 * kPairs + p] += wax * uby;
                    sacc[7 * kPairs + p] += way * ubx;
                    sacc[8 * kPairs + p] += way * uby;
                } else {
                    sacc[(9 + fs) * kPairs + p] += wq * ua * ub;
                }
            }
            if (tid < nS) {
                double ua = tU[tid * kChunk + qk];
                if (fs < 0) {
                    vq0 += wq * ua;
                    vqx += wq * tUx[tid * kChunk + qk];
                    vqy += wq * tUy[tid * kChunk + qk];
                } else if (fs == 0) {
                    vb0 += wq * ua;
                } else {
                    vb1 += wq * ua;
                }
            }
        }
        __syncthreads();
    }
    // scatter into the pattern: entry (a, b) and, for a != b, entry (b, a)
    const double st = A.sig_t[i], ss = A.sig_s[i], qi = A.q[i];
    const int64_t nnz = A.nnz, n = A.n;
    auto put = [&](int32_t ra, int32_t cb, double v, double m0, double gx, double gy, double kxx, double kxy,
                   double kyx, double kyy, double f0, double f1) {
        int pos = find_col(A.col, A.rowptr[ra], A.rowptr[ra + 1], cb);
        if (pos < 0) {
            atomicOr(A.flag, 8);
            return;
        }
        m0 *= v;
        atomicAdd(&A.mats[0 * nnz + pos], m0);
        atomicAdd(&A.mats[1 * nnz + pos], st * m0);
        atomicAdd(&A.mats[2 * nnz + pos], ss * m0);
        gx *= v;
        gy *= v;
        atomicAdd(&A.mats[3 * nnz + pos], gx);
        atomicAdd(&A.mats[4 * nnz + pos], gy);
        atomicAdd(&A.mats[5 * nnz + pos], st * gx);
        atomicAdd(&A.mats[6 * nnz + pos], st * gy);
        atomicAdd(&A.mats[7 * nnz + pos], ss * gx);
        atomicAdd(&A.mats[8 * nnz + pos], ss * gy);
        atomicAdd(&A.mats[9 * nnz + pos], kxx * v);
        atomicAdd(&A.mats[10 * nnz + pos], kxy * v);
        atomicAdd(&A.mats[11 * nnz + pos], kyx * v);
        atomicAdd(&A.mats[12 * nnz + pos], kyy * v);
        if (face_slot[0] >= 0 && f0 != 0.0) atomicAdd(&A.mats[(13 + face_slot[0]) * nnz + pos], f0 * v);
        if (face_slot[1] >= 0 && f1 != 0.0) atomicAdd(&A.mats[(13 + face_slot[1]) * nnz + pos], f1 * v);
    };
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
        int p = tid + k * kThreads;
        if (p >= nP) break;
        const int a = pairA[p], b = pairB[p];
        double acc[kAcc];
        bool any = false;
#pragma unroll
        for (int f = 0; f < kAcc; ++f) {
            acc[f] = sacc[f * kPairs + p];
            any |= acc[f] != 0.0;
        }
        if (!any) continue;
        // (a, b): trial function b carries V_b; (b, a): G from the (b, a) sums, K^xy and K^yx swap
        put(fidx[a], fidx[b], fV[b], acc[0], acc[1], acc[2], acc[5], acc[6], acc[7], acc[8], acc[9], acc[10]);
        if (a != b)
            put(fidx[b], fidx[a], fV[a], acc[0], acc[3], acc[4], acc[5], acc[7], acc[6], acc[8], acc[9], acc[10]);
    }
    if (tid < nS) {
        int32_t a = fidx[tid];
        if (vq0 != 0.0) atomicAdd(&A.vecs[a], qi * vq0);
        if (vqx != 0.0) atomicAdd(&A.vecs[n + a], qi * vqx);
        if (vqy != 0.0) atomicAdd(&A.vecs[2 * n + a], qi * vqy);
        if (face_slot[0] >= 0 && vb0 != 0.0) atomicAdd(&A.vecs[(3 + face_slot[0]) * n + a], vb0);
        if (face_slot[1] >= 0 && vb1 != 0.0) atomicAdd(&A.vecs[(3 + face_slot[1]) * n + a], vb1);
    }
}

// RK point interpolation at the centres: interp[pos(i, j)] = V_j U_j(x_i).
template <int ORD>
__global__ void k_interp_2d(int64_t n, const double *__restrict__ x, const double *__restrict__ R,
                            const double *__restrict__ V, const int32_t *__restrict__ rowptr,
                            const int32_t *__restrict__ col, double *__restrict__ interp,
                            int *__restrict__ flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t s0 = rowptr[i], len = rowptr[i + 1] - s0;
    double fx[kMaxS * 2], fy[kMaxS * 2], fR[kMaxS * 2], fV[kMaxS * 2];
    int32_t fp[kMaxS * 2];
    const double px = x[2 * i], py = x[2 * i + 1];
    int S = 0;
    for (int32_t p = 0; p < len; ++p) {
        int32_t j = col[s0 + p];
        double dx = px - x[2 * j], dy = py - x[2 * j + 1];
        if (sqrt(dx * dx + dy * dy) < R[j]) {
            if (S < 2 * kMaxS) {
                fx[S] = x[2 * j]; fy[S] = x[2 * j + 1]; fR[S] = R[j]; fV[S] = V[j]; fp[S] = s0 + p;
            }
            ++S;
        }
    }
    if (S > 2 * kMaxS) { atomicOr(flag, 2); return; }
    double U[kMaxS * 2], Ux[kMaxS * 2], Uy[kMaxS * 2];
    bool ok;
    if constexpr (ORD == 1) {
        ok = rk_point(px, py, 0.5 * R[i], S, fx, fy, fR, fV, U, Ux, Uy, 1);
    } else {
        double fR2[kMaxS * 2], finvh[kMaxS * 2];
        for (int a = 0; a < S; ++a) {
            fR2[a] = fR[a] * fR[a];
            finvh[a] = 2.0 / fR[a];
        }
        ok = S <= 64 && rk_point_gen<ORD>(px, py, 0.5 * R[i], S, fx, fy, fR2, finvh, fV, U, Ux, Uy, 1) != 0;
    }
    if (!ok) {
        atomicOr(flag, 1);
        return;
    }
    for (int a = 0; a < S; ++a) interp[fp[a]] = fV[a] * U[a];
}

}  // namespace

static mlpg_status upload_rules(mlpg_ctx *ctx, int ntri1d, int nline) {
    double xi[2 * kMaxTri], w[kMaxTri], t[kMaxLine], lw[kMaxLine];
    triangle_rule(ntri1d, xi, w);
    line_rule(nline, t, lw);
    CU(ctx, cudaMemcpyToSymbolAsync(c_tri_xi, xi, sizeof(double) * 2 * ntri1d * ntri1d, 0,
                                    cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, cudaMemcpyToSymbolAsync(c_tri_w, w, sizeof(double) * ntri1d * ntri1d, 0,
                                    cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, cudaMemcpyToSymbolAsync(c_line_t, t, sizeof(double) * nline, 0, cudaMemcpyHostToDevice,
                                    ctx->stream));
    CU(ctx, cudaMemcpyToSymbolAsync(c_line_w, lw, sizeof(double) * nline, 0, cudaMemcpyHostToDevice,
                                    ctx->stream));
    return MLPG_OK;
}

static mlpg_status check_flag(mlpg_ctx *ctx, const char *stage) {
    int flag = 0;
    CU(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag & 1) return set_err(ctx, MLPG_ERR_RK_SINGULAR, std::string(stage) + ": RK moment matrix singular");
    if (flag & 2) return set_err(ctx, MLPG_ERR_ARG, std::string(stage) + ": too many functions reach one cell");
    if (flag & 4) return set_err(ctx, MLPG_ERR_GEOMETRY, std::string(stage) + ": a cell touches more than two faces");
    if (flag & 8) return set_err(ctx, MLPG_ERR_GEOMETRY, std::string(stage) + ": support pair outside the overlap pattern");
    return MLPG_OK;
}

mlpg_status run_interp(mlpg_ctx *ctx) {
    MLPG_TRY(dalloc(ctx, &ctx->interp, ctx->nnz));
    if (!ctx->d_flag) MLPG_TRY(dalloc(ctx, &ctx->d_flag, 1));
    CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    CU(ctx, cudaMemsetAsync(ctx->interp, 0, ctx->nnz * sizeof(double), ctx->stream));
    int B = 128;
    const int ord = ctx->opt.rk_order;
    auto launch = [&](auto kern) {
        kern<<<(ctx->n + B - 1) / B, B, 0, ctx->stream>>>(ctx->n, ctx->x, ctx->R, ctx->V, ctx->rowptr, ctx->col,
                                                          ctx->interp, ctx->d_flag);
    };
    if (ord == 0) launch(k_interp_2d<0>);
    else if (ord == 2) launch(k_interp_2d<2>);
    else launch(k_interp_2d<1>);
    CU_LAUNCH(ctx);
    return check_flag(ctx, "interpolation");
}

mlpg_status run_assemble(mlpg_ctx *ctx) {
    const int tri1d = 5, nline = 5;
    MLPG_TRY(upload_rules(ctx, tri1d, nline));
    ctx->nmats = mlpg_n_matrices(2);
    ctx->nvecs = mlpg_n_vectors(2);
    if (!ctx->mats) MLPG_TRY(dalloc(ctx, &ctx->mats, (size_t)ctx->nmats * ctx->nnz));
    if (!ctx->vecs) MLPG_TRY(dalloc(ctx, &ctx->vecs, (size_t)ctx->nvecs * ctx->n));
    CU(ctx, cudaMemsetAsync(ctx->mats, 0, sizeof(double) * ctx->nmats * ctx->nnz, ctx->stream));
    CU(ctx, cudaMemsetAsync(ctx->vecs, 0, sizeof(double) * ctx->nvecs * ctx->n, ctx->stream));
    CU(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
    AsmArgs a;
    a.n = ctx->n; a.nnz = ctx->nnz;
    a.x = ctx->x; a.R = ctx->R; a.V = ctx->V; a.sig_t = ctx->sig_t; a.sig_s = ctx->sig_s; a.q = ctx->q;
    a.rowptr = ctx->rowptr; a.col = ctx->col; a.cptr = ctx->cptr; a.labels = ctx->labels;
    a.verts = ctx->verts;
    a.ntri = tri1d * tri1d; a.nline = nline;
    a.mats = ctx->mats; a.vecs = ctx->vecs; a.flag = ctx->d_flag;
    // shared table + weights + faces + pair sums for <ORD, MAXS, CHUNK>
    auto run = [&](auto kern, int maxs, int chunk) -> mlpg_status {
        size_t smem = sizeof(double) * (3 * (size_t)chunk * maxs + chunk + chunk / 2 + 1 +
                                        11 * (size_t)maxs * (maxs + 1) / 2);
        CU(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<ctx->n, kThreads, smem, ctx->stream>>>(a);
        CU_LAUNCH(ctx);
        return MLPG_OK;
    };
    if (ctx->opt.rk_order == 0) MLPG_TRY(run(k_assemble_2d<0, 48, 32>, 48, 32));
    else if (ctx->opt.rk_order == 2) MLPG_TRY(run(k_assemble_2d<2, 48, 32>, 48, 32));
    else MLPG_TRY(run(k_assemble_2d<1, kMaxS, kChunk>, kMaxS, kChunk));
    return check_flag(ctx, "assembly");
}

}  // namespace mlpg
