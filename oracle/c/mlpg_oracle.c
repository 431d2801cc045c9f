/*
 * Plain FP64 CPU oracle for the meshless (MLPG / reproducing-kernel / Voronoi
 * cell) discretisation of the discrete-ordinates transport equation of
 * Bassett & Owen, "Meshless discretization of the discrete-ordinates transport
 * equation with integration based on Voronoi cells" (arXiv 2008.02205).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of the method that the CUDA library is checked against.  Only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or generator with the CUDA library.
 *
 * What lives here (the loop-heavy parts; the linear algebra is in
 * oracle/mlpg_oracle.py):
 *   A. reference quadrature rules (Gauss-Jacobi by Golub-Welsch)   App. A, Sec. 3.2
 *   B. overlap connectivity by brute force                           Sec. 3.4
 *   C. Voronoi-like cells by half-plane clipping of the kernel box   Sec. 3.1
 *   D. quadrature points of the fan triangles and boundary edges     Sec. 3.1-3.2, App. A
 *   C3/D3. the same in 3D: polyhedral cells, fan tetrahedra, boundary
 *      triangles                                                    Sec. 3.1-3.2, App. A
 *   E. cubic-spline kernel and linear reproducing-kernel functions   Sec. 2.1-2.2
 *   F. quadrature-outermost integration of the bilinear forms        Sec. 3.2 (Alg. 1), Sec. 4.1
 *
 * Conventions (readings of the paper, shared by contract with the CUDA path):
 *   - kernel support radius R_j, smoothing length h_j = R_j / 2, cubic spline
 *     W(chi) with support chi < 2, chi = |x - x_j| / h_j (normalisation constant
 *     dropped: it cancels in the RK functions).
 *   - overlap neighbours of i: all j (including i) with |x_i - x_j| < R_i + R_j.
 *   - functions supported at x: all j with |x - x_j| < R_j.
 *   - the cell of i is [x_i - R_i, x_i + R_i]^d intersected with the domain box,
 *     clipped by the bisector half-planes of every overlap neighbour j != i.
 *   - 2D cells are fanned into triangles (x_i, v_k, v_{k+1}) from the generator,
 *     vertices counter-clockwise; the reference rule is mapped with p0 = x_i.
 *   - 3D cells are fanned into tetrahedra (x_i, c_f, f_k, f_{k+1}), one per edge
 *     of every face f, c_f the average of f's vertices; boundary faces into
 *     triangles (c_f, f_k, f_{k+1}).
 *   - RK basis P_j(x): the monomials of (x - x_j)/s up to the RK order (linear:
 *     [1, (x - x_j)/s]) with s = h of the point owning the evaluation point (any
 *     common scale gives the same U in exact arithmetic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_CAP -2
#define ORC_ERR_SINGULAR -6

#define LABEL_EXTENT (-100)

/* ======================================================================
 * A. Reference quadrature rules (Sec. 3.2 and Sec. 5; mapped onto the cells as in App. A)
 * ====================================================================== */

/* Eigen-decomposition of a small dense symmetric matrix a[n*n] by cyclic
 * Jacobi rotations.  On return the diagonal of a holds the eigenvalues and the
 * columns of v the eigenvectors. */
static void sym_eig_jacobi(int n, double *a, double *v)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) v[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += a[i * n + j] * a[i * n + j];
                if (i != j) off += a[i * n + j] * a[i * n + j];
            }
        if (off <= 1e-32 * tot) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a[p * n + q];
                if (apq == 0.0) continue;
                double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) { /* A <- A J */
                    double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - s * akq;
                    a[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) { /* A <- J^T A */
                    double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - s * aqk;
                    a[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = v[k * n + p], vkq = v[k * n + q];
                    v[k * n + p] = c * vkp - s * vkq;
                    v[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

/* (Sec. 3.2, App. A) Gauss-Jacobi rule on [-1, 1] for the weight (1 - t)^a (1 + t)^b, n points,
 * by Golub-Welsch: nodes are the eigenvalues of the symmetric tridiagonal
 * matrix of the Jacobi three-term recurrence, weights mu0 * (v_0k)^2.
 * Nodes returned in increasing order. */
int orc_gauss_jacobi(int n, double a, double b, double *t, double *wt)
{
    if (n < 1 || n > 64) return ORC_ERR_ARG;
    double *J = calloc((size_t)n * n, sizeof(double));
    double *V = calloc((size_t)n * n, sizeof(double));
    for (int k = 0; k < n; ++k) {
        double s = 2.0 * k + a + b;
        double diag;
        if (k == 0) diag = (b - a) / (a + b + 2.0);
        else diag = (b * b - a * a) / (s * (s + 2.0));
        J[k * n + k] = diag;
        if (k >= 1) {
            double kk = k;
            double beta = 4.0 * kk * (kk + a) * (kk + b) * (kk + a + b) /
                          (s * s * (s + 1.0) * (s - 1.0));
            J[k * n + (k - 1)] = J[(k - 1) * n + k] = sqrt(beta);
        }
    }
    sym_eig_jacobi(n, J, V);
    double mu0 = pow(2.0, a + b + 1.0) * tgamma(a + 1.0) * tgamma(b + 1.0) / tgamma(a + b + 2.0);
    for (int k = 0; k < n; ++k) {
        t[k] = J[k * n + k];
        wt[k] = mu0 * V[0 * n + k] * V[0 * n + k];
    }
    /* sort ascending (selection sort; n is tiny) */
    for (int i = 0; i < n; ++i) {
        int m = i;
        for (int j = i + 1; j < n; ++j) if (t[j] < t[m]) m = j;
        double tt = t[i]; t[i] = t[m]; t[m] = tt;
        double ww = wt[i]; wt[i] = wt[m]; wt[m] = ww;
    }
    free(J); free(V);
    return ORC_OK;
}

/* (Sec. 3.2, Sec. 5.1) Reference triangle {xi1, xi2 >= 0, xi1 + xi2 <= 1}: conical product of an
 * n-point Gauss-Jacobi(1,0) rule in u and an n-point Gauss-Legendre rule in v,
 * xi1 = u, xi2 = (1 - u) v, exact for total degree 2n - 1.  Point k = iu*n + iv.
 * xi[2*k], w[k]; sum(w) = 1/2. */
int orc_triangle_rule(int n, double *xi, double *w)
{
    double tu[64], wu[64], tv[64], wv[64];
    if (orc_gauss_jacobi(n, 1.0, 0.0, tu, wu) || orc_gauss_jacobi(n, 0.0, 0.0, tv, wv))
        return ORC_ERR_ARG;
    for (int iu = 0; iu < n; ++iu)
        for (int iv = 0; iv < n; ++iv) {
            double u = 0.5 * (tu[iu] + 1.0), v = 0.5 * (tv[iv] + 1.0);
            int k = iu * n + iv;
            xi[2 * k + 0] = u;
            xi[2 * k + 1] = (1.0 - u) * v;
            w[k] = 0.25 * wu[iu] * 0.5 * wv[iv];
        }
    return ORC_OK;
}

/* Gauss-Legendre on [-1, 1] (App. A line map x = p0 + (p1 - p0)(xi + 1)/2). */
int orc_line_rule(int n, double *t, double *w) { return orc_gauss_jacobi(n, 0.0, 0.0, t, w); }

/* (Sec. 3.2, Sec. 5) Reference tetrahedron {xi >= 0, xi1 + xi2 + xi3 <= 1}: conical product of
 * n-point Gauss-Jacobi(2,0) in u, Gauss-Jacobi(1,0) in v and Gauss-Legendre in
 * s, xi1 = u, xi2 = (1 - u) v, xi3 = (1 - u)(1 - v) s (Jacobian
 * (1 - u)^2 (1 - v), carried by the Jacobi weights), exact for total degree
 * 2n - 1.  Point k = (iu*n + iv)*n + is.  xi[3*k], w[k]; sum(w) = 1/6. */
int orc_tet_rule(int n, double *xi, double *w)
{
    double tu[64], wu[64], tv[64], wv[64], ts[64], ws[64];
    if (orc_gauss_jacobi(n, 2.0, 0.0, tu, wu) || orc_gauss_jacobi(n, 1.0, 0.0, tv, wv) ||
        orc_gauss_jacobi(n, 0.0, 0.0, ts, ws))
        return ORC_ERR_ARG;
    for (int iu = 0; iu < n; ++iu)
        for (int iv = 0; iv < n; ++iv)
            for (int is = 0; is < n; ++is) {
                double u = 0.5 * (tu[iu] + 1.0), v = 0.5 * (tv[iv] + 1.0), r = 0.5 * (ts[is] + 1.0);
                int k = (iu * n + iv) * n + is;
                xi[3 * k + 0] = u;
                xi[3 * k + 1] = (1.0 - u) * v;
                xi[3 * k + 2] = (1.0 - u) * (1.0 - v) * r;
                w[k] = (wu[iu] / 8.0) * (wv[iv] / 4.0) * (ws[is] / 2.0);
            }
    return ORC_OK;
}

/* ======================================================================
 * B. Overlap connectivity (Sec. 3.4): j is a neighbour of i when the kernel
 * supports overlap, |x_i - x_j| < R_i + R_j.  Brute force over all pairs.
 * Pass col == NULL to get the row counts only (rowptr filled, returns nnz).
 * ====================================================================== */
static double dist(int dim, const double *a, const double *b)
{
    double s = 0.0;
    for (int k = 0; k < dim; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
    return sqrt(s);
}

/* (Sec. 3.4) Overlap rows of all points, columns sorted; see section B. */
int64_t orc_neighbors(int dim, int64_t n, const double *x, const double *R, int64_t *rowptr,
                      int32_t *col)
{
    rowptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = rowptr[i];
        for (int64_t j = 0; j < n; ++j) {
            if (dist(dim, x + i * dim, x + j * dim) < R[i] + R[j]) {
                if (col) col[c] = (int32_t)j;
                ++c;
            }
        }
        rowptr[i + 1] = c;
    }
    return rowptr[n];
}

/* ======================================================================
 * C. Cells in 2D (Sec. 3.1): start from the kernel-extent box intersected with
 * the domain, clip by the bisector of every overlap neighbour.
 * A vertex label describes the edge that starts at that vertex:
 *   label >= 0      : bisector with point `label`
 *   label = -(f+1)  : domain face f (0:-x 1:+x 2:-y 3:+y)
 *   LABEL_EXTENT    : side of the kernel-extent box inside the domain
 * ====================================================================== */
static int clip_polygon(int nv, double *vx, double *vy, int32_t *lab, double *wx, double *wy,
                        int32_t *wl, const double *xi, const double *xj, int32_t j)
{
    double dx = xj[0] - xi[0], dy = xj[1] - xi[1];
    double mx = 0.5 * (xi[0] + xj[0]), my = 0.5 * (xi[1] + xj[1]);
    int out = 0;
    int all_in = 1;
    for (int k = 0; k < nv; ++k)
        if ((vx[k] - mx) * dx + (vy[k] - my) * dy > 0.0) { all_in = 0; break; }
    if (all_in) return nv;
    for (int k = 0; k < nv; ++k) {
        int k1 = (k + 1) % nv;
        double sk = (vx[k] - mx) * dx + (vy[k] - my) * dy;
        double sk1 = (vx[k1] - mx) * dx + (vy[k1] - my) * dy;
        int ink = sk <= 0.0, ink1 = sk1 <= 0.0;
        if (ink) { wx[out] = vx[k]; wy[out] = vy[k]; wl[out] = lab[k]; ++out; }
        if (ink != ink1) {
            double f = sk / (sk - sk1);
            wx[out] = vx[k] + (vx[k1] - vx[k]) * f;
            wy[out] = vy[k] + (vy[k1] - vy[k]) * f;
            wl[out] = ink ? j : lab[k];
            ++out;
        }
    }
    memcpy(vx, wx, sizeof(double) * out);
    memcpy(vy, wy, sizeof(double) * out);
    memcpy(lab, wl, sizeof(int32_t) * out);
    return out;
}

/* (Sec. 3.1, Fig. 1) Cells of all points.  cptr[n+1]; verts[2*cap]; labels[cap]; vol[n].
 * Pass verts == NULL to get the vertex counts only.  Returns total vertices. */
int64_t orc_cells_2d(int64_t n, const double *x, const double *R, const double *lo,
                     const double *hi, const int64_t *rowptr, const int32_t *col, int64_t *cptr,
                     double *verts, int32_t *labels, double *vol)
{
    int64_t maxrow = 0;
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] - rowptr[i] > maxrow) maxrow = rowptr[i + 1] - rowptr[i];
    int cap = (int)(2 * maxrow + 16);
    double *vx = malloc(sizeof(double) * cap), *vy = malloc(sizeof(double) * cap);
    double *wx = malloc(sizeof(double) * cap), *wy = malloc(sizeof(double) * cap);
    int32_t *lab = malloc(sizeof(int32_t) * cap), *wl = malloc(sizeof(int32_t) * cap);
    cptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double *xi = x + 2 * i;
        double x0 = xi[0] - R[i], x1 = xi[0] + R[i], y0 = xi[1] - R[i], y1 = xi[1] + R[i];
        int fx0 = x0 <= lo[0], fx1 = x1 >= hi[0], fy0 = y0 <= lo[1], fy1 = y1 >= hi[1];
        if (fx0) x0 = lo[0];
        if (fx1) x1 = hi[0];
        if (fy0) y0 = lo[1];
        if (fy1) y1 = hi[1];
        /* counter-clockwise from the lower-left corner */
        vx[0] = x0; vy[0] = y0; lab[0] = fy0 ? -(2 + 1) : LABEL_EXTENT; /* bottom */
        vx[1] = x1; vy[1] = y0; lab[1] = fx1 ? -(1 + 1) : LABEL_EXTENT; /* right  */
        vx[2] = x1; vy[2] = y1; lab[2] = fy1 ? -(3 + 1) : LABEL_EXTENT; /* top    */
        vx[3] = x0; vy[3] = y1; lab[3] = fx0 ? -(0 + 1) : LABEL_EXTENT; /* left   */
        int nv = 4;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (j == i) continue;
            nv = clip_polygon(nv, vx, vy, lab, wx, wy, wl, xi, x + 2 * (int64_t)j, j);
        }
        double area = 0.0;
        for (int k = 0; k < nv; ++k) {
            int k1 = (k + 1) % nv;
            area += vx[k] * vy[k1] - vx[k1] * vy[k];
        }
        if (vol) vol[i] = 0.5 * area;
        if (verts) {
            for (int k = 0; k < nv; ++k) {
                verts[2 * (cptr[i] + k) + 0] = vx[k];
                verts[2 * (cptr[i] + k) + 1] = vy[k];
                labels[cptr[i] + k] = lab[k];
            }
        }
        cptr[i + 1] = cptr[i] + nv;
    }
    free(vx); free(vy); free(wx); free(wy); free(lab); free(wl);
    return cptr[n];
}

/* ======================================================================
 * D. Quadrature points (Sec. 3.2, App. A).
 * Volume: for each cell i, each fan triangle (x_i, v_k, v_{k+1}), each point of
 * the reference triangle rule: x = p0 + (p1 - p0) xi1 + (p2 - p0) xi2,
 * weight w_ref |J| with |J| = |det[p1 - p0, p2 - p0]|.
 * Boundary: each cell edge labelled as a domain face, Gauss-Legendre points
 * x = p0 + (p1 - p0)(t + 1)/2, weight w_ref |p1 - p0| / 2.
 * Outputs are optional (NULL = count only).  Returns the number of points.
 * ====================================================================== */
int64_t orc_volume_qps_2d(int64_t n, const double *x, const int64_t *cptr, const double *verts,
                          int nref, double *xq, double *wq, int32_t *owner)
{
    double xi[2 * 4096], w[4096];
    int nq = nref * nref;
    orc_triangle_rule(nref, xi, w);
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
        int nv = (int)(cptr[i + 1] - cptr[i]);
        const double *p0 = x + 2 * i;
        for (int k = 0; k < nv; ++k) {
            const double *p1 = verts + 2 * (cptr[i] + k);
            const double *p2 = verts + 2 * (cptr[i] + (k + 1) % nv);
            double e1x = p1[0] - p0[0], e1y = p1[1] - p0[1];
            double e2x = p2[0] - p0[0], e2y = p2[1] - p0[1];
            double det = fabs(e1x * e2y - e1y * e2x);
            for (int q = 0; q < nq; ++q) {
                if (xq) {
                    xq[2 * c + 0] = p0[0] + e1x * xi[2 * q] + e2x * xi[2 * q + 1];
                    xq[2 * c + 1] = p0[1] + e1y * xi[2 * q] + e2y * xi[2 * q + 1];
                    wq[c] = w[q] * det;
                    owner[c] = (int32_t)i;
                }
                ++c;
            }
        }
    }
    return c;
}

/* (Sec. 3.2, App. A) Boundary points: the Gauss-Legendre rule on every cell edge that
 * lies on the domain boundary, with the edge's face index; see section D. */
int64_t orc_boundary_qps_2d(int64_t n, const int64_t *cptr, const double *verts,
                            const int32_t *labels, int nref, double *xb, double *wb, int32_t *face,
                            int32_t *owner)
{
    double t[64], w[64];
    orc_line_rule(nref, t, w);
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
        int nv = (int)(cptr[i + 1] - cptr[i]);
        for (int k = 0; k < nv; ++k) {
            int32_t L = labels[cptr[i] + k];
            if (L >= 0 || L == LABEL_EXTENT) continue;
            const double *p0 = verts + 2 * (cptr[i] + k);
            const double *p1 = verts + 2 * (cptr[i] + (k + 1) % nv);
            double len = sqrt((p1[0] - p0[0]) * (p1[0] - p0[0]) + (p1[1] - p0[1]) * (p1[1] - p0[1]));
            for (int q = 0; q < nref; ++q) {
                if (xb) {
                    double s = 0.5 * (t[q] + 1.0);
                    xb[2 * c + 0] = p0[0] + (p1[0] - p0[0]) * s;
                    xb[2 * c + 1] = p0[1] + (p1[1] - p0[1]) * s;
                    wb[c] = w[q] * 0.5 * len;
                    face[c] = -L - 1;
                    owner[c] = (int32_t)i;
                }
                ++c;
            }
        }
    }
    return c;
}

/* ======================================================================
 * C3/D3. Cells and quadrature points in 3D (Sec. 3.1-3.2, App. A).
 * The cell of i is the box [x_i - R_i, x_i + R_i]^3 intersected with the domain,
 * clipped by the bisector half-space {y : (y - m).(x_j - x_i) <= 0},
 * m = (x_i + x_j)/2, of every overlap neighbour j != i.  A cell is a list of
 * planar polygonal faces, each counter-clockwise seen from outside, with the
 * labels of the 2D cells (domain faces 0:-x 1:+x 2:-y 3:+y 4:-z 5:+z).
 * Clipping by one half-space: every face polygon is clipped (Sutherland-
 * Hodgman); the points where face edges cross the plane and the vertices on
 * it, taken once each, ordered by angle about the plane normal, form the new
 * face on the plane.  A vertex whose signed distance is within eps of the
 * plane counts as on it (planes through existing edges, vertices or faces, as
 * in unjittered lattices); a plane with no vertex beyond eps cuts nothing.
 * A neighbour whose plane lies beyond the farthest vertex cuts nothing and is
 * skipped.  Every face is fanned from its centre c_f (the average of its
 * vertices), so that the split does not depend on where a face's vertex list
 * starts: the cell into tetrahedra (x_i, c_f, v_k, v_k+1), one per face edge,
 * and boundary faces into triangles (c_f, v_k, v_k+1).
 * ====================================================================== */
typedef struct {
    int nf, cap_f, cap_v;
    int *nv;       /* [cap_f] vertices of each face */
    int32_t *lab;  /* [cap_f] label of each face */
    double *v;     /* [cap_f][cap_v][3] */
} poly3;

static int poly3_alloc(poly3 *P, int cap_f, int cap_v)
{
    P->nf = 0; P->cap_f = cap_f; P->cap_v = cap_v;
    P->nv = malloc(sizeof(int) * cap_f);
    P->lab = malloc(sizeof(int32_t) * cap_f);
    P->v = malloc(sizeof(double) * 3 * (size_t)cap_f * cap_v);
    return P->nv && P->lab && P->v ? ORC_OK : ORC_ERR_CAP;
}

static void poly3_free(poly3 *P) { free(P->nv); free(P->lab); free(P->v); }

static double *pv(const poly3 *P, int f, int k) { return P->v + 3 * ((size_t)f * P->cap_v + k); }

static void poly3_box(poly3 *P, const double *b0, const double *b1, const int *on_lo, const int *on_hi)
{
    /* corners c[ix + 2 iy + 4 iz]; faces listed counter-clockwise from outside */
    static const int F[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4},
                                {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};
    double c[8][3];
    for (int k = 0; k < 8; ++k) {
        c[k][0] = (k & 1) ? b1[0] : b0[0];
        c[k][1] = (k & 2) ? b1[1] : b0[1];
        c[k][2] = (k & 4) ? b1[2] : b0[2];
    }
    P->nf = 6;
    for (int f = 0; f < 6; ++f) {
        int a = f / 2, hi = f % 2;
        int dom = hi ? on_hi[a] : on_lo[a];
        P->lab[f] = dom ? -(f + 1) : LABEL_EXTENT;
        P->nv[f] = 4;
        for (int k = 0; k < 4; ++k) memcpy(pv(P, f, k), c[F[f][k]], sizeof(double) * 3);
    }
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double poly3_rmax(const poly3 *P, const double *g)
{
    double r2 = 0.0;
    for (int f = 0; f < P->nf; ++f)
        for (int k = 0; k < P->nv[f]; ++k) {
            const double *q = pv(P, f, k);
            double d[3] = {q[0] - g[0], q[1] - g[1], q[2] - g[2]};
            if (dot3(d, d) > r2) r2 = dot3(d, d);
        }
    return sqrt(r2);
}

/* (Sec. 3.1) Clip P by the bisector of (xi, xj) into W, then copy back.  cut[] holds up
 * to 2 cap_v cap_f points.  tol: length scale of "the same point".  Returns 0,
 * or ORC_ERR_CAP when a capacity is exceeded. */
static int poly3_clip(poly3 *P, poly3 *W, double *cut, const double *xi, const double *xj, int32_t j,
                      double tol)
{
    double d[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
    double m[3] = {0.5 * (xi[0] + xj[0]), 0.5 * (xi[1] + xj[1]), 0.5 * (xi[2] + xj[2])};
    const double eps = tol * sqrt(dot3(d, d));   /* signed distances s carry a factor |d| */
    int any_out = 0;
    for (int f = 0; f < P->nf && !any_out; ++f)
        for (int k = 0; k < P->nv[f]; ++k) {
            const double *a = pv(P, f, k);
            double am[3] = {a[0] - m[0], a[1] - m[1], a[2] - m[2]};
            if (dot3(am, d) > eps) { any_out = 1; break; }
        }
    if (!any_out) return ORC_OK;
    int nc = 0;
    W->nf = 0;
    for (int f = 0; f < P->nf; ++f) {
        int nv = P->nv[f], out = 0;
        if (W->nf >= W->cap_f) return ORC_ERR_CAP;
        for (int k = 0; k < nv; ++k) {
            const double *a = pv(P, f, k), *b = pv(P, f, (k + 1) % nv);
            double am[3] = {a[0] - m[0], a[1] - m[1], a[2] - m[2]};
            double bm[3] = {b[0] - m[0], b[1] - m[1], b[2] - m[2]};
            double sa = dot3(am, d), sb = dot3(bm, d);
            if (out + 2 > W->cap_v || nc + 2 > 2 * P->cap_v * P->cap_f) return ORC_ERR_CAP;
            if (sa <= eps) {                       /* inside or on the plane: kept */
                memcpy(pv(W, W->nf, out++), a, sizeof(double) * 3);
                if (sa >= -eps) memcpy(cut + 3 * nc++, a, sizeof(double) * 3);
            }
            if ((sa < -eps && sb > eps) || (sa > eps && sb < -eps)) {   /* strict crossing */
                double t = sa / (sa - sb), *q = pv(W, W->nf, out++);
                for (int e = 0; e < 3; ++e) q[e] = a[e] + (b[e] - a[e]) * t;
                memcpy(cut + 3 * nc++, q, sizeof(double) * 3);
            }
        }
        if (out >= 3) {
            W->nv[W->nf] = out;
            W->lab[W->nf] = P->lab[f];
            ++W->nf;
        }
    }
    /* the new face: distinct cut points ordered counter-clockwise about +d */
    int nu = 0;
    for (int c = 0; c < nc; ++c) {
        int dup = 0;
        for (int u = 0; u < nu && !dup; ++u) {
            double e[3] = {cut[3 * c] - cut[3 * u], cut[3 * c + 1] - cut[3 * u + 1], cut[3 * c + 2] - cut[3 * u + 2]};
            dup = sqrt(dot3(e, e)) <= tol;
        }
        if (!dup) {
            memmove(cut + 3 * nu, cut + 3 * c, sizeof(double) * 3);
            ++nu;
        }
    }
    if (nu >= 3) {
        if (W->nf >= W->cap_f || nu > W->cap_v) return ORC_ERR_CAP;
        double dl = sqrt(dot3(d, d)), n[3] = {d[0] / dl, d[1] / dl, d[2] / dl};
        int a = 0;
        for (int e = 1; e < 3; ++e)
            if (fabs(n[e]) < fabs(n[a])) a = e;
        double e1[3] = {-n[a] * n[0], -n[a] * n[1], -n[a] * n[2]}, e2[3];
        e1[a] += 1.0;
        double l1 = sqrt(dot3(e1, e1));
        for (int e = 0; e < 3; ++e) e1[e] /= l1;
        cross3(n, e1, e2);
        double cen[3] = {0, 0, 0};
        for (int u = 0; u < nu; ++u)
            for (int e = 0; e < 3; ++e) cen[e] += cut[3 * u + e] / nu;
        double *ang = malloc(sizeof(double) * nu);
        int *ord = malloc(sizeof(int) * nu);
        for (int u = 0; u < nu; ++u) {
            double r[3] = {cut[3 * u] - cen[0], cut[3 * u + 1] - cen[1], cut[3 * u + 2] - cen[2]};
            ang[u] = atan2(dot3(r, e2), dot3(r, e1));
            ord[u] = u;
        }
        for (int u = 1; u < nu; ++u) {   /* insertion sort by angle */
            int o = ord[u], k = u;
            while (k > 0 && ang[ord[k - 1]] > ang[o]) { ord[k] = ord[k - 1]; --k; }
            ord[k] = o;
        }
        for (int u = 0; u < nu; ++u) memcpy(pv(W, W->nf, u), cut + 3 * ord[u], sizeof(double) * 3);
        W->nv[W->nf] = nu;
        W->lab[W->nf] = j;
        ++W->nf;
        free(ang); free(ord);
    }
    P->nf = W->nf;
    for (int f = 0; f < W->nf; ++f) {
        P->nv[f] = W->nv[f];
        P->lab[f] = W->lab[f];
        memcpy(pv(P, f, 0), pv(W, f, 0), sizeof(double) * 3 * W->nv[f]);
    }
    return ORC_OK;
}

/* centre of face f: the average of its vertices */
static void face_centre(const double *v, int nv, double *c)
{
    c[0] = c[1] = c[2] = 0.0;
    for (int k = 0; k < nv; ++k)
        for (int e = 0; e < 3; ++e) c[e] += v[3 * k + e];
    for (int e = 0; e < 3; ++e) c[e] /= nv;
}

/* volume of a cell: sum of |det(c_f - g, vk - g, vk+1 - g)| / 6 over the fans */
static double poly3_volume(const poly3 *P, const double *g)
{
    double vol = 0.0;
    for (int f = 0; f < P->nf; ++f) {
        double v0[3];
        face_centre(pv(P, f, 0), P->nv[f], v0);
        for (int k = 0; k < P->nv[f]; ++k) {
            const double *v1 = pv(P, f, k), *v2 = pv(P, f, (k + 1) % P->nv[f]);
            double a[3] = {v0[0] - g[0], v0[1] - g[1], v0[2] - g[2]};
            double b[3] = {v1[0] - g[0], v1[1] - g[1], v1[2] - g[2]};
            double c[3] = {v2[0] - g[0], v2[1] - g[1], v2[2] - g[2]}, bc[3];
            cross3(b, c, bc);
            vol += fabs(dot3(a, bc)) / 6.0;
        }
    }
    return vol;
}

/* (Sec. 3.1) Cells of all points.  fptr[n+1] (faces of each cell), vol[n], *nfaces = all
 * faces; with vptr/verts/labels NULL only the counts are produced.  Otherwise
 * vptr[nfaces+1] (vertices of each face), verts[3 * total], labels[nfaces].
 * Returns the total number of face vertices, or a negative error. */
int64_t orc_cells_3d(int64_t n, const double *x, const double *R, const double *lo, const double *hi,
                     const int64_t *rowptr, const int32_t *col, int64_t *fptr, int64_t *vptr,
                     double *verts, int32_t *labels, double *vol, int64_t *nfaces)
{
    int64_t maxrow = 0;
    for (int64_t i = 0; i < n; ++i)
        if (rowptr[i + 1] - rowptr[i] > maxrow) maxrow = rowptr[i + 1] - rowptr[i];
    int cap_f = (int)maxrow + 8, cap_v = (int)maxrow + 16;
    poly3 P, W;
    if (poly3_alloc(&P, cap_f, cap_v) || poly3_alloc(&W, cap_f, cap_v)) return ORC_ERR_CAP;
    double *cut = malloc(sizeof(double) * 6 * (size_t)cap_f * cap_v);
    int64_t nv_tot = 0, nf_tot = 0;
    int rc = ORC_OK;
    fptr[0] = 0;
    if (vptr) vptr[0] = 0;
    for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
        const double *xi = x + 3 * i;
        double b0[3], b1[3];
        int on_lo[3], on_hi[3];
        for (int a = 0; a < 3; ++a) {
            b0[a] = xi[a] - R[i];
            b1[a] = xi[a] + R[i];
            on_lo[a] = b0[a] <= lo[a];
            on_hi[a] = b1[a] >= hi[a];
            if (on_lo[a]) b0[a] = lo[a];
            if (on_hi[a]) b1[a] = hi[a];
        }
        poly3_box(&P, b0, b1, on_lo, on_hi);
        double rmax = poly3_rmax(&P, xi);
        for (int64_t p = rowptr[i]; p < rowptr[i + 1] && rc == ORC_OK; ++p) {
            int32_t j = col[p];
            if (j == i) continue;
            const double *xj = x + 3 * (int64_t)j;
            double dd[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
            if (0.5 * sqrt(dot3(dd, dd)) >= rmax) continue;   /* plane beyond every vertex */
            rc = poly3_clip(&P, &W, cut, xi, xj, j, 1e-12 * R[i]);
            rmax = poly3_rmax(&P, xi);
        }
        if (rc != ORC_OK) break;
        if (vol) vol[i] = poly3_volume(&P, xi);
        for (int f = 0; f < P.nf; ++f) {
            if (vptr) {
                vptr[nf_tot + f + 1] = vptr[nf_tot + f] + P.nv[f];
                labels[nf_tot + f] = P.lab[f];
                memcpy(verts + 3 * vptr[nf_tot + f], pv(&P, f, 0), sizeof(double) * 3 * P.nv[f]);
            }
            nv_tot += P.nv[f];
        }
        nf_tot += P.nf;
        fptr[i + 1] = nf_tot;
    }
    poly3_free(&P); poly3_free(&W); free(cut);
    if (nfaces) *nfaces = nf_tot;
    return rc == ORC_OK ? nv_tot : rc;
}

/* Volume points: tetrahedra (x_i, c_f, vk, vk+1) of every face fan, reference
 * rule mapped by x = p0 + (p_a - p0) xi_a (App. A), weight w_ref |det J|. */
int64_t orc_volume_qps_3d(int64_t n, const double *x, const int64_t *fptr, const int64_t *vptr,
                          const double *verts, int nref, double *xq, double *wq, int32_t *owner)
{
    double xi[3 * 4096], w[4096];
    if (nref < 1 || nref > 16 || orc_tet_rule(nref, xi, w)) return ORC_ERR_ARG;
    int nq = nref * nref * nref;
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double *g = x + 3 * i;
        for (int64_t f = fptr[i]; f < fptr[i + 1]; ++f) {
            int nv = (int)(vptr[f + 1] - vptr[f]);
            double v0[3];
            face_centre(verts + 3 * vptr[f], nv, v0);
            for (int k = 0; k < nv; ++k) {
                const double *v1 = verts + 3 * (vptr[f] + k), *v2 = verts + 3 * (vptr[f] + (k + 1) % nv);
                double e1[3] = {v0[0] - g[0], v0[1] - g[1], v0[2] - g[2]};
                double e2[3] = {v1[0] - g[0], v1[1] - g[1], v1[2] - g[2]};
                double e3[3] = {v2[0] - g[0], v2[1] - g[1], v2[2] - g[2]}, c23[3];
                cross3(e2, e3, c23);
                double det = fabs(dot3(e1, c23));
                for (int q = 0; q < nq; ++q) {
                    if (xq) {
                        for (int e = 0; e < 3; ++e)
                            xq[3 * c + e] = g[e] + e1[e] * xi[3 * q] + e2[e] * xi[3 * q + 1] + e3[e] * xi[3 * q + 2];
                        wq[c] = w[q] * det;
                        owner[c] = (int32_t)i;
                    }
                    ++c;
                }
            }
        }
    }
    return c;
}

/* Boundary points: triangles (c_f, vk, vk+1) of every face on the domain
 * boundary, x = p0 + (p_a - p0) xi_a, weight w_ref |e1 x e2| (App. A). */
int64_t orc_boundary_qps_3d(int64_t n, const int64_t *fptr, const int64_t *vptr, const double *verts,
                            const int32_t *labels, int nref, double *xb, double *wb, int32_t *face,
                            int32_t *owner)
{
    double xi[2 * 4096], w[4096];
    if (nref < 1 || nref > 64 || orc_triangle_rule(nref, xi, w)) return ORC_ERR_ARG;
    int nq = nref * nref;
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t f = fptr[i]; f < fptr[i + 1]; ++f) {
            int32_t L = labels[f];
            if (L >= 0 || L == LABEL_EXTENT) continue;
            int nv = (int)(vptr[f + 1] - vptr[f]);
            double p0[3];
            face_centre(verts + 3 * vptr[f], nv, p0);
            for (int k = 0; k < nv; ++k) {
                const double *p1 = verts + 3 * (vptr[f] + k), *p2 = verts + 3 * (vptr[f] + (k + 1) % nv);
                double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
                double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]}, cr[3];
                cross3(e1, e2, cr);
                double K = sqrt(dot3(cr, cr));
                for (int q = 0; q < nq; ++q) {
                    if (xb) {
                        for (int e = 0; e < 3; ++e) xb[3 * c + e] = p0[e] + e1[e] * xi[2 * q] + e2[e] * xi[2 * q + 1];
                        wb[c] = w[q] * K;
                        face[c] = -L - 1;
                        owner[c] = (int32_t)i;
                    }
                    ++c;
                }
            }
        }
    return c;
}

/* ======================================================================
 * E. Kernel and reproducing-kernel functions (Sec. 2.1-2.2).
 * ====================================================================== */
/* cubic spline base kernel, support chi < 2 (normalisation dropped) */
static double kernel_w(double chi)
{
    if (chi < 1.0) return 1.0 - 1.5 * chi * chi + 0.75 * chi * chi * chi;
    if (chi < 2.0) return 0.25 * (2.0 - chi) * (2.0 - chi) * (2.0 - chi);
    return 0.0;
}
/* (Sec. 2.1) derivative of the cubic spline in chi */
static double kernel_dw(double chi)
{
    if (chi < 1.0) return -3.0 * chi + 2.25 * chi * chi;
    if (chi < 2.0) return -0.75 * (2.0 - chi) * (2.0 - chi);
    return 0.0;
}

/* Solve A y = b for a small dense matrix (Gaussian elimination, partial
 * pivoting).  A is destroyed.  Returns nonzero when a pivot vanishes. */
static int dense_solve(int n, double *A, double *b)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r) if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (!(fabs(A[p * n + c]) > 1e-300)) return 1;
        if (p != c) {
            for (int k = 0; k < n; ++k) { double t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return 0;
}

/* Basis of the RK correction (Sec. 2.2): all monomials of xi = (x - x_j)/s up
 * to total degree `order` (0, 1 or 2), ordered 1, xi_a, xi_a xi_b (a <= b).
 * P[np] and its derivatives dP[g][np] = d P / d xi_g.  Returns np. */
static int rk_basis(int dim, int order, const double *xi, double *P, double dP[3][10])
{
    int k = 0;
    P[k] = 1.0;
    for (int g = 0; g < dim; ++g) dP[g][k] = 0.0;
    ++k;
    if (order >= 1)
        for (int a = 0; a < dim; ++a, ++k) {
            P[k] = xi[a];
            for (int g = 0; g < dim; ++g) dP[g][k] = (g == a) ? 1.0 : 0.0;
        }
    if (order >= 2)
        for (int a = 0; a < dim; ++a)
            for (int b = a; b < dim; ++b, ++k) {
                P[k] = xi[a] * xi[b];
                for (int g = 0; g < dim; ++g) dP[g][k] = (g == a ? xi[b] : 0.0) + (g == b ? xi[a] : 0.0);
            }
    return k;
}

/* (Sec. 2.2, Eq. rk-matrix and its gradient) RK functions at the point xe from
 * the candidate list cand[ncand].
 * Supported j: |xe - x_j| < R_j.  Writes idx[ns], U[ns], dU[ns*dim]; returns
 * ns, or ORC_ERR_SINGULAR if the moment matrix cannot be inverted.
 *   M = sum_j V_j W_j P_j P_j^T,   C = M^{-1} e_1
 *   d_g M = sum_j V_j [(d_g P_j P_j^T + P_j d_g P_j^T) W_j + P_j P_j^T d_g W_j]
 *   d_g C = -M^{-1} (d_g M) C
 *   U_j = W_j P_j^T C,  d_g U_j = W_j (d_g P_j^T C + P_j^T d_g C) + P_j^T C d_g W_j
 * with d_g P = (d P / d xi_g) / s. */
static int rk_eval(int dim, int order, const double *xe, double s, int ncand, const int32_t *cand,
                   const double *x, const double *R, const double *V, int32_t *idx, double *U,
                   double *dU)
{
    /* per-call work arrays kept in static storage (about 330 KB): the oracle is
     * single-threaded (process pools start separate processes), so one copy serves */
    static double W[1024], dW[1024][3], P[1024][10], dPa[1024][3][10];
    double M[100] = {0}, dM[3][100] = {{0}};
    int ns = 0, np = 1;
    if (order < 0 || order > 2) return ORC_ERR_ARG;
    for (int c = 0; c < ncand; ++c) {
        int32_t j = cand[c];
        double d[3] = {0, 0, 0}, r2 = 0.0;
        for (int k = 0; k < dim; ++k) { d[k] = xe[k] - x[(int64_t)j * dim + k]; r2 += d[k] * d[k]; }
        double r = sqrt(r2);
        if (!(r < R[j])) continue;
        if (ns >= 1024) return ORC_ERR_CAP;
        double h = 0.5 * R[j];
        double chi = r / h;
        idx[ns] = j;
        W[ns] = kernel_w(chi);
        double g = (r > 0.0) ? kernel_dw(chi) / (r * h) : 0.0;
        for (int k = 0; k < dim; ++k) dW[ns][k] = g * d[k];
        double xi[3] = {d[0] / s, d[1] / s, d[2] / s};
        np = rk_basis(dim, order, xi, P[ns], dPa[ns]);
        for (int gg = 0; gg < dim; ++gg)
            for (int k = 0; k < np; ++k) dPa[ns][gg][k] /= s;   /* d/dx = (d/dxi) / s */
        ++ns;
    }
    if (ns == 0) return ORC_ERR_SINGULAR;
    for (int a = 0; a < ns; ++a) {
        double v = V[idx[a]];
        for (int r = 0; r < np; ++r)
            for (int c = 0; c < np; ++c) {
                M[r * np + c] += v * W[a] * P[a][r] * P[a][c];
                for (int g = 0; g < dim; ++g)
                    dM[g][r * np + c] += v * ((dPa[a][g][r] * P[a][c] + P[a][r] * dPa[a][g][c]) * W[a] +
                                              P[a][r] * P[a][c] * dW[a][g]);
            }
    }
    double A[100], C[10];
    memcpy(A, M, sizeof(A));
    for (int r = 0; r < np; ++r) C[r] = (r == 0) ? 1.0 : 0.0;
    if (dense_solve(np, A, C)) return ORC_ERR_SINGULAR;
    double dC[3][10];
    for (int g = 0; g < dim; ++g) {
        for (int r = 0; r < np; ++r) {
            double t = 0.0;
            for (int c = 0; c < np; ++c) t += dM[g][r * np + c] * C[c];
            dC[g][r] = -t;
        }
        memcpy(A, M, sizeof(A));
        if (dense_solve(np, A, dC[g])) return ORC_ERR_SINGULAR;
    }
    for (int a = 0; a < ns; ++a) {
        double PC = 0.0;
        for (int r = 0; r < np; ++r) PC += P[a][r] * C[r];
        U[a] = W[a] * PC;
        for (int g = 0; g < dim; ++g) {
            double dPC = 0.0, PdC = 0.0;
            for (int r = 0; r < np; ++r) {
                dPC += dPa[a][g][r] * C[r];
                PdC += P[a][r] * dC[g][r];
            }
            dU[a * dim + g] = W[a] * (dPC + PdC) + PC * dW[a][g];
        }
    }
    return ns;
}

/* (Sec. 2.2) RK functions at npts points; the candidates of point p are the overlap row of
 * owner[p] and the basis scale is h_owner = R_owner / 2.  CSR output: sptr[npts+1],
 * sidx, U, dU[*dim].  Pass sidx == NULL to count only.  Returns total entries or
 * a negative error. */
int64_t orc_rk_at_points(int dim, int order, int64_t n, const double *x, const double *R, const double *V,
                         const int64_t *rowptr, const int32_t *col, int64_t npts,
                         const double *pts, const int32_t *owner, int64_t *sptr, int32_t *sidx,
                         double *U, double *dU)
{
    int32_t idx[1024];
    double u[1024], du[3 * 1024];
    sptr[0] = 0;
    for (int64_t p = 0; p < npts; ++p) {
        int32_t o = owner[p];
        int ns = rk_eval(dim, order, pts + p * dim, 0.5 * R[o], (int)(rowptr[o + 1] - rowptr[o]),
                         col + rowptr[o], x, R, V, idx, u, du);
        if (ns < 0) return ns;
        if (sidx) {
            for (int a = 0; a < ns; ++a) {
                sidx[sptr[p] + a] = idx[a];
                U[sptr[p] + a] = u[a];
                for (int g = 0; g < dim; ++g) dU[(sptr[p] + a) * dim + g] = du[a * dim + g];
            }
        }
        sptr[p + 1] = sptr[p] + ns;
    }
    (void)n;
    return sptr[npts];
}

/* ======================================================================
 * F. Integration of the bilinear and linear forms (Alg. 1 with the forms of
 * the SUPG weak transport equation, Sec. 4.1).  Test function U_i (row),
 * trial function N_j = V_j U_j (column).  Matrices (each nnz long, in this
 * order in `mats`):
 *   M0   <U_i, N_j>            Mt  <U_i, st N_j>          Ms  <U_i, ss N_j>
 *   G^a  <d_a U_i, N_j>        Gt^a <d_a U_i, st N_j>     Gs^a <d_a U_i, ss N_j>
 *   K^ab <d_a U_i, d_b N_j>  (a-major, dim*dim arrays)
 *   S_f  (U_i, N_j) on domain face f (2*dim arrays)
 * Vectors (each n long, in `vecs`):
 *   Q0 <U_i, q>,  Q^a <d_a U_i, q>,  B_f (U_i, 1) on face f.
 * sigma_t, sigma_s, q are given per volume quadrature point (in the order of
 * orc_volume_qps_2d / orc_volume_qps_3d).  Returns 0 or a negative error.
 * ====================================================================== */
static int64_t find_pos(const int64_t *rowptr, const int32_t *col, int32_t a, int32_t b)
{
    int64_t lo = rowptr[a], hi = rowptr[a + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (col[mid] == b) return mid;
        if (col[mid] < b) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* (Sec. 4.1) numbers of integrated matrices and vectors; layout in section F */
int orc_n_mats(int dim) { return 3 + 3 * dim + dim * dim + 2 * dim; }
int orc_n_vecs(int dim) { return 1 + dim + 2 * dim; }

int orc_assemble(int dim, int order, int64_t n, const double *x, const double *R, const double *V,
                 const int64_t *rowptr, const int32_t *col, int64_t nvq, const double *xq,
                 const double *wq, const int32_t *qowner, const double *sig_t_q,
                 const double *sig_s_q, const double *q_q, int64_t nbq, const double *xb,
                 const double *wb, const int32_t *bface, const int32_t *bowner, double *mats,
                 double *vecs)
{
    if (dim != 2 && dim != 3) return ORC_ERR_ARG;
    const int64_t nnz = rowptr[n];
    const int nm = orc_n_mats(dim), nvv = orc_n_vecs(dim);
    memset(mats, 0, sizeof(double) * (size_t)nm * nnz);
    memset(vecs, 0, sizeof(double) * (size_t)nvv * n);
    double *M0 = mats, *Mt = mats + nnz, *Ms = mats + 2 * nnz;
    double *G = mats + 3 * nnz, *Gt = G + dim * nnz, *Gs = Gt + dim * nnz;
    double *K = Gs + dim * nnz, *S = K + dim * dim * nnz;
    double *Q0 = vecs, *Qa = vecs + n, *B = Qa + dim * n;
    int32_t idx[1024];
    double U[1024], dU[3 * 1024];
    for (int64_t p = 0; p < nvq; ++p) {
        int32_t o = qowner[p];
        int ns = rk_eval(dim, order, xq + p * dim, 0.5 * R[o], (int)(rowptr[o + 1] - rowptr[o]),
                         col + rowptr[o], x, R, V, idx, U, dU);
        if (ns < 0) return ns;
        double w = wq[p], st = sig_t_q[p], ss = sig_s_q[p], qv = q_q[p];
        for (int a = 0; a < ns; ++a) {
            int32_t i = idx[a];
            Q0[i] += w * qv * U[a];
            for (int g = 0; g < dim; ++g) Qa[g * n + i] += w * qv * dU[a * dim + g];
            for (int b = 0; b < ns; ++b) {
                int32_t j = idx[b];
                int64_t pos = find_pos(rowptr, col, i, j);
                if (pos < 0) return ORC_ERR_ARG; /* support pair outside the overlap pattern */
                double Nj = V[j] * U[b];
                M0[pos] += w * U[a] * Nj;
                Mt[pos] += w * st * U[a] * Nj;
                Ms[pos] += w * ss * U[a] * Nj;
                for (int g = 0; g < dim; ++g) {
                    double dUi = dU[a * dim + g];
                    G[g * nnz + pos] += w * dUi * Nj;
                    Gt[g * nnz + pos] += w * st * dUi * Nj;
                    Gs[g * nnz + pos] += w * ss * dUi * Nj;
                    for (int e = 0; e < dim; ++e)
                        K[(g * dim + e) * nnz + pos] += w * dUi * V[j] * dU[b * dim + e];
                }
            }
        }
    }
    for (int64_t p = 0; p < nbq; ++p) {
        int32_t o = bowner[p];
        int ns = rk_eval(dim, order, xb + p * dim, 0.5 * R[o], (int)(rowptr[o + 1] - rowptr[o]),
                         col + rowptr[o], x, R, V, idx, U, dU);
        if (ns < 0) return ns;
        int f = bface[p];
        double w = wb[p];
        for (int a = 0; a < ns; ++a) {
            int32_t i = idx[a];
            B[f * n + i] += w * U[a];
            for (int b = 0; b < ns; ++b) {
                int32_t j = idx[b];
                int64_t pos = find_pos(rowptr, col, i, j);
                if (pos < 0) return ORC_ERR_ARG;
                S[f * nnz + pos] += w * U[a] * V[j] * U[b];
            }
        }
    }
    return ORC_OK;
}
