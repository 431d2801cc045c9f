// Reference quadrature rules (Sec. 3.2, App. A), generated at run time.
//
// Gauss-Jacobi nodes are the roots of the Jacobi polynomial P_n^{(a,b)}, found
// by Newton iteration with deflation of the roots already found; weights from
// the closed form
//   w_k = 2^{a+b+1} G(n+a+1) G(n+b+1) / (G(n+a+b+1) n!) / ((1 - t_k^2) P_n'(t_k)^2).
// The triangle rule is the conical product of Gauss-Jacobi(1,0) (collapsed
// direction) and Gauss-Legendre, exact for total degree 2 n1d - 1; the paper's
// 2D runs use a 25-point rule, which here is n1d = 5 (degree 9).
#include <cmath>

#include "internal.h"

namespace mlpg {

// P_n^{(a,b)}(t) by the three-term recurrence.
static double jacobi_p(int n, double a, double b, double t) {
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * (a - b) + 0.5 * (a + b + 2.0) * t;
    for (int k = 2; k <= n; ++k) {
        double s = 2.0 * k + a + b;
        double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
        double c2 = (s - 1.0) * (s * (s - 2.0) * t + a * a - b * b);
        double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
        double p2 = (c2 * p1 - c3 * p0) / c1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// d/dt P_n^{(a,b)} = (n + a + b + 1)/2 * P_{n-1}^{(a+1,b+1)}
static double jacobi_dp(int n, double a, double b, double t) {
    if (n == 0) return 0.0;
    return 0.5 * (n + a + b + 1.0) * jacobi_p(n - 1, a + 1.0, b + 1.0, t);
}

void gauss_jacobi_newton(int n, double a, double b, double *t, double *w) {
    for (int k = 0; k < n; ++k) {
        // start near the k-th Chebyshev point (descending), refine with deflation
        double z = std::cos(M_PI * (k + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p = jacobi_p(n, a, b, z), dp = jacobi_dp(n, a, b, z);
            double defl = 0.0;
            for (int j = 0; j < k; ++j) defl += 1.0 / (z - t[j]);
            double step = p / (dp - p * defl);
            z -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        t[k] = z;
    }
    // ascending order
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (t[j] < t[i]) std::swap(t[i], t[j]);
    double lc = (a + b + 1.0) * std::log(2.0) + std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) -
                std::lgamma(n + a + b + 1.0) - std::lgamma(n + 1.0);
    double c = std::exp(lc);
    for (int k = 0; k < n; ++k) {
        double dp = jacobi_dp(n, a, b, t[k]);
        w[k] = c / ((1.0 - t[k] * t[k]) * dp * dp);
    }
}

void line_rule(int n, double *t, double *w) { gauss_jacobi_newton(n, 0.0, 0.0, t, w); }

void triangle_rule(int n1d, double *xi, double *w) {
    double tu[64], wu[64], tv[64], wv[64];
    gauss_jacobi_newton(n1d, 1.0, 0.0, tu, wu);
    gauss_jacobi_newton(n1d, 0.0, 0.0, tv, wv);
    for (int i = 0; i < n1d; ++i) {
        double u = 0.5 * (1.0 + tu[i]);
        for (int j = 0; j < n1d; ++j) {
            double v = 0.5 * (1.0 + tv[j]);
            int k = i * n1d + j;
            xi[2 * k] = u;
            xi[2 * k + 1] = v * (1.0 - u);
            w[k] = 0.125 * wu[i] * wv[j];
        }
    }
}

// Reference tetrahedron: collapsed coordinates u (Gauss-Jacobi(2,0)),
// v (Gauss-Jacobi(1,0)), r (Gauss-Legendre) on [0, 1]; xi = (u, v(1-u),
// r(1-u)(1-v)); the Jacobi weights carry the Jacobian (1-u)^2 (1-v).  Exact for
// total degree 2 n1d - 1 (n1d = 2: the paper's 3D order 3 with 8 points).
void tet_rule(int n1d, double *xi, double *w) {
    double tu[64], wu[64], tv[64], wv[64], tr[64], wr[64];
    gauss_jacobi_newton(n1d, 2.0, 0.0, tu, wu);
    gauss_jacobi_newton(n1d, 1.0, 0.0, tv, wv);
    gauss_jacobi_newton(n1d, 0.0, 0.0, tr, wr);
    int k = 0;
    for (int i = 0; i < n1d; ++i)
        for (int j = 0; j < n1d; ++j)
            for (int l = 0; l < n1d; ++l, ++k) {
                double u = 0.5 * (1.0 + tu[i]), v = 0.5 * (1.0 + tv[j]), r = 0.5 * (1.0 + tr[l]);
                xi[3 * k] = u;
                xi[3 * k + 1] = v * (1.0 - u);
                xi[3 * k + 2] = r * (1.0 - u) * (1.0 - v);
                w[k] = wu[i] * wv[j] * wr[l] / 64.0;
            }
}

}  // namespace mlpg
