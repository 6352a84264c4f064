// Per-N operator matrices of the fiber discretisation, built on the host in
// FP64 (Sec. 3.1.3-3.1.4; Eq. cheb-basis):
//   * nodal values -> Chebyshev coefficients by the DCT-I formula on the
//     points alpha_k = cos(k pi/(N-1)),
//   * derivatives and integrals by the coefficient recurrences,
//   * evaluation by Clenshaw's recurrence,
//   * Clenshaw-Curtis weights as the integrals of the cardinal functions.
// Matrix meanings (row-major):
//   Vy  [(N-4) x N] : velocity basis at the first-kind points y_i
//   V2, V3 [2 x N]  : 2nd, 3rd alpha-derivative of the velocity basis at alpha = +1, -1
//   Sig [N x N]     : 4th derivative of the velocity basis at the nodes (sigma)
//   Tn  [N x N]     : tension basis at the nodes; Vn [N x N] velocity basis at the nodes
//   Dm  [N x N]     : m-th derivative of the nodal interpolant at the nodes
//   Py  [(N-4) x N] : nodal interpolant at y;  Dz [(N-2) x N]: its derivative at z
// Velocity basis: I^4 T_0 .. I^4 T_{N-5}, T_0..T_3; tension basis: I^2 T_0 ..
// I^2 T_{N-3}, T_0, T_1 (I^m: m-fold integral from alpha = -1).
#include <cmath>

#include "context.h"

namespace fs {
namespace {

using Vec = std::vector<double>;

// d/dalpha of a Chebyshev series (length n -> n, top coefficient zero).
Vec cheb_deriv(const Vec &c)
{
    const int n = static_cast<int>(c.size());
    Vec d(n, 0.0);
    if (n < 2) return d;
    // d_{k-1} = d_{k+1} + 2 k c_k, then d_0 halved
    Vec e(n + 2, 0.0);
    for (int k = n - 1; k >= 1; --k) e[k - 1] = e[k + 1] + 2.0 * k * c[k];
    for (int k = 0; k < n; ++k) d[k] = e[k];
    d[0] *= 0.5;
    d[n - 1] = 0.0;
    return d;
}

// Antiderivative vanishing at alpha = -1 (length n -> n + 1).
Vec cheb_integ(const Vec &c)
{
    const int n = static_cast<int>(c.size());
    Vec C(n + 1, 0.0);
    auto cc = [&](int k) { return (k >= 0 && k < n) ? c[k] : 0.0; };
    if (n >= 1) C[1] = cc(0) - 0.5 * cc(2);
    for (int k = 2; k <= n; ++k) C[k] = (cc(k - 1) - cc(k + 1)) / (2.0 * k);
    double s = 0.0;  // value at -1 of sum_{k>=1} C_k T_k is sum C_k (-1)^k
    for (int k = 1; k <= n; ++k) s += (k % 2 ? -C[k] : C[k]);
    C[0] = -s;
    return C;
}

double clenshaw(const Vec &c, double x)
{
    double b1 = 0.0, b2 = 0.0;
    for (int k = static_cast<int>(c.size()) - 1; k >= 1; --k) {
        const double b0 = c[k] + 2.0 * x * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return (c.empty() ? 0.0 : c[0]) + x * b1 - b2;
}

double eval_deriv(Vec c, int m, double x)
{
    for (int i = 0; i < m; ++i) c = cheb_deriv(c);
    return clenshaw(c, x);
}

Vec unit(int j, int len)
{
    Vec e(len, 0.0);
    e[j] = 1.0;
    return e;
}

Vec integ_m(Vec c, int m)
{
    for (int i = 0; i < m; ++i) c = cheb_integ(c);
    return c;
}

}  // namespace

std::vector<double> build_ops(int N)
{
    const OpsLayout lay(N);
    std::vector<double> A(lay.total, 0.0);
    const double pi = M_PI;
    Vec a(N), y(N - 4), z(N - 2);
    for (int k = 0; k < N; ++k) a[k] = std::cos(k * pi / (N - 1));
    for (int i = 0; i < N - 4; ++i) y[i] = std::cos((2.0 * i + 1.0) * pi / (2.0 * (N - 4)));
    for (int i = 0; i < N - 2; ++i) z[i] = std::cos((2.0 * i + 1.0) * pi / (2.0 * (N - 2)));
    for (int k = 0; k < N; ++k) A[lay.alpha + k] = a[k];

    // DCT-I: coefficients from nodal values, Cm[j][k]
    std::vector<double> Cm(static_cast<size_t>(N) * N);
    for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k) {
            double v = 2.0 / (N - 1) * std::cos(double(j) * k * pi / (N - 1));
            if (k == 0 || k == N - 1) v *= 0.5;
            if (j == 0 || j == N - 1) v *= 0.5;
            Cm[size_t(j) * N + k] = v;
        }
    // Clenshaw-Curtis: omega_k = sum_j Cm[j][k] int_{-1}^{1} T_j
    for (int k = 0; k < N; ++k) {
        double s = 0.0;
        for (int j = 0; j < N; j += 2) s += Cm[size_t(j) * N + k] * 2.0 / (1.0 - double(j) * j);
        A[lay.omega + k] = s;
    }
    // nodal derivative / interpolation matrices: E(x) * Cm with E[i][j] = T_j^(m)(x_i)
    auto nodal = [&](const Vec &pts, int m, int64_t off) {
        const int P = static_cast<int>(pts.size());
        std::vector<double> E(static_cast<size_t>(P) * N);
        for (int j = 0; j < N; ++j) {
            Vec cj = unit(j, N);
            for (int i = 0; i < m; ++i) cj = cheb_deriv(cj);
            for (int i = 0; i < P; ++i) E[size_t(i) * N + j] = clenshaw(cj, pts[i]);
        }
        for (int i = 0; i < P; ++i)
            for (int k = 0; k < N; ++k) {
                double s = 0.0;
                for (int j = 0; j < N; ++j) s += E[size_t(i) * N + j] * Cm[size_t(j) * N + k];
                A[off + int64_t(i) * N + k] = s;
            }
    };
    nodal(a, 1, lay.D1);
    nodal(a, 2, lay.D2);
    nodal(a, 3, lay.D3);
    nodal(a, 4, lay.D4);
    nodal(y, 0, lay.Py);
    nodal(z, 1, lay.Dz);

    // unknown bases
    std::vector<Vec> BV, BT;
    for (int j = 0; j < N - 4; ++j) BV.push_back(integ_m(unit(j, j + 1), 4));
    for (int k = 0; k < 4; ++k) BV.push_back(unit(k, k + 1));
    for (int j = 0; j < N - 2; ++j) BT.push_back(integ_m(unit(j, j + 1), 2));
    for (int k = 0; k < 2; ++k) BT.push_back(unit(k, k + 1));
    for (int j = 0; j < N; ++j) {
        for (int i = 0; i < N - 4; ++i) A[lay.Vy + int64_t(i) * N + j] = clenshaw(BV[j], y[i]);
        for (int r = 0; r < 2; ++r) {
            const double x = r == 0 ? 1.0 : -1.0;
            A[lay.V2 + int64_t(r) * N + j] = eval_deriv(BV[j], 2, x);
            A[lay.V3 + int64_t(r) * N + j] = eval_deriv(BV[j], 3, x);
        }
        for (int k = 0; k < N; ++k) {
            // 4th derivative of I^4 T_j is T_j exactly; of T_0..T_3 it is 0
            A[lay.Sig + int64_t(k) * N + j] = j < N - 4 ? std::cos(double(j) * k * pi / (N - 1)) : 0.0;
            A[lay.Tn + int64_t(k) * N + j] = clenshaw(BT[j], a[k]);
            A[lay.Vn + int64_t(k) * N + j] = clenshaw(BV[j], a[k]);
        }
    }
    return A;
}

}  // namespace fs
