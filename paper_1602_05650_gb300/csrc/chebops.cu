// Per-N operator matrices of the fiber discretisation, built on the host in
// long double and rounded (Sec. 3.1.3-3.1.4; Eq. cheb-basis):
//   * nodal values -> Chebyshev coefficients by the DCT-I formula on the
//     points alpha_k = cos(k pi/(N-1)),
//   * derivatives and integrals by the coefficient recurrences,
//   * evaluation by Clenshaw's recurrence,
//   * Clenshaw-Curtis weights as the integrals of the cardinal functions.
// Matrix meanings (row-major):
//   Vy  [(N-4) x N] : velocity basis at the first-kind points y_i
//   Vgy [(N-4) x N] : (y_i + 1) x alpha-derivative of the velocity basis at y_i
//   V2, V3 [2 x N]  : 2nd, 3rd alpha-derivative of the velocity basis at alpha = +1, -1
//   V1 [2 x N]      : 1st alpha-derivative of the velocity basis at alpha = +1, -1
//   Sig [N x N]     : 4th derivative of the velocity basis at the nodes (sigma)
//   Tn  [N x N]     : tension basis at the nodes; Vn [N x N] velocity basis at the nodes
//   Dm  [N x N]     : m-th derivative of the nodal interpolant at the nodes
//   Py  [(N-4) x N] : nodal interpolant at y;  Dz [(N-2) x N]: its derivative at z
//   G1, Gz, G2, G3, G4: D1, Dz, the alpha = +-1 rows of D2, D3, and D4 as
//                    double-double pairs for the geometry (derivatives of the
//                    node positions amplify rounding by up to ~N^8).
// Velocity basis: I^4 T_0 .. I^4 T_{N-5}, T_0..T_3; tension basis: I^2 T_0 ..
// I^2 T_{N-3}, T_0, T_1 (I^m: m-fold integral from alpha = -1).
#include <cmath>
#include <map>
#include <memory>
#include <mutex>

#include "context.h"

namespace fs {
namespace {

using R = long double;
using Vec = std::vector<R>;
const R kPiL = 3.141592653589793238462643383279502884197L;

// d/dalpha of a Chebyshev series (length n -> n, top coefficient zero).
Vec cheb_deriv(const Vec &c)
{
    const int n = static_cast<int>(c.size());
    Vec d(n, 0.0L);
    if (n < 2) return d;
    // d_{k-1} = d_{k+1} + 2 k c_k, then d_0 halved
    Vec e(n + 2, 0.0L);
    for (int k = n - 1; k >= 1; --k) e[k - 1] = e[k + 1] + 2.0L * k * c[k];
    for (int k = 0; k < n - 1; ++k) d[k] = e[k];
    d[0] *= 0.5L;
    return d;
}

// Antiderivative vanishing at alpha = -1 (length n -> n + 1).
Vec cheb_integ(const Vec &c)
{
    const int n = static_cast<int>(c.size());
    Vec C(n + 1, 0.0L);
    auto cc = [&](int k) { return (k >= 0 && k < n) ? c[k] : 0.0L; };
    if (n >= 1) C[1] = cc(0) - 0.5L * cc(2);
    for (int k = 2; k <= n; ++k) C[k] = (cc(k - 1) - cc(k + 1)) / (2.0L * k);
    R s = 0.0L;  // value at -1 of sum_{k>=1} C_k T_k is sum C_k (-1)^k
    for (int k = 1; k <= n; ++k) s += (k % 2 ? -C[k] : C[k]);
    C[0] = -s;
    return C;
}

R clenshaw(const Vec &c, R x)
{
    R b1 = 0.0L, b2 = 0.0L;
    for (int k = static_cast<int>(c.size()) - 1; k >= 1; --k) {
        const R b0 = c[k] + 2.0L * x * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return (c.empty() ? 0.0L : c[0]) + x * b1 - b2;
}

R eval_deriv(Vec c, int m, R x)
{
    for (int i = 0; i < m; ++i) c = cheb_deriv(c);
    return clenshaw(c, x);
}

Vec unit(int j, int len)
{
    Vec e(len, 0.0L);
    e[j] = 1.0L;
    return e;
}

Vec integ_m(Vec c, int m)
{
    for (int i = 0; i < m; ++i) c = cheb_integ(c);
    return c;
}

std::vector<double> compute_ops(int N);

}  // namespace

// The tables depend on N only and take long-double work to build: built once
// per N per process (every context, batch and serving request reuses them).
std::vector<double> build_ops(int N)
{
    static std::mutex mu;
    static std::map<int, std::shared_ptr<const std::vector<double>>> cache;
    std::shared_ptr<const std::vector<double>> t;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(N);
        if (it != cache.end()) t = it->second;
    }
    if (!t) {
        auto built = std::make_shared<const std::vector<double>>(compute_ops(N));
        std::lock_guard<std::mutex> lk(mu);
        t = cache.emplace(N, built).first->second;
    }
    return *t;
}

namespace {

std::vector<double> compute_ops(int N)
{
    const OpsLayout lay(N);
    std::vector<double> A(lay.total, 0.0);
    Vec a(N), y(N - 4), z(N - 2);
    for (int k = 0; k < N; ++k) a[k] = std::cos(k * kPiL / (N - 1));
    for (int i = 0; i < N - 4; ++i) y[i] = std::cos((2.0L * i + 1.0L) * kPiL / (2.0L * (N - 4)));
    for (int i = 0; i < N - 2; ++i) z[i] = std::cos((2.0L * i + 1.0L) * kPiL / (2.0L * (N - 2)));
    for (int k = 0; k < N; ++k) A[lay.alpha + k] = static_cast<double>(a[k]);

    // DCT-I: coefficients from nodal values, Cm[j][k]
    std::vector<R> Cm(static_cast<size_t>(N) * N);
    for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k) {
            R v = 2.0L / (N - 1) * std::cos(R(j) * k * kPiL / (N - 1));
            if (k == 0 || k == N - 1) v *= 0.5L;
            if (j == 0 || j == N - 1) v *= 0.5L;
            Cm[size_t(j) * N + k] = v;
        }
    // Clenshaw-Curtis: omega_k = sum_j Cm[j][k] int_{-1}^{1} T_j
    for (int k = 0; k < N; ++k) {
        R s = 0.0L;
        for (int j = 0; j < N; j += 2) s += Cm[size_t(j) * N + k] * 2.0L / (1.0L - R(j) * j);
        A[lay.omega + k] = static_cast<double>(s);
    }
    // nodal derivative / interpolation matrices: E(x) * Cm with E[i][j] = T_j^(m)(x_i)
    auto nodal = [&](const Vec &pts, int m) {
        const int P = static_cast<int>(pts.size());
        std::vector<R> E(static_cast<size_t>(P) * N), D(static_cast<size_t>(P) * N);
        for (int j = 0; j < N; ++j) {
            Vec cj = unit(j, N);
            for (int i = 0; i < m; ++i) cj = cheb_deriv(cj);
            for (int i = 0; i < P; ++i) E[size_t(i) * N + j] = clenshaw(cj, pts[i]);
        }
        for (int i = 0; i < P; ++i)
            for (int k = 0; k < N; ++k) {
                R s = 0.0L;
                for (int j = 0; j < N; ++j) s += E[size_t(i) * N + j] * Cm[size_t(j) * N + k];
                D[size_t(i) * N + k] = s;
            }
        return D;
    };
    auto put = [&](const std::vector<R> &M, int64_t off) {
        for (size_t i = 0; i < M.size(); ++i) A[off + int64_t(i)] = static_cast<double>(M[i]);
    };
    auto put_dd = [&](const std::vector<R> &M, int64_t hi, int64_t lo, int row0, int nrows) {
        for (int r = 0; r < nrows; ++r)
            for (int k = 0; k < N; ++k) {
                const R v = M[size_t(row0 + r) * N + k];
                const double h = static_cast<double>(v);
                A[hi + int64_t(r) * N + k] = h;
                A[lo + int64_t(r) * N + k] = static_cast<double>(v - static_cast<R>(h));
            }
    };
    const std::vector<R> D1 = nodal(a, 1), D2 = nodal(a, 2), D3 = nodal(a, 3), D4 = nodal(a, 4);
    const std::vector<R> Py = nodal(y, 0), Dz = nodal(z, 1);
    put(D1, lay.D1);
    put(D2, lay.D2);
    put(D3, lay.D3);
    put(D4, lay.D4);
    put(Py, lay.Py);
    put(Dz, lay.Dz);
    put_dd(D1, lay.G1h, lay.G1l, 0, N);
    put_dd(Dz, lay.Gzh, lay.Gzl, 0, N - 2);
    put_dd(D4, lay.G4h, lay.G4l, 0, N);
    // rows at alpha = +1 (node 0) and alpha = -1 (node N-1)
    std::vector<R> D2e(2 * static_cast<size_t>(N)), D3e(2 * static_cast<size_t>(N));
    for (int k = 0; k < N; ++k) {
        D2e[k] = D2[k];
        D2e[N + k] = D2[size_t(N - 1) * N + k];
        D3e[k] = D3[k];
        D3e[N + k] = D3[size_t(N - 1) * N + k];
    }
    put_dd(D2e, lay.G2h, lay.G2l, 0, 2);
    put_dd(D3e, lay.G3h, lay.G3l, 0, 2);

    // unknown bases
    std::vector<Vec> BV, BT;
    for (int j = 0; j < N - 4; ++j) BV.push_back(integ_m(unit(j, j + 1), 4));
    for (int k = 0; k < 4; ++k) BV.push_back(unit(k, k + 1));
    for (int j = 0; j < N - 2; ++j) BT.push_back(integ_m(unit(j, j + 1), 2));
    for (int k = 0; k < 2; ++k) BT.push_back(unit(k, k + 1));
    for (int j = 0; j < N; ++j) {
        for (int i = 0; i < N - 4; ++i) {
            A[lay.Vy + int64_t(i) * N + j] = static_cast<double>(clenshaw(BV[j], y[i]));
            A[lay.Vgy + int64_t(i) * N + j] = static_cast<double>((y[i] + 1.0L) * eval_deriv(BV[j], 1, y[i]));
        }
        for (int r = 0; r < 2; ++r) {
            const R x = r == 0 ? 1.0L : -1.0L;
            A[lay.V2 + int64_t(r) * N + j] = static_cast<double>(eval_deriv(BV[j], 2, x));
            A[lay.V3 + int64_t(r) * N + j] = static_cast<double>(eval_deriv(BV[j], 3, x));
            A[lay.V1 + int64_t(r) * N + j] = static_cast<double>(eval_deriv(BV[j], 1, x));
        }
        for (int k = 0; k < N; ++k) {
            // 4th derivative of I^4 T_j is T_j exactly; of T_0..T_3 it is 0
            A[lay.Sig + int64_t(k) * N + j] =
                j < N - 4 ? static_cast<double>(std::cos(R(j) * k * kPiL / (N - 1))) : 0.0;
            A[lay.Tn + int64_t(k) * N + j] = static_cast<double>(clenshaw(BT[j], a[k]));
            A[lay.Vn + int64_t(k) * N + j] = static_cast<double>(clenshaw(BV[j], a[k]));
        }
    }
    return A;
}

}  // namespace

}  // namespace fs
