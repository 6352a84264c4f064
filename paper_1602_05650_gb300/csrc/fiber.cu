// Per-fiber FP64 kernels of the implicit step (one CTA per fiber):
//
//   k_geometry    explicit geometry (Sec. 3.2): X_s = g D_alpha X at the nodes and
//                 at the tension points, f_known = f^E - E g^4 D_alpha^4 X, the
//                 free-end data of Eq. bc-free, Clenshaw-Curtis weights, the
//                 local operator M (Eq. main-sb-local) and the K_delta pair
//                 records (Eq. sb-stokes-reg), g = 2/L.
//   k_force       f = -E dt g^4 sigma + g D_alpha(T X_s) at the nodes from the
//                 unknowns (Sec. 3.2 discrete force), and W f for the far field.
//   k_rows        w = M f + K_delta[f] + ubar at the nodes and the 4N rows:
//                 velocity rows -V(y) + P_y w, free-end rows, tension rows
//                 X_s(z) . D_z w (Eq. main-inextensibility), T(+-1) = 0.
//   k_block_build the self block of Eq. prec, column by column: the same
//                 force/velocity/row map applied to unit vectors with ubar = 0,
//                 written column-major.
//   k_lu / k_lu_solve  batched LU with partial pivoting and its triangular
//                 solves (the preconditioner apply, Sec. 3.3).
//   k_update      V, T at the nodes and X <- X + dt V.
//
// Unknowns of fiber m at unk_ptr[m]: [c_x, c_y, c_z, d] (N each), V_a = Phi_V c_a
// with Phi_V = [I^4 T_0..I^4 T_{N-5}, T_0..T_3], T = Phi_T d with
// Phi_T = [I^2 T_0..I^2 T_{N-3}, T_0, T_1].  Rows of fiber m at unk_ptr[m]:
// for a = 0..2: N-4 velocity rows, V_a''(+1), V_a''(-1), V_a'''(+1), V_a'''(-1);
// then N-2 tension rows, T(+1), T(-1).
#include <cmath>

#include "context.h"

namespace fs {
namespace {

constexpr double kPi = 3.14159265358979323846;

struct Fib {
    int m, N;
    int64_t n0, u0, z0, kp0, blk0;
    const double *op;
    OpsLayout lay;
    double L, g;
    __device__ Fib(const FiberTable &F, int mm)
        : m(mm), N(F.N[mm]), n0(F.node_ptr[mm]), u0(F.unk_ptr[mm]), z0(F.z_ptr[mm]),
          kp0(F.kp_ptr[mm]), blk0(F.blk_ptr[mm]), op(F.ops + F.ops_off[mm]), lay(F.N[mm]),
          L(F.L[mm]), g(2.0 / F.L[mm])
    {
    }
    __device__ const double *M_(int64_t off) const { return op + off; }
};

// ---------------------------------------------------------------- geometry
// Double-double accumulation (Knuth's TwoSum, FMA-based TwoProduct; the
// compensated dot product of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 2005):
// derivatives of the node positions multiply O(N^2m) matrix entries by
// positions, so they are summed with ~2^-104 relative rounding and rounded to
// double once.
__device__ __forceinline__ void two_sum_d(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (sh, sl) += (dh + dl) * (xh + xl)
__device__ __forceinline__ void dd_acc(double &sh, double &sl, double dh, double dl, double xh,
                                       double xl)
{
    const double p = dh * xh;
    const double pe = fma(dh, xh, -p) + (dh * xl + dl * xh);
    double s, e;
    two_sum_d(sh, p, s, e);
    e += sl + pe;
    sh = s + e;
    sl = e - (sh - s);
}

// sum_j G[row][j] (X_j - X_0)_a with G = Gh + Gl and X_j - X_0 = Xh + Xl
__device__ __forceinline__ double dd_row(const double *__restrict__ Gh, const double *__restrict__ Gl,
                                         const double *Xh, const double *Xl, int N, int row, int a)
{
    double sh = 0.0, sl = 0.0;
    for (int j = 0; j < N; ++j)
        dd_acc(sh, sl, Gh[row * N + j], Gl[row * N + j], Xh[3 * j + a], Xl[3 * j + a]);
    return sh + sl;
}

__global__ void __launch_bounds__(128) k_geometry(FiberTable F, const double *__restrict__ X,
                                                  const double *__restrict__ fext)
{
    extern __shared__ double gsm[];
    const Fib fb(F, blockIdx.x);
    const int N = fb.N;
    double *Xh = gsm;           // [N][3] X_j - X_0, high part
    double *Xlo = gsm + 3 * N;  // [N][3] X_j - X_0, low part (exact difference)
    double *Ws = gsm + 6 * N;   // [N]
    const double *x0 = X + 3 * fb.n0;
    for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) two_sum_d(x0[i], -x0[i % 3], Xh[i], Xlo[i]);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        Ws[k] = fb.op[fb.lay.omega + k] * fb.L * 0.5;
        F.W[fb.n0 + k] = Ws[k];
    }
    __syncthreads();
    const double g = fb.g, g4 = g * g * g * g;
    const double *G1h = fb.M_(fb.lay.G1h), *G1l = fb.M_(fb.lay.G1l);
    const double *G4h = fb.M_(fb.lay.G4h), *G4l = fb.M_(fb.lay.G4l);
    for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) {
        const int k = i / 3, a = i % 3;
        F.t[3 * fb.n0 + i] = g * dd_row(G1h, G1l, Xh, Xlo, N, k, a);
        const double x4 = dd_row(G4h, G4l, Xh, Xlo, N, k, a);
        F.fknown[3 * fb.n0 + i] = (fext ? fext[3 * fb.n0 + i] : 0.0) - F.E * g4 * x4;
    }
    const double *Gzh = fb.M_(fb.lay.Gzh), *Gzl = fb.M_(fb.lay.Gzl);
    for (int i = threadIdx.x; i < 3 * (N - 2); i += blockDim.x)
        F.tz[3 * fb.z0 + i] = g * dd_row(Gzh, Gzl, Xh, Xlo, N, i / 3, i % 3);
    if (threadIdx.x < 12) {
        // which: 0 = X''(+1), 1 = X''(-1), 2 = X'''(+1), 3 = X'''(-1)
        const int which = threadIdx.x / 3, a = threadIdx.x % 3;
        const double *Gh = fb.M_(which < 2 ? fb.lay.G2h : fb.lay.G3h);
        const double *Gl = fb.M_(which < 2 ? fb.lay.G2l : fb.lay.G3l);
        F.bc[12 * fb.m + threadIdx.x] = dd_row(Gh, Gl, Xh, Xlo, N, which & 1, a) / F.dt;
    }
    __syncthreads();
    const double c8 = 1.0 / (8.0 * kPi * F.mu);
    const double clog = -log(F.eps * F.eps * 2.718281828459045235);
    const double delta = F.delta_over_L * fb.L;
    const double *alpha = fb.M_(fb.lay.alpha);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double beta = 0.0;
        if (!F.lsb) {
            const double sk = (alpha[k] + 1.0) * fb.L * 0.5;
            for (int j = 0; j < N; ++j) {
                if (j == k) continue;
                const double ds = sk - (alpha[j] + 1.0) * fb.L * 0.5;
                beta += Ws[j] * c8 / sqrt(ds * ds + delta * delta);
            }
        }
        // M f - beta (I + tt) f = cA (f + t t.f) + cB (f - t t.f)
        const double cA = clog * c8 - beta, cB = 2.0 * c8;
        F.mloc[2 * (fb.n0 + k) + 0] = cA + cB;
        F.mloc[2 * (fb.n0 + k) + 1] = cA - cB;
    }
    if (!F.lsb) {
        for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
            const int k = i / N, j = i % N;
            double4_32a rec = make_double4_32a(0.0, 0.0, 0.0, 0.0);
            if (j != k) {
                const double rx = Xh[3 * k] - Xh[3 * j], ry = Xh[3 * k + 1] - Xh[3 * j + 1],
                             rz = Xh[3 * k + 2] - Xh[3 * j + 2];
                const double r2 = rx * rx + ry * ry + rz * rz;
                const double rn = sqrt(r2);
                rec.x = Ws[j] * c8 / sqrt(r2 + delta * delta);
                rec.y = rx / rn;
                rec.z = ry / rn;
                rec.w = rz / rn;
            }
            reinterpret_cast<double4_32a *>(F.kp)[fb.kp0 + i] = rec;
        }
    }
}

// ------------------------------------------------------- shared building blocks
// sigma_a and T at the nodes for nb column vectors us[c][4N]:
//   sig[c][k][a] = sum_{j < N-4} Sig[k][j] c_a[j],  Tn_[c][k] = sum_j Tn[k][j] d[j]
__device__ void dev_sigma_T(const Fib &fb, const double *us, int nb, double *sig, double *Tv)
{
    const int N = fb.N;
    const double *Sig = fb.M_(fb.lay.Sig), *Tn = fb.M_(fb.lay.Tn);
    for (int idx = threadIdx.x; idx < nb * N * 4; idx += blockDim.x) {
        const int c = idx / (4 * N), r = idx % (4 * N), k = r / 4, comp = r % 4;
        const double *u = us + c * 4 * N;
        double s = 0.0;
        if (comp < 3) {
            const double *ca = u + comp * N;
            for (int j = 0; j < N - 4; ++j) s += Sig[k * N + j] * ca[j];
            sig[(c * N + k) * 3 + comp] = s;
        } else {
            const double *d = u + 3 * N;
            for (int j = 0; j < N; ++j) s += Tn[k * N + j] * d[j];
            Tv[c * N + k] = s;
        }
    }
}

// f[c][k][a] = -E dt g^4 sig + g sum_j D1[k][j] T[j] t[j][a]
__device__ void dev_force_from(const FiberTable &F, const Fib &fb, const double *sig,
                               const double *Tv, int nb, double *q, double *f)
{
    const int N = fb.N;
    const double *t = F.t + 3 * fb.n0;
    for (int idx = threadIdx.x; idx < nb * N * 3; idx += blockDim.x) {
        const int c = idx / (3 * N), r = idx % (3 * N);
        q[idx] = Tv[c * N + r / 3] * t[r];
    }
    __syncthreads();
    const double g = fb.g, bend = -F.E * F.dt * g * g * g * g;
    const double *D1 = fb.M_(fb.lay.D1);
    for (int idx = threadIdx.x; idx < nb * N * 3; idx += blockDim.x) {
        const int c = idx / (3 * N), r = idx % (3 * N), k = r / 3, a = r % 3;
        const double *qc = q + c * 3 * N;
        double s = 0.0;
        for (int j = 0; j < N; ++j) s += D1[k * N + j] * qc[3 * j + a];
        f[idx] = bend * sig[idx] + g * s;
    }
}

// w[c][k] = mloc(f_k) + sum_{j != k} a_kj (f_j + rhat (rhat . f_j)) [+ ubar_k]
__device__ void dev_selfvel(const FiberTable &F, const Fib &fb, const double *f, int nb,
                            const double *ubar, double *w)
{
    const int N = fb.N;
    const double *t = F.t + 3 * fb.n0;
    const double *ml = F.mloc + 2 * fb.n0;
    const double4_32a *kp = reinterpret_cast<const double4_32a *>(F.kp) + fb.kp0;
    for (int idx = threadIdx.x; idx < nb * N; idx += blockDim.x) {
        const int c = idx / N, k = idx % N;
        const double *fc = f + c * 3 * N;
        const double fx = fc[3 * k], fy = fc[3 * k + 1], fz = fc[3 * k + 2];
        const double tx = t[3 * k], ty = t[3 * k + 1], tz = t[3 * k + 2];
        const double tf = tx * fx + ty * fy + tz * fz;
        double wx = ml[2 * k] * fx + ml[2 * k + 1] * tx * tf;
        double wy = ml[2 * k] * fy + ml[2 * k + 1] * ty * tf;
        double wz = ml[2 * k] * fz + ml[2 * k + 1] * tz * tf;
        if (!F.lsb) {
            for (int j = 0; j < N; ++j) {
                const double4_32a p = kp[k * N + j];   // zero record for j == k
                const double gx = fc[3 * j], gy = fc[3 * j + 1], gz = fc[3 * j + 2];
                const double hf = p.y * gx + p.z * gy + p.w * gz;
                wx += p.x * (gx + p.y * hf);
                wy += p.x * (gy + p.z * hf);
                wz += p.x * (gz + p.w * hf);
            }
        }
        if (ubar) {
            wx += ubar[3 * (fb.n0 + k)];
            wy += ubar[3 * (fb.n0 + k) + 1];
            wz += ubar[3 * (fb.n0 + k) + 2];
        }
        w[3 * idx] = wx;
        w[3 * idx + 1] = wy;
        w[3 * idx + 2] = wz;
    }
}

// rows[c][r] for r < 4N; out[c * ostride + r] = sign * row (+ const when rhs)
__device__ void dev_rows(const FiberTable &F, const Fib &fb, const double *us, const double *w,
                         int nb, bool rhs, double *out, int64_t ostride)
{
    const int N = fb.N;
    const double *Vy = fb.M_(fb.lay.Vy), *V2 = fb.M_(fb.lay.V2), *V3 = fb.M_(fb.lay.V3),
                 *Py = fb.M_(fb.lay.Py), *Dz = fb.M_(fb.lay.Dz), *Tn = fb.M_(fb.lay.Tn);
    const double *tz = F.tz + 3 * fb.z0;
    const double *bc = F.bc + 12 * fb.m;
    for (int idx = threadIdx.x; idx < nb * 4 * N; idx += blockDim.x) {
        const int c = idx / (4 * N), r = idx % (4 * N);
        const double *u = us + c * 4 * N;
        const double *wc = w + c * 3 * N;
        double val = 0.0;
        if (r < 3 * N) {
            const int a = r / N, i = r % N;
            const double *ca = u + a * N;
            if (i < N - 4) {
                double s = 0.0;
                for (int j = 0; j < N; ++j) s += Py[i * N + j] * wc[3 * j + a] - Vy[i * N + j] * ca[j];
                val = s;
            } else if (i < N - 2) {
                const int rr = i - (N - 4);
                double s = 0.0;
                for (int j = 0; j < N; ++j) s += V2[rr * N + j] * ca[j];
                val = s + (rhs ? bc[rr * 3 + a] : 0.0);
            } else {
                const int rr = i - (N - 2);
                double s = 0.0;
                for (int j = 0; j < N; ++j) s += V3[rr * N + j] * ca[j];
                val = s + (rhs ? bc[(2 + rr) * 3 + a] : 0.0);
            }
        } else {
            const int i = r - 3 * N;
            if (i < N - 2) {
                double sx = 0.0, sy = 0.0, sz = 0.0;
                for (int j = 0; j < N; ++j) {
                    const double d = Dz[i * N + j];
                    sx += d * wc[3 * j];
                    sy += d * wc[3 * j + 1];
                    sz += d * wc[3 * j + 2];
                }
                val = tz[3 * i] * sx + tz[3 * i + 1] * sy + tz[3 * i + 2] * sz;
            } else {
                const int node = (i == N - 2) ? 0 : N - 1;   // T(+1), T(-1)
                const double *d = u + 3 * N;
                double s = 0.0;
                for (int j = 0; j < N; ++j) s += Tn[node * N + j] * d[j];
                val = s;
            }
        }
        out[c * ostride + r] = rhs ? -val : val;
    }
}

// ---------------------------------------------------------------- kernels
// f = force of u (or the known force when u is NULL), wf = W f.  add_known:
// f = the known force, wf = W (known force + force of u) -- the density whose
// far field is the coupling of the known force plus that of u.
__global__ void __launch_bounds__(128) k_force(FiberTable F, const double *__restrict__ u,
                                               double *__restrict__ f, double *__restrict__ wf, int add_known)
{
    extern __shared__ double fsm[];
    const Fib fb(F, blockIdx.x);
    const int N = fb.N;
    double *us = fsm, *sig = us + 4 * N, *Tv = sig + 3 * N, *q = Tv + N, *fl = q + 3 * N;
    if (u) {
        for (int i = threadIdx.x; i < 4 * N; i += blockDim.x) us[i] = u[fb.u0 + i];
        __syncthreads();
        dev_sigma_T(fb, us, 1, sig, Tv);
        __syncthreads();
        dev_force_from(F, fb, sig, Tv, 1, q, fl);
        __syncthreads();
    } else {
        for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) fl[i] = F.fknown[3 * fb.n0 + i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) {
        if (u && add_known) {
            const double fk = F.fknown[3 * fb.n0 + i];
            f[3 * fb.n0 + i] = fk;
            wf[3 * fb.n0 + i] = F.W[fb.n0 + i / 3] * (fk + fl[i]);
        } else {
            f[3 * fb.n0 + i] = fl[i];
            wf[3 * fb.n0 + i] = F.W[fb.n0 + i / 3] * fl[i];
        }
    }
}

// mode 0: rows of A u (self + coupling); 1: right-hand side (known force,
// free-end data, negated; u unused); 2: coupling rows only, Rw(ubar) (the
// off-diagonal part A - P of Eq. prec for the fiber blocks).
__global__ void __launch_bounds__(128) k_rows(FiberTable F, const double *__restrict__ u,
                                              const double *__restrict__ f,
                                              const double *__restrict__ ubar,
                                              double *__restrict__ out, int mode)
{
    extern __shared__ double rsm[];
    const Fib fb(F, blockIdx.x);
    const int N = fb.N;
    double *us = rsm, *fs_ = us + 4 * N, *w = fs_ + 3 * N;
    for (int i = threadIdx.x; i < 4 * N; i += blockDim.x) us[i] = (u && mode == 0) ? u[fb.u0 + i] : 0.0;
    if (mode == 2) {
        for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) w[i] = ubar[3 * fb.n0 + i];
    } else {
        for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) fs_[i] = f[3 * fb.n0 + i];
        __syncthreads();
        dev_selfvel(F, fb, fs_, 1, ubar, w);
    }
    __syncthreads();
    dev_rows(F, fb, us, w, 1, mode == 1, out + fb.u0, 0);
}

// One CTA per (fiber, chunk of nb columns): B[:, col] = rows(e_col) with ubar = 0.
// The inputs are unit vectors, so the generic force/velocity maps are
// specialised by column type:
//   sigma_a,j (j < N-4): f = -E dt g^4 T_j(alpha) e_a  (one component, no D_alpha)
//   p_a,k              : f = 0 -> w = 0 (only the direct rows)
//   tension            : T = column of Tn, f = g D_alpha(T X_s) (three components)
__global__ void __launch_bounds__(256) k_block_build(FiberTable F, double *__restrict__ B, int nb)
{
    extern __shared__ double bsm[];
    const Fib fb(F, blockIdx.x);
    const int N = fb.N, n = 4 * N;
    const int col0 = blockIdx.y * nb;
    if (col0 >= n) return;
    const int cnt = min(nb, n - col0);
    double *us = bsm, *Tv = us + nb * 4 * N, *q = Tv + nb * N, *f = q + nb * 3 * N, *w = f + nb * 3 * N;
    const double *Sig = fb.M_(fb.lay.Sig), *Tn = fb.M_(fb.lay.Tn), *D1 = fb.M_(fb.lay.D1);
    const double *t = F.t + 3 * fb.n0;
    const double g = fb.g, bend = -F.E * F.dt * g * g * g * g;
    for (int i = threadIdx.x; i < cnt * n; i += blockDim.x) {
        const int c = i / n, r = i % n;
        us[i] = (r == col0 + c) ? 1.0 : 0.0;
    }
    // tension columns: T at the nodes and the product T X_s
    for (int i = threadIdx.x; i < cnt * N; i += blockDim.x) {
        const int c = i / N, k = i % N, col = col0 + c;
        const double Tk = col >= 3 * N ? Tn[k * N + (col - 3 * N)] : 0.0;
        Tv[i] = Tk;
        q[3 * i] = Tk * t[3 * k];
        q[3 * i + 1] = Tk * t[3 * k + 1];
        q[3 * i + 2] = Tk * t[3 * k + 2];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * N * 3; i += blockDim.x) {
        const int c = i / (3 * N), r = i % (3 * N), k = r / 3, a = r % 3, col = col0 + c;
        double v = 0.0;
        if (col < 3 * N) {
            const int ca = col / N, j = col % N;
            if (ca == a && j < N - 4) v = bend * Sig[k * N + j];
        } else {
            const double *qc = q + c * 3 * N;
            double s = 0.0;
            for (int jj = 0; jj < N; ++jj) s += D1[k * N + jj] * qc[3 * jj + a];
            v = g * s;
        }
        f[i] = v;
    }
    __syncthreads();
    // w = M f + K_delta[f], skipping p columns (f = 0) and using the single
    // nonzero component of sigma columns
    const double *ml = F.mloc + 2 * fb.n0;
    const double4_32a *kp = reinterpret_cast<const double4_32a *>(F.kp) + fb.kp0;
    for (int i = threadIdx.x; i < cnt * N; i += blockDim.x) {
        const int c = i / N, k = i % N, col = col0 + c;
        const double *fc = f + c * 3 * N;
        double wx = 0.0, wy = 0.0, wz = 0.0;
        const bool pcol = col < 3 * N && (col % N) >= N - 4;
        if (!pcol) {
            const double fx = fc[3 * k], fy = fc[3 * k + 1], fz = fc[3 * k + 2];
            const double tx = t[3 * k], ty = t[3 * k + 1], tz = t[3 * k + 2];
            const double tf = tx * fx + ty * fy + tz * fz;
            wx = ml[2 * k] * fx + ml[2 * k + 1] * tx * tf;
            wy = ml[2 * k] * fy + ml[2 * k + 1] * ty * tf;
            wz = ml[2 * k] * fz + ml[2 * k + 1] * tz * tf;
            if (!F.lsb) {
                if (col < 3 * N) {
                    const int a = col / N;   // f = fa e_a
                    for (int j = 0; j < N; ++j) {
                        const double4_32a p = kp[k * N + j];
                        const double fa = fc[3 * j + a];
                        const double ha = a == 0 ? p.y : (a == 1 ? p.z : p.w);
                        const double s = p.x * ha * fa;
                        wx += s * p.y;
                        wy += s * p.z;
                        wz += s * p.w;
                        if (a == 0) wx += p.x * fa; else if (a == 1) wy += p.x * fa; else wz += p.x * fa;
                    }
                } else {
                    for (int j = 0; j < N; ++j) {
                        const double4_32a p = kp[k * N + j];
                        const double gx = fc[3 * j], gy = fc[3 * j + 1], gz = fc[3 * j + 2];
                        const double hf = p.y * gx + p.z * gy + p.w * gz;
                        wx += p.x * (gx + p.y * hf);
                        wy += p.x * (gy + p.z * hf);
                        wz += p.x * (gz + p.w * hf);
                    }
                }
            }
        }
        w[3 * i] = wx;
        w[3 * i + 1] = wy;
        w[3 * i + 2] = wz;
    }
    __syncthreads();
    dev_rows(F, fb, us, w, cnt, false, B + fb.blk0 + static_cast<int64_t>(col0) * n, n);
    (void)Tv;
}

// Batched LU with partial pivoting, column-major n x n blocks, n = 4 N.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_lu(FiberTable F, double *__restrict__ B, int *__restrict__ piv,
                                            int *__restrict__ status)
{
    extern __shared__ double lsm[];
    __shared__ double rv[8];
    __shared__ int ri[8];
    __shared__ int s_p;
    const Fib fb(F, blockIdx.x);
    const int n = 4 * fb.N;
    double *Ag = B + fb.blk0;
    double *A = SMEM ? lsm : Ag;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (SMEM) {
        for (int i = tid; i < n * n; i += nt) A[i] = Ag[i];
        __syncthreads();
    }
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < n; i += nt) {
            const double v = fabs(A[static_cast<int64_t>(k) * n + i]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if ((tid & 31) == 0) {
            rv[tid >> 5] = best;
            ri[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double b = rv[0];
            int p = ri[0];
            for (int wv = 1; wv < nt / 32; ++wv)
                if (rv[wv] > b || (rv[wv] == b && ri[wv] < p)) {
                    b = rv[wv];
                    p = ri[wv];
                }
            s_p = p;
            piv[fb.u0 + k] = p;
            if (!(b > 0.0)) atomicOr(status, DEV_ERR_NUMERIC);
        }
        __syncthreads();
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < n; j += nt) {
                const int64_t cj = static_cast<int64_t>(j) * n;
                const double tmp = A[cj + k];
                A[cj + k] = A[cj + p];
                A[cj + p] = tmp;
            }
        __syncthreads();
        const double pv = A[static_cast<int64_t>(k) * n + k];
        const double inv = pv != 0.0 ? 1.0 / pv : 0.0;
        for (int i = k + 1 + tid; i < n; i += nt) A[static_cast<int64_t>(k) * n + i] *= inv;
        __syncthreads();
        const int m2 = n - k - 1;
        for (int idx = tid; idx < m2 * m2; idx += nt) {
            const int j = k + 1 + idx / m2, i = k + 1 + idx % m2;
            A[static_cast<int64_t>(j) * n + i] -=
                A[static_cast<int64_t>(k) * n + i] * A[static_cast<int64_t>(j) * n + k];
        }
        __syncthreads();
    }
    if (SMEM)
        for (int i = tid; i < n * n; i += nt) Ag[i] = A[i];
}

__global__ void __launch_bounds__(256) k_lu_solve(FiberTable F, const double *__restrict__ B,
                                                  const int *__restrict__ piv,
                                                  const double *__restrict__ in,
                                                  double *__restrict__ out)
{
    extern __shared__ double ssm[];
    const Fib fb(F, blockIdx.x);
    const int n = 4 * fb.N;
    const double *A = B + fb.blk0;
    double *y = ssm;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < n; i += nt) y[i] = in[fb.u0 + i];
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < n; ++k) {
            const int p = piv[fb.u0 + k];
            if (p != k) {
                const double tmp = y[k];
                y[k] = y[p];
                y[p] = tmp;
            }
        }
    __syncthreads();
    for (int k = 0; k < n - 1; ++k) {
        const double yk = y[k];
        const double *col = A + static_cast<int64_t>(k) * n;
        for (int i = k + 1 + tid; i < n; i += nt) y[i] -= col[i] * yk;
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        const double *col = A + static_cast<int64_t>(k) * n;
        if (tid == 0) y[k] = col[k] != 0.0 ? y[k] / col[k] : 0.0;
        __syncthreads();
        const double yk = y[k];
        for (int i = tid; i < k; i += nt) y[i] -= col[i] * yk;
        __syncthreads();
    }
    for (int i = tid; i < n; i += nt) out[fb.u0 + i] = y[i];
}

__global__ void __launch_bounds__(128) k_update(FiberTable F, const double *__restrict__ u,
                                                double *__restrict__ X, double *__restrict__ V,
                                                double *__restrict__ T)
{
    const Fib fb(F, blockIdx.x);
    const int N = fb.N;
    const double *Vn = fb.M_(fb.lay.Vn), *Tn = fb.M_(fb.lay.Tn);
    const double *us = u + fb.u0;
    for (int idx = threadIdx.x; idx < 4 * N; idx += blockDim.x) {
        const int k = idx / 4, comp = idx % 4;
        double s = 0.0;
        if (comp < 3) {
            for (int j = 0; j < N; ++j) s += Vn[k * N + j] * us[comp * N + j];
            V[3 * (fb.n0 + k) + comp] = s;
            X[3 * (fb.n0 + k) + comp] += F.dt * s;
        } else {
            for (int j = 0; j < N; ++j) s += Tn[k * N + j] * us[3 * N + j];
            T[fb.n0 + k] = s;
        }
    }
}

int build_cols(int N)
{
    // columns per CTA so that 14 N doubles per column stay within ~96 KB
    int nb = static_cast<int>(96 * 1024 / (14 * 8 * static_cast<int64_t>(N)));
    if (nb < 1) nb = 1;
    if (nb > 16) nb = 16;
    return nb;
}

}  // namespace

fs_status launch_geometry(fs_ctx *c)
{
    if (c->M == 0) return FS_OK;
    const size_t sm = static_cast<size_t>(7 * c->max_N) * sizeof(double);
    k_geometry<<<c->M, 128, sm, c->stream>>>(c->table(), c->d_X, c->d_fext);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_force(fs_ctx *c, const double *u, double *f, double *wf, bool add_known)
{
    if (c->M == 0) return FS_OK;
    const size_t sm = static_cast<size_t>(14 * c->max_N) * sizeof(double);
    k_force<<<c->M, 128, sm, c->stream>>>(c->table(), u, f, wf, add_known ? 1 : 0);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_rows(fs_ctx *c, const double *u, const double *f, const double *ubar, double *out,
                      int mode)
{
    if (c->M == 0) return FS_OK;
    const size_t sm = static_cast<size_t>(10 * c->max_N) * sizeof(double);
    k_rows<<<c->M, 128, sm, c->stream>>>(c->table(), u, f, ubar, out, mode);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_block_build(fs_ctx *c)
{
    if (c->M == 0) return FS_OK;
    const int nb = build_cols(c->max_N);
    const size_t sm = static_cast<size_t>(14) * nb * c->max_N * sizeof(double);
    if (sm > 48 * 1024)
        FS_CUDA(cudaFuncSetAttribute(k_block_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(sm)));
    const dim3 grid(c->M, (4 * c->max_N + nb - 1) / nb);
    k_block_build<<<grid, 256, sm, c->stream>>>(c->table(), c->d_B, nb);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_lu_factor(fs_ctx *c)
{
    if (c->M == 0) return FS_OK;
    const int n = 4 * c->max_N;
    const size_t sm = static_cast<size_t>(n) * n * sizeof(double);
    if (sm <= 200 * 1024) {
        FS_CUDA(cudaFuncSetAttribute(k_lu<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(sm)));
        k_lu<true><<<c->M, 256, sm, c->stream>>>(c->table(), c->d_B, c->d_piv, c->d_status);
    } else {
        k_lu<false><<<c->M, 256, 0, c->stream>>>(c->table(), c->d_B, c->d_piv, c->d_status);
    }
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_lu_solve(fs_ctx *c, const double *in, double *out)
{
    if (c->M == 0) return FS_OK;
    const size_t sm = static_cast<size_t>(4 * c->max_N) * sizeof(double);
    k_lu_solve<<<c->M, 256, sm, c->stream>>>(c->table(), c->d_B, c->d_piv, in, out);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_update(fs_ctx *c, const double *u)
{
    if (c->M == 0) return FS_OK;
    k_update<<<c->M, 128, 0, c->stream>>>(c->table(), u, c->d_X, c->d_V, c->d_T);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

}  // namespace fs
