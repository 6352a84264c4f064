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
//   k_build_*     the self block of Eq. prec for unit columns with ubar = 0,
//                 column-major, as GEMM-shaped products (see "block build").
//   k_lu / k_lu_solve  batched LU with partial pivoting and its triangular
//                 solves (the preconditioner apply, Sec. 3.3).
//   k_update      V, T at the nodes and X <- X + dt V.
//
// Unknowns of fiber m at unk_ptr[m]: [c_x, c_y, c_z, d] (N each), V_a = Phi_V c_a
// with Phi_V = [I^4 T_0..I^4 T_{N-5}, T_0..T_3], T = Phi_T d with
// Phi_T = [I^2 T_0..I^2 T_{N-3}, T_0, T_1].  Rows of fiber m at unk_ptr[m]:
// for a = 0..2: N-4 velocity rows, V_a''(+1), V_a''(-1), V_a'''(+1), V_a'''(-1);
// then N-2 tension rows, T(+1), T(-1).  A minus end attached to the rigid body
// (Sec. 2.3, Eqs. BC2-1, BC2-2, BC2-T) replaces V_a'''(-1) by V_a(-1) (its
// value U + Omega x r enters through the coupling rows), for a clamped end
// V_a''(-1) by g V_a'(-1) (= Omega x X_s), and T(-1) by X_s(-1) . w(-1), the
// tangential velocity expression at the end node.
#include <cmath>

#include <cuda_bf16.h>

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
                         int nb, bool rhs, double *out, int64_t ostride, const double *wv = nullptr)
{
    const int N = fb.N;
    const double *Vy = fb.M_(fb.lay.Vy), *V2 = fb.M_(fb.lay.V2), *V3 = fb.M_(fb.lay.V3),
                 *Py = fb.M_(fb.lay.Py), *Dz = fb.M_(fb.lay.Dz), *Tn = fb.M_(fb.lay.Tn);
    const double *tz = F.tz + 3 * fb.z0;
    const double *bc = F.bc + 12 * fb.m;
    const int att = F.attach ? F.attach[fb.m] : FS_END_FREE;
    const double *Vn = fb.M_(fb.lay.Vn), *V1 = fb.M_(fb.lay.V1);
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
                if (wv)   // velocity-row-only nodal field (the growth term)
                    for (int j = 0; j < N; ++j) s += Py[i * N + j] * wv[3 * j + a];
                val = s;
            } else if (i < N - 2) {
                const int rr = i - (N - 4);
                double s = 0.0;
                if (rr == 1 && att == FS_END_CLAMPED) {   // g V_a'(-1)
                    for (int j = 0; j < N; ++j) s += V1[N + j] * ca[j];
                    val = fb.g * s;
                } else {
                    for (int j = 0; j < N; ++j) s += V2[rr * N + j] * ca[j];
                    val = s + (rhs ? bc[rr * 3 + a] : 0.0);
                }
            } else {
                const int rr = i - (N - 2);
                double s = 0.0;
                if (rr == 1 && att != FS_END_FREE) {      // V_a(-1)
                    for (int j = 0; j < N; ++j) s += Vn[(N - 1) * N + j] * ca[j];
                    val = s;
                } else {
                    for (int j = 0; j < N; ++j) s += V3[rr * N + j] * ca[j];
                    val = s + (rhs ? bc[(2 + rr) * 3 + a] : 0.0);
                }
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
            } else if (i == N - 1 && att != FS_END_FREE) {   // X_s(-1) . w(-1)
                const double *te = F.t + 3 * (fb.n0 + N - 1);
                const double *we = wc + 3 * (N - 1);
                val = te[0] * we[0] + te[1] * we[1] + te[2] * we[2];
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
    double *us = rsm, *fs_ = us + 4 * N, *w = fs_ + 3 * N, *wv = w + 3 * N;
    for (int i = threadIdx.x; i < 4 * N; i += blockDim.x) us[i] = (u && mode == 0) ? u[fb.u0 + i] : 0.0;
    // growth (Sec. 2.4, Eq. chain-rule): the nodes sit at fixed alpha, so the
    // velocity rows carry the reparametrisation term R = (alpha + 1) k X_alpha
    // = (alpha + 1) k (L / 2) X_s.  Explicit (Eq. discrete-rhs): k = Ldot / L,
    // all of it on the right-hand side.  Implicit: k = kappa = Ldot / (L + dt
    // Ldot) on X+_alpha; its known part is this one, its dt V_alpha part sits
    // in the self block.
    const double ldot = (mode == 1 && F.Ldot) ? F.Ldot[fb.m] : 0.0;
    if (ldot != 0.0) {
        const double *al = fb.M_(fb.lay.alpha);
        const double *t = F.t + 3 * fb.n0;
        const double kl2 = (F.growth_implicit ? ldot / (fb.L + F.dt * ldot) : ldot / fb.L) * 0.5 * fb.L;
        for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) wv[i] = (al[i / 3] + 1.0) * kl2 * t[i];
    }
    if (mode == 2) {
        for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) w[i] = ubar[3 * fb.n0 + i];
    } else {
        for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) fs_[i] = f[3 * fb.n0 + i];
        __syncthreads();
        dev_selfvel(F, fb, fs_, 1, ubar, w);
    }
    __syncthreads();
    dev_rows(F, fb, us, w, 1, mode == 1, out + fb.u0, 0, ldot != 0.0 ? wv : nullptr);
}

// ------------------------------------------------------------- block build
// The self block of Eq. prec, B = Rd + Rw W with W = S F for the unit columns:
//   F  force at the nodes of each unknown (Sec. 3.2 discrete force):
//      sigma_a,j  f = -E dt g^4 (Sig column j) e_a   (one component)
//      p_a,k      f = 0
//      tension j  f = g D_alpha (T_j X_s),  T_j = column j of Tn   (three)
//   S  velocity at the nodes of a nodal force density: the local operator M
//      (Eq. main-sb-local) on the diagonal and the K_delta pair records
//      a_kl (I + rhat rhat) off it (Eq. sb-stokes-reg);
//   Rw velocity rows P_y w_a and tension rows X_s(z) . D_z w;
//   Rd the unknowns' direct rows: -V(y), the free-end rows, T at the ends.
// Three GEMM-shaped kernels with 64 x 64 output tiles, 4 x 4 FP64 register
// tiles per thread and the inner dimension staged through shared memory in
// chunks of 32: k_build_ftau (tension-column forces), k_build_w (W, with S
// generated on the fly from the pair records), k_build_rows (Rw W + Rd in the
// epilogue); k_build_direct writes the rows that do not involve w.
constexpr int kBT = 64, kBK = 32;

// S[(k,b),(l,a)] of the fiber (rows and columns component-major, b N + k).
__device__ __forceinline__ double s_entry(const FiberTable &F, const Fib &fb, int k, int b, int l, int a)
{
    if (k == l) {
        const double *ml = F.mloc + 2 * (fb.n0 + k);
        const double *t = F.t + 3 * (fb.n0 + k);
        return (a == b ? ml[0] : 0.0) + ml[1] * t[b] * t[a];
    }
    if (F.lsb) return 0.0;
    const double4_32a p = reinterpret_cast<const double4_32a *>(F.kp)[fb.kp0 + static_cast<int64_t>(k) * fb.N + l];
    const double rb = b == 0 ? p.y : (b == 1 ? p.z : p.w);
    const double ra = a == 0 ? p.y : (a == 1 ? p.z : p.w);
    return p.x * ((a == b ? 1.0 : 0.0) + rb * ra);
}

// One 64 x 64 tile of C += A B with A and B supplied element-wise by the
// callables; inner dimension K in chunks of kBK through shared memory.
// Thread (cg, rg) = (tid % 16, tid / 16) owns rows 4 rg.., columns 4 cg...
// B_KFAST: consecutive threads fetch consecutive inner indices of one B
// column (B stored column by column), else consecutive columns.
template <bool B_KFAST, class FA, class FB>
__device__ __forceinline__ void tile_gemm(int K, FA a_of, FB b_of, double (&acc)[4][4], double *sA, double *sB)
{
    const int tid = threadIdx.x, cg = tid & 15, rg = tid >> 4;
    for (int k0 = 0; k0 < K; k0 += kBK) {
        for (int idx = tid; idx < kBT * kBK; idx += 256) {
            const int r = idx / kBK, kk = idx - r * kBK;
            sA[kk * (kBT + 1) + r] = k0 + kk < K ? a_of(r, k0 + kk) : 0.0;
        }
        for (int idx = tid; idx < kBK * kBT; idx += 256) {
            int kk, cc;
            if (B_KFAST) {
                cc = idx / kBK;
                kk = idx - cc * kBK;
            } else {
                kk = idx / kBT;
                cc = idx - kk * kBT;
            }
            sB[kk * (kBT + 1) + cc] = k0 + kk < K ? b_of(k0 + kk, cc) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kBK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = sA[kk * (kBT + 1) + 4 * rg + i];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) bv[jj] = sB[kk * (kBT + 1) + 4 * cg + jj];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(av[i], bv[jj], acc[i][jj]);
        }
        __syncthreads();
    }
}

// F_tau[a][l][j] = g sum_q D1[l][q] t_{q,a} Tn[q][j]; grid (M, 3 nt^2) with
// nt = ceil(N / 64) output tiles per dimension.
__global__ void __launch_bounds__(256) k_build_ftau(FiberTable F)
{
    __shared__ double sA[kBK * (kBT + 1)], sB[kBK * (kBT + 1)];
    const Fib fb(F, blockIdx.x);
    const int N = fb.N, nt = (N + kBT - 1) / kBT;
    const int a = blockIdx.y / (nt * nt), rem = blockIdx.y - a * nt * nt;
    if (a >= 3) return;
    const int l0 = (rem / nt) * kBT, j0 = (rem % nt) * kBT;
    const double *D1 = fb.M_(fb.lay.D1), *Tn = fb.M_(fb.lay.Tn);
    const double *t = F.t + 3 * fb.n0;
    auto a_of = [&](int r, int q) -> double {
        const int l = l0 + r;
        return (l < N && q < N) ? D1[l * N + q] * t[3 * q + a] : 0.0;
    };
    auto b_of = [&](int q, int cc) -> double {
        const int j = j0 + cc;
        return (q < N && j < N) ? Tn[q * N + j] : 0.0;
    };
    double acc[4][4] = {};
    tile_gemm<false>(N, a_of, b_of, acc, sA, sB);
    const int tid = threadIdx.x, cg = tid & 15, rg = tid >> 4;
    double *out = F.ftau + fb.blk0 / 16 * 3 + static_cast<int64_t>(a) * N * N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int l = l0 + 4 * rg + i, j = j0 + 4 * cg + jj;
            if (l < N && j < N) out[l * N + j] = fb.g * acc[i][jj];
        }
}

// W = S F for the sigma and tension columns; grid (M, row tiles of 3N,
// column tiles): tiles below 3 ct_s hold the sigma columns of component
// ap = tile / ct_s, the others the tension columns.
__global__ void __launch_bounds__(256) k_build_w(FiberTable F)
{
    __shared__ double sA[kBK * (kBT + 1)], sB[kBK * (kBT + 1)];
    const Fib fb(F, blockIdx.x);
    const int N = fb.N;
    const int r0 = blockIdx.y * kBT;
    const int ct_s = (N - 4 + kBT - 1) / kBT, ct_t = (N + kBT - 1) / kBT;
    const int ct = blockIdx.z;
    if (r0 >= 3 * N || ct >= 3 * ct_s + ct_t) return;
    const bool sig = ct < 3 * ct_s;
    const int ap = sig ? ct / ct_s : 0;
    const int j0 = sig ? (ct - ap * ct_s) * kBT : (ct - 3 * ct_s) * kBT;
    const int ncol = sig ? N - 4 : N;
    const double bend = -F.E * F.dt * fb.g * fb.g * fb.g * fb.g;
    const double *Sig = fb.M_(fb.lay.Sig);
    const double *ftau = F.ftau + fb.blk0 / 16 * 3;
    double acc[4][4] = {};
    if (sig) {
        // inner l over N: S[(k,b),(l,ap)] Phi[l][j],  Phi = bend Sig
        auto a_of = [&](int r, int l) -> double {
            const int row = r0 + r;
            if (row >= 3 * N || l >= N) return 0.0;
            return s_entry(F, fb, row % N, row / N, l, ap);
        };
        auto b_of = [&](int l, int cc) -> double {
            const int jj = j0 + cc;
            return (l < N && jj < ncol) ? bend * Sig[l * N + jj] : 0.0;
        };
        tile_gemm<false>(N, a_of, b_of, acc, sA, sB);
    } else {
        // inner (a, l) over 3N: S[(k,b),(l,a)] F_tau[a][l][j]
        auto a_of = [&](int r, int q) -> double {
            const int row = r0 + r;
            if (row >= 3 * N || q >= 3 * N) return 0.0;
            return s_entry(F, fb, row % N, row / N, q % N, q / N);
        };
        auto b_of = [&](int q, int cc) -> double {
            const int jj = j0 + cc;
            return (q < 3 * N && jj < ncol) ? ftau[static_cast<int64_t>(q) * N + jj] : 0.0;
        };
        tile_gemm<false>(3 * N, a_of, b_of, acc, sA, sB);
    }
    const int tid = threadIdx.x, cg = tid & 15, rg = tid >> 4;
    double *W = F.wsc + fb.blk0 / 4 * 3;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int row = r0 + 4 * rg + i, j = j0 + 4 * cg + jj;
            if (row < 3 * N && j < ncol) {
                const int col = sig ? ap * N + j : 3 * N + j;
                W[static_cast<int64_t>(col) * 3 * N + row] = acc[i][jj];
            }
        }
}

// Rows that involve w, for all 4N columns: velocity rows (a, i < N-4):
//   P_y w_a - [col is c_a,j] V_y[i][j];  tension rows i < N-2: X_s(z_i) . D_z w.
// Grid (M, row tiles, column tiles of 4N): row tiles below 3 rt_v hold the
// velocity rows of component a = tile / rt_v (inner N), the others tension
// rows (inner 3N).
__global__ void __launch_bounds__(256) k_build_rows(FiberTable F, double *__restrict__ B)
{
    __shared__ double sA[kBK * (kBT + 1)], sB[kBK * (kBT + 1)];
    const Fib fb(F, blockIdx.x);
    const int N = fb.N, n = 4 * N;
    const int rt_v = (N - 4 + kBT - 1) / kBT, rt_t = (N - 2 + kBT - 1) / kBT;
    const int rt = blockIdx.y, c0 = blockIdx.z * kBT;
    if (rt >= 3 * rt_v + rt_t || c0 >= n) return;
    const bool vel = rt < 3 * rt_v;
    const int a = vel ? rt / rt_v : 0;
    const int i0 = vel ? (rt - a * rt_v) * kBT : (rt - 3 * rt_v) * kBT;
    const int nrow = vel ? N - 4 : N - 2;
    const double *W = F.wsc + fb.blk0 / 4 * 3;
    const double *Py = fb.M_(fb.lay.Py), *Vy = fb.M_(fb.lay.Vy), *Dz = fb.M_(fb.lay.Dz);
    const double *Vgy = fb.M_(fb.lay.Vgy);
    // growth at the new time (implicit variant only): (y + 1) kappa dt V_alpha(y),
    // kappa = Ldot / (L + dt Ldot); the explicit term has no part in the block
    const double ldot = (F.Ldot && F.growth_implicit) ? F.Ldot[fb.m] : 0.0;
    const double gdt = ldot != 0.0 ? F.dt * ldot / (fb.L + F.dt * ldot) : 0.0;
    const double *tz = F.tz + 3 * fb.z0;
    double acc[4][4] = {};
    auto b_of_w = [&](int q, int cc) -> double {   // W[col][q], q component-major
        const int col = c0 + cc;
        return col < n ? W[static_cast<int64_t>(col) * 3 * N + q] : 0.0;
    };
    if (vel) {
        auto a_of = [&](int r, int k) -> double {
            const int i = i0 + r;
            return (i < nrow && k < N) ? Py[i * N + k] : 0.0;
        };
        auto b_of = [&](int k, int cc) -> double { return b_of_w(a * N + k, cc); };
        tile_gemm<true>(N, a_of, b_of, acc, sA, sB);
    } else {
        auto a_of = [&](int r, int q) -> double {
            const int i = i0 + r;
            if (i >= nrow || q >= 3 * N) return 0.0;
            const int b = q / N, k = q - b * N;
            return tz[3 * i + b] * Dz[i * N + k];
        };
        tile_gemm<true>(3 * N, a_of, b_of_w, acc, sA, sB);
    }
    const int tid = threadIdx.x, cg = tid & 15, rg = tid >> 4;
    double *Bm = B + fb.blk0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int r = i0 + 4 * rg + i, col = c0 + 4 * cg + jj;
            if (r >= nrow || col >= n) continue;
            double v = acc[i][jj];
            int row;
            if (vel) {
                row = a * N + r;
                if (col < 3 * N && col / N == a) v += gdt * Vgy[r * N + (col - a * N)] - Vy[r * N + (col - a * N)];
            } else {
                row = 3 * N + r;
            }
            Bm[static_cast<int64_t>(col) * n + row] = v;
        }
}

// ------------------------------------------- block build on the tensor cores
// The two large products of the block build, W = S F and the w rows Rw W,
// in FP64-grade arithmetic on the bf16 tensor cores by operand splitting
// (the error-free product scheme of Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 2012, with row / column scaling):
//   * every row of the left operand X is scaled by 2^e (e: the row's largest
//     magnitude rounds below 2^e) and rounded to a 62-bit integer, written as
//     nine balanced base-128 digits x = 2^e sum_s a_s 2^-(6+7s), |a_s| <= 65;
//     the columns of the right operand Y likewise (2^f, digits b_t);
//   * every digit is an integer a bf16 holds exactly, every digit product an
//     integer FP32 holds exactly; for the products of one diagonal s + t = d
//     the sum over K <= 192 stays below 2^24 (9 x 192 x 65 x 64 < 2^23), so
//     the tensor cores' FP32 accumulation of a diagonal is exact;
//   * C = 2^(e+f) sum_{d<=8} 2^-(12+7d) acc_d: each exact acc_d is added as
//     an integer into one of two 64-bit sums (d <= 3 and d >= 4, each at its
//     relative power of 128), and the two become one FP64 value with a single
//     rounding.  The dropped diagonals d >= 9 weigh below 2^-52 of 2^(e+f);
//     entries down to 2^-62 of their row's largest keep their digits, so
//     products whose large factors sit at different k (cancelling sums of
//     small terms) stay within a few FP64 roundings of their own magnitude.
// mma.sync m16n8k16 (bf16 in, FP32 accumulate); CTA tile 64 x 32, eight warps
// of 16 x 16, every A fragment multiplied into all the diagonals it enters;
// inner dimension in chunks of 192.
constexpr int kOzDigits = 9;
constexpr int kOzKChunk = 192;

// Planes of one matrix operand: [digit][rows_p][kp] bf16 (k contiguous) and a
// per-row exponent, for `fibers` fibers of a chunk.
struct OzOperand {
    __nv_bfloat16 *d;   // [fiber][digit][rows_p][kp]
    int *e;             // [fiber][rows_p]
    int rows_p, kp;
    __device__ __nv_bfloat16 *plane(int f, int s) const
    {
        return d + ((static_cast<int64_t>(f) * kOzDigits + s) * rows_p) * kp;
    }
};

// Digits of x in the frame 2^e of its row (|x| < 2^e): nine balanced
// base-128 digits of round(x 2^(62-e)), most significant first.
__device__ __forceinline__ void oz_digits(double x, int e, float (&a)[kOzDigits])
{
    // round(x 2^(62-e)) from the bits of x (integer work only): the 53-bit
    // significand shifted by its exponent, rounded half up when bits drop
    const long long bits = __double_as_longlong(x);
    const int ex = static_cast<int>((bits >> 52) & 0x7ff);
    long long r = 0;
    if (ex > 0) {
        const long long mant = (bits & ((1LL << 52) - 1)) | (1LL << 52);
        const int sh = ex - 1075 + 62 - e;   // x 2^(62-e) = mant 2^sh
        if (sh >= 0) r = mant << sh;
        else if (sh > -54) r = (mant + (1LL << (-sh - 1))) >> (-sh);
        if (bits < 0) r = -r;
    }
#pragma unroll
    for (int s = kOzDigits - 1; s >= 1; --s) {
        int dg = static_cast<int>(r & 127);
        if (dg >= 64) dg -= 128;
        r = (r - dg) >> 7;
        a[s] = static_cast<float>(dg);
    }
    a[0] = static_cast<float>(r);
}

// One warp per row of a chunk fiber's operand X (rows < nrows, k < K, given
// by `get(f, row, k)`): the row's exponent and its digit planes; padding rows
// and columns are zero.  Grid (fibers of the chunk, ceil(rows_p / 4)), 128
// threads.
template <class Get>
__device__ __forceinline__ void oz_slice_row(const OzOperand &O, int f, int row, int nrows, int K, Get get)
{
    const int lane = threadIdx.x & 31;
    // the row's largest magnitude through bit patterns (monotone for
    // non-negative doubles; integer work, not the FP64 pipe)
    long long mb = 0;
    if (row < nrows)
        for (int k = lane; k < K; k += 32) mb = max(mb, __double_as_longlong(get(row, k)) & 0x7fffffffffffffffLL);
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    int e = 0;
    // frexp's exponent from the bits: max < 2^e (normal; a row of
    // subnormals only keeps e = 0 and rounds to zero digits)
    if (mb > 0) e = static_cast<int>(mb >> 52) - 1022;
    if (lane == 0) O.e[static_cast<int64_t>(f) * O.rows_p + row] = e;
    for (int k = lane; k < O.kp; k += 32) {
        float a[kOzDigits];
        if (row < nrows && k < K && mb > 0) {
            oz_digits(get(row, k), e, a);
        } else {
#pragma unroll
            for (int s = 0; s < kOzDigits; ++s) a[s] = 0.0f;
        }
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) O.plane(f, s)[static_cast<int64_t>(row) * O.kp + k] = __float2bfloat16_rn(a[s]);
    }
}

// S rows (left operand of W = S F): S[(k,b),(l,a)], rows b N + k, columns a N + l.
__global__ void __launch_bounds__(128) k_oz_slice_S(FiberTable F, int f0, OzOperand O)
{
    const int f = blockIdx.x, row = blockIdx.y * 4 + (threadIdx.x >> 5);
    if (row >= O.rows_p) return;
    const Fib fb(F, f0 + f);
    const int N = fb.N;
    oz_slice_row(O, f, row, 3 * N, 3 * N,
                 [&](int r, int q) { return s_entry(F, fb, r % N, r / N, q % N, q / N); });
}

// F columns (right operand of W = S F), one "row" per column c of F: sigma
// columns c = a N + j (j < N - 4): bend Sig[l][j] at q = a N + l; the p
// columns j >= N - 4 stay zero; tension columns c = 3N + j: F_tau[q][j].
__global__ void __launch_bounds__(128) k_oz_slice_F(FiberTable F, int f0, OzOperand O)
{
    const int f = blockIdx.x, col = blockIdx.y * 4 + (threadIdx.x >> 5);
    if (col >= O.rows_p) return;
    const Fib fb(F, f0 + f);
    const int N = fb.N;
    const double bend = -F.E * F.dt * fb.g * fb.g * fb.g * fb.g;
    const double *Sig = fb.M_(fb.lay.Sig);
    const double *ftau = F.ftau + fb.blk0 / 16 * 3;
    oz_slice_row(O, f, col, 4 * N, 3 * N, [&](int c, int q) -> double {
        if (c < 3 * N) {
            const int a = c / N, j = c - a * N;
            return (j < N - 4 && q / N == a) ? bend * Sig[(q - a * N) * N + j] : 0.0;
        }
        return ftau[static_cast<int64_t>(q) * N + (c - 3 * N)];
    });
}

// Rows of the w-row product: the velocity rows of component a at
// R = a vp + i (i < N - 4, vp = N - 4 rounded up to 64, so that a 64-row
// tile holds one component and needs only its N inner columns), the tension
// rows at R = 3 vp + i (i < N - 2); -1 for padding.
__device__ __forceinline__ int oz_w_row(int R, int N, bool &vel, int &a, int &i)
{
    const int vp = (N - 4 + 63) / 64 * 64;
    vel = R < 3 * vp;
    if (vel) {
        a = R / vp;
        i = R - a * vp;
        return i < N - 4 ? a * N + i : -1;
    }
    a = 0;
    i = R - 3 * vp;
    return i < N - 2 ? 3 * N + i : -1;
}

// Rw rows (left operand of the w rows, rows as oz_w_row): velocity rows
// P_y[i][k] at q = a N + k; tension rows X_s(z_i)_b D_z[i][k] at q = b N + k.
__global__ void __launch_bounds__(128) k_oz_slice_Rw(FiberTable F, int f0, OzOperand O)
{
    const int f = blockIdx.x, row = blockIdx.y * 4 + (threadIdx.x >> 5);
    if (row >= O.rows_p) return;
    const Fib fb(F, f0 + f);
    const int N = fb.N;
    const double *Py = fb.M_(fb.lay.Py), *Dz = fb.M_(fb.lay.Dz);
    const double *tz = F.tz + 3 * fb.z0;
    const int vp = (N - 4 + 63) / 64 * 64;
    oz_slice_row(O, f, row, 3 * vp + N - 2, 3 * N, [&](int R, int q) -> double {
        bool vel;
        int a, i;
        if (oz_w_row(R, N, vel, a, i) < 0) return 0.0;
        const int b = q / N, k = q - b * N;
        if (vel) return b == a ? Py[i * N + k] : 0.0;
        return tz[3 * i + b] * Dz[i * N + k];
    });
}

// W columns (right operand of the w rows): W[c][q], column-major.
__global__ void __launch_bounds__(128) k_oz_slice_W(FiberTable F, int f0, OzOperand O)
{
    const int f = blockIdx.x, col = blockIdx.y * 4 + (threadIdx.x >> 5);
    if (col >= O.rows_p) return;
    const Fib fb(F, f0 + f);
    const int N = fb.N;
    const double *W = F.wsc + fb.blk0 / 4 * 3;
    oz_slice_row(O, f, col, 4 * N, 3 * N,
                 [&](int c, int q) { return W[static_cast<int64_t>(c) * 3 * N + q]; });
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// 2^E as a double (0 below the normal range).
__device__ __forceinline__ double pow2(int E)
{
    return E < -1022 ? 0.0 : __longlong_as_double(static_cast<long long>(E + 1023) << 52);
}

// The split product's value 2^E (hi 2^-21 + lo 2^-56) from the two integer
// sums of its diagonals (hi: 0..3, lo: 4..8): hi converts exactly (|hi| <
// 2^53), lo rounds only beyond 2^53, and the FMA rounds once more.
__device__ __forceinline__ double oz_fold(long long hi, long long lo, int E)
{
    return fma(static_cast<double>(hi), pow2(E - 21), static_cast<double>(lo) * pow2(E - 56));
}

// Shared-memory staging of the digit planes: a 64-row x 32-k slab of one
// plane per operand, rows 80 bytes apart (conflict-free ldmatrix), two
// stages filled by cp.async while the other is consumed.
constexpr int kOzKs = 32, kOzLd = 40;   // k per stage, bf16 per staged row

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))));
}

// C = X Y^T-planes product of a chunk fiber: X planes (rows = output rows),
// Y planes (rows = output columns), both k-contiguous.  EPI 1: W (rows 3N,
// columns 4N) column-major into the block-build scratch; EPI 2: the w rows of
// the block (velocity rows with -V_y and the growth term, tension rows).
// Grid (fibers of the chunk, rows_p / 64, cols_p / 32), 256 threads: eight
// warps of 16 x 16.  Per k-slab of 32, all nine digit slabs of both
// operands pass through shared memory once (cp.async, two stages); per k-step
// of 16 a warp loads the nine B fragments, then each A fragment once and
// multiplies it into every diagonal it enters (9 + 9 ldmatrix for 90 mma).
// The nine diagonals accumulate in FP32, exactly, over at most kOzKChunk of
// k; each chunk's sums are added, as integers, into two 64-bit accumulators
// (diagonals 0..3 and 4..8 at their relative powers of 128), which become
// FP64 once at the end.
constexpr size_t kOzGemmSmem = size_t(2) * kOzDigits * (64 + 32) * kOzLd * sizeof(__nv_bfloat16);

template <int EPI>
__global__ void __launch_bounds__(256, 1) k_oz_gemm(FiberTable F, int f0, OzOperand X, OzOperand Y,
                                                    double *__restrict__ B)
{
    extern __shared__ __align__(128) unsigned char ozg_raw[];
    __nv_bfloat16 *sx = reinterpret_cast<__nv_bfloat16 *>(ozg_raw);   // [stage][digit][64][kOzLd]
    __nv_bfloat16 *sy = sx + 2 * kOzDigits * 64 * kOzLd;               // [stage][digit][32][kOzLd]
    const int f = blockIdx.x;
    const Fib fb(F, f0 + f);
    const int N = fb.N;
    const int K = 3 * N;
    const int vp = (N - 4 + 63) / 64 * 64;
    const int nrow = EPI == 1 ? 3 * N : 3 * vp + N - 2, ncol = 4 * N;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.z * 32;
    if (m0 >= nrow || n0 >= ncol) return;
    // inner range where the tile's operands are not zero: the sigma columns
    // of component a (W = S F) and the velocity rows of component a (w rows)
    // touch only k in [a N, a N + N)
    int k_lo = 0, k_hi = K;
    if (EPI == 1) {
        const int c1 = min(n0 + 31, ncol - 1);
        if (c1 < 3 * N) {
            k_lo = (n0 / N) * N;
            k_hi = (c1 / N + 1) * N;
        }
    } else if (m0 + 63 < 3 * vp) {
        k_lo = (m0 / vp) * N;
        k_hi = ((m0 + 63) / vp + 1) * N;
    }
    k_lo &= ~15;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
    const int wr = (warp >> 1) * 16, wc = (warp & 1) * 16;   // warp tile inside the CTA tile
    const int wm = m0 + wr, wn = n0 + wc;
    // slabs of kOzKs k each; the last may run past k_hi into zero padding
    // (planes hold kp >= K columns, zero beyond K) -- but never past kp
    const int nslab = (k_hi - k_lo + kOzKs - 1) / kOzKs;
    // 16-byte pieces: X 9 x 64 rows x 4, Y 9 x 32 rows x 4
    auto stage = [&](int buf, int k0) {
        for (int pc = tid; pc < kOzDigits * 64 * 4; pc += 256) {
            const int sd = pc >> 8, r = (pc >> 2) & 63, kk = 8 * (pc & 3);
            __nv_bfloat16 *dst = &sx[((buf * kOzDigits + sd) * 64 + r) * kOzLd + kk];
            if (k0 + kk < X.kp)
                cp_async16(dst, X.plane(f, sd) + static_cast<int64_t>(m0 + r) * X.kp + k0 + kk);
            else
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
        }
        for (int pc = tid; pc < kOzDigits * 32 * 4; pc += 256) {
            const int sd = pc >> 7, r = (pc >> 2) & 31, kk = 8 * (pc & 3);
            __nv_bfloat16 *dst = &sy[((buf * kOzDigits + sd) * 32 + r) * kOzLd + kk];
            if (k0 + kk < Y.kp)
                cp_async16(dst, Y.plane(f, sd) + static_cast<int64_t>(n0 + r) * Y.kp + k0 + kk);
            else
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0, 0, 0, 0);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    float acc[kOzDigits][2][4];
#pragma unroll
    for (int d = 0; d < kOzDigits; ++d)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int t = 0; t < 4; ++t) acc[d][j][t] = 0.0f;
    long long hi[2][4] = {}, lo[2][4] = {};
    stage(0, k_lo);
    for (int q = 0; q < nslab; ++q) {
        const int buf = q & 1;
        if (q + 1 < nslab) {
            stage(buf ^ 1, k_lo + (q + 1) * kOzKs);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        const __nv_bfloat16 *xs = sx + buf * kOzDigits * 64 * kOzLd, *ys = sy + buf * kOzDigits * 32 * kOzLd;
#pragma unroll
        for (int ks = 0; ks < kOzKs; ks += 16) {
            uint32_t bq[kOzDigits][4];
#pragma unroll
            for (int t = 0; t < kOzDigits; ++t)
                ldsm_x4(bq[t], &ys[(t * 32 + wc + (lane & 7) + 8 * (lane >> 4)) * kOzLd + ks + 8 * ((lane >> 3) & 1)]);
#pragma unroll
            for (int sd = 0; sd < kOzDigits; ++sd) {
                uint32_t a[4];
                ldsm_x4(a, &xs[(sd * 64 + wr + (lane & 15)) * kOzLd + ks + 8 * (lane >> 4)]);
#pragma unroll
                for (int t = 0; t + sd < kOzDigits; ++t) {
                    const uint32_t b0[2] = {bq[t][0], bq[t][1]}, b1[2] = {bq[t][2], bq[t][3]};
                    mma_bf16(acc[sd + t][0], a, b0);
                    mma_bf16(acc[sd + t][1], a, b1);
                }
            }
        }
        __syncthreads();   // the stage is refilled next
        if ((q + 1) % (kOzKChunk / kOzKs) == 0 || q + 1 == nslab) {
            // the chunk's exact diagonal sums into the integers
#pragma unroll
            for (int d = 0; d < kOzDigits; ++d)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const long long v = __float2int_rn(acc[d][j][t]);
                        if (d < 4) hi[j][t] += v << (7 * (3 - d));
                        else lo[j][t] += v << (7 * (8 - d));
                        acc[d][j][t] = 0.0f;
                    }
        }
    }
    // out = 2^(e_row + e_col - 12) (hi 2^-21 + lo 2^-56)
    double out[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int er = X.e[static_cast<int64_t>(f) * X.rows_p + wm + gid + 8 * (t >> 1)];
            const int ec = Y.e[static_cast<int64_t>(f) * Y.rows_p + wn + 8 * j + 2 * tig + (t & 1)];
            out[j][t] = oz_fold(hi[j][t], lo[j][t], er + ec - 12);
        }
    // epilogue
    const double *Vy = fb.M_(fb.lay.Vy), *Vgy = fb.M_(fb.lay.Vgy);
    const double ldot = (F.Ldot && F.growth_implicit) ? F.Ldot[fb.m] : 0.0;
    const double gdt = ldot != 0.0 ? F.dt * ldot / (fb.L + F.dt * ldot) : 0.0;
    const int n = 4 * N;
    double *W = F.wsc + fb.blk0 / 4 * 3;
    double *Bm = B + fb.blk0;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            {
                const int R = wm + gid + 8 * (q >> 1), col = wn + 8 * j + 2 * tig + (q & 1);
                if (R >= nrow || col >= ncol) continue;
                double v = out[j][q];
                if (EPI == 1) {
                    W[static_cast<int64_t>(col) * 3 * N + R] = v;
                } else {
                    bool vel;
                    int a, r;
                    const int row = oz_w_row(R, N, vel, a, r);
                    if (row < 0) continue;
                    if (vel && col < 3 * N && col / N == a) v += gdt * Vgy[r * N + (col - a * N)] - Vy[r * N + (col - a * N)];
                    Bm[static_cast<int64_t>(col) * n + row] = v;
                }
            }
        }
}

// Rows without the velocity rows' w: the end rows (second and third
// derivative of V_a at alpha = +1 and -1, Eq. bc-free, or the attached-end
// rows) and T(+1), T(-1) (or X_s(-1) . w(-1) of an attached end, read from
// the w columns k_build_w wrote); grid M.
__global__ void __launch_bounds__(256) k_build_direct(FiberTable F, double *__restrict__ B)
{
    const Fib fb(F, blockIdx.x);
    const int N = fb.N, n = 4 * N;
    const double *V2 = fb.M_(fb.lay.V2), *V3 = fb.M_(fb.lay.V3), *Tn = fb.M_(fb.lay.Tn);
    const double *Vn = fb.M_(fb.lay.Vn), *V1 = fb.M_(fb.lay.V1);
    const int att = F.attach ? F.attach[fb.m] : FS_END_FREE;
    const double *W = F.wsc + fb.blk0 / 4 * 3;
    const double *te = F.t + 3 * (fb.n0 + N - 1);
    double *Bm = B + fb.blk0;
    for (int idx = threadIdx.x; idx < 14 * n; idx += blockDim.x) {
        const int rr = idx / n, col = idx - rr * n;
        double v = 0.0;
        int row;
        if (rr < 12) {
            const int a = rr / 4, q = rr % 4;   // row a N + N-4 + q
            row = a * N + N - 4 + q;
            if (col < 3 * N && col / N == a) {
                const int j = col - a * N;
                if (q == 3 && att != FS_END_FREE) v = Vn[(N - 1) * N + j];
                else if (q == 1 && att == FS_END_CLAMPED) v = fb.g * V1[N + j];
                else v = q < 2 ? V2[q * N + j] : V3[(q - 2) * N + j];
            }
        } else if (rr == 13 && att != FS_END_FREE) {
            row = 4 * N - 1;
            const double *wc = W + static_cast<int64_t>(col) * 3 * N;
            v = te[0] * wc[N - 1] + te[1] * wc[2 * N - 1] + te[2] * wc[3 * N - 1];
        } else {
            const int node = rr == 12 ? 0 : N - 1;
            row = 3 * N + N - 2 + (rr - 12);
            if (col >= 3 * N) v = Tn[node * N + (col - 3 * N)];
        }
        Bm[static_cast<int64_t>(col) * n + row] = v;
    }
}

// Batched LU with partial pivoting of the column-major n x n fiber blocks
// (n = 4 N), one CTA per fiber, blocked right-looking: for each panel of BW
// columns,
//   1. factor the (n - k0) x BW panel in shared memory (pivot search, row
//      swap, scaling and rank-1 updates within the panel);
//   2. apply the panel's row swaps to the other columns;
//   3. U12 = L11^-1 A12 (unit lower triangle of the panel);
//   4. A22 -= L21 U12 in 64 x 64 tiles, 4 x 4 register tiles per thread.
// The trailing matrix is read and written once per panel instead of once per
// column; the pivots (and so the factors) are those of the column-by-column
// algorithm.  On return piv holds the composed row permutation: row i of the
// factored block is row piv[i] of the original, so the solve gathers
// y_i = b_{piv[i]}; dinv holds 1 / U_ii (the solve multiplies instead of
// dividing: a division is a multi-instruction FP64 sequence, and one lane at a
// time would pay it for the whole warp).
constexpr int kLuTC = 64;   // trailing-update tile width

template <int BW>
__global__ void __launch_bounds__(256) k_lu(FiberTable F, double *__restrict__ B, int *__restrict__ piv,
                                            double *__restrict__ dinv, int *__restrict__ status)
{
    constexpr int TC = kLuTC, UL = TC + 1;
    extern __shared__ double lsm[];
    __shared__ double rv[8];
    __shared__ int ri[8];
    __shared__ int s_piv[BW];
    __shared__ double s_inv;
    const Fib fb(F, blockIdx.x);
    const int n = 4 * fb.N;
    double *A = B + fb.blk0;
    int *pv = piv + fb.u0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double *P = lsm;                                   // panel, column-major, ld m
    double *U = lsm + static_cast<size_t>(n) * BW;     // U12 tile [BW][UL]
    int *perm = reinterpret_cast<int *>(U + BW * UL);  // [n] row permutation
    for (int i = tid; i < n; i += 256) perm[i] = i;
    for (int k0 = 0; k0 < n; k0 += BW) {
        const int kb = min(BW, n - k0), m = n - k0;
        for (int idx = tid; idx < kb * m; idx += 256) {
            const int c = idx / m, r = idx - c * m;
            P[idx] = A[static_cast<int64_t>(k0 + c) * n + k0 + r];
        }
        __syncthreads();
        // 1. the panel
        for (int j = 0; j < kb; ++j) {
            double best = -1.0;
            int bi = j;
            for (int r = j + tid; r < m; r += 256) {
                const double v = fabs(P[j * m + r]);
                if (v > best) {
                    best = v;
                    bi = r;
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
            if (lane == 0) {
                rv[wid] = best;
                ri[wid] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                double b = rv[0];
                int p = ri[0];
                for (int wv = 1; wv < 8; ++wv)
                    if (rv[wv] > b || (rv[wv] == b && ri[wv] < p)) {
                        b = rv[wv];
                        p = ri[wv];
                    }
                s_piv[j] = p;
                const double pvv = P[j * m + p];   // the pivot, row p before the exchange
                s_inv = pvv != 0.0 ? 1.0 / pvv : 0.0;
                const int t = perm[k0 + j];
                perm[k0 + j] = perm[k0 + p];
                perm[k0 + p] = t;
                if (!(b > 0.0)) atomicOr(status, DEV_ERR_NUMERIC);
            }
            __syncthreads();
            const int p = s_piv[j];
            if (p != j)
                for (int c = tid; c < kb; c += 256) {
                    const double t = P[c * m + j];
                    P[c * m + j] = P[c * m + p];
                    P[c * m + p] = t;
                }
            __syncthreads();
            const double inv = s_inv;
            for (int r = j + 1 + tid; r < m; r += 256) P[j * m + r] *= inv;
            __syncthreads();
            const int rows = m - j - 1, cols = kb - j - 1;
            for (int idx = tid; idx < rows * cols; idx += 256) {
                const int c = j + 1 + idx / rows, r = j + 1 + idx % rows;
                P[c * m + r] -= P[j * m + r] * P[c * m + j];
            }
            __syncthreads();
        }
        for (int idx = tid; idx < kb * m; idx += 256) {
            const int c = idx / m, r = idx - c * m;
            A[static_cast<int64_t>(k0 + c) * n + k0 + r] = P[idx];
        }
        // 2. the panel's swaps on the columns left and right of it
        for (int col = tid; col < n; col += 256) {
            if (col >= k0 && col < k0 + kb) continue;
            double *Ac = A + static_cast<int64_t>(col) * n + k0;
            for (int j = 0; j < kb; ++j) {
                const int p = s_piv[j];
                if (p != j) {
                    const double t = Ac[j];
                    Ac[j] = Ac[p];
                    Ac[p] = t;
                }
            }
        }
        __syncthreads();
        const int nr = n - k0 - kb;
        if (nr > 0) {
            // 3. U12 = L11^-1 A12, one column per thread
            for (int col = k0 + kb + tid; col < n; col += 256) {
                double *Ac = A + static_cast<int64_t>(col) * n + k0;   // this thread's column only
                for (int c = 0; c + 1 < kb; ++c) {
                    const double uc = Ac[c];
                    for (int r = c + 1; r < kb; ++r) Ac[r] = fma(-P[c * m + r], uc, Ac[r]);
                }
            }
            __syncthreads();
            // 4. A22 -= L21 U12
            const int cg = tid & 15, rg = tid >> 4;
            double *A22 = A + static_cast<int64_t>(k0 + kb) * n + k0 + kb;
            for (int c0 = 0; c0 < nr; c0 += TC) {
                const int tcn = min(TC, nr - c0);
                for (int idx = tid; idx < kb * TC; idx += 256) {
                    const int cc = idx / kb, kk = idx - cc * kb;
                    U[kk * UL + cc] = cc < tcn ? A[static_cast<int64_t>(k0 + kb + c0 + cc) * n + k0 + kk] : 0.0;
                }
                __syncthreads();
                for (int r0 = 0; r0 < nr; r0 += 64) {
                    const int rb = r0 + 4 * rg, cb = c0 + 4 * cg;
                    double acc[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj)
                            acc[i][jj] = (rb + i < nr && cb + jj < nr)
                                             ? A22[static_cast<int64_t>(cb + jj) * n + rb + i] : 0.0;
                    for (int kk = 0; kk < kb; ++kk) {
                        double a[4], w[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) a[i] = rb + i < nr ? P[kk * m + kb + rb + i] : 0.0;
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) w[jj] = U[kk * UL + 4 * cg + jj];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fma(-a[i], w[jj], acc[i][jj]);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj)
                            if (rb + i < nr && cb + jj < nr)
                                A22[static_cast<int64_t>(cb + jj) * n + rb + i] = acc[i][jj];
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += 256) {
        pv[i] = perm[i];
        // reciprocals of U's diagonal for the solve (a zero pivot gives 0, as
        // flagged in status above)
        const double d = A[static_cast<int64_t>(i) * n + i];
        dinv[fb.u0 + i] = d != 0.0 ? 1.0 / d : 0.0;
    }
}

// ------------------------------------------- LU with tensor-core updates
// The same factorisation (partial pivoting, right-looking, panels of
// kLuTcBW = 32 columns) as one launch per panel over a chunk of fibers:
//   k_lu_panel: the panel (pivot search, swaps, scaling, rank-1 updates) on
//     the FP64 pipe, the panel's swaps on the other columns, U12 = L11^-1 A12,
//     and the digit planes of L21 (one plane row per trailing row) and of U12
//     (one plane row per trailing column), 32 digits of k each;
//   k_lu_trail: A22 -= L21 U12 on the bf16 tensor cores by the split of the
//     block build (nine balanced base-128 digits of each row / column scaled
//     by its power of two, exact FP32 sums per diagonal for K = 32: at most
//     9 x 32 x 65 x 65 < 2^24), the diagonals summed as integers and folded
//     into FP64, then subtracted.
// The product's error is a few units of 2^-62 of (row max of L21) x (column
// max of U12): on that row-and-column scale no larger than the rounding of
// the FP64 update it replaces (entry by entry it can be, where an entry's
// large l and large u sit at different k).  The pivots are chosen by the same
// rule as k_lu from the same column values up to that rounding; piv and dinv
// as k_lu.
constexpr int kLuTcBW = 32;

// Rows of one operand's digit planes: trailing rows (or columns) of a panel,
// at most 4 N - 32, padded to 64.
__host__ __device__ inline int lu_tc_rows(int max_N) { return (4 * max_N + 63) / 64 * 64; }

// One plane row from a thread's own 32 values (k = 0..31): the row's
// exponent from the largest magnitude (bit patterns, integer work), then the
// nine digits of each value, written 8 bf16 (16 bytes) at a time.
__device__ __forceinline__ void oz_slice_regs(const OzOperand &O, int f, int row, const double (&v)[kLuTcBW])
{
    long long mb = 0;
#pragma unroll
    for (int c = 0; c < kLuTcBW; ++c) mb = max(mb, __double_as_longlong(v[c]) & 0x7fffffffffffffffLL);
    const bool nz = mb > 0;
    const int e = nz ? static_cast<int>(mb >> 52) - 1022 : 0;
    O.e[static_cast<int64_t>(f) * O.rows_p + row] = e;
#pragma unroll
    for (int g = 0; g < kLuTcBW; g += 8) {
        uint32_t w[kOzDigits][4];
#pragma unroll
        for (int h = 0; h < 8; h += 2) {
            float d0[kOzDigits], d1[kOzDigits];
            oz_digits(nz ? v[g + h] : 0.0, e, d0);
            oz_digits(nz ? v[g + h + 1] : 0.0, e, d1);
#pragma unroll
            for (int s2 = 0; s2 < kOzDigits; ++s2) {
                const __nv_bfloat162 pr = __floats2bfloat162_rn(d0[s2], d1[s2]);
                w[s2][h / 2] = *reinterpret_cast<const uint32_t *>(&pr);
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < kOzDigits; ++s2)
            *reinterpret_cast<uint4 *>(O.plane(f, s2) + static_cast<int64_t>(row) * O.kp + g) =
                make_uint4(w[s2][0], w[s2][1], w[s2][2], w[s2][3]);
    }
}

// Zero plane row (padding of the trailing tiles).
__device__ __forceinline__ void oz_zero_row(const OzOperand &O, int f, int row)
{
    O.e[static_cast<int64_t>(f) * O.rows_p + row] = 0;
#pragma unroll
    for (int s2 = 0; s2 < kOzDigits; ++s2)
#pragma unroll
        for (int g = 0; g < kLuTcBW; g += 8)
            *reinterpret_cast<uint4 *>(O.plane(f, s2) + static_cast<int64_t>(row) * O.kp + g) = make_uint4(0, 0, 0, 0);
}

// Panel k0 of every fiber of the chunk: one CTA of NT >= 4 N - k0 threads
// per fiber (64 to 512, the smallest that holds the step's largest panel),
// thread r holding row r of the panel (rows k0.. of its 32 columns) in
// registers.  Per column j: the pivot (largest |a_rj| over r >= j, lowest r
// on ties, as k_lu) by a block-wide argmax; rows j and p exchanged through
// shared memory, which also broadcasts the pivot row and its reciprocal; each
// row below scales its multiplier and updates its own entries -- two
// barriers per column, the rank-1 update in registers.  Then the panel's
// swaps on the other columns, U12, and the digit planes.  Fibers with
// 4 N <= k0 are done; a fiber's last panel writes dinv.
template <int NT>
__global__ void __launch_bounds__(NT, NT >= 256 ? 512 / NT : 4) k_lu_panel(FiberTable F, int f0, int k0, double *__restrict__ B,
                                                           int *__restrict__ piv, double *__restrict__ dinv,
                                                           int *__restrict__ status, OzOperand X, OzOperand Y)
{
    constexpr int BW = kLuTcBW, NW = NT / 32;
    __shared__ double rowp[BW + 1], rowj[BW];
    __shared__ double L11[BW][BW + 1];
    __shared__ long long s_rv[NW];
    __shared__ int s_ri[NW];
    __shared__ int s_perm[NT], s_src[NT], s_touch[2 * BW], s_nt;
    const int f = blockIdx.x;
    const Fib fb(F, f0 + f);
    const int n = 4 * fb.N;
    if (k0 >= n) return;
    double *A = B + fb.blk0;
    int *pv = piv + fb.u0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int kb = min(BW, n - k0), m = n - k0;
    const int r = tid;
    const bool own = r < m;
    double a[BW];
#pragma unroll
    for (int c = 0; c < BW; ++c) a[c] = (own && c < kb) ? A[static_cast<int64_t>(k0 + c) * n + k0 + r] : 0.0;
    if (own) {
        s_perm[r] = k0 == 0 ? r : pv[k0 + r];
        s_src[r] = r;
    }
#pragma unroll
    for (int j = 0; j < BW; ++j) {
        if (j >= kb) break;
        // |a_rj| compared through its bit pattern (monotone for non-negative
        // doubles): integer work, not the FP64 pipe
        long long v = (own && r >= j) ? (__double_as_longlong(a[j]) & 0x7fffffffffffffffLL) : -1LL;
        int bi = r;
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > v || (ov == v && oi < bi)) {
                v = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_rv[wid] = v;
            s_ri[wid] = bi;
        }
        __syncthreads();
        long long best = s_rv[0];
        int p = s_ri[0];
#pragma unroll
        for (int w = 1; w < NW; ++w)
            if (s_rv[w] > best || (s_rv[w] == best && s_ri[w] < p)) {
                best = s_rv[w];
                p = s_ri[w];
            }
        if (r == p) {
#pragma unroll
            for (int c = 0; c < BW; ++c) rowp[c] = a[c];
            rowp[BW] = a[j] != 0.0 ? 1.0 / a[j] : 0.0;
        }
        if (r == j && p != j) {
#pragma unroll
            for (int c = 0; c < BW; ++c) rowj[c] = a[c];
        }
        if (tid == 0) {
            if (best <= 0 || best >= 0x7ff0000000000000LL) atomicOr(status, DEV_ERR_NUMERIC);
            int t = s_perm[j];
            s_perm[j] = s_perm[p];
            s_perm[p] = t;
            t = s_src[j];
            s_src[j] = s_src[p];
            s_src[p] = t;
        }
        __syncthreads();
        if (r == j) {
#pragma unroll
            for (int c = 0; c < BW; ++c) a[c] = rowp[c];
        } else if (r == p) {
#pragma unroll
            for (int c = 0; c < BW; ++c) a[c] = rowj[c];
        }
        if (own && r > j) {
            const double l = a[j] * rowp[BW];
            a[j] = l;
#pragma unroll
            for (int c = j + 1; c < BW; ++c) a[c] = fma(-l, rowp[c], a[c]);
        }
    }
    __syncthreads();
    if (own) {
#pragma unroll
        for (int c = 0; c < BW; ++c)
            if (c < kb) A[static_cast<int64_t>(k0 + c) * n + k0 + r] = a[c];
        pv[k0 + r] = s_perm[r];
    }
    if (r < BW) {
#pragma unroll
        for (int c = 0; c < BW; ++c) L11[r][c] = a[c];
    }
    // the panel's swaps on the columns left and right of it, as one gather
    // per column: row i of the panel's rows takes row src[i] (the composed
    // swaps), for the at most 2 kb rows that move; whole columns per round so
    // that every read precedes the writes of its column
    if (wid == 0) {
        int cnt = 0;
        for (int base = 0; base < m; base += 32) {
            const int i = base + lane;
            const bool moved = i < m && s_src[i] != i;
            const unsigned bal = __ballot_sync(0xffffffffu, moved);
            if (moved) s_touch[cnt + __popc(bal & ((1u << lane) - 1u))] = i;
            cnt += __popc(bal);
        }
        if (lane == 0) s_nt = cnt;
    }
    __syncthreads();
    const int nt = s_nt, ncol = n - kb;
    if (nt > 0) {
        constexpr int Q = NT <= 64 ? 16 : (NT <= 128 ? 8 : 4);   // loads in flight per thread
        const int cpr = max(1, NT * Q / nt);   // whole columns per round
        for (int c0 = 0; c0 < ncol; c0 += cpr) {
            const int items = min(cpr, ncol - c0) * nt;
            double v[Q];
            int at[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int id = q * NT + tid;
                at[q] = -1;
                if (id < items) {
                    const int ci = c0 + id / nt, i = s_touch[id % nt];
                    const int col = ci < k0 ? ci : ci + kb;
                    at[q] = col * n + k0 + i;
                    v[q] = A[static_cast<int64_t>(col) * n + k0 + s_src[i]];
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (at[q] >= 0) A[at[q]] = v[q];
            __syncthreads();
        }
    }
    const int nr = m - kb;
    if (nr <= 0) {
        // the fiber's last panel: reciprocals of U's diagonal for the solve
        for (int i = tid; i < n; i += NT) {
            const double d = A[static_cast<int64_t>(i) * n + i];
            dinv[fb.u0 + i] = d != 0.0 ? 1.0 / d : 0.0;
        }
        return;
    }
    // digit planes of L21: thread r >= BW slices its own row i = r - BW;
    // padding rows up to the tiles' 64 are zero (both operands)
    if (own && r >= BW) oz_slice_regs(X, f, r - BW, a);
    const int rows = (nr + 63) / 64 * 64;   // the rows the trailing tiles read
    for (int i = nr + tid; i < rows; i += NT) {
        oz_zero_row(X, f, i);
        oz_zero_row(Y, f, i);
    }
    // U12 = L11^-1 A12 (kb == BW == 32 here): one column per thread in
    // registers, forward substitution with the unit lower triangle of L11
    // (shared memory, the same entry for all threads: broadcast; read
    // through a volatile view: one shared load per use, not 496
    // loop-invariant registers); the thread then slices its column into
    // U12's digit planes
    const volatile double(*Lv)[BW + 1] = L11;
    for (int col = k0 + BW + tid; col < n; col += NT) {
        double *Ac = A + static_cast<int64_t>(col) * n + k0;
        double u[BW];
#pragma unroll
        for (int q = 0; q < BW; q += 2) {
            const double2 t = *reinterpret_cast<const double2 *>(Ac + q);
            u[q] = t.x;
            u[q + 1] = t.y;
        }
#pragma unroll
        for (int c = 0; c + 1 < BW; ++c)
#pragma unroll
            for (int r2 = c + 1; r2 < BW; ++r2) u[r2] = fma(-Lv[r2][c], u[c], u[r2]);
#pragma unroll
        for (int q = 0; q < BW; q += 2) *reinterpret_cast<double2 *>(Ac + q) = make_double2(u[q], u[q + 1]);
        oz_slice_regs(Y, f, col - k0 - BW, u);
    }
}

// A22 -= L21 U12 for panel k0: grid (fibers of the chunk, tiles, tiles) of
// 64 x 64 trailing tiles, 256 threads (eight warps of 32 x 16), all nine
// digit slabs of both operands in shared memory (2 x 9 x 64 x 40 bf16).
constexpr size_t kLuTrailSmem = size_t(2) * kOzDigits * 64 * kOzLd * sizeof(__nv_bfloat16);

__global__ void __launch_bounds__(256, 2) k_lu_trail(FiberTable F, int f0, int k0, double *__restrict__ B,
                                                     OzOperand X, OzOperand Y)
{
    extern __shared__ __align__(128) unsigned char lts_raw[];
    __nv_bfloat16 *sx = reinterpret_cast<__nv_bfloat16 *>(lts_raw);
    __nv_bfloat16 *sy = sx + kOzDigits * 64 * kOzLd;
    const int f = blockIdx.x;
    const Fib fb(F, f0 + f);
    const int n = 4 * fb.N;
    const int nr = n - k0 - kLuTcBW;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.z * 64;
    if (nr <= 0 || m0 >= nr || n0 >= nr) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gid = lane >> 2, tig = lane & 3;
    {
        // one 16-byte piece per thread and plane: row tid >> 2, k offset 8 (tid & 3)
        const int r = tid >> 2, kk = 8 * (tid & 3);
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) {
            cp_async16(&sx[(s * 64 + r) * kOzLd + kk], X.plane(f, s) + static_cast<int64_t>(m0 + r) * X.kp + kk);
            cp_async16(&sy[(s * 64 + r) * kOzLd + kk], Y.plane(f, s) + static_cast<int64_t>(n0 + r) * Y.kp + kk);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
    }
    const int wr = (warp >> 2) * 32, wc = (warp & 3) * 16;
    long long hi[2][2][4] = {}, lo[2][2][4] = {};
    for (int d = 0; d < kOzDigits; ++d) {
        float acc[2][2][4] = {};
        for (int s = 0; s <= d; ++s) {
            const __nv_bfloat16 *xs = sx + s * 64 * kOzLd, *ys = sy + (d - s) * 64 * kOzLd;
#pragma unroll
            for (int ks = 0; ks < kLuTcBW; ks += 16) {
                uint32_t a[2][4], bq[4];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    ldsm_x4(a[i], &xs[(wr + 16 * i + (lane & 15)) * kOzLd + ks + 8 * (lane >> 4)]);
                ldsm_x4(bq, &ys[(wc + (lane & 7) + 8 * (lane >> 4)) * kOzLd + ks + 8 * ((lane >> 3) & 1)]);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t b2[2] = {bq[2 * j], bq[2 * j + 1]};
                        mma_bf16(acc[i][j], a[i], b2);
                    }
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const long long v = __float2int_rn(acc[i][j][t]);
                    if (d < 4) hi[i][j][t] += v << (7 * (3 - d));
                    else lo[i][j][t] += v << (7 * (8 - d));
                }
    }
    double *A22 = B + fb.blk0 + static_cast<int64_t>(k0 + kLuTcBW) * n + k0 + kLuTcBW;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int R = m0 + wr + 16 * i + gid + 8 * (t >> 1), C = n0 + wc + 8 * j + 2 * tig + (t & 1);
                if (R >= nr || C >= nr) continue;
                const int E = X.e[static_cast<int64_t>(f) * X.rows_p + R] + Y.e[static_cast<int64_t>(f) * Y.rows_p + C] - 12;
                A22[static_cast<int64_t>(C) * n + R] -= oz_fold(hi[i][j][t], lo[i][j][t], E);
            }
}

// x = P^-1 in with the factors of k_lu, one CTA per fiber: row permutation, then
// blocked forward (unit L) and backward (U) substitution -- one warp solves
// each BW x BW diagonal block from shared memory, all threads update the
// remaining entries with the block's columns (coalesced column reads).
template <int BW>
__global__ void __launch_bounds__(256) k_lu_solve(FiberTable F, const double *__restrict__ B,
                                                  const int *__restrict__ piv,
                                                  const double *__restrict__ dinv,
                                                  const double *__restrict__ in,
                                                  double *__restrict__ out)
{
    constexpr int DL = BW + 1;
    extern __shared__ double ssm[];
    const Fib fb(F, blockIdx.x);
    const int n = 4 * fb.N;
    const double *A = B + fb.blk0;
    double *y = ssm, *D = ssm + n;
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) y[i] = in[fb.u0 + piv[fb.u0 + i]];
    __syncthreads();
    for (int j0 = 0; j0 < n; j0 += BW) {
        const int jb = min(BW, n - j0);
        for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
            const int c = idx / jb, r = idx - c * jb;
            D[c * DL + r] = A[static_cast<int64_t>(j0 + c) * n + j0 + r];
        }
        __syncthreads();
        if (tid < 32) {
            double v = tid < jb ? y[j0 + tid] : 0.0;
            for (int c = 0; c < jb; ++c) {
                const double yc = __shfl_sync(0xffffffffu, v, c);
                if (tid > c && tid < jb) v -= D[c * DL + tid] * yc;
            }
            if (tid < jb) y[j0 + tid] = v;
        }
        __syncthreads();
        for (int i = j0 + jb + tid; i < n; i += blockDim.x) {
            const double *Ai = A + static_cast<int64_t>(j0) * n + i;
            double sum = y[i];
            if (jb == BW) {   // full block: the BW column loads issued together
                double av[BW];
#pragma unroll
                for (int c = 0; c < BW; ++c) av[c] = Ai[static_cast<int64_t>(c) * n];
#pragma unroll
                for (int c = 0; c < BW; ++c) sum = fma(-av[c], y[j0 + c], sum);
            } else {
                for (int c = 0; c < jb; ++c) sum = fma(-Ai[static_cast<int64_t>(c) * n], y[j0 + c], sum);
            }
            y[i] = sum;
        }
        __syncthreads();
    }
    for (int j1 = n; j1 > 0; j1 -= BW) {
        const int j0 = max(0, j1 - BW), jb = j1 - j0;
        for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
            const int c = idx / jb, r = idx - c * jb;
            D[c * DL + r] = A[static_cast<int64_t>(j0 + c) * n + j0 + r];
        }
        __syncthreads();
        if (tid < 32) {
            double v = tid < jb ? y[j0 + tid] : 0.0;
            for (int c = jb - 1; c >= 0; --c) {
                if (tid == c) v *= dinv[fb.u0 + j0 + c];
                const double yc = __shfl_sync(0xffffffffu, v, c);
                if (tid < c) v -= D[c * DL + tid] * yc;
            }
            if (tid < jb) y[j0 + tid] = v;
        }
        __syncthreads();
        for (int i = tid; i < j0; i += blockDim.x) {
            const double *Ai = A + static_cast<int64_t>(j0) * n + i;
            double sum = y[i];
            if (jb == BW) {   // full block: the BW column loads issued together
                double av[BW];
#pragma unroll
                for (int c = 0; c < BW; ++c) av[c] = Ai[static_cast<int64_t>(c) * n];
#pragma unroll
                for (int c = 0; c < BW; ++c) sum = fma(-av[c], y[j0 + c], sum);
            } else {
                for (int c = 0; c < jb; ++c) sum = fma(-Ai[static_cast<int64_t>(c) * n], y[j0 + c], sum);
            }
            y[i] = sum;
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += blockDim.x) out[fb.u0 + i] = y[i];
}

// V, T at the nodes; X <- X + dt V; L <- L + dt Ldot (growth)
__global__ void __launch_bounds__(128) k_update(FiberTable F, const double *__restrict__ u,
                                                double *__restrict__ X, double *__restrict__ V,
                                                double *__restrict__ T, double *__restrict__ L)
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
    if (F.Ldot) {
        __syncthreads();   // every thread has read L (in fb) before it changes
        if (threadIdx.x == 0) L[fb.m] += F.dt * F.Ldot[fb.m];
    }
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
    const size_t sm = static_cast<size_t>(13 * c->max_N) * sizeof(double);
    k_rows<<<c->M, 128, sm, c->stream>>>(c->table(), u, f, ubar, out, mode);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_block_build(fs_ctx *c)
{
    if (c->M == 0) return FS_OK;
    const int N = c->max_N;
    const FiberTable T = c->table();
    const int nt = (N + kBT - 1) / kBT;
    k_build_ftau<<<dim3(c->M, 3 * nt * nt), 256, 0, c->stream>>>(T);
    FS_LAUNCH_CHECK();
    if (c->oz_chunk > 0) {
        // W = S F and the w rows on the tensor cores (split bf16 operands),
        // a chunk of fibers at a time through the digit-plane scratch
        const OzDims D(N);
        OzOperand X1{c->d_ozx, c->d_ozxe, D.r1, D.kp}, X2{c->d_ozx, c->d_ozxe, D.r2, D.kp},
            Y{c->d_ozy, c->d_ozye, D.ry, D.kp};
        FS_CUDA(cudaFuncSetAttribute(k_oz_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(kOzGemmSmem)));
        FS_CUDA(cudaFuncSetAttribute(k_oz_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(kOzGemmSmem)));
        for (int f0 = 0; f0 < c->M; f0 += c->oz_chunk) {
            const unsigned nf = static_cast<unsigned>(std::min(c->oz_chunk, c->M - f0));
            k_oz_slice_S<<<dim3(nf, D.r1 / 4), 128, 0, c->stream>>>(T, f0, X1);
            FS_LAUNCH_CHECK();
            k_oz_slice_F<<<dim3(nf, D.ry / 4), 128, 0, c->stream>>>(T, f0, Y);
            FS_LAUNCH_CHECK();
            k_oz_gemm<1><<<dim3(nf, D.r1 / 64, D.ry / 32), 256, kOzGemmSmem, c->stream>>>(T, f0, X1, Y, c->d_B);
            FS_LAUNCH_CHECK();
            k_oz_slice_Rw<<<dim3(nf, D.r2 / 4), 128, 0, c->stream>>>(T, f0, X2);
            FS_LAUNCH_CHECK();
            k_oz_slice_W<<<dim3(nf, D.ry / 4), 128, 0, c->stream>>>(T, f0, Y);
            FS_LAUNCH_CHECK();
            k_oz_gemm<2><<<dim3(nf, D.r2 / 64, D.ry / 32), 256, kOzGemmSmem, c->stream>>>(T, f0, X2, Y, c->d_B);
            FS_LAUNCH_CHECK();
        }
    } else {
        const int ct = 3 * ((N - 4 + kBT - 1) / kBT) + (N + kBT - 1) / kBT;
        k_build_w<<<dim3(c->M, (3 * N + kBT - 1) / kBT, ct), 256, 0, c->stream>>>(T);
        FS_LAUNCH_CHECK();
        const int rt = 3 * ((N - 4 + kBT - 1) / kBT) + (N - 2 + kBT - 1) / kBT;
        k_build_rows<<<dim3(c->M, rt, (4 * N + kBT - 1) / kBT), 256, 0, c->stream>>>(T, c->d_B);
        FS_LAUNCH_CHECK();
    }
    k_build_direct<<<c->M, 256, 0, c->stream>>>(T, c->d_B);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

// Panel width of the blocked LU: 32 while the panel (n x 32 doubles) and the
// trailing tile fit comfortably in shared memory, else 16.
int lu_panel(int n) { return n <= 128 ? 32 : 16; }

fs_status launch_lu_factor(fs_ctx *c)
{
    if (c->M == 0) return FS_OK;
    if (c->lu_chunk > 0) {
        // trailing updates on the tensor cores, a chunk of fibers at a time
        // through the digit-plane scratch of the block build
        const int maxn = 4 * c->max_N, rp = lu_tc_rows(c->max_N);
        const FiberTable T = c->table();
        OzOperand X{c->d_ozx, c->d_ozxe, rp, kLuTcBW}, Y{c->d_ozy, c->d_ozye, rp, kLuTcBW};
        FS_CUDA(cudaFuncSetAttribute(k_lu_trail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(kLuTrailSmem)));
        for (int f0 = 0; f0 < c->M; f0 += c->lu_chunk) {
            const unsigned nf = static_cast<unsigned>(std::min(c->lu_chunk, c->M - f0));
            for (int k0 = 0; k0 < maxn; k0 += kLuTcBW) {
                // one thread per panel row: the smallest CTA that holds the
                // largest panel of this step
                const int mrows = maxn - k0;
                if (mrows <= 64)
                    k_lu_panel<64><<<nf, 64, 0, c->stream>>>(T, f0, k0, c->d_B, c->d_piv, c->d_dinv, c->d_status, X, Y);
                else if (mrows <= 128)
                    k_lu_panel<128><<<nf, 128, 0, c->stream>>>(T, f0, k0, c->d_B, c->d_piv, c->d_dinv, c->d_status, X, Y);
                else if (mrows <= 256)
                    k_lu_panel<256><<<nf, 256, 0, c->stream>>>(T, f0, k0, c->d_B, c->d_piv, c->d_dinv, c->d_status, X, Y);
                else
                    k_lu_panel<512><<<nf, 512, 0, c->stream>>>(T, f0, k0, c->d_B, c->d_piv, c->d_dinv, c->d_status, X, Y);
                FS_LAUNCH_CHECK();
                const int nr = maxn - k0 - kLuTcBW;
                if (nr > 0) {
                    const unsigned tiles = static_cast<unsigned>((nr + 63) / 64);
                    k_lu_trail<<<dim3(nf, tiles, tiles), 256, kLuTrailSmem, c->stream>>>(T, f0, k0, c->d_B, X, Y);
                    FS_LAUNCH_CHECK();
                }
            }
        }
        return FS_OK;
    }
    const int n = 4 * c->max_N, bw = lu_panel(n);
    const size_t sm = (static_cast<size_t>(n) * bw + static_cast<size_t>(bw) * (kLuTC + 1)) * sizeof(double) +
                      static_cast<size_t>(n) * sizeof(int);
    if (bw == 32) {
        FS_CUDA(cudaFuncSetAttribute(k_lu<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
        k_lu<32><<<c->M, 256, sm, c->stream>>>(c->table(), c->d_B, c->d_piv, c->d_dinv, c->d_status);
    } else {
        FS_CUDA(cudaFuncSetAttribute(k_lu<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));
        k_lu<16><<<c->M, 256, sm, c->stream>>>(c->table(), c->d_B, c->d_piv, c->d_dinv, c->d_status);
    }
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_lu_solve(fs_ctx *c, const double *in, double *out)
{
    if (c->M == 0) return FS_OK;
    const size_t sm = (static_cast<size_t>(4 * c->max_N) + 32 * 33) * sizeof(double);
    k_lu_solve<32><<<c->M, 256, sm, c->stream>>>(c->table(), c->d_B, c->d_piv, c->d_dinv, in, out);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status launch_update(fs_ctx *c, const double *u)
{
    if (c->M == 0) return FS_OK;
    k_update<<<c->M, 128, 0, c->stream>>>(c->table(), u, c->d_X, c->d_V, c->d_T, c->d_L);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

}  // namespace fs
