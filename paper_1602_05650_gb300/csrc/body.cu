// The rigid body (Sec. 2.2) and the fibers attached to it (Sec. 2.3).
//
//   body_load        Stokeslet and rotlet strengths F, L of the body: the
//                    external load plus, for every attached end, the force
//                    and torque the rod's balance laws give (Eqs. f-ext,
//                    t-ext): with X+ = X + dt V at the end s = 0 (alpha = -1),
//                      F_m = -E g^3 X+_aaa + T X_s,
//                      L_m = (X - X^P) x F_m + E g^2 X_s x X+_aa.
//                    One CTA, fixed summation order (deterministic).
//   body_point_flow  G(x - X^P) F + R(x - X^P) L at any points (Eqs. oseen,
//                    rotlet), the part of the body's flow outside its double
//                    layer (Eq. main-nsb-vel).
//   body_rigid_rows  the attached-end rows' terms in U, Omega: -(U + Omega x
//                    r) in the position rows, -Omega x X_s in the clamped
//                    rows, -X_s . (U + Omega x r) in the tension row.
//   body_constraints mean of q1 - U and mean of (y - X^P) x q1 - Omega over
//                    the body's surface (Eqs. main-nsb-rgbt, main-nsb-rgbr).
//   body_update      X^P and the body's nodes move by dt U.
#include <cmath>

#include "context.h"

namespace fs {
namespace {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Sum of six values over a 256-thread CTA in a fixed order; result in
// thread 0's acc.
__device__ void block_sum6(double (&acc)[6], double (*red)[6])
{
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 6; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 6; ++k) red[threadIdx.x >> 5][k] = acc[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 6; ++k) acc[k] = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w)
            for (int k = 0; k < 6; ++k) acc[k] += red[w][k];
    }
}

__global__ void __launch_bounds__(256) k_body_load(FiberTable F, const int *__restrict__ att_list, int n_att,
                                                   const double *__restrict__ X, const double *__restrict__ u,
                                                   int mode, double *__restrict__ rb)
{
    __shared__ double red[8][6];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double cx = rb[kRbCenter], cy = rb[kRbCenter + 1], cz = rb[kRbCenter + 2];
    for (int k = threadIdx.x; k < n_att; k += blockDim.x) {
        const int m = att_list[k];
        const int N = F.N[m];
        const OpsLayout lay(N);
        const double *op = F.ops + F.ops_off[m];
        const double g = 2.0 / F.L[m];
        const int64_t n0 = F.node_ptr[m], u0 = F.unk_ptr[m];
        const double *te = F.t + 3 * (n0 + N - 1);
        const double *xe = X + 3 * (n0 + N - 1);
        double x2[3] = {0.0, 0.0, 0.0}, x3[3] = {0.0, 0.0, 0.0}, Tm = 0.0;
        if (mode != LOAD_LIN) {
            // free-end data holds X''(-1) / dt and X'''(-1) / dt
            for (int a = 0; a < 3; ++a) {
                x2[a] = F.dt * F.bc[12 * m + 3 + a];
                x3[a] = F.dt * F.bc[12 * m + 9 + a];
            }
        }
        if (mode != LOAD_KNOWN) {
            const double *V2m = op + lay.V2 + N, *V3m = op + lay.V3 + N, *Tm_ = op + lay.Tn + int64_t(N - 1) * N;
            const double *us = u + u0;
            for (int a = 0; a < 3; ++a) {
                double s2 = 0.0, s3 = 0.0;
                for (int j = 0; j < N; ++j) {
                    s2 += V2m[j] * us[a * N + j];
                    s3 += V3m[j] * us[a * N + j];
                }
                x2[a] += F.dt * s2;
                x3[a] += F.dt * s3;
            }
            for (int j = 0; j < N; ++j) Tm += Tm_[j] * us[3 * N + j];
        }
        const double g2 = g * g, g3 = g2 * g;
        double f[3], r[3] = {xe[0] - cx, xe[1] - cy, xe[2] - cz}, rf[3], tb[3];
        for (int a = 0; a < 3; ++a) f[a] = -F.E * g3 * x3[a] + Tm * te[a];
        cross3(r, f, rf);
        cross3(te, x2, tb);
        for (int a = 0; a < 3; ++a) {
            acc[a] += f[a];
            acc[3 + a] += rf[a] + F.E * g2 * tb[a];
        }
    }
    block_sum6(acc, red);
    if (threadIdx.x == 0) {
        const bool ext = mode != LOAD_LIN;
        for (int a = 0; a < 3; ++a) {
            rb[kRbF + a] = acc[a] + (ext ? rb[kRbFext + a] : 0.0);
            rb[kRbL + a] = acc[3 + a] + (ext ? rb[kRbLext + a] : 0.0);
        }
    }
}

__global__ void k_point_flow(const double *__restrict__ x, int64_t n, const double *__restrict__ rb, double c8,
                             double *__restrict__ out)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    const double r[3] = {x[3 * i] - rb[kRbCenter], x[3 * i + 1] - rb[kRbCenter + 1], x[3 * i + 2] - rb[kRbCenter + 2]};
    const double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const double h[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    const double *Fv = rb + kRbF, *Lv = rb + kRbL;
    const double hf = h[0] * Fv[0] + h[1] * Fv[1] + h[2] * Fv[2];
    double lh[3];
    cross3(Lv, h, lh);
    for (int a = 0; a < 3; ++a) out[3 * i + a] += c8 * ((Fv[a] + h[a] * hf) / rn + lh[a] / (rn * rn));
}

__global__ void k_rigid_rows(FiberTable F, const int *__restrict__ att_list, int n_att, const double *__restrict__ X,
                             const double *__restrict__ rb, const double *__restrict__ rigid, double sign,
                             double *__restrict__ rows)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_att) return;
    const int m = att_list[k];
    const int N = F.N[m];
    const int64_t n0 = F.node_ptr[m], u0 = F.unk_ptr[m];
    const double *te = F.t + 3 * (n0 + N - 1);
    const double *xe = X + 3 * (n0 + N - 1);
    const double r[3] = {xe[0] - rb[kRbCenter], xe[1] - rb[kRbCenter + 1], xe[2] - rb[kRbCenter + 2]};
    double om_r[3], om_t[3], v[3];
    cross3(rigid + 3, r, om_r);
    cross3(rigid + 3, te, om_t);
    for (int a = 0; a < 3; ++a) v[a] = rigid[a] + om_r[a];
    double *out = rows + u0;
    for (int a = 0; a < 3; ++a) out[a * N + N - 1] -= sign * v[a];
    if (F.attach[m] == FS_END_CLAMPED)
        for (int a = 0; a < 3; ++a) out[a * N + N - 3] -= sign * om_t[a];
    out[4 * N - 1] -= sign * (te[0] * v[0] + te[1] * v[1] + te[2] * v[2]);
}

__global__ void __launch_bounds__(256) k_body_constraints(const double *__restrict__ y, const double *__restrict__ w,
                                                          const double *__restrict__ q, int n,
                                                          const double *__restrict__ rb,
                                                          const double *__restrict__ rigid, double *__restrict__ out)
{
    __shared__ double red[8][6];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double r[3] = {y[3 * i] - rb[kRbCenter], y[3 * i + 1] - rb[kRbCenter + 1], y[3 * i + 2] - rb[kRbCenter + 2]};
        double rq[3];
        cross3(r, q + 3 * i, rq);
        for (int a = 0; a < 3; ++a) {
            acc[a] += w[i] * q[3 * i + a];
            acc[3 + a] += w[i] * rq[a];
        }
    }
    block_sum6(acc, red);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) out[k] = acc[k] / rb[kRbArea] - rigid[k];
}

__global__ void k_body_move(double *__restrict__ y, int n, double *__restrict__ rb, const double *__restrict__ rigid,
                            double dt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        for (int a = 0; a < 3; ++a) y[3 * i + a] += dt * rigid[a];
    if (i == 0)
        for (int a = 0; a < 3; ++a) {
            rb[kRbCenter + a] += dt * rigid[a];
            rb[kRbU + a] = rigid[a];
            rb[kRbOm + a] = rigid[3 + a];
        }
}

}  // namespace

fs_status body_load(fs_ctx *c, const double *u, int mode)
{
    if (!c->body.on) return FS_OK;
    k_body_load<<<1, 256, 0, c->stream>>>(c->table(), c->body.att_list, c->body.n_att, c->d_X, u, mode, c->body.rb);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status body_point_flow(fs_ctx *c, const double *x, int64_t n, double *out)
{
    if (!c->body.on || n == 0) return FS_OK;
    k_point_flow<<<static_cast<unsigned>((n + 127) / 128), 128, 0, c->stream>>>(x, n, c->body.rb,
                                                                              1.0 / (8.0 * kPi * c->mu), out);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status body_rigid_rows(fs_ctx *c, const double *v, double *rows, double sign)
{
    if (!c->body.on || c->body.n_att == 0) return FS_OK;
    const double *rigid = v + c->n_fib_unk + 3 * int64_t(c->surf.n);
    k_rigid_rows<<<(c->body.n_att + 127) / 128, 128, 0, c->stream>>>(c->table(), c->body.att_list, c->body.n_att,
                                                                      c->d_X, c->body.rb, rigid, sign, rows);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status body_constraints(fs_ctx *c, const double *q1, const double *rigid, double *out)
{
    const int p = c->surf.n_per;
    k_body_constraints<<<1, 256, 0, c->stream>>>(c->surf.y + 3 * int64_t(p), c->surf.w + p, q1, c->body.n,
                                                  c->body.rb, rigid, out);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status body_update(fs_ctx *c, const double *rigid)
{
    if (!c->body.on) return FS_OK;
    const int p = c->surf.n_per;
    k_body_move<<<(c->body.n + 127) / 128, 128, 0, c->stream>>>(c->surf.y + 3 * int64_t(p), c->body.n, c->body.rb,
                                                                 rigid, c->dt);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

}  // namespace fs

using namespace fs;

extern "C" {

fs_status fs_get_body(fs_ctx *c, double *center, double *U, double *Omega)
{
    if (!c || !c->body.on) {
        set_error("fs_get_body: context without a body");
        return FS_EINVAL;
    }
    double h[kRbSize];
    FS_CUDA(cudaMemcpyAsync(h, c->body.rb, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    for (int a = 0; a < 3; ++a) {
        if (center) center[a] = h[kRbCenter + a];
        if (U) U[a] = h[kRbU + a];
        if (Omega) Omega[a] = h[kRbOm + a];
    }
    return FS_OK;
}

fs_status fs_set_body_load(fs_ctx *c, const double *force, const double *torque)
{
    if (!c || !c->body.on || !force || !torque) {
        set_error("fs_set_body_load: context without a body or NULL load");
        return FS_EINVAL;
    }
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(force[a]) || !std::isfinite(torque[a])) {
            set_error("fs_set_body_load: non-finite load");
            return FS_EINVAL;
        }
    double h[6] = {force[0], force[1], force[2], torque[0], torque[1], torque[2]};
    FS_CUDA(cudaMemcpyAsync(c->body.rb + kRbFext, h, 6 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));   // h is a host staging array
    return FS_OK;
}

}  // extern "C"
