// Confined suspensions: the no-slip spherical periphery (Sec. 2.1, Eqs.
// main-cortex-vel, main-cortex-density; Sec. 3.1.1-3.1.2), and the surface of
// a rigid body (Sec. 2.2, Eq. main-nsb-second-kind).  Both surfaces form one
// node set (periphery first) for the double-layer sums; each keeps its own
// subtraction matrices and limit:
//
// Periphery rows (3 per surface node y_i), fluid-side limit of the double layer
// with singularity subtraction and the rank completion N:
//   sum_{j != i} w_j T(y_i - y_j):((q_j - q_i) n_j) + q_i + n_i sum_j w_j n_j.q_j
//     + sum_{fibers} G(y_i - X) W f = 0
// where the subtraction term is -A_i q_i with the geometric 3x3 matrix
//   A_i[a][b] = sum_{j != i} w_j T_abc(y_i - y_j) n_jc
// computed once per context.  Fiber nodes feel u^c = T[q] (Eq. cortex-vel).
// Body rows (fluid outside: the limit has no +q_i term, and no N):
//   sum_{j != i} w_j T(y_i - y_j):((q_j - q_i) n_j) - U - Omega x (y_i - X^P)
//     + (fiber Stokeslets, periphery double layer, G F + R L at y_i) = 0
// followed by the six rigid-motion constraint rows.
// Preconditioner: the scalar diagonal of each surface's self block (Eq.
// prec), -1 on the U, Omega rows.
#include <cmath>

#include "context.h"

namespace fs {
namespace {

constexpr double kStressC = -3.0 / (4.0 * 3.14159265358979323846);

// A_i and the Jacobi diagonal, FP64, one thread per node.
__global__ void k_surface_geom(const double *__restrict__ y, const double *__restrict__ nrm,
                               const double *__restrict__ w, int n, double *__restrict__ A,
                               double *__restrict__ diag, int interior)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double yx = y[3 * i], yy = y[3 * i + 1], yz = y[3 * i + 2];
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        const double r[3] = {yx - y[3 * j], yy - y[3 * j + 1], yz - y[3 * j + 2]};
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double ri = 1.0 / sqrt(r2);
        const double ri5 = ri * ri * ri * ri * ri;
        const double rn = r[0] * nrm[3 * j] + r[1] * nrm[3 * j + 1] + r[2] * nrm[3 * j + 2];
        const double s = kStressC * w[j] * rn * ri5;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) M[3 * a + b] += s * r[a] * r[b];
    }
    for (int k = 0; k < 9; ++k) A[9 * i + k] = M[k];
    for (int a = 0; a < 3; ++a)
        diag[3 * i + a] = -M[4 * a] + (interior ? 1.0 + w[i] * nrm[3 * i + a] * nrm[3 * i + a] : 0.0);
}

// s = sum_j w_j n_j . q_j  (one CTA)
__global__ void __launch_bounds__(512) k_normal_flux(const double *__restrict__ nrm,
                                                     const double *__restrict__ w,
                                                     const double *__restrict__ q, int n,
                                                     double *__restrict__ s)
{
    __shared__ double red[16];
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        acc += w[j] * (nrm[3 * j] * q[3 * j] + nrm[3 * j + 1] * q[3 * j + 1] + nrm[3 * j + 2] * q[3 * j + 2]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) t += red[k];
        *s = t;
    }
}

// periphery node (i < n_per): out_i = dl_i - A_i q_i + q_i + n_i s + usurf_i
// body node:                   out_i = dl_i - A_i q_i - U - Omega x (y_i - X^P) + usurf_i
__global__ void k_surface_combine(const double *__restrict__ dl, const double *__restrict__ A,
                                  const double *__restrict__ q, const double *__restrict__ nrm,
                                  const double *__restrict__ s, const double *__restrict__ usurf,
                                  int n, int n_per, const double *__restrict__ y,
                                  const double *__restrict__ rb, const double *__restrict__ rigid,
                                  double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool per = i < n_per;
    const double flux = per ? *s : 0.0;
    double rig[3] = {0.0, 0.0, 0.0};
    if (!per) {
        const double r[3] = {y[3 * i] - rb[kRbCenter], y[3 * i + 1] - rb[kRbCenter + 1],
                             y[3 * i + 2] - rb[kRbCenter + 2]};
        const double *U = rigid, *Om = rigid + 3;
        rig[0] = U[0] + Om[1] * r[2] - Om[2] * r[1];
        rig[1] = U[1] + Om[2] * r[0] - Om[0] * r[2];
        rig[2] = U[2] + Om[0] * r[1] - Om[1] * r[0];
    }
    for (int a = 0; a < 3; ++a) {
        double v = dl[3 * i + a] + (per ? q[3 * i + a] + nrm[3 * i + a] * flux : -rig[a]);
        for (int b = 0; b < 3; ++b) v -= A[9 * i + 3 * a + b] * q[3 * i + b];
        out[3 * i + a] = v + (usurf ? usurf[3 * i + a] : 0.0);
    }
}

__global__ void k_neg(const double *__restrict__ in, double *__restrict__ out, int64_t n)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) out[i] = -in[i];
}

__global__ void k_div(const double *__restrict__ in, const double *__restrict__ d,
                      double *__restrict__ out, int64_t n)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) out[i] = in[i] / d[i];
}

fs_status run_sum(fs_ctx *c, PairSumArgs &a)
{
    a.pairs = double(a.n_src) * double(a.n_tgt);
    a.prof = c->opt.profile ? &c->prof : nullptr;
    FS_TRY(c->scratch.reserve(pairsum_scratch_bytes(a.kind, a.n_src, a.n_tgt, a.sum_prec,
                                                    a.shape_override),
                              c->stream));
    return pairsum(a, c->scratch.ptr, c->scratch.bytes, c->d_status, c->stream);
}

}  // namespace

fs_status surface_diag(fs_ctx *c)
{
    const int n = c->surf.n;
    if (!n) return FS_OK;
    std::vector<int2> ex(n);
    for (int i = 0; i < n; ++i) ex[i] = make_int2(i, i + 1);
    FS_CUDA(cudaMemcpyAsync(c->surf.excl, ex.data(), n * sizeof(int2), cudaMemcpyHostToDevice, c->stream));
    const int p = c->surf.n_per, nb = n - p;
    if (p > 0) {
        k_surface_geom<<<(p + 127) / 128, 128, 0, c->stream>>>(c->surf.y, c->surf.nrm, c->surf.w, p, c->surf.A,
                                                                c->surf.diag, 1);
        FS_LAUNCH_CHECK();
    }
    if (nb > 0) {
        k_surface_geom<<<(nb + 127) / 128, 128, 0, c->stream>>>(c->surf.y + 3 * int64_t(p), c->surf.nrm + 3 * int64_t(p),
                                                                 c->surf.w + p, nb, c->surf.A + 9 * int64_t(p),
                                                                 c->surf.diag + 3 * int64_t(p), 0);
        FS_LAUNCH_CHECK();
    }
    FS_CUDA(cudaStreamSynchronize(c->stream));   // `ex` is a host staging vector
    return FS_OK;
}

// ubar_fibers += T[q] at the fiber nodes (q != nullptr); d_usurf = fiber
// Stokeslets at the surface nodes; with a body, both += G F + R L of the
// strengths body_load left in the body record.
fs_status surface_couplings(fs_ctx *c, const double *q, double *ubar_fibers, int sum_prec,
                            bool hilo)
{
    if (q && c->M > 0) {
        PairSumArgs a;
        a.kind = PAIR_STRESSLET;
        a.src_xyz = c->surf.y;
        a.src_dens = q;
        a.src_w = c->surf.w;
        a.src_nrm = c->surf.nrm;
        a.n_src = c->surf.n;
        a.tgt_xyz = c->d_X;
        a.n_tgt = c->n_tot;
        a.out = ubar_fibers;
        a.scale = kStressC;
        a.sum_prec = sum_prec;
        a.hilo = hilo;
        a.accumulate = true;
        a.shape_override = c->opt.tile_override;
        FS_TRY(run_sum(c, a));
        c->pairs_last += c->n_tot * int64_t(c->surf.n);
    }
    PairSumArgs b;
    b.kind = PAIR_STOKESLET;
    b.src_xyz = c->d_X;
    b.src_dens = c->d_wf;
    b.n_src = c->n_tot;
    b.tgt_xyz = c->surf.y;
    b.n_tgt = c->surf.n;
    b.out = c->d_usurf;
    b.scale = 1.0 / (8.0 * M_PI * c->mu);
    b.sum_prec = sum_prec;
    b.hilo = hilo;
    b.shape_override = c->opt.tile_override;
    FS_TRY(run_sum(c, b));
    c->pairs_last += c->n_tot * int64_t(c->surf.n);
    if (c->body.on) {
        FS_TRY(body_point_flow(c, c->d_X, c->n_tot, ubar_fibers));
        FS_TRY(body_point_flow(c, c->surf.y, c->surf.n, c->d_usurf));
    }
    return FS_OK;
}

// out = surface rows (matvec) or -usurf (rhs); with a body, q is followed by
// U, Omega and out by the six constraint rows (0 in the rhs)
fs_status surface_rows(fs_ctx *c, const double *q, const double *usurf, double *out, bool rhs,
                       int sum_prec, bool hilo)
{
    const int n = c->surf.n;
    if (rhs || !q) {
        k_neg<<<(3 * n + 255) / 256, 256, 0, c->stream>>>(usurf, out, 3 * int64_t(n));
        FS_LAUNCH_CHECK();
        if (c->body.on) FS_CUDA(cudaMemsetAsync(out + 3 * int64_t(n), 0, 6 * sizeof(double), c->stream));
        return FS_OK;
    }
    PairSumArgs a;
    a.kind = PAIR_STRESSLET;
    a.src_xyz = c->surf.y;
    a.src_dens = q;
    a.src_w = c->surf.w;
    a.src_nrm = c->surf.nrm;
    a.n_src = n;
    a.excl = c->surf.excl;
    a.tgt_xyz = c->surf.y;
    a.n_tgt = n;
    a.out = c->surf.tmp;
    a.scale = kStressC;
    a.sum_prec = sum_prec;
    a.hilo = hilo;
    a.shape_override = c->opt.tile_override;
    FS_TRY(run_sum(c, a));
    c->pairs_last += int64_t(n) * n;
    const int p = c->surf.n_per;
    if (p > 0) {
        k_normal_flux<<<1, 512, 0, c->stream>>>(c->surf.nrm, c->surf.w, q, p, c->surf.flux);
        FS_LAUNCH_CHECK();
    }
    const double *rigid = c->body.on ? q + 3 * int64_t(n) : nullptr;
    k_surface_combine<<<(n + 127) / 128, 128, 0, c->stream>>>(c->surf.tmp, c->surf.A, q, c->surf.nrm,
                                                               c->surf.flux, usurf, n, p, c->surf.y,
                                                               c->body.rb, rigid, out);
    FS_LAUNCH_CHECK();
    if (c->body.on) FS_TRY(body_constraints(c, q + 3 * int64_t(p), rigid, out + 3 * int64_t(n)));
    return FS_OK;
}

fs_status surface_precond(fs_ctx *c, const double *in, double *out)
{
    const int64_t n3 = 3 * int64_t(c->surf.n);
    k_div<<<static_cast<unsigned>((n3 + 255) / 256), 256, 0, c->stream>>>(in, c->surf.diag, out, n3);
    FS_LAUNCH_CHECK();
    if (c->body.on) {
        k_neg<<<1, 32, 0, c->stream>>>(in + n3, out + n3, 6);
        FS_LAUNCH_CHECK();
    }
    return FS_OK;
}

}  // namespace fs

using namespace fs;

extern "C" {

fs_status fs_stresslet_apply(fs_ctx *c, const double *src_xyz, const double *src_nrm,
                             const double *src_w, const double *src_q, int64_t n_src,
                             const double *tgt_xyz, int64_t n_tgt, double *out_u,
                             int32_t sum_precision)
{
    if (!c || n_src < 0 || n_tgt < 0 ||
        (n_src > 0 && (!src_xyz || !src_nrm || !src_w || !src_q)) || (n_tgt > 0 && (!tgt_xyz || !out_u))) {
        set_error("fs_stresslet_apply: bad arguments");
        return FS_EINVAL;
    }
    if (sum_precision != FS_SUM_FP32 && sum_precision != FS_SUM_FP64 && sum_precision != FS_SUM_FF) {
        set_error("fs_stresslet_apply: unknown precision %d", sum_precision);
        return FS_EINVAL;
    }
    if (n_src >= (1LL << 31) - 1 || n_tgt >= (1LL << 31) - 1) {
        set_error("fs_stresslet_apply: at most 2^31-2 sources and targets");
        return FS_EINVAL;
    }
    PairSumArgs a;
    a.kind = PAIR_STRESSLET;
    a.src_xyz = src_xyz;
    a.src_dens = src_q;
    a.src_w = src_w;
    a.src_nrm = src_nrm;
    a.n_src = n_src;
    a.tgt_xyz = tgt_xyz;
    a.n_tgt = n_tgt;
    a.out = out_u;
    a.scale = kStressC;
    a.sum_prec = sum_precision;
    a.hilo = true;
    a.shape_override = c->opt.tile_override;
    return run_sum(c, a);
}

fs_status fs_surface_apply(fs_ctx *c, const double *q, double *out, int32_t sum_precision)
{
    // with a body, q and out span all surface unknowns (densities, then U, Omega)
    if (!c || c->surf.n == 0 || !q || !out) {
        set_error("fs_surface_apply: context without periphery or NULL arrays");
        return FS_EINVAL;
    }
    if (sum_precision != FS_SUM_FP32 && sum_precision != FS_SUM_FP64 && sum_precision != FS_SUM_FF) {
        set_error("fs_surface_apply: unknown precision %d", sum_precision);
        return FS_EINVAL;
    }
    return surface_rows(c, q, nullptr, out, false, sum_precision, true);
}

}  // extern "C"
