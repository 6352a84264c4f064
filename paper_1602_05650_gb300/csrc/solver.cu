// Context setup, Krylov kernels and the implicit step driver.
//
// One step (Sec. 3.2-3.3): geometry, per-fiber self blocks + LU (Eq. prec),
// right-hand side with an FP64 far field, then
//   FS_FP64 : left-preconditioned GMRES on A u = b with the FP64 far field;
//   FS_MIXED: iterative refinement -- r = b - A u with the FP64 far field,
//             GMRES on A e = r with the FP32 far field to inner_tol, u += e --
//             until ||P^-1 r|| <= tol ||P^-1 b||.
// GMRES: x0 = 0, classical Gram-Schmidt with one re-orthogonalisation (CGS2),
// Givens rotations on the host (one small device->host copy per iteration).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "context.h"

namespace fs {
namespace {

constexpr int kDotBlocks = 64;

__global__ void k_multidot(const double *__restrict__ V, int64_t ld, int k,
                           const double *__restrict__ w, int64_t n, double *__restrict__ part)
{
    // part[i * kDotBlocks + b] = sum over chunk b of V_i . w
    __shared__ double red[8];
    const int i = blockIdx.y;
    const int64_t chunk = (n + kDotBlocks - 1) / kDotBlocks;
    const int64_t e0 = blockIdx.x * chunk, e1 = min(n, e0 + chunk);
    const double *v = V + i * ld;
    double s = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) s += v[e] * w[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int wv = 0; wv < static_cast<int>(blockDim.x >> 5); ++wv) t += red[wv];
        part[i * kDotBlocks + blockIdx.x] = t;
    }
}

// h[i] (+)= sum_b part[i][b]; if do_sqrt, h[0] = sqrt(h[0]) (norm)
__global__ void k_finish_dots(const double *__restrict__ part, int k, double *__restrict__ h, int add,
                              int do_sqrt)
{
    const int i = threadIdx.x;
    if (i >= k) return;
    double s = 0.0;
    for (int b = 0; b < kDotBlocks; ++b) s += part[i * kDotBlocks + b];
    if (do_sqrt) s = sqrt(s);
    h[i] = add ? h[i] + s : s;
}

// w -= sum_i h[i] V_i
__global__ void k_axpy_multi(double *__restrict__ w, const double *__restrict__ V, int64_t ld,
                             const double *__restrict__ h, int k, int64_t n)
{
    const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (e >= n) return;
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += h[i] * V[i * ld + e];
    w[e] -= s;
}

// out = in / (*nrm)  (zero if the norm is zero)
__global__ void k_scale_by(const double *__restrict__ in, const double *__restrict__ nrm,
                           double *__restrict__ out, int64_t n)
{
    const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (e >= n) return;
    const double d = *nrm;
    out[e] = d > 0.0 ? in[e] / d : 0.0;
}

// x += sum_i y[i] V_i
__global__ void k_lincomb(double *__restrict__ x, const double *__restrict__ V, int64_t ld,
                          const double *__restrict__ y, int k, int64_t n)
{
    const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (e >= n) return;
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += y[i] * V[i * ld + e];
    x[e] += s;
}

// out = a - b
__global__ void k_sub(const double *__restrict__ a, const double *__restrict__ b,
                      double *__restrict__ out, int64_t n)
{
    const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (e < n) out[e] = a[e] - b[e];
}

__global__ void k_add(double *__restrict__ x, const double *__restrict__ e, int64_t n)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) x[i] += e[i];
}

unsigned blocks_for(int64_t n) { return static_cast<unsigned>((n + 255) / 256); }

template <class T>
fs_status dalloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return FS_OK;
    if (cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("device allocation of %zu bytes failed", n * sizeof(T));
        return FS_ENOMEM;
    }
    return FS_OK;
}

// ||v|| into d_h[slot] (device) -- uses d_part
fs_status dev_norm(fs_ctx *c, const double *v, int64_t n, double *dst)
{
    k_multidot<<<dim3(kDotBlocks, 1), 256, 0, c->stream>>>(v, 0, 1, v, n, c->d_part);
    FS_LAUNCH_CHECK();
    k_finish_dots<<<1, 32, 0, c->stream>>>(c->d_part, 1, dst, 0, 1);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status read_scalar(fs_ctx *c, const double *d, double *h)
{
    FS_CUDA(cudaMemcpyAsync(c->h_pinned, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    *h = c->h_pinned[0];
    return FS_OK;
}

// Far field at the fiber nodes: ubar = (1/8 pi mu) sum_{other fibers} G0 W f
fs_status far_field(fs_ctx *c, int sum_prec, bool hilo)
{
    PairSumArgs a;
    a.kind = PAIR_STOKESLET;
    a.src_xyz = c->d_X;
    a.src_dens = c->d_wf;
    a.n_src = c->n_tot;
    a.excl = c->d_excl;
    a.tgt_xyz = c->d_X;
    a.n_tgt = c->n_tot;
    a.out = c->d_ubar;
    a.scale = 1.0 / (8.0 * M_PI * c->mu);
    a.sum_prec = sum_prec;
    a.hilo = hilo;
    a.shape_override = c->opt.tile_override;
    int64_t self = 0;
    for (int m = 0; m < c->M; ++m) self += int64_t(c->Nm[m]) * c->Nm[m];
    a.pairs = double(c->n_tot) * double(c->n_tot) - double(self);
    a.prof = c->opt.profile ? &c->prof : nullptr;
    FS_TRY(c->scratch.reserve(pairsum_scratch_bytes(a.kind, a.n_src, a.n_tgt, sum_prec, a.shape_override),
                              c->stream));
    FS_TRY(pairsum(a, c->scratch.ptr, c->scratch.bytes, c->d_status, c->stream));
    c->pairs_last += c->n_tot * c->n_tot - self;
    return FS_OK;
}

// Preconditioned operator of Eq. prec, out = P^-1 A v, evaluated as
//   fibers : v + P^-1 (A - P) v  -- P is exactly the self block, so only the
//            coupling rows Rw(ubar) pass through the block solves (the block's
//            own rounding is never amplified by its inverse, cond ~1e9);
//   surface: D^-1 (S q + fiber Stokeslets)  -- D the Jacobi diagonal.
// sum_prec selects the far-field arithmetic.
fs_status apply_pa(fs_ctx *c, const double *v, double *out, int sum_prec)
{
    FS_TRY(launch_force(c, v, c->d_f, c->d_wf));
    FS_TRY(far_field(c, sum_prec, false));
    const double *q = c->surf.n ? v + c->n_fib_unk : nullptr;
    if (c->surf.n) FS_TRY(surface_couplings(c, q, c->d_ubar, sum_prec, false));
    FS_TRY(launch_rows(c, nullptr, c->d_f, c->d_ubar, c->d_e, ROWS_COUPLING));
    FS_TRY(launch_lu_solve(c, c->d_e, out));
    k_add<<<blocks_for(c->n_fib_unk), 256, 0, c->stream>>>(out, v, c->n_fib_unk);
    FS_LAUNCH_CHECK();
    if (c->surf.n) {
        FS_TRY(surface_rows(c, q, c->d_usurf, c->d_e + c->n_fib_unk, false, sum_prec, false));
        FS_TRY(surface_precond(c, c->d_e + c->n_fib_unk, out + c->n_fib_unk));
    }
    return FS_OK;
}

// Far-field arithmetic of the accurate sums (right-hand side, refinement
// residuals): FP64 on the plain FP64 path, float-float on the mixed path.
int accurate_prec(const fs_ctx *c) { return c->opt.prec == FS_FP64 ? FS_SUM_FP64 : FS_SUM_FF; }

// b (Eq. sche-linear-eq right-hand side) with the accurate far field, then pb = P^-1 b
fs_status rhs(fs_ctx *c, double *b, double *pb)
{
    const int ap = accurate_prec(c);
    FS_TRY(launch_force(c, nullptr, c->d_f, c->d_wf));
    FS_TRY(far_field(c, ap, false));
    if (c->surf.n) FS_TRY(surface_couplings(c, nullptr, c->d_ubar, ap, false));
    FS_TRY(launch_rows(c, nullptr, c->d_f, c->d_ubar, b, ROWS_RHS));
    if (c->surf.n) FS_TRY(surface_rows(c, nullptr, c->d_usurf, b + c->n_fib_unk, true, ap, false));
    FS_TRY(launch_lu_solve(c, b, pb));
    if (c->surf.n) FS_TRY(surface_precond(c, b + c->n_fib_unk, pb + c->n_fib_unk));
    return FS_OK;
}

struct GmresResult {
    int iters = 0;          // Arnoldi steps (outer steps for the flexible solver)
    int inner_iters = 0;    // flexible solver: inner GMRES iterations in total
    double rel = 0.0;       // |g| / beta0 estimate
    bool converged = false;
};

// Storage of one Krylov space: basis V [(R+1) x n], optional flexible
// directions Z [R x n], Hessenberg / norm scratch on the device and a pinned
// host copy.
struct Space {
    int R;
    double *V, *Z, *h, *part, *w, *r, *hpin;
};

Space inner_space(fs_ctx *c)
{
    return Space{c->kdim - 1, c->d_basis, nullptr, c->d_h, c->d_part, c->d_w, c->d_r, c->h_pinned};
}

Space outer_space(fs_ctx *c)
{
    return Space{c->okdim - 1, c->d_obasis, c->d_oz, c->d_oh, c->d_opart, c->d_ow, c->d_or, c->oh_pinned};
}

fs_status dev_norm_s(fs_ctx *c, const Space &sp, const double *v, int64_t n, double *dst)
{
    k_multidot<<<dim3(kDotBlocks, 1), 256, 0, c->stream>>>(v, 0, 1, v, n, sp.part);
    FS_LAUNCH_CHECK();
    k_finish_dots<<<1, 32, 0, c->stream>>>(sp.part, 1, dst, 0, 1);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status read_scalar_s(fs_ctx *c, const Space &sp, const double *d, double *h)
{
    FS_CUDA(cudaMemcpyAsync(sp.hpin, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    *h = sp.hpin[0];
    return FS_OK;
}

// out = operator(v): the preconditioned operator with the far field of `prec`
struct Op {
    int sum_prec;
};

// GMRES core for (P^-1 A) x = pb, x0 = 0, restarted after R steps, CGS2 and
// Givens rotations.  With a flexible preconditioner (inner_prec >= 0) each
// direction is z_j = an inner GMRES solve of (P^-1 A_inner) z = v_j to
// inner_tol, the basis is built from (P^-1 A) z_j and x = Z y (FGMRES).
fs_status gmres_core(fs_ctx *c, const Space &sp, const double *pb, double *x, double tol, int max_iter,
                     int sum_prec, int inner_prec, double inner_tol, GmresResult *res);

fs_status gmres(fs_ctx *c, const double *pb, double *x, double tol, int max_iter, int sum_prec,
                GmresResult *res)
{
    return gmres_core(c, inner_space(c), pb, x, tol, max_iter, sum_prec, -1, 0.0, res);
}

fs_status gmres_core(fs_ctx *c, const Space &sp, const double *pb, double *x, double tol, int max_iter,
                     int sum_prec, int inner_prec, double inner_tol, GmresResult *res)
{
    const int64_t n = c->n_unk;
    const int R = sp.R;
    const int hs = R + 1;   // stride of the h buffer blocks
    double *V = sp.V;
    const bool flexible = inner_prec >= 0;
    *res = GmresResult();
    FS_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), c->stream));
    FS_CUDA(cudaMemcpyAsync(sp.r, pb, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    double *d_beta = sp.h + 2 * hs + 2;
    FS_TRY(dev_norm_s(c, sp, sp.r, n, d_beta));
    double beta0;
    FS_TRY(read_scalar_s(c, sp, d_beta, &beta0));
    if (!(beta0 > 0.0)) {
        res->converged = true;
        return FS_OK;
    }
    if (!std::isfinite(beta0)) {
        set_error("gmres: non-finite right-hand side");
        return FS_ENUMERIC;
    }
    double beta = beta0;
    std::vector<double> H(static_cast<size_t>(R + 1) * R), cs(R), sn(R), g(R + 1), y(R);
    int total = 0;
    while (true) {
        k_scale_by<<<blocks_for(n), 256, 0, c->stream>>>(sp.r, d_beta, V, n);
        FS_LAUNCH_CHECK();
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int kcols = 0;
        bool done = false;
        for (int j = 0; j < R; ++j) {
            double *Vj = V + j * n, *Vn = V + (j + 1) * n;
            if (flexible) {
                GmresResult ir;
                double *Zj = sp.Z + j * n;
                FS_TRY(gmres_core(c, inner_space(c), Vj, Zj, inner_tol, c->opt.max_iter, inner_prec, -1, 0.0,
                                  &ir));
                res->inner_iters += ir.iters;
                FS_TRY(apply_pa(c, Zj, sp.w, sum_prec));
            } else {
                FS_TRY(apply_pa(c, Vj, sp.w, sum_prec));
            }
            double *h = sp.h;
            for (int pass = 0; pass < 2; ++pass) {   // CGS2
                double *hp = h + (pass ? hs : 0);
                k_multidot<<<dim3(kDotBlocks, j + 1), 256, 0, c->stream>>>(V, n, j + 1, sp.w, n, sp.part);
                FS_LAUNCH_CHECK();
                k_finish_dots<<<1, 256, 0, c->stream>>>(sp.part, j + 1, hp, 0, 0);
                FS_LAUNCH_CHECK();
                k_axpy_multi<<<blocks_for(n), 256, 0, c->stream>>>(sp.w, V, n, hp, j + 1, n);
                FS_LAUNCH_CHECK();
            }
            FS_TRY(dev_norm_s(c, sp, sp.w, n, h + 2 * hs));
            k_scale_by<<<blocks_for(n), 256, 0, c->stream>>>(sp.w, h + 2 * hs, Vn, n);
            FS_LAUNCH_CHECK();
            FS_CUDA(cudaMemcpyAsync(sp.hpin, h, (2 * hs + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
            FS_CUDA(cudaStreamSynchronize(c->stream));
            double *hc = &H[static_cast<size_t>(j) * (R + 1)];   // column j, length R+1
            for (int i = 0; i <= j; ++i) hc[i] = sp.hpin[i] + sp.hpin[hs + i];
            const double hn = sp.hpin[2 * hs];
            hc[j + 1] = hn;
            if (!std::isfinite(hn)) {
                set_error("gmres: non-finite Arnoldi vector");
                return FS_ENUMERIC;
            }
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
                hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
                hc[i] = t;
            }
            const double d = std::hypot(hc[j], hc[j + 1]);
            cs[j] = d > 0.0 ? hc[j] / d : 1.0;
            sn[j] = d > 0.0 ? hc[j + 1] / d : 0.0;
            hc[j] = d;
            hc[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++total;
            kcols = j + 1;
            res->rel = std::fabs(g[j + 1]) / beta0;
            if (res->rel <= tol) {
                res->converged = true;
                done = true;
                break;
            }
            if (hn == 0.0 || total >= max_iter) {
                done = true;
                break;
            }
        }
        // y = H^-1 g (upper triangular kcols x kcols), x += (V or Z) y
        for (int i = kcols - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < kcols; ++l) s -= H[static_cast<size_t>(l) * (R + 1) + i] * y[l];
            const double dii = H[static_cast<size_t>(i) * (R + 1) + i];
            y[i] = dii != 0.0 ? s / dii : 0.0;
        }
        std::memcpy(sp.hpin, y.data(), kcols * sizeof(double));
        double *d_y = sp.h + 3 * hs + 4;
        FS_CUDA(cudaMemcpyAsync(d_y, sp.hpin, kcols * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        k_lincomb<<<blocks_for(n), 256, 0, c->stream>>>(x, flexible ? sp.Z : V, n, d_y, kcols, n);
        FS_LAUNCH_CHECK();
        FS_CUDA(cudaStreamSynchronize(c->stream));   // hpin is reused below
        if (done) break;
        // restart: r = pb - P^-1 A x
        FS_TRY(apply_pa(c, x, sp.w, sum_prec));
        k_sub<<<blocks_for(n), 256, 0, c->stream>>>(pb, sp.w, sp.r, n);
        FS_LAUNCH_CHECK();
        FS_TRY(dev_norm_s(c, sp, sp.r, n, d_beta));
        FS_TRY(read_scalar_s(c, sp, d_beta, &beta));
        res->rel = beta / beta0;
        if (res->rel <= tol) {
            res->converged = true;
            break;
        }
    }
    res->iters = total;
    return FS_OK;
}

fs_status check_status(fs_ctx *c)
{
    int h = 0;
    FS_CUDA(cudaMemcpyAsync(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    if (h & DEV_ERR_TIMEOUT) {
        set_error("a bounded device-side wait gave up (status 0x%x)", h);
        FS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
        return FS_ETIMEOUT;
    }
    if (h & DEV_ERR_NUMERIC) {
        set_error("zero pivot or non-finite value in a fiber block (status 0x%x)", h);
        FS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
        return FS_ENUMERIC;
    }
    return FS_OK;
}

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

fs_status context_init(fs_ctx *c, int M, const int32_t *ppf, const fs_boundary *bd)
{
    c->M = M;
    c->Nm.assign(ppf, ppf + M);
    c->node_ptr.assign(M + 1, 0);
    c->unk_ptr.assign(M + 1, 0);
    c->blk_ptr.assign(M + 1, 0);
    std::vector<int64_t> kp(M + 1, 0), zp(M + 1, 0);
    for (int m = 0; m < M; ++m) {
        const int N = ppf[m];
        c->node_ptr[m + 1] = c->node_ptr[m] + N;
        c->unk_ptr[m + 1] = c->unk_ptr[m] + 4 * N;
        c->blk_ptr[m + 1] = c->blk_ptr[m] + int64_t(16) * N * N;
        kp[m + 1] = kp[m] + int64_t(N) * N;
        zp[m + 1] = zp[m] + (N - 2);
        c->max_N = std::max(c->max_N, N);
    }
    c->n_tot = c->node_ptr[M];
    c->n_fib_unk = c->unk_ptr[M];
    c->n_blk = c->blk_ptr[M];
    c->n_kp = kp[M];
    c->n_z = zp[M];
    c->surf.n = bd ? bd->n_nodes : 0;
    c->n_unk = c->n_fib_unk + 3 * int64_t(c->surf.n);
    if (c->n_tot >= (1LL << 31) - 1) {
        set_error("fs_create: at most 2^31-2 points");
        return FS_EINVAL;
    }
    FS_TRY(dalloc(&c->d_status, 1));
    FS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    FS_CUDA(cudaMallocHost(&c->h_pinned, 4096 * sizeof(double)));
    if (M == 0) return FS_OK;

    // op sets
    std::vector<double> ops;
    for (int m = 0; m < M; ++m) {
        const int N = ppf[m];
        if (c->ops_offset.count(N)) continue;
        c->ops_offset[N] = static_cast<int64_t>(ops.size());
        const std::vector<double> o = build_ops(N);
        ops.insert(ops.end(), o.begin(), o.end());
    }
    std::vector<int64_t> off(M);
    for (int m = 0; m < M; ++m) off[m] = c->ops_offset[ppf[m]];
    std::vector<int2> excl(c->n_tot);
    for (int m = 0; m < M; ++m)
        for (int64_t i = c->node_ptr[m]; i < c->node_ptr[m + 1]; ++i)
            excl[i] = make_int2(static_cast<int>(c->node_ptr[m]), static_cast<int>(c->node_ptr[m + 1]));

    FS_TRY(dalloc(&c->d_N, M));
    FS_TRY(dalloc(&c->d_node_ptr, M + 1));
    FS_TRY(dalloc(&c->d_unk_ptr, M + 1));
    FS_TRY(dalloc(&c->d_blk_ptr, M + 1));
    FS_TRY(dalloc(&c->d_kp_ptr, M + 1));
    FS_TRY(dalloc(&c->d_z_ptr, M + 1));
    FS_TRY(dalloc(&c->d_ops_off, M));
    FS_TRY(dalloc(&c->d_ops, ops.size()));
    FS_TRY(dalloc(&c->d_excl, c->n_tot));
    FS_CUDA(cudaMemcpy(c->d_N, ppf, M * sizeof(int), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->d_node_ptr, c->node_ptr.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->d_unk_ptr, c->unk_ptr.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->d_blk_ptr, c->blk_ptr.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->d_kp_ptr, kp.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->d_z_ptr, zp.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->d_ops_off, off.data(), M * sizeof(int64_t), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->d_ops, ops.data(), ops.size() * sizeof(double), cudaMemcpyHostToDevice));
    FS_CUDA(cudaMemcpy(c->d_excl, excl.data(), c->n_tot * sizeof(int2), cudaMemcpyHostToDevice));

    const int64_t P = c->n_tot;
    FS_TRY(dalloc(&c->d_X, 3 * P));
    FS_TRY(dalloc(&c->d_L, M));
    FS_TRY(dalloc(&c->d_fext, 3 * P));
    FS_TRY(dalloc(&c->d_t, 3 * P));
    FS_TRY(dalloc(&c->d_tz, 3 * c->n_z));
    FS_TRY(dalloc(&c->d_fknown, 3 * P));
    FS_TRY(dalloc(&c->d_W, P));
    FS_TRY(dalloc(&c->d_mloc, 2 * P));
    FS_TRY(dalloc(&c->d_bc, 12 * M));
    FS_TRY(dalloc(&c->d_kp, 4 * c->n_kp));
    FS_TRY(dalloc(&c->d_B, c->n_blk));
    FS_TRY(dalloc(&c->d_piv, c->n_fib_unk));
    FS_TRY(dalloc(&c->d_V, 3 * P));
    FS_TRY(dalloc(&c->d_T, P));
    FS_TRY(dalloc(&c->d_f, 3 * P));
    FS_TRY(dalloc(&c->d_wf, 3 * P));
    FS_TRY(dalloc(&c->d_ubar, 3 * P));
    FS_CUDA(cudaMemset(c->d_kp, 0, 4 * c->n_kp * sizeof(double)));
    FS_CUDA(cudaMemset(c->d_V, 0, 3 * P * sizeof(double)));
    FS_CUDA(cudaMemset(c->d_T, 0, P * sizeof(double)));

    const int R = std::max(2, std::min(c->opt.restart, 250));   // k_finish_dots uses 256 threads
    c->kdim = R + 1;
    const int64_t n = c->n_unk;
    FS_TRY(dalloc(&c->d_basis, static_cast<size_t>(c->kdim) * n));
    FS_TRY(dalloc(&c->d_b, n));
    FS_TRY(dalloc(&c->d_x, n));
    FS_TRY(dalloc(&c->d_r, n));
    FS_TRY(dalloc(&c->d_w, n));
    FS_TRY(dalloc(&c->d_e, n));
    FS_TRY(dalloc(&c->d_pb, n));
    FS_TRY(dalloc(&c->d_h, 4 * c->kdim + 8));
    FS_TRY(dalloc(&c->d_part, static_cast<size_t>(c->kdim) * kDotBlocks));
    if (c->opt.prec == FS_MIXED) {
        c->okdim = 17;   // outer (flexible) restart length 16
        FS_TRY(dalloc(&c->d_obasis, static_cast<size_t>(c->okdim) * n));
        FS_TRY(dalloc(&c->d_oz, static_cast<size_t>(c->okdim - 1) * n));
        FS_TRY(dalloc(&c->d_oh, 4 * c->okdim + 8));
        FS_TRY(dalloc(&c->d_opart, static_cast<size_t>(c->okdim) * kDotBlocks));
        FS_TRY(dalloc(&c->d_ow, n));
        FS_TRY(dalloc(&c->d_or, n));
        FS_CUDA(cudaMallocHost(&c->oh_pinned, 4096 * sizeof(double)));
    }
    if (c->surf.n) {
        const int ns = c->surf.n;
        FS_TRY(dalloc(&c->surf.y, 3 * ns));
        FS_TRY(dalloc(&c->surf.nrm, 3 * ns));
        FS_TRY(dalloc(&c->surf.w, ns));
        FS_TRY(dalloc(&c->surf.diag, 3 * ns));
        FS_TRY(dalloc(&c->d_usurf, 3 * ns));
        FS_TRY(dalloc(&c->surf.A, 9 * ns));
        FS_TRY(dalloc(&c->surf.tmp, 3 * ns));
        FS_TRY(dalloc(&c->surf.flux, 1));
        FS_TRY(dalloc(&c->surf.excl, ns));
        FS_CUDA(cudaMemcpy(c->surf.y, bd->nodes, 3 * ns * sizeof(double), cudaMemcpyHostToDevice));
        FS_CUDA(cudaMemcpy(c->surf.nrm, bd->normals, 3 * ns * sizeof(double), cudaMemcpyHostToDevice));
        FS_CUDA(cudaMemcpy(c->surf.w, bd->weights, ns * sizeof(double), cudaMemcpyHostToDevice));
        FS_TRY(surface_diag(c));
    }
    FS_CUDA(cudaDeviceSynchronize());
    return FS_OK;
}

void context_free(fs_ctx *c)
{
    if (c->stream) cudaStreamSynchronize(c->stream);
    void *ptrs[] = {c->d_status, c->d_N, c->d_node_ptr, c->d_unk_ptr, c->d_blk_ptr, c->d_kp_ptr,
                    c->d_z_ptr, c->d_ops_off, c->d_ops, c->d_excl, c->d_X, c->d_L, c->d_fext,
                    c->d_t, c->d_tz, c->d_fknown, c->d_W, c->d_mloc, c->d_bc, c->d_kp, c->d_B,
                    c->d_piv, c->d_V, c->d_T, c->d_f, c->d_wf, c->d_ubar, c->d_basis, c->d_b,
                    c->d_x, c->d_r, c->d_w, c->d_e, c->d_pb, c->d_obasis, c->d_oz, c->d_oh, c->d_opart, c->d_ow, c->d_or, c->d_h, c->d_part, c->surf.y, c->surf.nrm,
                    c->surf.w, c->surf.diag, c->d_usurf, c->surf.A, c->surf.tmp, c->surf.flux, c->surf.excl};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->oh_pinned) cudaFreeHost(c->oh_pinned);
    c->oh_pinned = nullptr;
    c->prof.release_all();
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    c->prof.pool.clear();
    c->h_pinned = nullptr;
    c->scratch.release();
}

}  // namespace fs

fs::FiberTable fs_ctx::table() const
{
    fs::FiberTable F;
    F.M = M;
    F.N = d_N;
    F.node_ptr = d_node_ptr;
    F.unk_ptr = d_unk_ptr;
    F.blk_ptr = d_blk_ptr;
    F.kp_ptr = d_kp_ptr;
    F.z_ptr = d_z_ptr;
    F.ops_off = d_ops_off;
    F.ops = d_ops;
    F.L = d_L;
    F.mu = mu;
    F.eps = eps;
    F.E = E;
    F.dt = dt;
    F.delta_over_L = opt.delta_over_L;
    F.lsb = opt.lsb;
    F.t = d_t;
    F.tz = d_tz;
    F.fknown = d_fknown;
    F.W = d_W;
    F.mloc = d_mloc;
    F.bc = d_bc;
    F.kp = d_kp;
    return F;
}

using namespace fs;

extern "C" {

fs_status fs_set_state(fs_ctx *c, const double *X, const double *L, const double *f_ext,
                       int32_t dev)
{
    if (!c || c->M == 0 || !X || !L) {
        set_error("fs_set_state: NULL argument or context without fibers");
        return FS_EINVAL;
    }
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    std::vector<double> hL(c->M);
    if (dev)
        FS_CUDA(cudaMemcpy(hL.data(), L, c->M * sizeof(double), cudaMemcpyDeviceToHost));
    else
        std::memcpy(hL.data(), L, c->M * sizeof(double));
    for (int m = 0; m < c->M; ++m)
        if (!(hL[m] > 0.0) || !std::isfinite(hL[m])) {
            set_error("fs_set_state: fiber %d has length %g", m, hL[m]);
            return FS_EINVAL;
        }
    FS_CUDA(cudaMemcpyAsync(c->d_X, X, 3 * c->n_tot * sizeof(double), kind, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_L, hL.data(), c->M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (f_ext)
        FS_CUDA(cudaMemcpyAsync(c->d_fext, f_ext, 3 * c->n_tot * sizeof(double), kind, c->stream));
    else
        FS_CUDA(cudaMemsetAsync(c->d_fext, 0, 3 * c->n_tot * sizeof(double), c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    c->have_state = true;
    c->geometry_ok = c->precond_ok = false;
    return FS_OK;
}

fs_status fs_get_state(fs_ctx *c, double *X, double *T, double *V, int32_t dev)
{
    if (!c || c->M == 0) {
        set_error("fs_get_state: NULL context or no fibers");
        return FS_EINVAL;
    }
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (X) FS_CUDA(cudaMemcpyAsync(X, c->d_X, 3 * c->n_tot * sizeof(double), kind, c->stream));
    if (T) FS_CUDA(cudaMemcpyAsync(T, c->d_T, c->n_tot * sizeof(double), kind, c->stream));
    if (V) FS_CUDA(cudaMemcpyAsync(V, c->d_V, 3 * c->n_tot * sizeof(double), kind, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

fs_status fs_build_precond(fs_ctx *c)
{
    if (!c || !c->have_state) {
        set_error("fs_build_precond: no state set");
        return FS_EINVAL;
    }
    if (!c->geometry_ok) {
        FS_TRY(launch_geometry(c));
        c->geometry_ok = true;
    }
    FS_TRY(launch_block_build(c));
    FS_TRY(launch_lu_factor(c));
    c->precond_ok = true;
    return FS_OK;
}

fs_status fs_step(fs_ctx *c, fs_step_info *info)
{
    if (!c || !c->have_state || c->M == 0) {
        set_error("fs_step: no state set");
        return FS_EINVAL;
    }
    const auto t0 = std::chrono::steady_clock::now();
    c->pairs_last = 0;
    double tms[8] = {0};
    if (!c->geometry_ok) {
        FS_TRY(launch_geometry(c));
        c->geometry_ok = true;
    }
    if (!c->precond_ok) FS_TRY(fs_build_precond(c));
    if (info) {
        FS_CUDA(cudaStreamSynchronize(c->stream));
        tms[1] = ms_since(t0);
    }
    FS_TRY(rhs(c, c->d_b, c->d_pb));
    FS_TRY(check_status(c));
    if (info) tms[0] = ms_since(t0) - tms[1];
    int iters = 0, sweeps = 0;
    double rel = 0.0;
    bool converged = false;
    if (c->opt.prec == FS_FP64) {
        GmresResult gr;
        FS_TRY(gmres(c, c->d_pb, c->d_x, c->opt.tol, c->opt.max_iter, FS_SUM_FP64, &gr));
        iters = gr.iters;
        rel = gr.rel;
        sweeps = 1;
        converged = gr.converged;
    } else {
        // mixed: flexible GMRES on the operator with the float-float far field,
        // each direction preconditioned by an FP32-far-field GMRES solve
        GmresResult gr;
        FS_TRY(gmres_core(c, outer_space(c), c->d_pb, c->d_x, c->opt.tol, c->opt.max_iter,
                          accurate_prec(c), FS_SUM_FP32, c->opt.inner_tol, &gr));
        iters = gr.inner_iters;
        sweeps = gr.iters;
        rel = gr.rel;
        converged = gr.converged;
    }
    FS_TRY(check_status(c));
    tms[2] = ms_since(t0) - tms[0] - tms[1];
    if (info) {
        info->iters = iters;
        info->refine_sweeps = sweeps;
        info->resid = rel;
        info->pairs = c->pairs_last;
    }
    if (!converged) {
        if (info) {
            tms[4] = ms_since(t0);
            std::memcpy(info->t_ms, tms, sizeof(tms));
        }
        set_error("fs_step: not converged (rel. residual %.3e after %d iterations)", rel, iters);
        return FS_ENOTCONV;
    }
    FS_TRY(launch_update(c, c->d_x));
    c->geometry_ok = c->precond_ok = false;
    if (info) {
        FS_CUDA(cudaStreamSynchronize(c->stream));
        tms[4] = ms_since(t0);
        tms[3] = tms[4] - tms[0] - tms[1] - tms[2];
        std::memcpy(info->t_ms, tms, sizeof(tms));
    }
    return FS_OK;
}

}  // extern "C"
