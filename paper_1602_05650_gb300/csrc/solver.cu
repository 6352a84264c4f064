// Context setup, Krylov kernels and the implicit step driver.
//
// One step (Sec. 3.2-3.3): geometry, per-fiber self blocks + LU (Eq. prec),
// right-hand side, then one of
//   FS_FP64            : left-preconditioned GMRES on A u = b, every far field
//                        in FP64;
//   FS_MIXED, relax = 1: GMRES on the operator with the plain FP32 far field and
//                        an FP32 hi/lo right-hand side to inner_tol; ONE true
//                        preconditioned residual r = P^-1 b - P^-1 A u whose far
//                        fields are float-float (FP64-grade, on the FP32 pipe);
//                        GMRES on the plain FP32 operator for the correction d
//                        until |r - P^-1 A d| <= tol |P^-1 b|, u += d (a residual
//                        too large for the FP32 operator's accuracy is reduced
//                        1e3-fold and r taken again, at most max_refine times);
//   FS_MIXED, relax = 0: flexible GMRES whose outer operator has float-float far
//                        fields, each direction preconditioned by a GMRES solve
//                        on the FP32-far-field operator to inner_tol.
// GMRES: x0 = 0, classical Gram-Schmidt with one re-orthogonalisation (CGS2),
// Givens rotations on the host (one small device->host copy per iteration).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "context.h"

namespace fs {
namespace {


__global__ void k_add(double *__restrict__ x, const double *__restrict__ e, int64_t n)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) x[i] += e[i];
}

unsigned blocks_for(int64_t n) { return static_cast<unsigned>((n + 255) / 256); }

// Pinned host buffer: from the context's region when it has one.
fs_status pinned_alloc(fs_ctx *c, double **p, size_t n)
{
    if (c->pool) {
        *p = static_cast<double *>(c->pool->take_host(n * sizeof(double)));
        if (!*p) {
            set_error("pinned host buffer of %zu bytes exceeds the preallocated region", n * sizeof(double));
            return FS_ENOMEM;
        }
        return FS_OK;
    }
    FS_CUDA(cudaMallocHost(p, n * sizeof(double)));
    return FS_OK;
}

template <class T>
fs_status dalloc(fs_ctx *c, T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) return FS_OK;
    if (c->pool) {
        *p = static_cast<T *>(c->pool->take_dev(n * sizeof(T)));
        if (!*p) {
            set_error("device allocation of %zu bytes exceeds the preallocated region", n * sizeof(T));
            return FS_ENOMEM;
        }
        c->dev_bytes += n * sizeof(T);
        return FS_OK;
    }
    if (cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("device allocation of %zu bytes failed", n * sizeof(T));
        return FS_ENOMEM;
    }
    c->dev_bytes += n * sizeof(T);
    return FS_OK;
}

// ------------------------------------------------------ segmented Krylov kernels
// Vectors hold several independent systems back to back.  Work is described by
// chunks (int4: first element, length <= kChunk, system, 0) covering the
// active systems only; per-system scalars live in h[s * SH + offset].
constexpr int kChunk = 4096;

// part[i * nch + c] = sum over chunk c of V_i . w
__global__ void k_seg_dot(const double *__restrict__ V, int64_t ld, const double *__restrict__ w,
                          const int4 *__restrict__ ch, int nch, double *__restrict__ part)
{
    __shared__ double red[8];
    const int c = blockIdx.x, i = blockIdx.y;
    const int4 q = ch[c];
    const double *v = V + i * ld;
    double s = 0.0;
    for (int e = threadIdx.x; e < q.y; e += blockDim.x) s += v[q.x + e] * w[q.x + e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int wv = 0; wv < static_cast<int>(blockDim.x >> 5); ++wv) t += red[wv];
        part[static_cast<int64_t>(i) * nch + c] = t;
    }
}

// h[s * SH + off + i] = sum of part[i][c] over the chunks of active system slot b
// (sch[b] = (system, first chunk, end chunk)); sqrt when do_sqrt
__global__ void k_seg_finish(const double *__restrict__ part, int k, int nch, const int4 *__restrict__ sch,
                             double *__restrict__ h, int SH, int off, int do_sqrt)
{
    const int4 q = sch[blockIdx.x];
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double s = 0.0;
        for (int c = q.y; c < q.z; ++c) s += part[static_cast<int64_t>(i) * nch + c];
        h[static_cast<int64_t>(q.x) * SH + off + i] = do_sqrt ? sqrt(s) : s;
    }
}

// w -= sum_{i<k} h[s SH + off + i] V_i  on active chunks
__global__ void k_seg_axpy(double *__restrict__ w, const double *__restrict__ V, int64_t ld,
                           const double *__restrict__ h, int SH, int off, int k,
                           const int4 *__restrict__ ch)
{
    const int4 q = ch[blockIdx.x];
    const double *hs = h + static_cast<int64_t>(q.z) * SH + off;
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < q.y; e += gridDim.y * blockDim.x) {
        const int64_t g = q.x + e;
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += hs[i] * V[i * ld + g];
        w[g] -= s;
    }
}

// out = in / h[s SH + off]  (0 if the norm is 0)
__global__ void k_seg_scale(const double *__restrict__ in, const double *__restrict__ h, int SH, int off,
                            double *__restrict__ out, const int4 *__restrict__ ch)
{
    const int4 q = ch[blockIdx.x];
    const double d = h[static_cast<int64_t>(q.z) * SH + off];
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < q.y; e += gridDim.y * blockDim.x)
        out[q.x + e] = d > 0.0 ? in[q.x + e] / d : 0.0;
}

// x += sum_{i < kk[s]} y[s SH + off + i] V_i
__global__ void k_seg_lincomb(double *__restrict__ x, const double *__restrict__ V, int64_t ld,
                              const double *__restrict__ h, int SH, int off, const int *__restrict__ kk,
                              const int4 *__restrict__ ch)
{
    const int4 q = ch[blockIdx.x];
    const double *ys = h + static_cast<int64_t>(q.z) * SH + off;
    const int k = kk[q.z];
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < q.y; e += gridDim.y * blockDim.x) {
        const int64_t g = q.x + e;
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += ys[i] * V[i * ld + g];
        x[g] += s;
    }
}

// mode 0: out = 0; 1: out = a; 2: out = a - b   (on active chunks)
__global__ void k_seg_set(double *__restrict__ out, const double *__restrict__ a,
                          const double *__restrict__ b, int mode, const int4 *__restrict__ ch)
{
    const int4 q = ch[blockIdx.x];
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < q.y; e += gridDim.y * blockDim.x) {
        const int64_t g = q.x + e;
        out[g] = mode == 0 ? 0.0 : (mode == 1 ? a[g] : a[g] - b[g]);
    }
}

// ------------------------------------------------ GMRES cycle as a CUDA graph
// With fs_options.use_graph = 1 a restart cycle of the (non-flexible) GMRES
// runs as ONE graph launch: a conditional WHILE node whose body is one
// iteration -- operator, CGS2, norm, scaling, and the Givens rotation of
// every system on the device, which also sets the loop condition (some
// system still running and the cycle not full).  The iteration index lives
// in device memory, so the body is the same graph for every iteration; the
// host synchronises once per cycle, not once per iteration.

// out = V_j on the active chunks, j = *jd
__global__ void k_copy_col_j(const double *__restrict__ V, int64_t ld, const int *__restrict__ jd,
                             double *__restrict__ out, const int4 *__restrict__ ch)
{
    const int4 q = ch[blockIdx.x];
    const double *v = V + static_cast<int64_t>(*jd) * ld;
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < q.y; e += gridDim.y * blockDim.x)
        out[q.x + e] = v[q.x + e];
}

// k_seg_dot for rows i <= *jd (the grid covers the cycle's largest row count)
__global__ void k_seg_dot_j(const double *__restrict__ V, int64_t ld, const double *__restrict__ w,
                            const int4 *__restrict__ ch, int nch, double *__restrict__ part,
                            const int *__restrict__ jd)
{
    const int c = blockIdx.x, i = blockIdx.y;
    if (i > *jd) return;
    __shared__ double red[8];
    const int4 q = ch[c];
    const double *v = V + i * ld;
    double s = 0.0;
    for (int e = threadIdx.x; e < q.y; e += blockDim.x) s += v[q.x + e] * w[q.x + e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int wv = 0; wv < static_cast<int>(blockDim.x >> 5); ++wv) t += red[wv];
        part[static_cast<int64_t>(i) * nch + c] = t;
    }
}

// k_seg_finish for rows i <= *jd
__global__ void k_seg_finish_j(const double *__restrict__ part, int nch, const int4 *__restrict__ sch,
                               double *__restrict__ h, int SH, int off, const int *__restrict__ jd)
{
    const int4 q = sch[blockIdx.x];
    const int k = *jd + 1;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double s = 0.0;
        for (int c = q.y; c < q.z; ++c) s += part[static_cast<int64_t>(i) * nch + c];
        h[static_cast<int64_t>(q.x) * SH + off + i] = s;
    }
}

// w -= sum_{i <= *jd} h[s SH + off + i] V_i
__global__ void k_seg_axpy_j(double *__restrict__ w, const double *__restrict__ V, int64_t ld,
                             const double *__restrict__ h, int SH, int off, const int4 *__restrict__ ch,
                             const int *__restrict__ jd)
{
    const int4 q = ch[blockIdx.x];
    const double *hs = h + static_cast<int64_t>(q.z) * SH + off;
    const int k = *jd + 1;
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < q.y; e += gridDim.y * blockDim.x) {
        const int64_t g = q.x + e;
        double s = 0.0;
        for (int i = 0; i < k; ++i) s += hs[i] * V[i * ld + g];
        w[g] -= s;
    }
}

// V_{j+1} = in / h[s SH + off] (0 if the norm is 0), j = *jd
__global__ void k_seg_scale_col_j(const double *__restrict__ in, const double *__restrict__ h, int SH, int off,
                                  double *__restrict__ V, int64_t ld, const int *__restrict__ jd,
                                  const int4 *__restrict__ ch)
{
    const int4 q = ch[blockIdx.x];
    const double d = h[static_cast<int64_t>(q.z) * SH + off];
    double *out = V + static_cast<int64_t>(*jd + 1) * ld;
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < q.y; e += gridDim.y * blockDim.x)
        out[q.x + e] = d > 0.0 ? in[q.x + e] / d : 0.0;
}

// Per-system Givens state of the device cycle.
struct GivensState {
    double *H;       // [S][R][R+1] rotated Hessenberg columns
    double *cs, *sn; // [S][R]
    double *g;       // [S][R+1]
    double *sc;      // [S][4]: beta, lim, res, rel
    int *st;         // [S][4]: its, kk, conv, done (done < 0: non-finite Arnoldi vector)
    int *jd;         // [1] iteration index of the cycle
    int R, max_iter;
};

// Cycle start for the systems of sch: g = (beta, 0, ...), kk = 0, running;
// beta from h[s SH + off_beta]; lim and its from the host (init[s] = lim, its).
__global__ void k_givens_init(GivensState G, const int4 *__restrict__ sch, int nsch,
                              const double *__restrict__ h, int SH, int off_beta, const double *__restrict__ init)
{
    for (int b = threadIdx.x; b < nsch; b += blockDim.x) {
        const int s = sch[b].x;
        double *g = G.g + static_cast<int64_t>(s) * (G.R + 1);
        for (int i = 0; i <= G.R; ++i) g[i] = 0.0;
        const double beta = h[static_cast<int64_t>(s) * SH + off_beta];
        g[0] = beta;
        G.sc[4 * s + 0] = beta;
        G.sc[4 * s + 1] = init[2 * s];
        G.sc[4 * s + 2] = beta;
        G.st[4 * s + 0] = static_cast<int>(init[2 * s + 1]);
        G.st[4 * s + 1] = 0;
        G.st[4 * s + 2] = 0;
        G.st[4 * s + 3] = 0;
    }
    if (threadIdx.x == 0) *G.jd = 0;
}

// Column j = *jd of every running system: the CGS2 coefficients (two passes)
// and the new norm, the earlier rotations, a new rotation, the residual
// estimate |g_{j+1}| and the convergence test; a system that converges, breaks
// down or reaches max_iter keeps its state from then on.  One block; sets the
// WHILE condition and advances *jd.
__global__ void __launch_bounds__(256) k_givens_step(GivensState G, const int4 *__restrict__ sch, int nsch,
                                                     const double *__restrict__ h, int SH, int hs,
                                                     cudaGraphConditionalHandle cond)
{
    const int j = *G.jd;
    int alive = 0;
    for (int b = threadIdx.x; b < nsch; b += blockDim.x) {
        const int s = sch[b].x;
        int *st = G.st + 4 * s;
        if (st[3]) continue;
        const double *hp = h + static_cast<int64_t>(s) * SH;
        double *hc = G.H + (static_cast<int64_t>(s) * G.R + j) * (G.R + 1);
        double *cs = G.cs + static_cast<int64_t>(s) * G.R, *sn = G.sn + static_cast<int64_t>(s) * G.R;
        double *g = G.g + static_cast<int64_t>(s) * (G.R + 1);
        for (int i = 0; i <= j; ++i) hc[i] = hp[i] + hp[hs + i];
        const double hn = hp[2 * hs];
        hc[j + 1] = hn;
        if (!isfinite(hn)) {
            st[3] = -1;
            continue;
        }
        for (int i = 0; i < j; ++i) {
            const double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
            hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
            hc[i] = t;
        }
        const double d = hypot(hc[j], hc[j + 1]);
        cs[j] = d > 0.0 ? hc[j] / d : 1.0;
        sn[j] = d > 0.0 ? hc[j + 1] / d : 0.0;
        hc[j] = d;
        hc[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        st[0] += 1;
        st[1] = j + 1;
        const double res = fabs(g[j + 1]);
        G.sc[4 * s + 2] = res;
        if (res <= G.sc[4 * s + 1]) {
            st[2] = 1;
            st[3] = 1;
        } else if (hn == 0.0 || st[0] >= G.max_iter) {
            st[3] = 1;
        } else {
            ++alive;
        }
    }
    __shared__ int red[8];
    for (int o = 16; o > 0; o >>= 1) alive += __shfl_xor_sync(0xffffffffu, alive, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = alive;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) tot += red[w];
        *G.jd = j + 1;
        cudaGraphSetConditional(cond, (tot > 0 && j + 1 < G.R) ? 1u : 0u);
    }
}

// y = H^-1 g (upper triangular, kk columns) per system of sch, into
// h[s SH + off_y + i]; kk[s] for the update x += V y.
__global__ void k_givens_backsub(GivensState G, const int4 *__restrict__ sch, int nsch, double *__restrict__ h,
                                 int SH, int off_y, int *__restrict__ kk)
{
    for (int b = threadIdx.x; b < nsch; b += blockDim.x) {
        const int s = sch[b].x;
        const int k = G.st[4 * s + 1];
        const double *H = G.H + static_cast<int64_t>(s) * G.R * (G.R + 1);
        const double *g = G.g + static_cast<int64_t>(s) * (G.R + 1);
        double *y = h + static_cast<int64_t>(s) * SH + off_y;
        for (int i = k - 1; i >= 0; --i) {
            double sum = g[i];
            for (int l = i + 1; l < k; ++l) sum -= H[static_cast<int64_t>(l) * (G.R + 1) + i] * y[l];
            const double dii = H[static_cast<int64_t>(i) * (G.R + 1) + i];
            y[i] = dii != 0.0 ? sum / dii : 0.0;
        }
        kk[s] = k;
    }
}

// ------------------------------------------------------ segmented GMRES (host)
struct SysState {
    double beta0 = 0.0, beta = 0.0, rel = 0.0, res = 0.0, lim = 0.0;
    int its = 0, inner = 0, kk = 0;
    bool conv = false, done = false;
    std::vector<double> H, cs, sn, g, y;
};

// One Krylov space: basis V [(R+1) x n], flexible directions Z [R x n],
// per-system scalars h [S x SH], reduction partials, work vectors, chunk lists.
struct Space {
    int R;
    double *V, *Z, *h, *part, *w, *r, *hpin;
    int4 *d_ch, *d_sch;
    int *d_kk;
    int nch = 0, nsch = 0;
};

Space inner_space(fs_ctx *c)
{
    return Space{c->kdim - 1, c->d_basis, nullptr, c->d_h, c->d_part, c->d_w, c->d_r, c->h_pinned,
                 c->d_ich, c->d_isch, c->d_ikk};
}

Space outer_space(fs_ctx *c)
{
    return Space{c->okdim - 1, c->d_obasis, c->d_oz, c->d_oh, c->d_opart, c->d_ow, c->d_or, c->oh_pinned,
                 c->d_och, c->d_osch, c->d_okk};
}

int SHof(const Space &sp) { return 4 * (sp.R + 1) + 8; }

// chunk lists of the given active systems
fs_status seg_build(fs_ctx *c, Space &sp, const std::vector<int> &act)
{
    std::vector<int4> ch, sch;
    for (int s : act) {
        const int64_t lo = c->sys_unk_ptr[s], hi = c->sys_unk_ptr[s + 1];
        const int first = static_cast<int>(ch.size());
        for (int64_t e = lo; e < hi; e += kChunk)
            ch.push_back(make_int4(static_cast<int>(e), static_cast<int>(std::min<int64_t>(kChunk, hi - e)), s, 0));
        sch.push_back(make_int4(s, first, static_cast<int>(ch.size()), 0));
    }
    if (static_cast<int64_t>(ch.size()) > c->chunk_cap || static_cast<int>(sch.size()) > c->S) {
        set_error("gmres: chunk list exceeds its capacity");
        return FS_EINVAL;
    }
    sp.nch = static_cast<int>(ch.size());
    sp.nsch = static_cast<int>(sch.size());
    if (sp.nch) {
        FS_CUDA(cudaMemcpyAsync(sp.d_ch, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream));
        FS_CUDA(cudaMemcpyAsync(sp.d_sch, sch.data(), sch.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                c->stream));
    }
    return FS_OK;
}

dim3 seg_grid(const Space &sp) { return dim3(static_cast<unsigned>(sp.nch), kChunk / 256); }

// h[s SH + off + i] = V_i . w  (i < k) for the active systems
fs_status seg_dots(fs_ctx *c, const Space &sp, const double *V, int64_t ld, int k, const double *w, int off,
                   bool do_sqrt)
{
    if (!sp.nch) return FS_OK;
    k_seg_dot<<<dim3(sp.nch, k), 256, 0, c->stream>>>(V, ld, w, sp.d_ch, sp.nch, sp.part);
    FS_LAUNCH_CHECK();
    k_seg_finish<<<sp.nsch, 128, 0, c->stream>>>(sp.part, k, sp.nch, sp.d_sch, sp.h, SHof(sp), off,
                                                  do_sqrt ? 1 : 0);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status seg_set(fs_ctx *c, const Space &sp, double *out, const double *a, const double *b, int mode)
{
    if (!sp.nch) return FS_OK;
    k_seg_set<<<seg_grid(sp), 256, 0, c->stream>>>(out, a, b, mode, sp.d_ch);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

fs_status fetch_h(fs_ctx *c, const Space &sp)
{
    FS_CUDA(cudaMemcpyAsync(sp.hpin, sp.h, static_cast<size_t>(c->S) * SHof(sp) * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

// Far field at the fiber nodes for the active systems (each target block sums
// its own system's sources only): ubar = (1/8 pi mu) sum_{other fibers} G0 W f
// Direct-sum arguments of the fiber far field (groups: the per-system work
// list's groups when the systems are summed separately).
PairSumArgs far_field_args(fs_ctx *c, int sum_prec, bool hilo, const std::vector<int> *act,
                           std::vector<int4> &groups)
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
    if (a.shape_override == 0 && c->opt.autotune) a.shape_override = c->tuned[2 * sum_prec + (hilo ? 1 : 0)];
    double pairs = 0.0;
    groups.clear();
    if ((c->S > 1 || c->worklist) && act) {
        for (int s : *act) {
            const int lo = static_cast<int>(c->sys_node_ptr[s]), hi = static_cast<int>(c->sys_node_ptr[s + 1]);
            groups.push_back(make_int4(lo, hi, lo, hi));
            pairs += double(hi - lo) * double(hi - lo) - c->sys_self_pairs[s];
        }
        a.groups = &groups;
        a.work_dev = c->d_work;
        a.work_cap = c->work_cap;
    } else {
        for (int s = 0; s < c->S; ++s) pairs += double(c->sys_node_ptr[s + 1] - c->sys_node_ptr[s]) *
                                                double(c->sys_node_ptr[s + 1] - c->sys_node_ptr[s]) -
                                                c->sys_self_pairs[s];
    }
    a.pairs = pairs;
    // event records cannot sit in a graph's loop body
    a.prof = (c->opt.profile && !c->capturing) ? &c->prof : nullptr;
    a.work_uploaded = c->capturing;
    return a;
}

// The autotuner: the far field of `a` once untimed and once timed (CUDA
// events on the context's stream) in every launch shape 1..3; *shape = the
// fastest.  Each run overwrites a.out (the caller's sum then writes the
// result), and none is recorded in the kernel profile.  Synchronises the
// stream once per shape.
fs_status tune_far_field(fs_ctx *c, PairSumArgs a, int *shape)
{
    a.prof = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FS_CUDA(cudaEventCreate(&e0));
    const cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        FS_CUDA(ce);
    }
    float best = 0.0f;
    fs_status st = FS_OK;
    for (int s = 1; s <= 3 && st == FS_OK; ++s) {
        a.shape_override = s;
        st = c->scratch.reserve(pairsum_scratch_bytes(a.kind, a.n_src, a.n_tgt, a.sum_prec, s), c->stream);
        if (st == FS_OK) st = pairsum(a, c->scratch.ptr, c->scratch.bytes, c->d_status, c->stream);
        if (st != FS_OK) break;
        float ms = 0.0f;
        if (cudaEventRecord(e0, c->stream) != cudaSuccess ||
            (st = pairsum(a, c->scratch.ptr, c->scratch.bytes, c->d_status, c->stream)) != FS_OK ||
            cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            if (st == FS_OK) {
                set_error("autotune: event timing failed: %s", cudaGetErrorString(cudaGetLastError()));
                st = FS_ECUDA;
            }
            break;
        }
        if (*shape == 0 || ms < best) {
            best = ms;
            *shape = s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FS_OK) *shape = 0;
    return st;
}

// Far field at the fiber nodes for the active systems (each target block sums
// its own system's sources only): ubar = (1/8 pi mu) sum_{other fibers} G0 W f
fs_status far_field(fs_ctx *c, int sum_prec, bool hilo, const std::vector<int> *act)
{
    if (c->opt.tree_order > 0) {
        // fast summation: the treecode at the chosen order, whatever the precision
        c->pairs_last += c->n_tot * c->n_tot;
        return tree_sum(c, c->d_X, c->d_wf, c->n_tot, nullptr, c->d_X, nullptr, c->n_tot, c->d_ubar,
                        c->opt.tree_order, c->opt.tree_theta, c->d_excl);
    }
    std::vector<int4> groups;
    PairSumArgs a = far_field_args(c, sum_prec, hilo, act, groups);
    if (a.shape_override == 0 && c->opt.autotune && !c->capturing) {
        // this class's first sum: time the shapes, keep the fastest
        int &shape = c->tuned[2 * sum_prec + (hilo ? 1 : 0)];
        FS_TRY(tune_far_field(c, a, &shape));
        a.shape_override = shape;
    }
    FS_TRY(c->scratch.reserve(pairsum_scratch_bytes(a.kind, a.n_src, a.n_tgt, sum_prec, a.shape_override),
                              c->stream));
    FS_TRY(pairsum(a, c->scratch.ptr, c->scratch.bytes, c->d_status, c->stream));
    c->pairs_last += static_cast<int64_t>(a.pairs);
    return FS_OK;
}

// Before a graph capture: the far field's scratch reserved and its work list
// (if any) uploaded, so that the captured sums neither allocate nor copy from
// the host; *items = the work list's length (0: one stream-K sum).
fs_status prepare_far_field(fs_ctx *c, int sum_prec, bool hilo, const std::vector<int> *act, int64_t *items)
{
    std::vector<int4> groups;
    PairSumArgs a = far_field_args(c, sum_prec, hilo, act, groups);
    a.work_uploaded = false;
    FS_TRY(c->scratch.reserve(pairsum_scratch_bytes(a.kind, a.n_src, a.n_tgt, sum_prec, a.shape_override),
                              c->stream));
    return pairsum_work_list(a, c->stream, items);
}

// Preconditioned operator of Eq. prec, out = P^-1 A v, evaluated as
//   fibers : v + P^-1 (A - P) v  -- P is exactly the self block, so only the
//            coupling rows Rw(ubar) (and an attached end's terms in the body's
//            U, Omega) pass through the block solves (the block's own
//            rounding is never amplified by its inverse, cond ~1e9);
//   surface: D^-1 (S q + fiber Stokeslets)  -- D the Jacobi diagonal (with a
//            body: its rows, Stokeslet and rotlet, and constraint rows).
// sum_prec selects the far-field arithmetic; act restricts the far field to
// those systems (results of other systems are not meaningful).
fs_status apply_pa(fs_ctx *c, const double *v, double *out, int sum_prec, const std::vector<int> *act,
                   bool hilo = false)
{
    FS_TRY(launch_force(c, v, c->d_f, c->d_wf));
    FS_TRY(body_load(c, v, LOAD_LIN));
    FS_TRY(far_field(c, sum_prec, hilo, act));
    const double *q = c->surf.n ? v + c->n_fib_unk : nullptr;
    if (c->surf.n) FS_TRY(surface_couplings(c, q, c->d_ubar, sum_prec, hilo));
    FS_TRY(launch_rows(c, nullptr, c->d_f, c->d_ubar, c->d_e, ROWS_COUPLING));
    FS_TRY(body_rigid_rows(c, v, c->d_e, 1.0));
    FS_TRY(launch_lu_solve(c, c->d_e, out));
    if (c->n_fib_unk) {
        k_add<<<blocks_for(c->n_fib_unk), 256, 0, c->stream>>>(out, v, c->n_fib_unk);
        FS_LAUNCH_CHECK();
    }
    if (c->surf.n) {
        FS_TRY(surface_rows(c, q, c->d_usurf, c->d_e + c->n_fib_unk, false, sum_prec, hilo));
        FS_TRY(surface_precond(c, c->d_e + c->n_fib_unk, out + c->n_fib_unk));
    }
    return FS_OK;
}

// Inexact-Krylov relaxation (mixed precision): an operator error of relative
// size eta on a correction taken when the residual is r adds at most about
// eta |r| to the final residual, so once eta |r| <= kRelaxShare tol |P^-1 b|
// an FP32 far field is accurate enough for the rest of the solve.  Bounds of
// the relative error: hi/lo coordinates kEtaFP32 (measured ~3e-7), plain
// coordinates kEtaFP32Plain (measured ~3e-6 over a whole sum; the bound
// allows for the nearest pairs, whose rounding is relative to their distance).
constexpr double kEtaFP32 = 1e-6;
constexpr double kEtaFP32Plain = 1e-4;
constexpr double kRelaxShare = 0.05;

// Far-field arithmetic of the accurate sums (right-hand side, outer operator):
// FP64 on the plain FP64 path, float-float on the mixed path.
int accurate_prec(const fs_ctx *c) { return c->opt.prec == FS_FP64 ? FS_SUM_FP64 : FS_SUM_FF; }

// b (Eq. sche-linear-eq right-hand side), then pb = P^-1 b; far field in
// `ap` arithmetic (the accurate one by default)
fs_status rhs(fs_ctx *c, double *b, double *pb, int ap = -1, bool hilo = false)
{
    if (ap < 0) ap = accurate_prec(c);
    FS_TRY(launch_force(c, nullptr, c->d_f, c->d_wf));
    FS_TRY(body_load(c, nullptr, LOAD_KNOWN));
    FS_TRY(far_field(c, ap, hilo, &c->all_sys));
    if (c->surf.n) FS_TRY(surface_couplings(c, nullptr, c->d_ubar, ap, hilo));
    FS_TRY(launch_rows(c, nullptr, c->d_f, c->d_ubar, b, ROWS_RHS));
    if (c->surf.n) FS_TRY(surface_rows(c, nullptr, c->d_usurf, b + c->n_fib_unk, true, ap, hilo));
    FS_TRY(launch_lu_solve(c, b, pb));
    if (c->surf.n) FS_TRY(surface_precond(c, b + c->n_fib_unk, pb + c->n_fib_unk));
    return FS_OK;
}

__global__ void k_sub(double *__restrict__ out, const double *__restrict__ v, int64_t n)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) out[i] -= v[i];
}

__global__ void k_negate(double *__restrict__ v, int64_t n)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) v[i] = -v[i];
}

// Preconditioned residual r = P^-1 b - (P^-1 A) x with ONE set of far
// fields: the couplings of the known force and of x's force are the fields of
// the sum of the two densities (they are linear in the density), so
//   fibers : r = P^-1 rows_rhs(f_known, ubar[W (f_known + f(x))] + T[q]) - x,
//   surface: r = -D^-1 (S q + G[W (f_known + f(x))]),
// q the surface density part of x; the body's Stokeslet and rotlet carry the
// known plus the linear end loads, and the attached ends' rigid terms of x
// are subtracted from their rows.
fs_status true_residual(fs_ctx *c, const double *x, double *r, int sum_prec)
{
    FS_TRY(launch_force(c, x, c->d_f, c->d_wf, true));
    FS_TRY(body_load(c, x, LOAD_BOTH));
    FS_TRY(far_field(c, sum_prec, false, &c->all_sys));
    const double *q = c->surf.n ? x + c->n_fib_unk : nullptr;
    if (c->surf.n) FS_TRY(surface_couplings(c, q, c->d_ubar, sum_prec, false));
    FS_TRY(launch_rows(c, nullptr, c->d_f, c->d_ubar, c->d_e, ROWS_RHS));
    FS_TRY(body_rigid_rows(c, x, c->d_e, -1.0));
    FS_TRY(launch_lu_solve(c, c->d_e, r));
    if (c->n_fib_unk) {
        k_sub<<<blocks_for(c->n_fib_unk), 256, 0, c->stream>>>(r, x, c->n_fib_unk);
        FS_LAUNCH_CHECK();
    }
    if (c->surf.n) {
        const int64_t n3 = c->n_surf_unk;
        FS_TRY(surface_rows(c, q, c->d_usurf, c->d_e + c->n_fib_unk, false, sum_prec, false));
        FS_TRY(surface_precond(c, c->d_e + c->n_fib_unk, r + c->n_fib_unk));
        k_negate<<<blocks_for(n3), 256, 0, c->stream>>>(r + c->n_fib_unk, n3);
        FS_LAUNCH_CHECK();
    }
    return FS_OK;
}

GivensState givens_state(fs_ctx *c)
{
    GivensState G;
    G.H = c->d_gH;
    G.cs = c->d_gcs;
    G.sn = c->d_gsn;
    G.g = c->d_gg;
    G.sc = c->d_gsc;
    G.st = c->d_gst;
    G.jd = c->d_gj;
    G.R = c->kdim - 1;
    G.max_iter = c->opt.max_iter;
    return G;
}

// One iteration of the cycle's body (the WHILE node), enqueued on the
// capturing stream: V_j -> operator -> CGS2 -> norm -> V_{j+1} -> Givens.
fs_status cycle_body(fs_ctx *c, Space &sp, const std::vector<int> &act, int sum_prec, bool hilo,
                     cudaGraphConditionalHandle cond)
{
    const int64_t n = c->n_unk;
    const int R = sp.R, hs = R + 1, SH = SHof(sp);
    const int *jd = c->d_gj;
    k_copy_col_j<<<seg_grid(sp), 256, 0, c->stream>>>(sp.V, n, jd, c->d_vcur, sp.d_ch);
    FS_LAUNCH_CHECK();
    FS_TRY(apply_pa(c, c->d_vcur, sp.w, sum_prec, &act, hilo));
    for (int pass = 0; pass < 2; ++pass) {   // CGS2
        const int off = pass ? hs : 0;
        k_seg_dot_j<<<dim3(sp.nch, R + 1), 256, 0, c->stream>>>(sp.V, n, sp.w, sp.d_ch, sp.nch, sp.part, jd);
        FS_LAUNCH_CHECK();
        k_seg_finish_j<<<sp.nsch, 128, 0, c->stream>>>(sp.part, sp.nch, sp.d_sch, sp.h, SH, off, jd);
        FS_LAUNCH_CHECK();
        k_seg_axpy_j<<<seg_grid(sp), 256, 0, c->stream>>>(sp.w, sp.V, n, sp.h, SH, off, sp.d_ch, jd);
        FS_LAUNCH_CHECK();
    }
    FS_TRY(seg_dots(c, sp, sp.w, 0, 1, sp.w, 2 * hs, true));
    k_seg_scale_col_j<<<seg_grid(sp), 256, 0, c->stream>>>(sp.w, sp.h, SH, 2 * hs, sp.V, n, jd, sp.d_ch);
    FS_LAUNCH_CHECK();
    k_givens_step<<<1, 256, 0, c->stream>>>(givens_state(c), sp.d_sch, sp.nsch, sp.h, SH, hs, cond);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

// One restart cycle of the inner GMRES as a CUDA graph (the chunk lists of
// `act` are on the device and V_0 is set): per-system start values, ONE
// launch of the graph whose WHILE node iterates until every system of the
// cycle has converged, stopped or filled the cycle, the back substitution
// y = H^-1 g per system, and one read of the systems' states.  Graphs are
// cached per launch shape (precision, chunk and work-list counts); the lists'
// contents are read at run time, so one graph serves every cycle of a shape.
fs_status cycle_graph(fs_ctx *c, Space &sp, const std::vector<int> &act, int sum_prec, bool hilo, int max_iter,
                      std::vector<SysState> &st)
{
    const int R = sp.R, hs = R + 1, SH = SHof(sp);
    // start values: lim and its per system
    for (int s : act) {
        c->h_ginit[2 * s] = st[s].lim;
        c->h_ginit[2 * s + 1] = st[s].its;
    }
    FS_CUDA(cudaMemcpyAsync(c->d_ginit, c->h_ginit, 2 * static_cast<size_t>(c->S) * sizeof(double),
                            cudaMemcpyHostToDevice, c->stream));
    GivensState G = givens_state(c);
    G.max_iter = max_iter;
    k_givens_init<<<1, 256, 0, c->stream>>>(G, sp.d_sch, sp.nsch, sp.h, SH, 2 * hs + 2, c->d_ginit);
    FS_LAUNCH_CHECK();
    // the far field's work list and scratch are set up before capture
    int64_t items = 0;
    FS_TRY(prepare_far_field(c, sum_prec, hilo, &act, &items));
    CycleGraph *cg = nullptr;
    for (CycleGraph &g : c->graphs)
        if (g.prec == sum_prec && g.hilo == hilo && g.nch == sp.nch && g.nsch == sp.nsch && g.items == items &&
            g.max_iter == max_iter)
            cg = &g;
    if (!cg) {
        CycleGraph g;
        g.prec = sum_prec;
        g.hilo = hilo;
        g.nch = sp.nch;
        g.nsch = sp.nsch;
        g.items = items;
        g.max_iter = max_iter;
        FS_CUDA(cudaGraphCreate(&g.graph, 0));
        cudaGraphConditionalHandle cond;
        FS_CUDA(cudaGraphConditionalHandleCreate(&cond, g.graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        FS_CUDA(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        // body kernels (G.max_iter is a kernel argument: part of the key)
        const int saved_iter = c->opt.max_iter;
        c->opt.max_iter = max_iter;
        const uint64_t l0 = g_launches;
        // capture on a stream of its own (the context's stream may be the
        // legacy default stream, which cannot capture); the graph itself is
        // launched on the context's stream
        if (!c->cap_stream) FS_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        FS_CUDA(cudaStreamSynchronize(c->stream));
        cudaStream_t own = c->stream;
        c->stream = c->cap_stream;
        const cudaError_t be =
            cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        fs_status bs = FS_ECUDA;
        cudaGraph_t got = nullptr;
        cudaError_t ce = be;
        if (be == cudaSuccess) {
            c->capturing = true;
            bs = cycle_body(c, sp, act, sum_prec, hilo, cond);
            c->capturing = false;
            ce = cudaStreamEndCapture(c->stream, &got);
        } else {
            set_error("gmres: cannot begin a graph capture: %s", cudaGetErrorString(be));
        }
        c->stream = own;
        c->opt.max_iter = saved_iter;
        if (bs != FS_OK) {
            cudaGraphDestroy(g.graph);
            return bs;
        }
        if (ce != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g.graph);
            set_error("gmres: graph capture failed: %s", cudaGetErrorString(ce));
            return FS_ECUDA;
        }
        g.body_launches = g_launches - l0;
        __atomic_sub_fetch(&g_launches, g.body_launches, __ATOMIC_RELAXED);   // counted per iteration below
        FS_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
        c->graphs.push_back(g);
        cg = &c->graphs.back();
    }
    FS_CUDA(cudaGraphLaunch(cg->exec, c->stream));
    k_givens_backsub<<<1, 256, 0, c->stream>>>(G, sp.d_sch, sp.nsch, sp.h, SH, 3 * hs + 4, sp.d_kk);
    FS_LAUNCH_CHECK();
    // the systems' states (and the iterations the loop ran) back to the host
    FS_CUDA(cudaMemcpyAsync(c->h_gst, c->d_gst, 4 * static_cast<size_t>(c->S) * sizeof(int), cudaMemcpyDeviceToHost,
                            c->stream));
    FS_CUDA(cudaMemcpyAsync(c->h_gsc, c->d_gsc, 4 * static_cast<size_t>(c->S) * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->h_gj, c->d_gj, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    __atomic_add_fetch(&g_launches, cg->body_launches * static_cast<uint64_t>(*c->h_gj), __ATOMIC_RELAXED);
    for (int s : act) {
        SysState &q = st[s];
        const int *gs = c->h_gst + 4 * s;
        if (gs[3] < 0) {
            set_error("gmres: non-finite Arnoldi vector (system %d)", s);
            return FS_ENUMERIC;
        }
        q.its = gs[0];
        q.kk = gs[1];
        q.conv = gs[2] != 0;
        q.done = gs[3] != 0 || q.its >= max_iter;
        q.res = c->h_gsc[4 * s + 2];
        q.rel = q.beta0 > 0.0 ? q.res / q.beta0 : 0.0;
    }
    return FS_OK;
}

// Restarted GMRES for (P^-1 A) x = pb, x0 = 0, on each system in `want`
// independently (lockstep: one operator application per iteration for all
// running systems), CGS2 and Givens rotations per system; x overwritten on
// those systems.  With inner_prec >= 0 each direction is z_j = an inner GMRES
// solve of (P^-1 A_inner) z = v_j to inner_tol and x = Z y (flexible GMRES).
fs_status gmres_seg(fs_ctx *c, Space &sp, const double *pb, double *x, double tol, int max_iter,
                    int sum_prec, int inner_prec, double inner_tol, const std::vector<int> &want,
                    std::vector<SysState> &st, bool hilo = false, const std::vector<double> *tol_abs = nullptr,
                    double partial_rel = 0.0)
{
    const int64_t n = c->n_unk;
    const int R = sp.R, hs = R + 1, SH = SHof(sp);
    const bool flexible = inner_prec >= 0;
    // device cycles: the inner Krylov space, direct far fields, no event
    // records (a graph's body holds kernels, copies and memsets only)
    const bool graph = c->opt.use_graph && !flexible && sp.V == c->d_basis && c->d_gH && !c->opt.profile &&
                       c->opt.tree_order == 0 && partial_rel == 0.0;
    double *V = sp.V;
    st.assign(c->S, SysState());
    std::vector<int> act = want;
    FS_TRY(seg_build(c, sp, act));
    FS_TRY(seg_set(c, sp, x, nullptr, nullptr, 0));
    FS_TRY(seg_set(c, sp, sp.r, pb, nullptr, 1));
    FS_TRY(seg_dots(c, sp, sp.r, 0, 1, sp.r, 2 * hs + 2, true));
    FS_TRY(fetch_h(c, sp));
    {
        std::vector<int> keep;
        for (int s : act) {
            SysState &q = st[s];
            q.beta0 = q.beta = sp.hpin[static_cast<int64_t>(s) * SH + 2 * hs + 2];
            if (!std::isfinite(q.beta0)) {
                set_error("gmres: non-finite right-hand side (system %d)", s);
                return FS_ENUMERIC;
            }
            // converged when |residual| <= lim (tol |pb| unless given per system)
            q.lim = tol_abs ? (*tol_abs)[s] : tol * q.beta0;
            // a correction too large for this operator's accuracy to finish the
            // solve is only taken part of the way (another true residual follows)
            if (partial_rel > 0.0 && (hilo ? kEtaFP32 : kEtaFP32Plain) * q.beta0 > kRelaxShare * q.lim)
                q.lim = std::max(q.lim, partial_rel * q.beta0);
            q.res = q.beta0;
            if (!(q.beta0 > 0.0) || q.beta0 <= q.lim) {
                q.conv = q.done = true;
                continue;
            }
            q.H.assign(static_cast<size_t>(R + 1) * R, 0.0);
            q.cs.assign(R, 0.0);
            q.sn.assign(R, 0.0);
            q.g.assign(R + 1, 0.0);
            q.y.assign(R, 0.0);
            keep.push_back(s);
        }
        act.swap(keep);
    }
    while (!act.empty()) {
        FS_TRY(seg_build(c, sp, act));
        k_seg_scale<<<seg_grid(sp), 256, 0, c->stream>>>(sp.r, sp.h, SH, 2 * hs + 2, V, sp.d_ch);
        FS_LAUNCH_CHECK();
        if (graph) {
            // the whole cycle on the device: one graph launch, one synchronisation
            FS_TRY(cycle_graph(c, sp, act, sum_prec, hilo, max_iter, st));
        } else {
        for (int s : act) {
            SysState &q = st[s];
            std::fill(q.g.begin(), q.g.end(), 0.0);
            q.g[0] = q.beta;
            q.kk = 0;
        }
        std::vector<int> running = act;
        for (int j = 0; j < R && !running.empty(); ++j) {
            double *Vj = V + j * n, *Vn = V + (j + 1) * n;
            if (flexible) {
                double *Zj = sp.Z + j * n;
                Space isp = inner_space(c);
                std::vector<SysState> ist;
                FS_TRY(gmres_seg(c, isp, Vj, Zj, inner_tol, c->opt.max_iter, inner_prec, -1, 0.0, running, ist));
                for (int s : running) st[s].inner += ist[s].its;
                FS_TRY(apply_pa(c, Zj, sp.w, sum_prec, &running));
            } else {
                FS_TRY(apply_pa(c, Vj, sp.w, sum_prec, &running, hilo));
            }
            for (int pass = 0; pass < 2; ++pass) {   // CGS2
                const int off = pass ? hs : 0;
                FS_TRY(seg_dots(c, sp, V, n, j + 1, sp.w, off, false));
                k_seg_axpy<<<seg_grid(sp), 256, 0, c->stream>>>(sp.w, V, n, sp.h, SH, off, j + 1, sp.d_ch);
                FS_LAUNCH_CHECK();
            }
            FS_TRY(seg_dots(c, sp, sp.w, 0, 1, sp.w, 2 * hs, true));
            k_seg_scale<<<seg_grid(sp), 256, 0, c->stream>>>(sp.w, sp.h, SH, 2 * hs, Vn, sp.d_ch);
            FS_LAUNCH_CHECK();
            FS_TRY(fetch_h(c, sp));
            std::vector<int> still;
            for (int s : running) {
                SysState &q = st[s];
                const double *hp = sp.hpin + static_cast<int64_t>(s) * SH;
                double *hc = &q.H[static_cast<size_t>(j) * (R + 1)];
                for (int i = 0; i <= j; ++i) hc[i] = hp[i] + hp[hs + i];
                const double hn = hp[2 * hs];
                hc[j + 1] = hn;
                if (!std::isfinite(hn)) {
                    set_error("gmres: non-finite Arnoldi vector (system %d)", s);
                    return FS_ENUMERIC;
                }
                for (int i = 0; i < j; ++i) {
                    const double t = q.cs[i] * hc[i] + q.sn[i] * hc[i + 1];
                    hc[i + 1] = -q.sn[i] * hc[i] + q.cs[i] * hc[i + 1];
                    hc[i] = t;
                }
                const double d = std::hypot(hc[j], hc[j + 1]);
                q.cs[j] = d > 0.0 ? hc[j] / d : 1.0;
                q.sn[j] = d > 0.0 ? hc[j + 1] / d : 0.0;
                hc[j] = d;
                hc[j + 1] = 0.0;
                q.g[j + 1] = -q.sn[j] * q.g[j];
                q.g[j] = q.cs[j] * q.g[j];
                ++q.its;
                q.kk = j + 1;
                q.res = std::fabs(q.g[j + 1]);
                q.rel = q.res / q.beta0;
                if (q.res <= q.lim) {
                    q.conv = q.done = true;
                } else if (hn == 0.0 || q.its >= max_iter) {
                    q.done = true;
                } else {
                    still.push_back(s);
                }
            }
            if (still.size() != running.size()) {
                running.swap(still);
                if (!running.empty()) FS_TRY(seg_build(c, sp, running));
            }
        }
        // y = H^-1 g per system; x += (V or Z) y on the systems of this cycle
        std::vector<int> kk(c->S, 0);
        for (int s : act) {
            SysState &q = st[s];
            const int k = q.kk;
            for (int i = k - 1; i >= 0; --i) {
                double sum = q.g[i];
                for (int l = i + 1; l < k; ++l) sum -= q.H[static_cast<size_t>(l) * (R + 1) + i] * q.y[l];
                const double dii = q.H[static_cast<size_t>(i) * (R + 1) + i];
                q.y[i] = dii != 0.0 ? sum / dii : 0.0;
            }
            kk[s] = k;
            std::memcpy(sp.hpin + static_cast<int64_t>(s) * SH + 3 * hs + 4, q.y.data(), k * sizeof(double));
        }
        FS_CUDA(cudaMemcpyAsync(sp.h, sp.hpin, static_cast<size_t>(c->S) * SH * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream));
        FS_CUDA(cudaMemcpyAsync(sp.d_kk, kk.data(), c->S * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        FS_TRY(seg_build(c, sp, act));
        k_seg_lincomb<<<seg_grid(sp), 256, 0, c->stream>>>(x, flexible ? sp.Z : V, n, sp.h, SH, 3 * hs + 4,
                                                           sp.d_kk, sp.d_ch);
        FS_LAUNCH_CHECK();
        FS_CUDA(cudaStreamSynchronize(c->stream));   // hpin and kk are reused below
        }
        if (graph) {
            k_seg_lincomb<<<seg_grid(sp), 256, 0, c->stream>>>(x, V, n, sp.h, SH, 3 * hs + 4, sp.d_kk, sp.d_ch);
            FS_LAUNCH_CHECK();
        }
        std::vector<int> again;
        for (int s : act)
            if (!st[s].done) again.push_back(s);
        if (again.empty()) break;
        // restart: r = pb - P^-1 A x on the systems that continue
        act.swap(again);
        FS_TRY(seg_build(c, sp, act));
        FS_TRY(apply_pa(c, x, sp.w, sum_prec, &act, hilo));
        FS_TRY(seg_set(c, sp, sp.r, pb, sp.w, 2));
        FS_TRY(seg_dots(c, sp, sp.r, 0, 1, sp.r, 2 * hs + 2, true));
        FS_TRY(fetch_h(c, sp));
        std::vector<int> keep;
        for (int s : act) {
            SysState &q = st[s];
            q.beta = sp.hpin[static_cast<int64_t>(s) * SH + 2 * hs + 2];
            q.res = q.beta;
            q.rel = q.beta / q.beta0;
            if (q.res <= q.lim) q.conv = q.done = true;
            else keep.push_back(s);
        }
        act.swap(keep);
    }
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

fs_status fiber_arrays(fs_ctx *c, int M, const int32_t *ppf, const std::vector<int64_t> &kp,
                       const std::vector<int64_t> &zp);
fs_status krylov_arrays(fs_ctx *c);
fs_status surface_arrays(fs_ctx *c, const fs_boundary *bd, const fs_body *body);

fs_status context_init(fs_ctx *c, int S, const int32_t *fps, int M, const int32_t *ppf,
                       const fs_boundary *bd, const fs_body *body, const int32_t *minus_end)
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
    c->surf.n_per = bd ? bd->n_nodes : 0;
    c->body.on = body != nullptr;
    c->body.n = body ? body->n_nodes : 0;
    c->surf.n = c->surf.n_per + c->body.n;
    c->n_surf_unk = 3 * int64_t(c->surf.n) + (c->body.on ? 6 : 0);
    c->n_unk = c->n_fib_unk + c->n_surf_unk;
    if (c->n_tot >= (1LL << 31) - 1 || c->n_unk >= (1LL << 31) - 1) {
        set_error("fs_create: at most 2^31-2 points and unknowns");
        return FS_EINVAL;
    }
    // independent systems: consecutive fiber ranges
    c->S = std::max(1, S);
    c->sys_fib_ptr.assign(c->S + 1, 0);
    if (S >= 1 && fps) {
        for (int s = 0; s < S; ++s) c->sys_fib_ptr[s + 1] = c->sys_fib_ptr[s] + fps[s];
        if (c->sys_fib_ptr[S] != M) {
            set_error("fs_create_batch: fibers per system sum to %d, not %d", c->sys_fib_ptr[S], M);
            return FS_EINVAL;
        }
    } else {
        c->sys_fib_ptr[1] = M;
    }
    c->sys_node_ptr.assign(c->S + 1, 0);
    c->sys_unk_ptr.assign(c->S + 1, 0);
    c->sys_self_pairs.assign(c->S, 0.0);
    c->all_sys.resize(c->S);
    for (int s = 0; s < c->S; ++s) {
        c->all_sys[s] = s;
        c->sys_node_ptr[s + 1] = c->node_ptr[c->sys_fib_ptr[s + 1]];
        c->sys_unk_ptr[s + 1] = c->unk_ptr[c->sys_fib_ptr[s + 1]];
        for (int m = c->sys_fib_ptr[s]; m < c->sys_fib_ptr[s + 1]; ++m)
            c->sys_self_pairs[s] += double(ppf[m]) * double(ppf[m]);
    }
    c->sys_unk_ptr[c->S] = c->n_unk;   // the periphery unknowns belong to the (single) system
    c->sys_iters.assign(c->S, 0);
    c->sys_outer.assign(c->S, 0);
    c->sys_resid.assign(c->S, 0.0);
    c->sys_conv.assign(c->S, 0);
    FS_TRY(dalloc(c, &c->d_status, 1));
    FS_CUDA(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    FS_TRY(pinned_alloc(c, &c->h_pinned, 4096));
    if (M == 0 && !c->body.on) return FS_OK;
    if (M > 0) FS_TRY(fiber_arrays(c, M, ppf, kp, zp));
    if (c->body.on) {
        std::vector<int> att(M, FS_END_FREE), list;
        for (int m = 0; m < M; ++m) {
            att[m] = minus_end ? minus_end[m] : FS_END_FREE;
            if (att[m] != FS_END_FREE) list.push_back(m);
        }
        c->body.n_att = static_cast<int>(list.size());
        c->body.radius = body->radius;
        double area = 0.0;
        for (int i = 0; i < body->n_nodes; ++i) area += body->weights[i];
        std::vector<double> rb(kRbSize, 0.0);
        for (int a = 0; a < 3; ++a) {
            rb[kRbCenter + a] = body->center[a];
            rb[kRbFext + a] = body->force[a];
            rb[kRbLext + a] = body->torque[a];
        }
        rb[kRbArea] = area;
        FS_TRY(dalloc(c, &c->body.rb, kRbSize));
        FS_TRY(dalloc(c, &c->body.attach, M));
        FS_TRY(dalloc(c, &c->body.att_list, list.size()));
        FS_CUDA(cudaMemcpyAsync(c->body.rb, rb.data(), kRbSize * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        if (M > 0)
            FS_CUDA(cudaMemcpyAsync(c->body.attach, att.data(), M * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        if (!list.empty())
            FS_CUDA(cudaMemcpyAsync(c->body.att_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    c->stream));
        FS_CUDA(cudaStreamSynchronize(c->stream));   // host staging vectors
        if (M == 0) c->have_state = true;   // a lone body needs no fiber state
    }
    FS_TRY(krylov_arrays(c));
    FS_TRY(surface_arrays(c, bd, body));
    // host staging vectors above go out of scope here; the context's stream
    // may be a non-blocking one that other contexts share the device with
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

// Fiber arrays of context_init: op sets, pointers, geometry and block storage.
fs_status fiber_arrays(fs_ctx *c, int M, const int32_t *ppf, const std::vector<int64_t> &kp,
                       const std::vector<int64_t> &zp)
{
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

    FS_TRY(dalloc(c, &c->d_N, M));
    FS_TRY(dalloc(c, &c->d_node_ptr, M + 1));
    FS_TRY(dalloc(c, &c->d_unk_ptr, M + 1));
    FS_TRY(dalloc(c, &c->d_blk_ptr, M + 1));
    FS_TRY(dalloc(c, &c->d_kp_ptr, M + 1));
    FS_TRY(dalloc(c, &c->d_z_ptr, M + 1));
    FS_TRY(dalloc(c, &c->d_ops_off, M));
    FS_TRY(dalloc(c, &c->d_ops, ops.size()));
    FS_TRY(dalloc(c, &c->d_excl, c->n_tot));
    FS_CUDA(cudaMemcpyAsync(c->d_N, ppf, M * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_node_ptr, c->node_ptr.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_unk_ptr, c->unk_ptr.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_blk_ptr, c->blk_ptr.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_kp_ptr, kp.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_z_ptr, zp.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_ops_off, off.data(), M * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_ops, ops.data(), ops.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaMemcpyAsync(c->d_excl, excl.data(), c->n_tot * sizeof(int2), cudaMemcpyHostToDevice, c->stream));

    const int64_t P = c->n_tot;
    FS_TRY(dalloc(c, &c->d_X, 3 * P));
    FS_TRY(dalloc(c, &c->d_L, M));
    FS_TRY(dalloc(c, &c->d_Ldot, M));
    FS_CUDA(cudaMemsetAsync(c->d_Ldot, 0, M * sizeof(double), c->stream));
    FS_TRY(dalloc(c, &c->d_fext, 3 * P));
    FS_TRY(dalloc(c, &c->d_t, 3 * P));
    FS_TRY(dalloc(c, &c->d_tz, 3 * c->n_z));
    FS_TRY(dalloc(c, &c->d_fknown, 3 * P));
    FS_TRY(dalloc(c, &c->d_W, P));
    FS_TRY(dalloc(c, &c->d_mloc, 2 * P));
    FS_TRY(dalloc(c, &c->d_bc, 12 * M));
    FS_TRY(dalloc(c, &c->d_kp, 4 * c->n_kp));
    FS_TRY(dalloc(c, &c->d_B, c->n_blk));
    FS_TRY(dalloc(c, &c->d_ftau, c->n_blk / 16 * 3));
    FS_TRY(dalloc(c, &c->d_wsc, c->n_blk / 4 * 3));
    // the p columns of w are never written: they stay zero (f = 0 there)
    FS_CUDA(cudaMemsetAsync(c->d_wsc, 0, static_cast<size_t>(c->n_blk / 4 * 3) * sizeof(double), c->stream));
    {
        const OzPlan q = oz_plan(M, c->max_N, c->opt);
        c->oz_chunk = q.oz_chunk;
        c->lu_chunk = q.lu_chunk;
        if (q.x > 0) {
            FS_TRY(dalloc(c, &c->d_ozx, static_cast<size_t>(q.x)));
            FS_TRY(dalloc(c, &c->d_ozy, static_cast<size_t>(q.y)));
            FS_TRY(dalloc(c, &c->d_ozxe, static_cast<size_t>(q.xe)));
            FS_TRY(dalloc(c, &c->d_ozye, static_cast<size_t>(q.ye)));
        }
    }
    FS_TRY(dalloc(c, &c->d_piv, c->n_fib_unk));
    FS_TRY(dalloc(c, &c->d_dinv, c->n_fib_unk));
    FS_TRY(dalloc(c, &c->d_V, 3 * P));
    FS_TRY(dalloc(c, &c->d_T, P));
    FS_TRY(dalloc(c, &c->d_f, 3 * P));
    FS_TRY(dalloc(c, &c->d_wf, 3 * P));
    FS_TRY(dalloc(c, &c->d_ubar, 3 * P));
    FS_CUDA(cudaMemsetAsync(c->d_kp, 0, 4 * c->n_kp * sizeof(double), c->stream));
    FS_CUDA(cudaMemsetAsync(c->d_V, 0, 3 * P * sizeof(double), c->stream));
    FS_CUDA(cudaMemsetAsync(c->d_T, 0, P * sizeof(double), c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));   // host staging vectors
    return FS_OK;
}

// Krylov workspace of context_init.
fs_status krylov_arrays(fs_ctx *c)
{
    const int R = std::max(2, std::min(c->opt.restart, 250));   // k_finish_dots uses 256 threads
    c->kdim = R + 1;
    const int64_t n = c->n_unk;
    FS_TRY(dalloc(c, &c->d_basis, static_cast<size_t>(c->kdim) * n));
    FS_TRY(dalloc(c, &c->d_b, n));
    FS_TRY(dalloc(c, &c->d_x, n));
    FS_TRY(dalloc(c, &c->d_r, n));
    FS_TRY(dalloc(c, &c->d_w, n));
    FS_TRY(dalloc(c, &c->d_e, n));
    FS_TRY(dalloc(c, &c->d_pb, n));
    c->chunk_cap = n / kChunk + c->S + 2;
    int64_t items = c->S;
    for (int s = 0; s < c->S; ++s) items += (c->sys_node_ptr[s + 1] - c->sys_node_ptr[s] + 127) / 128;
    c->work_cap = items;
    FS_TRY(dalloc(c, &c->d_work, static_cast<size_t>(c->work_cap)));
    const size_t SHi = 4 * size_t(c->kdim) + 8;
    FS_TRY(dalloc(c, &c->d_h, c->S * SHi));
    FS_TRY(dalloc(c, &c->d_part, static_cast<size_t>(c->kdim) * c->chunk_cap));
    FS_TRY(dalloc(c, &c->d_ich, static_cast<size_t>(c->chunk_cap)));
    FS_TRY(dalloc(c, &c->d_isch, static_cast<size_t>(c->S)));
    FS_TRY(dalloc(c, &c->d_ikk, static_cast<size_t>(c->S)));
    if (!c->pool) FS_CUDA(cudaFreeHost(c->h_pinned));
    c->h_pinned = nullptr;
    FS_TRY(pinned_alloc(c, &c->h_pinned, c->S * SHi));
    if (c->opt.use_graph) {
        const size_t S = c->S, R = c->kdim - 1;
        FS_TRY(dalloc(c, &c->d_gH, S * R * (R + 1)));
        FS_TRY(dalloc(c, &c->d_gcs, S * R));
        FS_TRY(dalloc(c, &c->d_gsn, S * R));
        FS_TRY(dalloc(c, &c->d_gg, S * (R + 1)));
        FS_TRY(dalloc(c, &c->d_gsc, 4 * S));
        FS_TRY(dalloc(c, &c->d_ginit, 2 * S));
        FS_TRY(dalloc(c, &c->d_gst, 4 * S));
        FS_TRY(dalloc(c, &c->d_gj, 1));
        FS_TRY(dalloc(c, &c->d_vcur, static_cast<size_t>(n)));
        // host mirrors: ginit [2S], gsc [4S] doubles, gst [4S] + gj ints
        FS_TRY(pinned_alloc(c, &c->h_gbuf, 6 * S + 2 * S + 2));
        c->h_ginit = c->h_gbuf;
        c->h_gsc = c->h_gbuf + 2 * S;
        c->h_gst = reinterpret_cast<int *>(c->h_gbuf + 6 * S);
        c->h_gj = c->h_gst + 4 * S;
    }
    if (c->opt.prec == FS_MIXED) {
        c->okdim = 17;   // outer (flexible) restart length 16
        const size_t SHo = 4 * size_t(c->okdim) + 8;
        FS_TRY(dalloc(c, &c->d_obasis, static_cast<size_t>(c->okdim) * n));
        FS_TRY(dalloc(c, &c->d_oz, static_cast<size_t>(c->okdim - 1) * n));
        FS_TRY(dalloc(c, &c->d_oh, c->S * SHo));
        FS_TRY(dalloc(c, &c->d_opart, static_cast<size_t>(c->okdim) * c->chunk_cap));
        FS_TRY(dalloc(c, &c->d_ow, n));
        FS_TRY(dalloc(c, &c->d_or, n));
        FS_TRY(dalloc(c, &c->d_och, static_cast<size_t>(c->chunk_cap)));
        FS_TRY(dalloc(c, &c->d_osch, static_cast<size_t>(c->S)));
        FS_TRY(dalloc(c, &c->d_okk, static_cast<size_t>(c->S)));
        FS_TRY(pinned_alloc(c, &c->oh_pinned, c->S * SHo));
    }
    return FS_OK;
}

// Surface arrays of context_init: periphery nodes, then the body's.
fs_status surface_arrays(fs_ctx *c, const fs_boundary *bd, const fs_body *body)
{
    if (!c->surf.n) return FS_OK;
    const int ns = c->surf.n, p = c->surf.n_per, nb = c->body.n;
    FS_TRY(dalloc(c, &c->surf.y, 3 * ns));
    FS_TRY(dalloc(c, &c->surf.nrm, 3 * ns));
    FS_TRY(dalloc(c, &c->surf.w, ns));
    FS_TRY(dalloc(c, &c->surf.diag, 3 * ns));
    FS_TRY(dalloc(c, &c->d_usurf, 3 * ns));
    FS_TRY(dalloc(c, &c->surf.A, 9 * ns));
    FS_TRY(dalloc(c, &c->surf.tmp, 3 * ns));
    FS_TRY(dalloc(c, &c->surf.flux, 1));
    FS_TRY(dalloc(c, &c->surf.excl, ns));
    FS_CUDA(cudaMemsetAsync(c->surf.flux, 0, sizeof(double), c->stream));
    const size_t d = sizeof(double);
    if (p > 0) {
        FS_CUDA(cudaMemcpyAsync(c->surf.y, bd->nodes, 3 * p * d, cudaMemcpyHostToDevice, c->stream));
        FS_CUDA(cudaMemcpyAsync(c->surf.nrm, bd->normals, 3 * p * d, cudaMemcpyHostToDevice, c->stream));
        FS_CUDA(cudaMemcpyAsync(c->surf.w, bd->weights, p * d, cudaMemcpyHostToDevice, c->stream));
    }
    if (nb > 0) {
        FS_CUDA(cudaMemcpyAsync(c->surf.y + 3 * int64_t(p), body->nodes, 3 * nb * d, cudaMemcpyHostToDevice, c->stream));
        FS_CUDA(cudaMemcpyAsync(c->surf.nrm + 3 * int64_t(p), body->normals, 3 * nb * d, cudaMemcpyHostToDevice,
                                c->stream));
        FS_CUDA(cudaMemcpyAsync(c->surf.w + p, body->weights, nb * d, cudaMemcpyHostToDevice, c->stream));
    }
    return surface_diag(c);
}

// Upper bound of the CTAs one wave of a direct sum may hold (SMs x resident
// CTAs per SM); lets the estimate run without asking a device.
constexpr int kSlotsBound = 8192;

// Digit-plane scratch of the tensor-core block build (tc_blocks) and LU
// (tc_lu): chunk sizes and element counts of the planes (bf16) and exponents
// (int); the LU reuses the build's planes, which it outgrows only when the
// build is off.  Shared by the allocation and the memory estimate.
OzPlan oz_plan(int M, int maxN, const fs_options &o)
{
    OzPlan q;
    if (M <= 0) return q;
    if (o.tc_blocks) {
        const OzDims D(maxN);
        const int64_t per = D.bytes_per_fiber();
        q.oz_chunk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>({int64_t(M), 512, (int64_t(1) << 30) / per})));
        const int64_t rx = std::max(D.r1, D.r2);
        q.x = int64_t(q.oz_chunk) * OzDims::digits * rx * D.kp;
        q.y = int64_t(q.oz_chunk) * OzDims::digits * D.ry * D.kp;
        q.xe = int64_t(q.oz_chunk) * rx;
        q.ye = int64_t(q.oz_chunk) * D.ry;
    }
    if (o.tc_lu && LuTcDims::fits(maxN)) {
        const LuTcDims L(maxN);
        const int64_t per = 2 * (L.plane_elems() * 2 + int64_t(L.rows) * 4);
        q.lu_chunk = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(int64_t(M), (int64_t(1) << 30) / per)));
        q.x = std::max(q.x, int64_t(q.lu_chunk) * L.plane_elems());
        q.y = std::max(q.y, int64_t(q.lu_chunk) * L.plane_elems());
        q.xe = std::max(q.xe, int64_t(q.lu_chunk) * L.rows);
        q.ye = std::max(q.ye, int64_t(q.lu_chunk) * L.rows);
    }
    return q;
}

// Device bytes context_init allocates for this problem, plus the largest
// direct-sum scratch a step reserves.  Each allocation is rounded up to the
// allocator's 512-byte granule; the result bounds what fs_device_bytes reports.
size_t estimate_bytes(int M, const int32_t *ppf, int n_surf, const fs_options &opt)
{
    size_t total = 0;
    auto add = [&](size_t bytes) { total += (bytes + 511) & ~size_t(511); };
    add(sizeof(int));   // status word
    if (M == 0) return total;
    int64_t P = 0, n_fib_unk = 0, n_blk = 0, n_kp = 0, n_z = 0, ops = 0;
    std::map<int, int> seen;
    for (int m = 0; m < M; ++m) {
        const int64_t N = ppf[m];
        P += N;
        n_fib_unk += 4 * N;
        n_blk += 16 * N * N;
        n_kp += N * N;
        n_z += N - 2;
        if (!seen.count(ppf[m])) {
            seen[ppf[m]] = 1;
            ops += OpsLayout(ppf[m]).total;
        }
    }
    const size_t d = sizeof(double);
    add(M * sizeof(int));
    for (int i = 0; i < 5; ++i) add((M + 1) * sizeof(int64_t));
    add(M * sizeof(int64_t));
    add(ops * d);
    add(P * sizeof(int2));
    for (int64_t k : {3 * P, int64_t(M), int64_t(M), 3 * P, 3 * P, 3 * n_z, 3 * P, P, 2 * P, 12 * int64_t(M), 4 * n_kp, n_blk,
                      n_blk / 16 * 3, n_blk / 4 * 3})
        add(k * d);
    {   // digit planes of the tensor-core block build and LU
        int maxN = 0;
        for (int m = 0; m < M; ++m) maxN = std::max(maxN, int(ppf[m]));
        const OzPlan q = oz_plan(M, maxN, opt);
        add(q.x * 2);
        add(q.y * 2);
        add(q.xe * 4);
        add(q.ye * 4);
    }
    add(n_fib_unk * sizeof(int));
    add(n_fib_unk * sizeof(double));
    for (int64_t k : {3 * P, P, 3 * P, 3 * P, 3 * P}) add(k * d);
    const int64_t n = n_fib_unk + 3 * int64_t(n_surf) + 6;   // + a rigid body's U, Omega
    const int R = std::max(2, std::min(opt.restart, 250));
    const int64_t kdim = R + 1;
    add(kdim * n * d);
    for (int i = 0; i < 6; ++i) add(n * d);
    const int64_t chunk_cap = n / kChunk + 1 + 2;
    add(((P + 127) / 128 + 1) * sizeof(int4));
    add((4 * kdim + 8) * d);
    add(kdim * chunk_cap * d);
    add(chunk_cap * sizeof(int4));
    add(sizeof(int4));
    add(sizeof(int));
    if (opt.use_graph) {   // device Givens state of one system, the current basis vector
        for (int64_t k : {kdim * (kdim - 1) + 4 * kdim, int64_t(4), int64_t(2), n}) add(k * d);
        add(4 * sizeof(int));
        add(sizeof(int));
    }
    if (opt.prec == FS_MIXED) {
        const int64_t ok = 17;
        add(ok * n * d);
        add((ok - 1) * n * d);
        add((4 * ok + 8) * d);
        add(ok * chunk_cap * d);
        add(n * d);
        add(n * d);
        add(chunk_cap * sizeof(int4));
        add(sizeof(int4));
        add(sizeof(int));
    }
    if (n_surf) {
        const int64_t ns = n_surf;
        for (int64_t k : {3 * ns, 3 * ns, ns, 3 * ns, 3 * ns, 9 * ns, 3 * ns, int64_t(1)}) add(k * d);
        add(ns * sizeof(int2));
        add(kRbSize * d);                   // a rigid body's record and fiber lists
        add(M * sizeof(int));
        add(M * sizeof(int));
    }
    // the scratch grows to 5/4 of the largest sum it has served
    size_t sc = 0;
    const int64_t sizes[4][2] = {{P, P}, {n_surf, P}, {P, n_surf}, {n_surf, n_surf}};
    for (int kind : {int(PAIR_STOKESLET), int(PAIR_STRESSLET)})
        for (int prec : {int(FS_SUM_FP64), int(FS_SUM_FP32), int(FS_SUM_FF)})
            for (auto &sz : sizes)
                if (sz[0] > 0 && sz[1] > 0)
                    sc = std::max(sc, pairsum_scratch_bytes(kind, sz[0], sz[1], prec, opt.tile_override,
                                                            kSlotsBound));
    total += sc + sc / 4 + 512;
    return total;
}

void context_free(fs_ctx *c)
{
    if (c->stream) cudaStreamSynchronize(c->stream);
    void *ptrs[] = {c->d_status, c->d_N, c->d_node_ptr, c->d_unk_ptr, c->d_blk_ptr, c->d_kp_ptr,
                    c->d_z_ptr, c->d_ops_off, c->d_ops, c->d_excl, c->d_X, c->d_L, c->d_Ldot, c->d_fext,
                    c->d_t, c->d_tz, c->d_fknown, c->d_W, c->d_mloc, c->d_bc, c->d_kp, c->d_B, c->d_ftau, c->d_wsc,
                    c->d_piv, c->d_dinv, c->d_V, c->d_T, c->d_f, c->d_wf, c->d_ubar, c->d_basis, c->d_b,
                    c->d_x, c->d_r, c->d_w, c->d_e, c->d_pb, c->d_obasis, c->d_oz, c->d_oh, c->d_opart, c->d_ow, c->d_or, c->d_work, c->d_ich, c->d_isch, c->d_ikk, c->d_och, c->d_osch, c->d_okk, c->d_h, c->d_part, c->surf.y, c->surf.nrm,
                    c->surf.w, c->surf.diag, c->d_usurf, c->surf.A, c->surf.tmp, c->surf.flux, c->surf.excl,
                    c->body.rb, c->body.attach, c->body.att_list};
    for (fs::CycleGraph &g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
    }
    c->graphs.clear();
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->cap_stream = nullptr;
    void *gptrs[] = {c->d_gH, c->d_gcs, c->d_gsn, c->d_gg, c->d_gsc, c->d_ginit, c->d_vcur, c->d_gst, c->d_gj,
                     c->d_ozx, c->d_ozy, c->d_ozxe, c->d_ozye};
    // buffers carved from a preallocated region go back with the region
    if (!c->pool) {
        for (void *p : gptrs)
            if (p) cudaFree(p);
        if (c->h_gbuf) cudaFreeHost(c->h_gbuf);
        for (void *p : ptrs)
            if (p) cudaFree(p);
        if (c->h_pinned) cudaFreeHost(c->h_pinned);
        if (c->oh_pinned) cudaFreeHost(c->oh_pinned);
    }
    c->oh_pinned = nullptr;
    c->prof.release_all();
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    c->prof.pool.clear();
    c->h_pinned = nullptr;
    c->scratch.release();
    c->tree_scratch.release();
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
    F.ftau = d_ftau;
    F.wsc = d_wsc;
    F.Ldot = growth ? d_Ldot : nullptr;
    F.growth_implicit = opt.growth_implicit;
    F.attach = body.on ? body.attach : nullptr;
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

fs_status fs_get_self_block(fs_ctx *c, int32_t fiber, double *out)
{
    if (!c || !c->have_state || fiber < 0 || fiber >= c->M || !out) {
        set_error("fs_get_self_block: no state, fiber out of range or NULL output");
        return FS_EINVAL;
    }
    if (!c->geometry_ok) {
        FS_TRY(launch_geometry(c));
        c->geometry_ok = true;
    }
    // the blocks are factored in place by the preconditioner build: assemble
    // them again, copy one out, and let the next step factor them anew
    FS_TRY(launch_block_build(c));
    c->precond_ok = false;
    const int64_t n = 4 * int64_t(c->Nm[fiber]);
    FS_CUDA(cudaMemcpyAsync(out, c->d_B + c->blk_ptr[fiber], static_cast<size_t>(n * n) * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

fs_status fs_get_tuned_shapes(const fs_ctx *c, int32_t *out)
{
    if (!c || !out) {
        set_error("fs_get_tuned_shapes: NULL context or output");
        return FS_EINVAL;
    }
    for (int i = 0; i < 8; ++i) out[i] = c->tuned[i];
    return FS_OK;
}

fs_status fs_get_block_lu(fs_ctx *c, int32_t fiber, double *lu, int32_t *piv)
{
    if (!c || !c->have_state || fiber < 0 || fiber >= c->M || !lu || !piv) {
        set_error("fs_get_block_lu: no state, fiber out of range or NULL output");
        return FS_EINVAL;
    }
    if (!c->precond_ok) FS_TRY(fs_build_precond(c));
    const int64_t n = 4 * int64_t(c->Nm[fiber]);
    FS_CUDA(cudaMemcpyAsync(lu, c->d_B + c->blk_ptr[fiber], static_cast<size_t>(n * n) * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaMemcpyAsync(piv, c->d_piv + c->unk_ptr[fiber], static_cast<size_t>(n) * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

fs_status fs_step(fs_ctx *c, fs_step_info *info)
{
    if (!c || !c->have_state || (c->M == 0 && !c->body.on)) {
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
    // mixed precision: solve with an FP32 right-hand side, then one
    // float-float true residual and a plain FP32 correction.  The right-hand
    // side's Stokeslet sum runs in the packed kernel (per-thread frames: the
    // hi/lo accuracy on fiber nodes); with a boundary the stresslets keep
    // hi/lo coordinates
    const bool split = c->opt.prec == FS_MIXED && c->opt.relax;
    if (split) FS_TRY(rhs(c, c->d_b, c->d_pb, FS_SUM_FP32, c->surf.n > 0));
    else FS_TRY(rhs(c, c->d_b, c->d_pb));
    FS_TRY(check_status(c));
    if (info) tms[0] = ms_since(t0) - tms[1];
    int iters = 0, sweeps = 0;
    double rel = 0.0;
    bool converged = false;
    std::vector<SysState> st;
    std::vector<int> its(c->S, 0), outer(c->S, 0);
    std::vector<double> resid(c->S, 0.0);
    std::vector<char> conv(c->S, 0);
    if (c->opt.prec == FS_FP64) {
        Space sp = inner_space(c);
        FS_TRY(gmres_seg(c, sp, c->d_pb, c->d_x, c->opt.tol, c->opt.max_iter, FS_SUM_FP64, -1, 0.0,
                         c->all_sys, st));
        for (int s = 0; s < c->S; ++s) {
            its[s] = st[s].its;
            outer[s] = 1;
            resid[s] = st[s].rel;
            conv[s] = st[s].conv;
        }
    } else if (split) {
        // (1) x1: GMRES on the FP32-far-field operator with the FP32 right-hand
        //     side, to the inner tolerance (or tol if tighter);
        // (2) r1 = P^-1 b - (P^-1 A) x1 with one float-float far field;
        // (3) d: GMRES on the plain FP32 operator for (P^-1 A) d = r1 until
        //     |r1 - (P^-1 A) d| <= tol |P^-1 b|.  Its operator error (relative
        //     ~3e-6, bounded by kEtaFP32Plain) acts on a correction of size
        //     |r1| (~inner tol |P^-1 b|).  A residual too large for that
        //     (kEtaFP32Plain |r1| > kRelaxShare tol |P^-1 b|) is reduced
        //     1e3-fold and the residual recomputed.
        Space sp = inner_space(c);
        std::vector<SysState> s1, s2;
        FS_TRY(gmres_seg(c, sp, c->d_pb, c->d_x, std::min(c->opt.inner_tol, 0.1), c->opt.max_iter, FS_SUM_FP32,
                         -1, 0.0, c->all_sys, s1));
        std::vector<double> lim(c->S, 0.0);
        for (int s = 0; s < c->S; ++s) {
            lim[s] = c->opt.tol * s1[s].beta0;
            its[s] = s1[s].its;
            outer[s] = 1;
        }
        const int sweeps_max = std::max(1, c->opt.max_refine);
        for (int sw = 0; sw < sweeps_max; ++sw) {
            FS_TRY(true_residual(c, c->d_x, c->d_b, accurate_prec(c)));
            const bool last = sw + 1 == sweeps_max;
            FS_TRY(gmres_seg(c, sp, c->d_b, c->d_pb, c->opt.tol, c->opt.max_iter, FS_SUM_FP32, -1, 0.0,
                             c->all_sys, s2, false, &lim, last ? 0.0 : 1e-3));
            k_add<<<blocks_for(c->n_unk), 256, 0, c->stream>>>(c->d_x, c->d_pb, c->n_unk);
            FS_LAUNCH_CHECK();
            bool again = false;
            for (int s = 0; s < c->S; ++s) {
                its[s] += s2[s].its;
                if (s2[s].its > 0) ++outer[s];
                resid[s] = s1[s].beta0 > 0.0 ? s2[s].res / s1[s].beta0 : 0.0;
                conv[s] = s2[s].conv && s2[s].res <= lim[s];
                if (!last && kEtaFP32Plain * s2[s].beta0 > kRelaxShare * lim[s]) again = true;
            }
            if (!again) break;
        }
    } else {
        // mixed: flexible GMRES on the operator with the float-float far field,
        // each direction preconditioned by an FP32-far-field GMRES solve
        Space sp = outer_space(c);
        FS_TRY(gmres_seg(c, sp, c->d_pb, c->d_x, c->opt.tol, c->opt.max_iter, accurate_prec(c), FS_SUM_FP32,
                         c->opt.inner_tol, c->all_sys, st));
        for (int s = 0; s < c->S; ++s) {
            its[s] = st[s].inner;
            outer[s] = st[s].its;
            resid[s] = st[s].rel;
            conv[s] = st[s].conv;
        }
    }
    converged = true;
    for (int s = 0; s < c->S; ++s) {
        iters = std::max(iters, its[s]);
        sweeps = std::max(sweeps, outer[s]);
        rel = std::max(rel, resid[s]);
        converged = converged && conv[s];
        c->sys_iters[s] = its[s];
        c->sys_outer[s] = outer[s];
        c->sys_resid[s] = resid[s];
        c->sys_conv[s] = conv[s] ? 1 : 0;
    }
    FS_TRY(check_status(c));
    tms[2] = ms_since(t0) - tms[0] - tms[1];
    if (info) {
        info->iters = iters;
        info->refine_sweeps = sweeps;
        info->resid = rel;
        info->pairs = c->pairs_last;
    }
    // a serving batch updates every system and reports convergence per
    // system (fs_batch_info); the others are not held back by one that failed
    if (!converged && !c->partial_ok) {
        if (info) {
            tms[4] = ms_since(t0);
            std::memcpy(info->t_ms, tms, sizeof(tms));
        }
        set_error("fs_step: not converged (rel. residual %.3e after %d iterations)", rel, iters);
        return FS_ENOTCONV;
    }
    FS_TRY(launch_update(c, c->d_x));
    FS_TRY(body_update(c, c->d_x + c->n_fib_unk + 3 * int64_t(c->surf.n)));
    c->geometry_ok = c->precond_ok = false;
    if (info) {
        FS_CUDA(cudaStreamSynchronize(c->stream));
        tms[4] = ms_since(t0);
        tms[3] = tms[4] - tms[0] - tms[1] - tms[2];
        std::memcpy(info->t_ms, tms, sizeof(tms));
    }
    return FS_OK;
}

fs_status fs_set_growth(fs_ctx *c, const double *Ldot, int32_t dev)
{
    if (!c || c->M == 0 || !Ldot) {
        set_error("fs_set_growth: NULL argument or context without fibers");
        return FS_EINVAL;
    }
    std::vector<double> hL(c->M), hD(c->M);
    FS_CUDA(cudaMemcpyAsync(hL.data(), c->d_L, c->M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (dev)
        FS_CUDA(cudaMemcpyAsync(hD.data(), Ldot, c->M * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    if (!dev) std::memcpy(hD.data(), Ldot, c->M * sizeof(double));
    bool any = false;
    for (int m = 0; m < c->M; ++m) {
        if (!std::isfinite(hD[m]) || !(hL[m] + c->dt * hD[m] > 0.0)) {
            set_error("fs_set_growth: fiber %d: length %g + dt x rate %g would not stay positive", m, hL[m],
                      hD[m]);
            return FS_EINVAL;
        }
        any = any || hD[m] != 0.0;
    }
    FS_CUDA(cudaMemcpyAsync(c->d_Ldot, hD.data(), c->M * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    c->growth = any;
    c->precond_ok = false;   // the self block carries the growth term
    return FS_OK;
}

fs_status fs_get_unknowns(fs_ctx *c, double *u, int32_t dev)
{
    if (!c || !u || c->n_unk == 0) {
        set_error("fs_get_unknowns: NULL argument or empty context");
        return FS_EINVAL;
    }
    FS_CUDA(cudaMemcpyAsync(u, c->d_x, static_cast<size_t>(c->n_unk) * sizeof(double),
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

fs_status fs_get_lengths(fs_ctx *c, double *L, int32_t dev)
{
    if (!c || c->M == 0 || !L) {
        set_error("fs_get_lengths: NULL argument or context without fibers");
        return FS_EINVAL;
    }
    FS_CUDA(cudaMemcpyAsync(L, c->d_L, c->M * sizeof(double), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            c->stream));
    FS_CUDA(cudaStreamSynchronize(c->stream));
    return FS_OK;
}

size_t fs_estimate_bytes(int32_t n_fibers, const int32_t *points_per_fiber, int32_t n_surface_nodes,
                         const fs_options *options)
{
    if (n_fibers < 0 || (n_fibers > 0 && !points_per_fiber) || n_surface_nodes < 0) return 0;
    for (int m = 0; m < n_fibers; ++m)
        if (points_per_fiber[m] < 6 || points_per_fiber[m] > 256) return 0;
    fs_options o;
    if (options) o = *options; else fs_options_default(&o);
    // options fs_create would refuse (an unknown precision, restart > 250, ...) estimate nothing
    if (check_options(o, "fs_estimate_bytes", 1) != FS_OK) return 0;
    return estimate_bytes(n_fibers, points_per_fiber, n_surface_nodes, o);
}

fs_status fs_device_bytes(const fs_ctx *c, size_t *bytes)
{
    if (!c || !bytes) {
        set_error("fs_device_bytes: NULL argument");
        return FS_EINVAL;
    }
    *bytes = c->dev_bytes + c->scratch.bytes;
    return FS_OK;
}

fs_status fs_batch_info(const fs_ctx *c, int32_t *iters, int32_t *outer, double *resid,
                        int32_t *converged)
{
    if (!c) {
        set_error("fs_batch_info: NULL context");
        return FS_EINVAL;
    }
    for (int s = 0; s < c->S; ++s) {
        if (iters) iters[s] = c->sys_iters[s];
        if (outer) outer[s] = c->sys_outer[s];
        if (resid) resid[s] = c->sys_resid[s];
        if (converged) converged[s] = c->sys_conv[s];
    }
    return FS_OK;
}

}  // extern "C"
