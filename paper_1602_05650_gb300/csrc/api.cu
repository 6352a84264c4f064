// C-ABI entry points: context lifetime, state transfer, direct sums, step.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "context.h"

namespace fs {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void *Pool::take_dev(size_t bytes)
{
    const size_t at = (dev_used + 255) & ~size_t(255);
    if (at + bytes > dev_cap) return nullptr;
    dev_used = at + bytes;
    return dev + at;
}

void *Pool::take_host(size_t bytes)
{
    const size_t at = (host_used + 255) & ~size_t(255);
    if (at + bytes > host_cap) return nullptr;
    host_used = at + bytes;
    return host + at;
}

fs_status Scratch::reserve(size_t need, cudaStream_t st)
{
    if (need <= bytes) return FS_OK;
    if (pool) {
        // the region was sized for the largest sum; an earlier, smaller piece
        // stays unused until the region is given back
        void *p = pool->take_dev(need);
        if (!p) {
            set_error("scratch: %zu bytes exceed the preallocated region", need);
            return FS_ENOMEM;
        }
        ptr = p;
        bytes = need;
        return FS_OK;
    }
    if (ptr) {
        FS_CUDA(cudaStreamSynchronize(st));
        FS_CUDA(cudaFree(ptr));
        ptr = nullptr;
        bytes = 0;
    }
    size_t want = need + need / 4;
    if (cudaMalloc(&ptr, want) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
        set_error("scratch: cudaMalloc of %zu bytes failed", want);
        return FS_ENOMEM;
    }
    bytes = want;
    return FS_OK;
}

void Scratch::release()
{
    if (ptr && !pool) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

fs_status check_options(const fs_options &o, const char *who, int n_systems)
{
    // the step dispatches on prec: any other value would reach the flexible
    // GMRES without its outer Krylov arrays (allocated for FS_MIXED only)
    if (o.prec != FS_FP64 && o.prec != FS_MIXED) {
        set_error("%s: prec must be FS_FP64 or FS_MIXED (got %d)", who, o.prec);
        return FS_EINVAL;
    }
    if (!(o.tol > 0.0 && o.tol < 1.0) || !(o.inner_tol > 0.0 && o.inner_tol < 1.0)) {
        set_error("%s: tol and inner_tol must lie in (0, 1)", who);
        return FS_EINVAL;
    }
    if (o.max_iter < 1 || o.restart < 1 || o.restart > 250 || o.max_refine < 1) {
        set_error("%s: need max_iter >= 1, 1 <= restart <= 250, max_refine >= 1", who);
        return FS_EINVAL;
    }
    if (!(o.delta_over_L >= 0.0) || !std::isfinite(o.delta_over_L)) {
        set_error("%s: delta_over_L must be finite and >= 0", who);
        return FS_EINVAL;
    }
    if ((o.lsb | o.relax | o.profile | o.growth_implicit | o.tc_blocks | o.tc_lu | o.autotune) & ~1) {
        set_error("%s: lsb, relax, profile, growth_implicit, tc_blocks, tc_lu and autotune are 0 or 1", who);
        return FS_EINVAL;
    }
    if (o.use_graph != 0 && o.use_graph != 1) {
        set_error("%s: use_graph is 0 or 1", who);
        return FS_EINVAL;
    }
    if (o.autotune && o.use_graph) {
        // a captured cycle keeps the shapes (and work lists) of its capture
        set_error("%s: autotune and use_graph exclude each other", who);
        return FS_EINVAL;
    }
    if (o.tile_override < 0 || o.tile_override > 3) {
        set_error("%s: tile_override must be 0 (measured default) or a shape id 1..3", who);
        return FS_EINVAL;
    }
    const int t = o.tree_order;
    if (t != 0 && t != 4 && t != 6 && t != 8 && t != 10) {
        set_error("%s: tree_order must be 0, 4, 6, 8 or 10 (got %d)", who, t);
        return FS_EINVAL;
    }
    if (t && !(o.tree_theta > 0.0 && o.tree_theta < 1.0)) {
        set_error("%s: tree_theta must lie in (0, 1)", who);
        return FS_EINVAL;
    }
    if (t && n_systems > 1) {
        set_error("%s: the treecode far field serves single-system contexts", who);
        return FS_EINVAL;
    }
    return FS_OK;
}

}  // namespace fs

using namespace fs;

extern "C" {

const char *fs_last_error(void) { return g_err; }

const char *fs_status_str(int32_t s)
{
    switch (s) {
    case FS_OK: return "FS_OK";
    case FS_EINVAL: return "FS_EINVAL";
    case FS_ENOMEM: return "FS_ENOMEM";
    case FS_ECUDA: return "FS_ECUDA";
    case FS_ENOTCONV: return "FS_ENOTCONV";
    case FS_ENUMERIC: return "FS_ENUMERIC";
    case FS_EAGAIN: return "FS_EAGAIN";
    case FS_EBUSY: return "FS_EBUSY";
    case FS_ETIMEOUT: return "FS_ETIMEOUT";
    default: return "FS_UNKNOWN";
    }
}

fs_status fs_options_default(fs_options *o)
{
    if (!o) {
        set_error("fs_options_default: NULL");
        return FS_EINVAL;
    }
    std::memset(o, 0, sizeof(*o));
    o->prec = FS_MIXED;
    o->tol = 1e-8;
    o->max_iter = 200;
    o->restart = 60;
    o->max_refine = 6;
    o->inner_tol = 1e-6;
    o->delta_over_L = 0.01;
    o->lsb = 0;
    o->use_graph = 0;
    o->tile_override = 0;
    o->profile = 0;
    o->relax = 1;
    o->tree_order = 0;
    o->tree_theta = 0.5;
    o->growth_implicit = 0;
    o->tc_blocks = 1;
    o->tc_lu = 1;
    o->autotune = 0;
    return FS_OK;
}

static fs_status create_impl(fs_ctx **out, int32_t n_systems, const int32_t *fps, int32_t n_fibers,
                             const int32_t *ppf, double mu, double eps, double E, double dt,
                             const fs_boundary *boundary, const fs_options *opt, void *cuda_stream,
                             const fs_body *body = nullptr, const int32_t *minus_end = nullptr,
                             Pool *pool = nullptr, bool serving = false)
{
    if (!out) {
        set_error("fs_create: out is NULL");
        return FS_EINVAL;
    }
    *out = nullptr;
    if (n_fibers < 0 || (n_fibers > 0 && !ppf)) {
        set_error("fs_create: bad fiber count or points_per_fiber");
        return FS_EINVAL;
    }
    if (!(mu > 0.0) || !(eps > 0.0 && eps < 1.0) || !(E >= 0.0) || !(dt > 0.0)) {
        set_error("fs_create: need mu > 0, 0 < eps < 1, E >= 0, dt > 0");
        return FS_EINVAL;
    }
    for (int m = 0; m < n_fibers; ++m)
        if (ppf[m] < 6 || ppf[m] > 256) {
            set_error("fs_create: points per fiber must be in [6, 256] (fiber %d has %d)", m, ppf[m]);
            return FS_EINVAL;
        }
    if (boundary && (boundary->n_nodes <= 0 || !boundary->nodes || !boundary->normals ||
                     !boundary->weights)) {
        set_error("fs_create: incomplete boundary description");
        return FS_EINVAL;
    }
    if (body && (body->n_nodes <= 0 || !body->nodes || !body->normals || !body->weights ||
                 !(body->radius > 0.0))) {
        set_error("fs_create_with_body: incomplete body description");
        return FS_EINVAL;
    }
    if (body)
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(body->center[a]) || !std::isfinite(body->force[a]) ||
                !std::isfinite(body->torque[a])) {
                set_error("fs_create_with_body: non-finite center or load");
                return FS_EINVAL;
            }
    if (minus_end)
        for (int m = 0; m < n_fibers; ++m) {
            if (minus_end[m] != FS_END_FREE && minus_end[m] != FS_END_CLAMPED && minus_end[m] != FS_END_HINGED) {
                set_error("fs_create_with_body: fiber %d has unknown end condition %d", m, minus_end[m]);
                return FS_EINVAL;
            }
            if (minus_end[m] != FS_END_FREE && !body) {
                set_error("fs_create_with_body: fiber %d is attached but there is no body", m);
                return FS_EINVAL;
            }
        }
    if (opt) FS_TRY(check_options(*opt, n_systems > 1 ? "fs_create_batch" : "fs_create", n_systems));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        set_error("fs_create: no CUDA device");
        return FS_ECUDA;
    }
    fs_ctx *c = new fs_ctx();
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->mu = mu;
    c->eps = eps;
    c->E = E;
    c->dt = dt;
    if (opt) c->opt = *opt; else fs_options_default(&c->opt);
    c->pool = pool;
    c->scratch.pool = c->tree_scratch.pool = pool;
    c->worklist = c->partial_ok = serving;
    fs_status s = context_init(c, n_systems, fps, n_fibers, ppf, boundary, body, minus_end);
    if (s != FS_OK) {
        context_free(c);
        delete c;
        return s;
    }
    *out = c;
    return FS_OK;
}

}  // extern "C"

namespace fs {
fs_status create_serving(fs_ctx **out, int32_t n_systems, const int32_t *fps, int32_t n_fibers, const int32_t *ppf,
                         double mu, double eps, double E, double dt, const fs_boundary *boundary,
                         const fs_options *opt, void *cuda_stream, Pool *pool)
{
    return create_impl(out, n_systems, fps, n_fibers, ppf, mu, eps, E, dt, boundary, opt, cuda_stream, nullptr,
                       nullptr, pool, true);
}
}  // namespace fs

extern "C" {

fs_status fs_create(fs_ctx **out, int32_t n_fibers, const int32_t *ppf, double mu, double eps,
                    double E, double dt, const fs_boundary *boundary, const fs_options *opt,
                    void *cuda_stream)
{
    return create_impl(out, 1, nullptr, n_fibers, ppf, mu, eps, E, dt, boundary, opt, cuda_stream);
}

fs_status fs_create_with_body(fs_ctx **out, int32_t n_fibers, const int32_t *ppf, const int32_t *minus_end,
                              double mu, double eps, double E, double dt, const fs_boundary *boundary,
                              const fs_body *body, const fs_options *opt, void *cuda_stream)
{
    return create_impl(out, 1, nullptr, n_fibers, ppf, mu, eps, E, dt, boundary, opt, cuda_stream, body,
                       minus_end);
}

fs_status fs_create_batch(fs_ctx **out, int32_t n_systems, const int32_t *fibers_per_system,
                          const int32_t *points_per_fiber, double mu, double eps, double E, double dt,
                          const fs_options *opt, void *cuda_stream)
{
    if (!out || n_systems < 1 || !fibers_per_system) {
        set_error("fs_create_batch: need at least one system and fibers_per_system");
        if (out) *out = nullptr;
        return FS_EINVAL;
    }
    int64_t M = 0;
    for (int s = 0; s < n_systems; ++s) {
        if (fibers_per_system[s] < 1) {
            set_error("fs_create_batch: system %d has no fiber", s);
            *out = nullptr;
            return FS_EINVAL;
        }
        M += fibers_per_system[s];
    }
    if (M >= (1LL << 31)) {
        set_error("fs_create_batch: too many fibers");
        *out = nullptr;
        return FS_EINVAL;
    }
    return create_impl(out, n_systems, fibers_per_system, static_cast<int32_t>(M), points_per_fiber, mu, eps,
                       E, dt, nullptr, opt, cuda_stream);
}

void fs_destroy(fs_ctx *c)
{
    if (!c) return;
    context_free(c);
    delete c;
}

fs_status fs_sizes(const fs_ctx *c, int64_t *n_points, int64_t *n_unknowns)
{
    if (!c) {
        set_error("fs_sizes: NULL context");
        return FS_EINVAL;
    }
    if (n_points) *n_points = c->n_tot;
    if (n_unknowns) *n_unknowns = c->n_unk;
    return FS_OK;
}

fs_status fs_stokeslet_apply(fs_ctx *c, const double *src_xyz, const double *src_wf, int64_t n_src,
                             const int32_t *src_fiber, const double *tgt_xyz,
                             const int32_t *tgt_fiber, int64_t n_tgt, double *out_u,
                             int32_t sum_precision)
{
    if (!c) {
        set_error("fs_stokeslet_apply: NULL context");
        return FS_EINVAL;
    }
    if (n_src < 0 || n_tgt < 0 || (n_src > 0 && (!src_xyz || !src_wf)) ||
        (n_tgt > 0 && (!tgt_xyz || !out_u))) {
        set_error("fs_stokeslet_apply: bad sizes or NULL arrays");
        return FS_EINVAL;
    }
    if (sum_precision != FS_SUM_FP32 && sum_precision != FS_SUM_FP64 && sum_precision != FS_SUM_FF &&
        sum_precision != FS_SUM_FP32_PLAIN) {
        set_error("fs_stokeslet_apply: unknown precision %d", sum_precision);
        return FS_EINVAL;
    }
    const bool plain = sum_precision == FS_SUM_FP32_PLAIN;
    if (plain) sum_precision = FS_SUM_FP32;
    if (n_src >= (1LL << 31) - 1 || n_tgt >= (1LL << 31) - 1) {
        set_error("fs_stokeslet_apply: at most 2^31-2 sources and targets");
        return FS_EINVAL;
    }
    const bool ids = src_fiber && tgt_fiber;
    const size_t need = pairsum_scratch_bytes(PAIR_STOKESLET, n_src, n_tgt, sum_precision,
                                              c->opt.tile_override) +
                        (ids ? static_cast<size_t>(n_tgt) * sizeof(int2) + 512 : 0);
    FS_TRY(c->scratch.reserve(need, c->stream));
    Carve cv(c->scratch.ptr, c->scratch.bytes);
    PairSumArgs a;
    if (ids) {
        int2 *excl = cv.take<int2>(n_tgt);
        FS_TRY(exclusion_from_ids(src_fiber, n_src, tgt_fiber, n_tgt, excl, c->stream));
        a.excl = excl;
    }
    cv.used = (cv.used + 255) & ~size_t(255);
    a.kind = PAIR_STOKESLET;
    a.src_xyz = src_xyz;
    a.src_dens = src_wf;
    a.n_src = n_src;
    a.tgt_xyz = tgt_xyz;
    a.n_tgt = n_tgt;
    a.out = out_u;
    a.scale = 1.0 / (8.0 * M_PI * c->mu);
    a.sum_prec = sum_precision;
    a.hilo = !plain;
    a.shape_override = c->opt.tile_override;
    a.pairs = double(n_src) * double(n_tgt);
    a.prof = c->opt.profile ? &c->prof : nullptr;
    return pairsum(a, cv.base + cv.used, cv.cap - cv.used, c->d_status, c->stream);
}

}  // extern "C"
