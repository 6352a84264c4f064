// Serving: independent fiber-suspension step requests, continuously batched.
//
// The server owns one region of device memory (the HBM budget, allocated
// once at creation) and two engine threads, each with its own CUDA stream and
// pinned staging buffer.  Requests (host arrays, copied at submit) wait in a
// FIFO.  A free engine takes the queue head and every other queued request
// that can share a step with it (same physical parameters, precision and
// tolerance, free space, up to max_slots requests, as long as the batch's
// memory estimate fits the largest free piece of the region), carves a piece
// of the region for them and runs ONE batched implicit step: every launch
// covers all of the batch's systems, each system keeps its own GMRES
// (fs_create_batch).  Requests that arrive while a batch is on the GPU join
// the next batch the other engine (or this one) forms, so the two engines'
// batches overlap on the device.  No request allocates: the batch context
// carves its buffers from the region, the operator tables are built once per
// point count, and the piece goes back to the region when the step ends.
//
// A request's arithmetic does not depend on its batch: the far fields run
// per system (work list) even for a batch of one, and every reduction of the
// Krylov solver is per system, so a request gives the same bits alone and in
// any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>

#include "context.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    std::vector<int32_t> ppf;
    std::vector<double> X, L, F;
    bool has_boundary = false;
    double R = 0.0;
    std::vector<double> bnodes, bnormals, bweights;
    double mu = 1, eps = 1e-3, E = 1, dt = 1e-3;
    fs_options opt{};
    double *out_X = nullptr, *out_V = nullptr, *out_T = nullptr;
    size_t bytes = 0;   // memory estimate of the request alone
    bool done = false;
    fs_status status = FS_OK;
    std::string err;
    fs_step_info info{};
    Clock::time_point t_submit, t_start, t_done;
};

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Requests that may share one batched step: the same physical parameters and
// solver options, no boundary.
bool same_step(const Req *a, const Req *b)
{
    return !a->has_boundary && !b->has_boundary && a->mu == b->mu && a->eps == b->eps && a->E == b->E &&
           a->dt == b->dt && std::memcmp(&a->opt, &b->opt, sizeof(fs_options)) == 0;
}

constexpr int kEngines = 2;
constexpr size_t kAlign = 256;

}  // namespace

namespace fs {

// Device memory a serving batch of these systems carves from the region:
// the context's arrays and its largest direct-sum scratch (as a context of
// all fibers), plus the per-system Krylov scalars and lists, plus slack for
// the 256-byte alignment of every piece.
size_t serving_batch_bytes(const std::vector<int32_t> &ppf, int n_systems, int n_surf, const fs_options &opt)
{
    size_t b = estimate_bytes(static_cast<int>(ppf.size()), ppf.data(), n_surf, opt);
    const int R = std::max(2, std::min(opt.restart, 250));
    b += static_cast<size_t>(n_systems) * (2 * (4 * size_t(R + 1) + 8) * sizeof(double) + 4096);
    return b + b / 50 + (1 << 20);
}

// Pinned host bytes a batch of n_systems carves (the GMRES scalars read back).
size_t serving_batch_host_bytes(int n_systems, const fs_options &opt)
{
    const int R = std::max(2, std::min(opt.restart, 250));
    return (4096 + static_cast<size_t>(n_systems) * (4 * size_t(R + 1) + 8 + 4 * 17 + 8)) * sizeof(double) +
           4 * kAlign;
}

}  // namespace fs

struct fs_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_slots = 1;
    char *region = nullptr;                  // the HBM budget, allocated once
    std::map<size_t, size_t> free_pieces;    // offset -> size, coalesced
    std::deque<Req *> pending;
    std::map<uint64_t, Req *> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> engines;
    bool stop = false;
    uint64_t next_ticket = 1;
    int64_t completed = 0, batches = 0;
    int running = 0;

    void engine_loop();
    size_t largest_free() const;
    bool take_piece(size_t bytes, size_t *off);
    void give_piece(size_t off, size_t bytes);
    bool form_batch(std::vector<Req *> &batch, size_t *off, size_t *bytes);
    void run_batch(std::vector<Req *> &batch, char *dev, size_t bytes, cudaStream_t st, char *pinned,
                   size_t pinned_cap);
};

size_t fs_server::largest_free() const
{
    size_t m = 0;
    for (auto &kv : free_pieces) m = std::max(m, kv.second);
    return m;
}

bool fs_server::take_piece(size_t bytes, size_t *off)
{
    bytes = (bytes + kAlign - 1) & ~(kAlign - 1);
    for (auto it = free_pieces.begin(); it != free_pieces.end(); ++it) {
        if (it->second < bytes) continue;
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_pieces.erase(it);
        if (rest) free_pieces[at] = rest;
        return true;
    }
    return false;
}

void fs_server::give_piece(size_t off, size_t bytes)
{
    bytes = (bytes + kAlign - 1) & ~(kAlign - 1);
    auto it = free_pieces.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_pieces.end() && it->first + it->second == next->first) {
        it->second += next->second;
        free_pieces.erase(next);
    }
    if (it != free_pieces.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            free_pieces.erase(it);
        }
    }
}

// Under the lock: the queue head and the queued requests that can share its
// step, as many as fit max_slots and the largest free piece.  False (nothing
// taken) when the queue is empty or the head alone does not fit yet.
bool fs_server::form_batch(std::vector<Req *> &batch, size_t *off, size_t *bytes)
{
    batch.clear();
    if (pending.empty()) return false;
    const size_t room = largest_free();
    Req *head = pending.front();
    std::vector<int32_t> ppf(head->ppf);
    const int n_surf = head->has_boundary ? static_cast<int>(head->bweights.size()) : 0;
    size_t need = fs::serving_batch_bytes(ppf, 1, n_surf, head->opt);
    if (need > room) return false;
    batch.push_back(head);
    const size_t scan = std::min(pending.size(), static_cast<size_t>(4 * max_slots + 4));
    for (size_t k = 1; k < scan && static_cast<int>(batch.size()) < max_slots; ++k) {
        Req *r = pending[k];
        if (!same_step(head, r)) continue;
        std::vector<int32_t> trial(ppf);
        trial.insert(trial.end(), r->ppf.begin(), r->ppf.end());
        const size_t b = fs::serving_batch_bytes(trial, static_cast<int>(batch.size()) + 1, 0, head->opt);
        if (b > room) continue;
        ppf.swap(trial);
        need = b;
        batch.push_back(r);
    }
    if (!take_piece(need, off)) {
        batch.clear();
        return false;
    }
    *bytes = need;
    for (Req *r : batch) pending.erase(std::find(pending.begin(), pending.end(), r));
    used += (need + kAlign - 1) & ~(kAlign - 1);
    running += static_cast<int>(batch.size());
    ++batches;
    return true;
}

void fs_server::run_batch(std::vector<Req *> &batch, char *dev, size_t bytes, cudaStream_t st, char *pinned,
                          size_t pinned_cap)
{
    const Clock::time_point t0 = Clock::now();
    for (Req *r : batch) r->t_start = t0;
    const int S = static_cast<int>(batch.size());
    const Req *h = batch.front();
    std::vector<int32_t> fps, ppf;
    std::vector<int64_t> node0(S + 1, 0);
    for (int s = 0; s < S; ++s) {
        fps.push_back(static_cast<int32_t>(batch[s]->ppf.size()));
        ppf.insert(ppf.end(), batch[s]->ppf.begin(), batch[s]->ppf.end());
        node0[s + 1] = node0[s] + static_cast<int64_t>(batch[s]->X.size() / 3);
    }
    const int64_t P = node0[S];
    std::vector<double> X(3 * P), L, F(3 * P), Xo(3 * P), Vo(3 * P), To(P);
    for (int s = 0; s < S; ++s) {
        std::copy(batch[s]->X.begin(), batch[s]->X.end(), X.begin() + 3 * node0[s]);
        std::copy(batch[s]->F.begin(), batch[s]->F.end(), F.begin() + 3 * node0[s]);
        L.insert(L.end(), batch[s]->L.begin(), batch[s]->L.end());
    }
    fs_boundary bd{};
    if (h->has_boundary) {
        bd.R = h->R;
        bd.n_nodes = static_cast<int32_t>(h->bweights.size());
        bd.nodes = h->bnodes.data();
        bd.normals = h->bnormals.data();
        bd.weights = h->bweights.data();
    }
    fs::Pool pool;
    pool.dev = dev;
    pool.dev_cap = bytes;
    pool.host = pinned;
    pool.host_cap = pinned_cap;
    fs_ctx *c = nullptr;
    fs_step_info inf{};
    fs_status s = fs::create_serving(&c, S, fps.data(), static_cast<int32_t>(ppf.size()), ppf.data(), h->mu, h->eps,
                                     h->E, h->dt, h->has_boundary ? &bd : nullptr, &h->opt, st, &pool);
    if (s == FS_OK) s = fs_set_state(c, X.data(), L.data(), F.data(), 0);
    if (s == FS_OK) s = fs_step(c, &inf);
    if (s == FS_OK) s = fs_get_state(c, Xo.data(), To.data(), Vo.data(), 0);
    std::vector<int32_t> its(S, 0), outer(S, 0), conv(S, 0);
    std::vector<double> resid(S, 0.0);
    if (s == FS_OK) s = fs_batch_info(c, its.data(), outer.data(), resid.data(), conv.data());
    const std::string err = s == FS_OK ? std::string() : std::string(fs_last_error());
    if (c) fs_destroy(c);   // region memory is not freed here: the piece goes back whole
    const Clock::time_point t1 = Clock::now();
    for (int k = 0; k < S; ++k) {
        Req *r = batch[k];
        r->status = s;
        r->err = err;
        r->info = inf;
        if (s == FS_OK) {
            const int64_t n0 = node0[k], n = node0[k + 1] - n0;
            std::memcpy(r->out_V, Vo.data() + 3 * n0, 3 * n * sizeof(double));
            if (r->out_X) std::memcpy(r->out_X, Xo.data() + 3 * n0, 3 * n * sizeof(double));
            if (r->out_T) std::memcpy(r->out_T, To.data() + n0, n * sizeof(double));
            r->info.iters = its[k];
            r->info.refine_sweeps = outer[k];
            r->info.resid = resid[k];
            double pairs = double(n) * double(n);
            for (int32_t q : r->ppf) pairs -= double(q) * double(q);
            r->info.pairs = static_cast<int64_t>(pairs);
            if (!conv[k]) {
                r->status = FS_ENOTCONV;
                char buf[160];
                std::snprintf(buf, sizeof(buf), "fs_step: not converged (rel. residual %.3e after %d iterations)",
                              resid[k], its[k]);
                r->err = buf;
            }
        }
        r->t_done = t1;
        r->info.t_ms[5] = ms_between(r->t_submit, r->t_start);
        r->info.t_ms[6] = ms_between(r->t_submit, r->t_done);
        r->info.t_ms[7] = static_cast<double>(S);   // requests in its batch
    }
}

void fs_server::engine_loop()
{
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    fs_options o;
    fs_options_default(&o);
    o.restart = 250;
    const size_t pinned_cap = fs::serving_batch_host_bytes(max_slots, o);
    char *pinned = nullptr;
    if (cudaMallocHost(&pinned, pinned_cap) != cudaSuccess) {
        cudaGetLastError();
        pinned = nullptr;
    }
    for (;;) {
        std::vector<Req *> batch;
        size_t off = 0, bytes = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || form_batch(batch, &off, &bytes); });
            if (stop) break;
        }
        if (pinned)
            run_batch(batch, region + off, bytes, st, pinned, pinned_cap);
        for (Req *r : batch)
            if (!pinned) {
                r->status = FS_ENOMEM;
                r->err = "serving: no pinned staging buffer";
            }
        {
            std::lock_guard<std::mutex> lk(mu);
            give_piece(off, bytes);
            used -= (bytes + kAlign - 1) & ~(kAlign - 1);
            running -= static_cast<int>(batch.size());
            for (Req *r : batch) {
                r->done = true;
                ++completed;
                // free copies of the inputs now; the ticket stays until polled
                std::vector<double>().swap(r->X);
                std::vector<double>().swap(r->F);
                std::vector<double>().swap(r->bnodes);
                std::vector<double>().swap(r->bnormals);
                std::vector<double>().swap(r->bweights);
            }
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
    if (pinned) cudaFreeHost(pinned);
    if (st) cudaStreamDestroy(st);
}

using namespace fs;

extern "C" {

fs_status fs_server_create(fs_server **out, size_t hbm_budget_bytes, int32_t max_slots, int32_t device)
{
    if (!out || max_slots < 1 || max_slots > 4096 || hbm_budget_bytes == 0) {
        set_error("fs_server_create: need a budget > 0 and 1..4096 slots");
        if (out) *out = nullptr;
        return FS_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_error("fs_server_create: no CUDA device %d", device);
        *out = nullptr;
        return FS_ECUDA;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    char *region = nullptr;
    const cudaError_t e = cudaMalloc(&region, hbm_budget_bytes);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("fs_server_create: cannot allocate the %zu-byte region: %s", hbm_budget_bytes,
                  cudaGetErrorString(e));
        *out = nullptr;
        return FS_ENOMEM;
    }
    fs_server *sv = new fs_server();
    sv->device = device;
    sv->budget = hbm_budget_bytes;
    sv->max_slots = max_slots;
    sv->region = region;
    sv->free_pieces[0] = hbm_budget_bytes & ~(kAlign - 1);
    for (int i = 0; i < kEngines; ++i) sv->engines.emplace_back([sv] { sv->engine_loop(); });
    *out = sv;
    return FS_OK;
}

fs_status fs_submit(fs_server *sv, const fs_request *rq, uint64_t *ticket)
{
    if (!sv || !rq || !ticket || rq->n_fibers < 1 || !rq->points_per_fiber || !rq->X || !rq->lengths ||
        !rq->out_V) {
        set_error("fs_submit: bad request");
        return FS_EINVAL;
    }
    if (!(rq->mu > 0.0) || !(rq->eps > 0.0 && rq->eps < 1.0) || !(rq->E >= 0.0) || !(rq->dt > 0.0)) {
        set_error("fs_submit: need mu > 0, 0 < eps < 1, E >= 0, dt > 0");
        return FS_EINVAL;
    }
    for (int32_t m = 0; m < rq->n_fibers; ++m)
        if (!(rq->lengths[m] > 0.0) || !std::isfinite(rq->lengths[m])) {
            set_error("fs_submit: fiber %d has length %g", m, rq->lengths[m]);
            return FS_EINVAL;
        }
    Req *r = new Req();
    r->ppf.assign(rq->points_per_fiber, rq->points_per_fiber + rq->n_fibers);
    int64_t ntot = 0;
    for (int32_t n : r->ppf) {
        if (n < 6 || n > 256) {
            delete r;
            set_error("fs_submit: points per fiber must be in [6, 256]");
            return FS_EINVAL;
        }
        ntot += n;
    }
    // a non-finite input would stop its whole batch's solve: refused here
    for (int64_t i = 0; i < 3 * ntot; ++i)
        if (!std::isfinite(rq->X[i]) || (rq->f_ext && !std::isfinite(rq->f_ext[i]))) {
            delete r;
            set_error("fs_submit: positions and forces must be finite (entry %lld)", static_cast<long long>(i));
            return FS_EINVAL;
        }
    r->X.assign(rq->X, rq->X + 3 * ntot);
    r->L.assign(rq->lengths, rq->lengths + rq->n_fibers);
    if (rq->f_ext) r->F.assign(rq->f_ext, rq->f_ext + 3 * ntot);
    else r->F.assign(3 * ntot, 0.0);
    if (rq->boundary) {
        const fs_boundary *b = rq->boundary;
        if (b->n_nodes <= 0 || !b->nodes || !b->normals || !b->weights) {
            delete r;
            set_error("fs_submit: incomplete boundary description");
            return FS_EINVAL;
        }
        r->has_boundary = true;
        r->R = b->R;
        r->bnodes.assign(b->nodes, b->nodes + 3 * int64_t(b->n_nodes));
        r->bnormals.assign(b->normals, b->normals + 3 * int64_t(b->n_nodes));
        r->bweights.assign(b->weights, b->weights + b->n_nodes);
    }
    r->mu = rq->mu;
    r->eps = rq->eps;
    r->E = rq->E;
    r->dt = rq->dt;
    fs_options_default(&r->opt);
    r->opt.prec = rq->prec;
    r->opt.tol = rq->tol > 0.0 ? rq->tol : r->opt.tol;
    if (check_options(r->opt, "fs_submit", 1) != FS_OK) {
        delete r;
        return FS_EINVAL;
    }
    r->out_X = rq->out_X;
    r->out_V = rq->out_V;
    r->out_T = rq->out_T;
    r->bytes = serving_batch_bytes(r->ppf, 1, r->has_boundary ? static_cast<int>(r->bweights.size()) : 0, r->opt);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (r->bytes > sv->budget) {
        const size_t need = r->bytes;
        delete r;
        set_error("fs_submit: the request needs ~%zu bytes, more than the server's budget", need);
        return FS_EBUSY;
    }
    r->ticket = sv->next_ticket++;
    r->t_submit = Clock::now();
    sv->reqs[r->ticket] = r;
    sv->pending.push_back(r);
    *ticket = r->ticket;
    sv->cv_work.notify_one();
    return FS_OK;
}

static fs_status finish(fs_server *sv, std::map<uint64_t, Req *>::iterator it, fs_step_info *info)
{
    Req *r = it->second;
    const fs_status s = r->status;
    if (info) *info = r->info;
    if (s != FS_OK) set_error("%s", r->err.c_str());
    sv->reqs.erase(it);
    delete r;
    return s;
}

fs_status fs_poll(fs_server *sv, uint64_t ticket, fs_step_info *info)
{
    if (!sv) {
        set_error("fs_poll: NULL server");
        return FS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
        set_error("fs_poll: unknown ticket %llu", static_cast<unsigned long long>(ticket));
        return FS_EINVAL;
    }
    if (!it->second->done) return FS_EAGAIN;
    return finish(sv, it, info);
}

fs_status fs_server_wait(fs_server *sv, uint64_t ticket, fs_step_info *info, double timeout_s)
{
    if (!sv) {
        set_error("fs_server_wait: NULL server");
        return FS_EINVAL;
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) {
        set_error("fs_server_wait: unknown ticket %llu", static_cast<unsigned long long>(ticket));
        return FS_EINVAL;
    }
    Req *r = it->second;
    const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
    if (!ok) {
        set_error("fs_server_wait: ticket %llu not done after %.3f s", static_cast<unsigned long long>(ticket),
                  timeout_s);
        return FS_ETIMEOUT;
    }
    return finish(sv, sv->reqs.find(ticket), info);
}

fs_status fs_server_stats(fs_server *sv, int32_t *pending, int32_t *running, size_t *bytes_in_use,
                          int64_t *completed)
{
    if (!sv) {
        set_error("fs_server_stats: NULL server");
        return FS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (pending) *pending = static_cast<int32_t>(sv->pending.size());
    if (running) *running = sv->running;
    if (bytes_in_use) *bytes_in_use = sv->used;
    if (completed) *completed = sv->completed;
    return FS_OK;
}

fs_status fs_server_batches(fs_server *sv, int64_t *batches)
{
    if (!sv || !batches) {
        set_error("fs_server_batches: NULL argument");
        return FS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    *batches = sv->batches;
    return FS_OK;
}

void fs_server_destroy(fs_server *sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        // requests never admitted are dropped with their tickets
        sv->pending.clear();
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->engines) t.join();
    for (auto &kv : sv->reqs) delete kv.second;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(sv->device);
    if (sv->region) cudaFree(sv->region);
    cudaSetDevice(prev);
    delete sv;
}

}  // extern "C"
