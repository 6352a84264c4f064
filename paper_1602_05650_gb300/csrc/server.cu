// Serving: independent fiber-suspension step requests admitted continuously.
//
// A server owns up to `max_slots` worker threads, each with its own CUDA
// stream.  Requests (host arrays) wait in a FIFO; a free worker admits the head
// of the queue as soon as its device-memory estimate fits the remaining HBM
// budget, builds its context on its stream, runs one implicit step and copies
// the result to the caller's host buffers.  Requests that arrive while others
// run are admitted as slots and memory free up, and their kernels overlap with
// the running ones on the GPU.  Each request computes exactly what fs_step
// computes for it alone (same kernels, same launch shapes), so results do not
// depend on the mix.
#include <algorithm>
#include <chrono>
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
    size_t bytes = 0;
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

}  // namespace

struct fs_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_slots = 1;
    std::deque<Req *> pending;
    std::map<uint64_t, Req *> reqs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    bool stop = false;
    uint64_t next_ticket = 1;
    int64_t completed = 0;

    void worker_loop();
};

void fs_server::worker_loop()
{
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    for (;;) {
        Req *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] {
                return stop || (!pending.empty() && used + pending.front()->bytes <= budget);
            });
            if (stop) break;
            r = pending.front();
            pending.pop_front();
            used += r->bytes;
        }
        r->t_start = Clock::now();
        fs_ctx *c = nullptr;
        fs_boundary bd{};
        if (r->has_boundary) {
            bd.R = r->R;
            bd.n_nodes = static_cast<int32_t>(r->bweights.size());
            bd.nodes = r->bnodes.data();
            bd.normals = r->bnormals.data();
            bd.weights = r->bweights.data();
        }
        fs_status s = fs_create(&c, static_cast<int32_t>(r->ppf.size()), r->ppf.data(), r->mu, r->eps, r->E,
                                r->dt, r->has_boundary ? &bd : nullptr, &r->opt, st);
        if (s == FS_OK) s = fs_set_state(c, r->X.data(), r->L.data(), r->F.data(), 0);
        fs_step_info inf{};
        if (s == FS_OK) s = fs_step(c, &inf);
        if (s == FS_OK) s = fs_get_state(c, r->out_X, r->out_T, r->out_V, 0);
        std::string err = s == FS_OK ? std::string() : std::string(fs_last_error());
        if (c) fs_destroy(c);
        {
            std::lock_guard<std::mutex> lk(mu);
            r->t_done = Clock::now();
            r->status = s;
            r->err = err;
            r->info = inf;
            r->info.t_ms[5] = ms_between(r->t_submit, r->t_start);
            r->info.t_ms[6] = ms_between(r->t_submit, r->t_done);
            r->done = true;
            used -= r->bytes;
            ++completed;
            // free copies of the inputs now; the ticket stays until polled
            std::vector<double>().swap(r->X);
            std::vector<double>().swap(r->F);
            std::vector<double>().swap(r->bnodes);
            std::vector<double>().swap(r->bnormals);
            std::vector<double>().swap(r->bweights);
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
}

using namespace fs;

extern "C" {

fs_status fs_server_create(fs_server **out, size_t hbm_budget_bytes, int32_t max_slots, int32_t device)
{
    if (!out || max_slots < 1 || max_slots > 256 || hbm_budget_bytes == 0) {
        set_error("fs_server_create: need a budget > 0 and 1..256 slots");
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
    fs_server *sv = new fs_server();
    sv->device = device;
    sv->budget = hbm_budget_bytes;
    sv->max_slots = max_slots;
    for (int i = 0; i < max_slots; ++i) sv->workers.emplace_back([sv] { sv->worker_loop(); });
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
    r->bytes = fs_estimate_bytes(rq->n_fibers, rq->points_per_fiber,
                                 r->has_boundary ? static_cast<int32_t>(r->bweights.size()) : 0, &r->opt);
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
    int run = 0;
    for (auto &kv : sv->reqs)
        if (!kv.second->done && std::find(sv->pending.begin(), sv->pending.end(), kv.second) == sv->pending.end())
            ++run;
    if (pending) *pending = static_cast<int32_t>(sv->pending.size());
    if (running) *running = run;
    if (bytes_in_use) *bytes_in_use = sv->used;
    if (completed) *completed = sv->completed;
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
    for (auto &t : sv->workers) t.join();
    for (auto &kv : sv->reqs) delete kv.second;
    delete sv;
}

}  // extern "C"
