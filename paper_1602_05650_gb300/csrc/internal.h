// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fibersolve.h"

namespace fs {

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);

#define FS_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::fs::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #call,                  \
                            cudaGetErrorString(e_));                                     \
            return FS_ECUDA;                                                             \
        }                                                                                \
    } while (0)

#define FS_TRY(expr)                                                                     \
    do {                                                                                 \
        fs_status s_ = (expr);                                                           \
        if (s_ != FS_OK) return s_;                                                      \
    } while (0)

extern unsigned long long g_launches;  // kernels launched by this library
#define FS_LAUNCH_CHECK()                                                                \
    do {                                                                                 \
        __atomic_add_fetch(&::fs::g_launches, 1ULL, __ATOMIC_RELAXED);                   \
        FS_CUDA(cudaGetLastError());                                                     \
    } while (0)

// Device status word bits written by kernels (never by faults).
enum : int {
    DEV_ERR_TIMEOUT = 1,   // a bounded mbarrier wait gave up
    DEV_ERR_NUMERIC = 2,   // non-finite value or zero pivot
};

// ---------------------------------------------------------------- scratch
// Grow-only device buffer owned by a context.
// A region of preallocated memory a context draws all of its buffers from
// instead of cudaMalloc / cudaMallocHost (serving: the server owns the
// memory, contexts only carve it).  Bump allocation, 256-byte pieces; the
// region is given back as a whole by its owner.
struct Pool {
    char *dev = nullptr;
    size_t dev_cap = 0, dev_used = 0;
    char *host = nullptr;   // pinned host memory
    size_t host_cap = 0, host_used = 0;
    void *take_dev(size_t bytes);    // nullptr when the region is exhausted
    void *take_host(size_t bytes);
};

struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
    Pool *pool = nullptr;   // draw from this region instead of cudaMalloc
    fs_status reserve(size_t need, cudaStream_t st);
    void release();
};

// Bump allocator over a caller-provided region (256-byte aligned pieces).
struct Carve {
    char *base;
    size_t used = 0, cap;
    Carve(void *b, size_t c) : base(static_cast<char *>(b)), cap(c) {}
    template <class T>
    T *take(size_t n) {
        used = (used + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base + used);
        used += n * sizeof(T);
        return p;
    }
};

// ---------------------------------------------------------------- direct sums
enum : int { PAIR_STOKESLET = 0, PAIR_STRESSLET = 1 };

// Launch plan of the tiled direct sums: nb target blocks of tb = tpt x
// threads targets, nt source tiles, W = nb x nt block-tile pairs shared out
// to `grid` CTAs (one wave) in equal contiguous runs.
struct SumPlan {
    int tpt;          // targets per thread
    int tile;         // sources per shared-memory stage
    int threads;      // threads per CTA
    int tb;           // targets per block
    int n_arr;        // packed per-source arrays
    size_t v4;        // bytes per packed array element
    size_t smem;      // dynamic shared memory per CTA
    int64_t nb, nt, W;
    int grid;
};

// CUDA-event records of direct-sum kernel launches (opt.profile).
struct Profiler {
    struct Rec {
        int cls;
        cudaEvent_t a, b;
        double pairs;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get();
    void release_all();
};

struct PairSumArgs {
    int kind = PAIR_STOKESLET;
    const double *src_xyz = nullptr;   // [n_src][3]
    const double *src_dens = nullptr;  // Stokeslet: W f [n_src][3]; stresslet: q [n_src][3]
    const double *src_w = nullptr;     // stresslet: quadrature weights [n_src] (else nullptr)
    const double *src_nrm = nullptr;   // stresslet: normals [n_src][3] (else nullptr)
    int64_t n_src = 0;
    const int2 *excl = nullptr;        // per target: skipped source index range [x, y)
    const double *tgt_xyz = nullptr;   // [n_tgt][3]
    int64_t n_tgt = 0;
    double *out = nullptr;             // [n_tgt][3]
    double scale = 1.0;                // applied to the kernel sum
    int sum_prec = FS_SUM_FP32;
    bool hilo = true;                  // FP32: hi/lo-split coordinates
    bool accumulate = false;           // out += scale * sum instead of out = ...
    int shape_override = 0;
    // batched systems: (target lo, target hi, source lo, source hi) per group;
    // each target block then sums only its group's sources (no source splits)
    const std::vector<int4> *groups = nullptr;
    int4 *work_dev = nullptr;          // device buffer for the work list
    int64_t work_cap = 0;
    Profiler *prof = nullptr;          // record the main kernel with CUDA events
    double pairs = 0.0;                // pairs evaluated (for the profiler)
    bool work_uploaded = false;        // the work list is on the device already (graph capture)
};

// slots > 0: CTAs one wave may hold (an upper bound will do); 0: ask the
// current device (SMs x resident CTAs of the chosen kernel).
SumPlan plan_pairsum(int kind, int64_t n_src, int64_t n_tgt, int sum_prec, bool hilo, int shape_override,
                     int slots);
size_t pairsum_scratch_bytes(int kind, int64_t n_src, int64_t n_tgt, int sum_prec, int shape_override,
                             int slots = 0);
// Enqueue the sum on `st`; scratch must hold pairsum_scratch_bytes(...) bytes.
fs_status pairsum(const PairSumArgs &a, void *scratch, size_t scratch_bytes, int *d_status,
                  cudaStream_t st);

// The work list of a.groups uploaded to a.work_dev (*items = its length;
// 0 without groups): what pairsum does before its launch, done ahead of a
// graph capture.
fs_status pairsum_work_list(const PairSumArgs &a, cudaStream_t st, int64_t *items);

// Exclusion ranges from non-decreasing source fiber ids (binary search per target).
fs_status exclusion_from_ids(const int32_t *src_fiber, int64_t n_src, const int32_t *tgt_fiber,
                             int64_t n_tgt, int2 *excl, cudaStream_t st);

int num_sms();

}  // namespace fs
