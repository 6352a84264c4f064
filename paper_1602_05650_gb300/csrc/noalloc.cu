// Direct Stokeslet sum that allocates nothing.
//
// Some callers cannot let this library call cudaMalloc: applications whose own
// allocator owns (or has reserved) all of the device's memory, so that a
// driver allocation here would fail or fragment their pool, and latency-bound
// loops that cannot absorb the implicit device-wide synchronisation of
// cudaMalloc / cudaFree.  For them, fs_stokeslet_apply_noalloc runs the same
// kernels as fs_stokeslet_apply with its scratch in a fixed, file-scope device
// array instead of context memory.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace fs {
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;   // 32 MiB, held by every GPU that loads the library

// [0, 256): status word; [256, kNoAllocBytes): exclusion ranges and the direct-sum scratch
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the array for the current device (host code cannot use
// the array's name as a device pointer).  Resolved once per device.
fs_status scratch_address(void **out)
{
    int dev = 0;
    FS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("fs_stokeslet_apply_noalloc: device ordinal %d out of range", dev);
        return FS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("fs_stokeslet_apply_noalloc: cudaGetSymbolAddress failed: %s",
                      cudaGetErrorString(e));
            return FS_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return FS_OK;
}

}  // namespace
}  // namespace fs

using namespace fs;

extern "C" {

fs_status fs_stokeslet_apply_noalloc(const double *src_xyz, const double *src_wf, int64_t n_src,
                                     const int32_t *src_fiber, const double *tgt_xyz,
                                     const int32_t *tgt_fiber, int64_t n_tgt, double *out_u,
                                     double mu, int32_t sum_precision, void *cuda_stream)
{
    if (n_src < 0 || n_tgt < 0 || (n_src > 0 && (!src_xyz || !src_wf)) ||
        (n_tgt > 0 && (!tgt_xyz || !out_u)) || !(mu > 0.0)) {
        set_error("fs_stokeslet_apply_noalloc: bad sizes, NULL arrays or mu <= 0");
        return FS_EINVAL;
    }
    if (sum_precision != FS_SUM_FP32 && sum_precision != FS_SUM_FP64 && sum_precision != FS_SUM_FF &&
        sum_precision != FS_SUM_FP32_PLAIN) {
        set_error("fs_stokeslet_apply_noalloc: unknown precision %d", sum_precision);
        return FS_EINVAL;
    }
    const bool plain = sum_precision == FS_SUM_FP32_PLAIN;
    if (plain) sum_precision = FS_SUM_FP32;
    if (n_src >= (1LL << 31) - 1 || n_tgt >= (1LL << 31) - 1) {
        set_error("fs_stokeslet_apply_noalloc: at most 2^31-2 sources and targets");
        return FS_EINVAL;
    }
    const bool ids = src_fiber && tgt_fiber;
    const size_t excl_bytes = ids ? ((static_cast<size_t>(n_tgt) * sizeof(int2) + 255) & ~size_t(255)) : 0;
    const size_t need = 256 + excl_bytes + pairsum_scratch_bytes(PAIR_STOKESLET, n_src, n_tgt, sum_precision, 0);
    if (need > kNoAllocBytes) {
        set_error("fs_stokeslet_apply_noalloc: %lld sources x %lld targets need %zu bytes of scratch, "
                  "more than the fixed %zu bytes; use fs_stokeslet_apply",
                  static_cast<long long>(n_src), static_cast<long long>(n_tgt), need, kNoAllocBytes);
        return FS_EINVAL;
    }
    void *base = nullptr;
    FS_TRY(scratch_address(&base));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    char *b = static_cast<char *>(base);
    int *d_status = reinterpret_cast<int *>(b);
    FS_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));   // the array keeps the last call's contents
    PairSumArgs a;
    if (ids) {
        int2 *excl = reinterpret_cast<int2 *>(b + 256);
        FS_TRY(exclusion_from_ids(src_fiber, n_src, tgt_fiber, n_tgt, excl, st));
        a.excl = excl;
    }
    a.kind = PAIR_STOKESLET;
    a.src_xyz = src_xyz;
    a.src_dens = src_wf;
    a.n_src = n_src;
    a.tgt_xyz = tgt_xyz;
    a.n_tgt = n_tgt;
    a.out = out_u;
    a.scale = 1.0 / (8.0 * M_PI * mu);
    a.sum_prec = sum_precision;
    a.hilo = !plain;
    return pairsum(a, b + 256 + excl_bytes, kNoAllocBytes - 256 - excl_bytes, d_status, st);
}

}  // extern "C"
