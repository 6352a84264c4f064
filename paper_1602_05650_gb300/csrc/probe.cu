// Measurement support: kernel launch counter, CUDA-event profiler of the
// direct sums, and an FMA-throughput probe of the CUDA-core pipes.
#include <cstring>

#include "context.h"

namespace fs {

unsigned long long g_launches = 0;

cudaEvent_t Profiler::get()
{
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
        e = pool.back();
        pool.pop_back();
        return e;
    }
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void Profiler::release_all()
{
    for (auto &r : recs) {
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

namespace {

// 8 independent FMA chains per thread keep the pipe busy; the result is
// stored so the loop is not removed.
template <class T>
__global__ void __launch_bounds__(256) k_fma_probe(T *out, int64_t iters, T seed)
{
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + T(threadIdx.x + k);
    const T m = T(0.999999), c = T(1e-7);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = a[k] * m + c;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace fs

using namespace fs;

extern "C" {

uint64_t fs_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

fs_status fs_kernel_stats(fs_ctx *c, fs_kernel_stat *out, int32_t reset)
{
    if (!c || !out) {
        set_error("fs_kernel_stats: NULL argument");
        return FS_EINVAL;
    }
    std::memset(out, 0, sizeof(fs_kernel_stat) * FS_KS_COUNT);
    FS_CUDA(cudaStreamSynchronize(c->stream));
    for (auto &r : c->prof.recs) {
        float ms = 0.0f;
        FS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
        if (r.cls >= 0 && r.cls < FS_KS_COUNT) {
            out[r.cls].launches += 1;
            out[r.cls].total_ms += ms;
            out[r.cls].pairs += r.pairs;
        }
    }
    if (reset) c->prof.release_all();
    return FS_OK;
}

fs_status fs_probe_fma(int32_t precision, double *flops_per_s)
{
    if (!flops_per_s || (precision != 0 && precision != 1)) {
        set_error("fs_probe_fma: bad arguments");
        return FS_EINVAL;
    }
    const int blocks = num_sms() * 8, threads = 256;
    const int64_t iters = precision == 1 ? (1 << 16) : (1 << 11);
    void *buf = nullptr;
    FS_CUDA(cudaMalloc(&buf, size_t(blocks) * threads * 8));
    cudaEvent_t e0, e1;
    FS_CUDA(cudaEventCreate(&e0));
    FS_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        FS_CUDA(cudaEventRecord(e0, 0));
        if (precision == 1)
            k_fma_probe<float><<<blocks, threads>>>(static_cast<float *>(buf), iters, 1.0f);
        else
            k_fma_probe<double><<<blocks, threads>>>(static_cast<double *>(buf), iters, 1.0);
        FS_LAUNCH_CHECK();
        FS_CUDA(cudaEventRecord(e1, 0));
        FS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        FS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best) best = ms;   // first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    *flops_per_s = 2.0 * 8.0 * double(iters) * blocks * threads / (double(best) * 1e-3);
    return FS_OK;
}

}  // extern "C"
