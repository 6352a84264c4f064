// Tiled all-pairs direct sums of the Stokes kernels.
//
//   Stokeslet (Eqs. oseen, single-layer, complementary-uf):
//     u(x_i) = sum_j G(x_i - y_j) wf_j,   G(r) = (I + rhat rhat) / (8 pi mu |r|),
//     evaluated as  u_i += rinv (wf + r (r.wf) rinv^2),  rinv = rsqrt(|r|^2);
//   stresslet double layer (Eqs. stresslet, double-layer, cortex-vel):
//     u(x_i) = sum_j w_j T(x_i - y_j):(q_j n_j),  T_abc = -(3/4 pi) rhat_a rhat_b rhat_c / |r|^2,
//     evaluated as  u_i += r (r.wq)(r.n) rinv^5  (the constant applied once at the end).
//
// Both are O(N^2) pair sums bound by the FP32 (or FP64) CUDA-core pipe -- not
// by memory and not dense contractions -- so they run on CUDA cores:
//   * each thread keeps T targets in registers;
//   * sources stream through shared memory in tiles copied by TMA bulk copies
//     (cp.async.bulk + mbarrier, two stages, non-multicast); all lanes read the
//     same source (broadcast), float4/double4_32a packed;
//   * FP32 path: optional hi/lo split of the centred coordinates so that
//     r = (xh - yh) + (xl - yl) keeps ~2^-48 relative accuracy in the difference;
//     FP32 per-tile partial sums, compensated (TwoSum) accumulation across tiles,
//     FP64 output;
//   * excluded pairs (same fiber / the target's own surface node) are skipped by
//     a per-pair index test only in the tiles that overlap a CTA's exclusions;
//   * sources may be split across CTAs so that small problems fill all SMs; the
//     partial sums are then reduced in FP64 in a fixed order (deterministic).
#include <algorithm>
#include <climits>
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>

#include "internal.h"

namespace fs {
namespace {

constexpr int kThreads = 128;
constexpr int kTile32 = 256;    // sources per stage, FP32 path
constexpr int kTile64 = 128;    // sources per stage, FP64 path
constexpr int kTileFF = 128;    // sources per stage, float-float path
constexpr int kWaitIters = 1 << 22;

// Per-source arrays: 0 = position (hi part), 1 = weighted density (W f or w q),
// 2 = normal (stresslet only), then the position lo part (FP32 hi/lo only).
template <int KIND, bool HILO>
struct Arr {
    static constexpr int base = KIND == PAIR_STRESSLET ? 3 : 2;
    static constexpr int n = base + (HILO ? 1 : 0);
};

// A CTA's share of a sum.  Default (stream-K) mode: a contiguous run of tiles
// g in [g0, g0 + n_run) of the flattened (target block, source tile) space,
// g = block * nt + tile, with g0 = c W / G for CTA c of G: every CTA of the
// single wave gets the same number of tiles to within one, whatever the
// problem's shape.  A run crosses target blocks; each block it touches is a
// "piece" whose partial sums go to slot (c + block) of the partial array.
// Work-list mode (batched systems): one item = one target block against its
// system's source range, written directly.
struct Run {
    int64_t g0 = 0, n_run = 0, nt = 0, n_src = 0;
    int4 wi = make_int4(0, 0, 0, 0);
    bool work = false;
    int tile = 0, tb = 0;

    __device__ Run(const int4 *work_list, int64_t nt_, int64_t W, int G, int64_t n_src_, int tile_, int tb_)
        : nt(nt_), n_src(n_src_), work(work_list != nullptr), tile(tile_), tb(tb_)
    {
        if (work) {
            wi = work_list[blockIdx.x];
            n_run = wi.w > wi.z ? (static_cast<int64_t>(wi.w) - wi.z + tile - 1) / tile : 0;
        } else {
            const int64_t c = blockIdx.x;
            g0 = c * W / G;
            n_run = (c + 1) * W / G - g0;
        }
    }
    // sources of tile `it` of the run: [j0, j0 + cnt)
    __device__ void src(int64_t it, int64_t &j0, int &cnt) const
    {
        int64_t end;
        if (work) {
            j0 = wi.z + it * tile;
            end = wi.w;
        } else {
            j0 = ((g0 + it) % nt) * tile;
            end = n_src;
        }
        cnt = static_cast<int>(min(static_cast<int64_t>(tile), end - j0));
    }
    // the piece starting at tile `it`: targets [tbase, t_end), length in tiles, target block
    __device__ void piece(int64_t it, int64_t n_tgt, int64_t &tbase, int64_t &t_end, int64_t &len,
                          int64_t &blk) const
    {
        if (work) {
            tbase = wi.x;
            t_end = static_cast<int64_t>(wi.x) + wi.y;
            len = n_run;
            blk = 0;
        } else {
            const int64_t g = g0 + it;
            blk = g / nt;
            len = min(nt - (g - blk * nt), n_run - it);
            tbase = blk * tb;
            t_end = n_tgt;
        }
    }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// TMA bulk copy global -> this CTA's shared memory, completing on `bar`.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for the phase with the given parity; false after kWaitIters polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < kWaitIters; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void two_sum(float &s, float &c, float b)
{
    const float a = s;
    const float t = a + b;
    const float bp = t - a;
    c += (a - (t - bp)) + (b - bp);
    s = t;
}

template <class V>
struct Vec4Of;
template <>
struct Vec4Of<float> {
    using type = float4;
};
template <>
struct Vec4Of<double> {
    using type = double4_32a;
};

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// One tile of sources against T register-resident targets.
template <class R, int T, int KIND, bool HILO, bool MASK>
__device__ __forceinline__ void tile_sum(const typename Vec4Of<R>::type *__restrict__ sp,
                                         const typename Vec4Of<R>::type *__restrict__ sw,
                                         const typename Vec4Of<R>::type *__restrict__ sn,
                                         const typename Vec4Of<R>::type *__restrict__ sl, int cnt,
                                         int j0, const R (&tx)[T], const R (&ty)[T], const R (&tz)[T],
                                         const R (&lx)[T], const R (&ly)[T], const R (&lz)[T],
                                         const int (&elo)[T], const int (&ecnt)[T], R (&ax)[T],
                                         R (&ay)[T], R (&az)[T])
{
    using V4 = typename Vec4Of<R>::type;
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
        const V4 p = sp[j];
        const V4 f = sw[j];
        V4 nn, pl;
        if constexpr (KIND == PAIR_STRESSLET) nn = sn[j];
        if constexpr (HILO) pl = sl[j];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            R dx, dy, dz;
            if constexpr (HILO) {
                dx = (tx[t] - p.x) + (lx[t] - pl.x);
                dy = (ty[t] - p.y) + (ly[t] - pl.y);
                dz = (tz[t] - p.z) + (lz[t] - pl.z);
            } else {
                dx = tx[t] - p.x;
                dy = ty[t] - p.y;
                dz = tz[t] - p.z;
            }
            const R r2 = fma_t(dz, dz, fma_t(dy, dy, dx * dx));
            R ri = rsqrt_t(r2);
            if constexpr (MASK) {
                if (static_cast<unsigned>(j0 + j - elo[t]) < static_cast<unsigned>(ecnt[t])) ri = R(0);
            }
            const R rf = fma_t(dz, f.z, fma_t(dy, f.y, dx * f.x));
            if constexpr (KIND == PAIR_STOKESLET) {
                const R s = rf * (ri * ri);
                ax[t] = fma_t(ri, fma_t(s, dx, f.x), ax[t]);
                ay[t] = fma_t(ri, fma_t(s, dy, f.y), ay[t]);
                az[t] = fma_t(ri, fma_t(s, dz, f.z), az[t]);
            } else {
                const R rn = fma_t(dz, nn.z, fma_t(dy, nn.y, dx * nn.x));
                const R ri2 = ri * ri;
                const R s = (rf * rn) * (ri2 * ri2 * ri);
                ax[t] = fma_t(s, dx, ax[t]);
                ay[t] = fma_t(s, dy, ay[t]);
                az[t] = fma_t(s, dz, az[t]);
            }
        }
    }
}

// Work-list mode: out[i] = (acc ? out[i] : 0) + scale * sum.  Stream-K mode:
// part[(c + block) * TB + local][3] = this CTA's partial sum (reduced by
// k_reduce_streamk).
template <class R, int T, int KIND, bool HILO>
__global__ void __launch_bounds__(kThreads)
    k_pairsum(const typename Vec4Of<R>::type *__restrict__ src, int64_t n_src, int64_t nt, int64_t W, int G,
              const double *__restrict__ tgt, const int2 *__restrict__ excl, int64_t n_tgt,
              const double *__restrict__ center, double *__restrict__ out, double *__restrict__ part,
              double scale, int acc, int *__restrict__ status, const int4 *__restrict__ work)
{
    using V4 = typename Vec4Of<R>::type;
    using A = Arr<KIND, HILO>;
    constexpr int TILE = sizeof(R) == 4 ? kTile32 : kTile64;
    constexpr int TB = T * kThreads;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V4 *smem = reinterpret_cast<V4 *>(smem_raw);   // [stage][array][TILE]
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_lo, s_hi;

    const int tid = threadIdx.x;
    const Run run(work, nt, W, G, n_src, TILE, TB);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto stage_ptr = [&](int stage, int arr) -> V4 * { return smem + (stage * A::n + arr) * TILE; };
    auto issue = [&](int64_t it) {
        int64_t j0;
        int cnt;
        run.src(it, j0, cnt);
        const int stage = static_cast<int>(it & 1);
        const uint32_t bytes = static_cast<uint32_t>(cnt) * static_cast<uint32_t>(sizeof(V4));
        mbar_expect_tx(&bars[stage], bytes * A::n);
#pragma unroll
        for (int a = 0; a < A::n; ++a) bulk_g2s(stage_ptr(stage, a), src + a * n_src + j0, bytes, &bars[stage]);
    };
    if (tid == 0) {
        if (run.n_run > 0) issue(0);
        if (run.n_run > 1) issue(1);
    }
    const double c0 = center[0], c1 = center[1], c2 = center[2];
    bool failed = false;
    int64_t it = 0;
    do {
        int64_t tbase, t_end, len, blk;
        run.piece(it, n_tgt, tbase, t_end, len, blk);
        // this piece's targets in registers, and the block's exclusion bounds
        if (tid == 0) {
            s_lo = INT_MAX;
            s_hi = INT_MIN;
        }
        R tx[T], ty[T], tz[T], lx[T], ly[T], lz[T];
        int elo[T], ecnt[T];
        int my_lo = INT_MAX, my_hi = INT_MIN;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = tbase + tid + static_cast<int64_t>(t) * kThreads;
            double x = 0.0, y = 0.0, z = 0.0;
            int2 e = make_int2(0, 0);
            if (i < t_end) {
                x = tgt[3 * i + 0] - c0;
                y = tgt[3 * i + 1] - c1;
                z = tgt[3 * i + 2] - c2;
                if (excl) e = excl[i];
            }
            tx[t] = static_cast<R>(x);
            ty[t] = static_cast<R>(y);
            tz[t] = static_cast<R>(z);
            lx[t] = static_cast<R>(x - static_cast<double>(tx[t]));
            ly[t] = static_cast<R>(y - static_cast<double>(ty[t]));
            lz[t] = static_cast<R>(z - static_cast<double>(tz[t]));
            elo[t] = e.x;
            ecnt[t] = e.y > e.x ? e.y - e.x : 0;
            if (e.y > e.x) {
                my_lo = min(my_lo, e.x);
                my_hi = max(my_hi, e.y);
            }
        }
        __syncthreads();
        if (my_hi > my_lo) {
            atomicMin(&s_lo, my_lo);
            atomicMax(&s_hi, my_hi);
        }
        __syncthreads();
        const int blo = s_lo, bhi = s_hi;

        // FP32: compensated cross-tile sums (s, c); FP64: plain accumulation in s
        R sx[T], sy[T], sz[T], cx[T], cy[T], cz[T];
#pragma unroll
        for (int t = 0; t < T; ++t) sx[t] = sy[t] = sz[t] = cx[t] = cy[t] = cz[t] = R(0);
        for (int64_t q = 0; q < len; ++q, ++it) {
            const int stage = static_cast<int>(it & 1);
            const bool ok = mbar_wait(&bars[stage], static_cast<uint32_t>((it >> 1) & 1));
            if (!__syncthreads_and(ok)) {
                failed = true;
                break;
            }
            // every thread has finished tile it-1, so its stage can be refilled
            if (tid == 0 && it >= 1 && it + 1 < run.n_run) issue(it + 1);
            int64_t j0;
            int cnt;
            run.src(it, j0, cnt);
            const bool masked = bhi > blo && j0 < bhi && j0 + cnt > blo;
            const V4 *p0 = stage_ptr(stage, 0), *p1 = stage_ptr(stage, 1);
            const V4 *pn = stage_ptr(stage, KIND == PAIR_STRESSLET ? 2 : 1);
            const V4 *pl = stage_ptr(stage, A::base < A::n ? A::base : 0);
            if constexpr (sizeof(R) == 4) {
                R ax[T], ay[T], az[T];
#pragma unroll
                for (int t = 0; t < T; ++t) ax[t] = ay[t] = az[t] = R(0);
                if (masked)
                    tile_sum<R, T, KIND, HILO, true>(p0, p1, pn, pl, cnt, static_cast<int>(j0), tx, ty, tz,
                                                     lx, ly, lz, elo, ecnt, ax, ay, az);
                else
                    tile_sum<R, T, KIND, HILO, false>(p0, p1, pn, pl, cnt, static_cast<int>(j0), tx, ty, tz,
                                                      lx, ly, lz, elo, ecnt, ax, ay, az);
#pragma unroll
                for (int t = 0; t < T; ++t) {
                    two_sum(sx[t], cx[t], ax[t]);
                    two_sum(sy[t], cy[t], ay[t]);
                    two_sum(sz[t], cz[t], az[t]);
                }
            } else {
                if (masked)
                    tile_sum<R, T, KIND, false, true>(p0, p1, pn, pl, cnt, static_cast<int>(j0), tx, ty, tz,
                                                      lx, ly, lz, elo, ecnt, sx, sy, sz);
                else
                    tile_sum<R, T, KIND, false, false>(p0, p1, pn, pl, cnt, static_cast<int>(j0), tx, ty, tz,
                                                       lx, ly, lz, elo, ecnt, sx, sy, sz);
            }
        }
        if (failed) break;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = tbase + tid + static_cast<int64_t>(t) * kThreads;
            if (i >= t_end) continue;
            const double ux = static_cast<double>(sx[t]) + static_cast<double>(cx[t]);
            const double uy = static_cast<double>(sy[t]) + static_cast<double>(cy[t]);
            const double uz = static_cast<double>(sz[t]) + static_cast<double>(cz[t]);
            if (work) {
                double *o = out + 3 * i;
                o[0] = (acc ? o[0] : 0.0) + scale * ux;
                o[1] = (acc ? o[1] : 0.0) + scale * uy;
                o[2] = (acc ? o[2] : 0.0) + scale * uz;
            } else {
                double *o = part + ((static_cast<int64_t>(blockIdx.x) + blk) * TB + tid + t * kThreads) * 3;
                o[0] = ux;
                o[1] = uy;
                o[2] = uz;
            }
        }
    } while (it < run.n_run);
    if (failed) {
        if (tid == 0) {
            atomicOr(status, DEV_ERR_TIMEOUT);
            // let copies already in flight land before the CTA exits (bounded)
            mbar_wait(&bars[0], 0);
            mbar_wait(&bars[1], 0);
        }
    }
}

// ------------------------------------------------- FP32 Stokeslet, packed pairs
// The FP32 Stokeslet sum in Blackwell's packed two-lane FP32 instructions
// (__fadd2_rn / __fmul2_rn / __ffma2_rn: one instruction evaluates the same
// source against two targets), so that the 17 FP32 operations of a pair take
// 8.5 issue slots and the kernel is bound by the FMA pipe, not by issue.
//
// Per pair: 16 FP32 operations (3 differences, 3 for |r|^2, 3 for r.(W f),
// one for (r.(W f))/|r|^2, 3 + 3 for the accumulation) plus two MUFU
// operations (rsqrt, rcp).
//
// Coordinates in a per-thread frame.  Each thread holds T consecutive
// targets (normally nodes of one fiber) and a frame origin g = (float) of its
// middle target's coordinates relative to the sources' bounding-box centre
// (exactly representable in FP32).  Targets are stored as t - g rounded once
// from FP64; a source arrives as hi + lo floats of s - centre and is moved
// into the frame once per thread as (g - s_hi) - s_lo.  For the sources near
// a thread's targets, g - s_hi is exact (Sterbenz), so the rounding of the
// pair difference is relative to the pair's own distance and the fiber's
// extent, not to the extent of the whole point set (the accuracy of the hi/lo
// kernel at the cost of 6 FP32 operations per source per thread, 0.75 per
// pair at T = 8).
// Approximate reciprocal on the MUFU unit (PTX rcp.approx.ftz.f32, about
// 1 ulp); used for 1/|r|^2 beside rsqrt's 1/|r|.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int T, bool MASK>
__device__ __forceinline__ void tile_x2(const float4 *__restrict__ sp, const float4 *__restrict__ sw,
                                        const float4 *__restrict__ sl, int cnt, int j0, float gx, float gy,
                                        float gz, const float2 (&tx)[T / 2], const float2 (&ty)[T / 2],
                                        const float2 (&tz)[T / 2], const int2 *__restrict__ ex,
                                        float2 (&ax)[T / 2], float2 (&ay)[T / 2], float2 (&az)[T / 2])
{
    // masked tiles (those that overlap some target's own fiber): the
    // targets' excluded source ranges, [lo, lo + cnt)
    int elo[MASK ? T : 1], ecnt[MASK ? T : 1];
    if constexpr (MASK) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int2 e = ex[t];
            elo[t] = e.x;
            ecnt[t] = e.y > e.x ? e.y - e.x : 0;
        }
    }
#pragma unroll 8
    for (int j = 0; j < cnt; ++j) {
        const float4 p = sp[j], f = sw[j], l = sl[j];
        // minus the source in the thread's frame
        const float nx = (gx - p.x) - l.x, ny = (gy - p.y) - l.y, nz = (gz - p.z) - l.z;
        const float2 NX = make_float2(nx, nx), NY = make_float2(ny, ny), NZ = make_float2(nz, nz);
        const float2 FX = make_float2(f.x, f.x), FY = make_float2(f.y, f.y), FZ = make_float2(f.z, f.z);
#pragma unroll
        for (int q = 0; q < T / 2; ++q) {
            const float2 dx = __fadd2_rn(tx[q], NX);
            const float2 dy = __fadd2_rn(ty[q], NY);
            const float2 dz = __fadd2_rn(tz[q], NZ);
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            // 1/|r| and 1/|r|^2 both on the MUFU unit (the FMA pipe is the bound)
            float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
            float2 ri2 = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
            if constexpr (MASK) {
                if (static_cast<unsigned>(j0 + j - elo[2 * q]) < static_cast<unsigned>(ecnt[2 * q]))
                    ri.x = ri2.x = 0.0f;
                if (static_cast<unsigned>(j0 + j - elo[2 * q + 1]) < static_cast<unsigned>(ecnt[2 * q + 1]))
                    ri.y = ri2.y = 0.0f;
            }
            float2 rf = __fmul2_rn(dx, FX);
            rf = __ffma2_rn(dy, FY, rf);
            rf = __ffma2_rn(dz, FZ, rf);
            const float2 s = __fmul2_rn(rf, ri2);
            ax[q] = __ffma2_rn(ri, __ffma2_rn(s, dx, FX), ax[q]);
            ay[q] = __ffma2_rn(ri, __ffma2_rn(s, dy, FY), ay[q]);
            az[q] = __ffma2_rn(ri, __ffma2_rn(s, dz, FZ), az[q]);
        }
    }
}

// Resident CTAs per SM the packed kernel is compiled for: 4 at 8 targets per
// thread (16 warps per SM; at 3 the FMA pipe idled for want of eligible warps).
template <int T>
struct X2Occ {
    static constexpr int value = T >= 8 ? 4 : 6;
};

// Shared memory of the packed kernel beyond its source stages: the
// compensated cross-tile sums (s, c) of x, y, z for T targets per thread.
__host__ __device__ constexpr size_t x2_sum_bytes(int T) { return size_t(6) * T * kThreads * sizeof(float); }

// Same schedule and outputs as k_pairsum (stream-K partials or work-list
// items); sources packed as [0] position hi, [1] W f, [2] position lo.
// Target i of a piece is tbase + tid T + t.  The cross-tile sums live in
// shared memory ([value][target][thread], conflict-free) to keep the
// registers within four CTAs per SM.
template <int T>
__global__ void __launch_bounds__(kThreads, X2Occ<T>::value)
    k_stokeslet_x2(const float4 *__restrict__ src, int64_t n_src, int64_t nt, int64_t W, int G,
                   const double *__restrict__ tgt, const int2 *__restrict__ excl, int64_t n_tgt,
                   const double *__restrict__ center, double *__restrict__ out, double *__restrict__ part,
                   double scale, int acc, int *__restrict__ status, const int4 *__restrict__ work)
{
    static_assert(T % 2 == 0, "targets per thread come in pairs");
    constexpr int NARR = 3, TILE = kTile32, TB = T * kThreads, NP = T / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *smem = reinterpret_cast<float4 *>(smem_raw);   // [stage][array][TILE]
    float *sums = reinterpret_cast<float *>(smem + 2 * NARR * TILE);   // [6][T][kThreads]
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_lo, s_hi;

    const int tid = threadIdx.x;
    const Run run(work, nt, W, G, n_src, TILE, TB);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto stage_ptr = [&](int stage, int arr) -> float4 * { return smem + (stage * NARR + arr) * TILE; };
    auto issue = [&](int64_t it) {
        int64_t j0;
        int cnt;
        run.src(it, j0, cnt);
        const int stage = static_cast<int>(it & 1);
        const uint32_t bytes = static_cast<uint32_t>(cnt) * 16u;
        mbar_expect_tx(&bars[stage], bytes * NARR);
#pragma unroll
        for (int a = 0; a < NARR; ++a) bulk_g2s(stage_ptr(stage, a), src + a * n_src + j0, bytes, &bars[stage]);
    };
    if (tid == 0) {
        if (run.n_run > 0) issue(0);
        if (run.n_run > 1) issue(1);
    }
    auto sum_at = [&](int v, int t) -> float & { return sums[(v * T + t) * kThreads + tid]; };
    const double c0 = center[0], c1 = center[1], c2 = center[2];
    bool failed = false;
    int64_t it = 0;
    do {
        int64_t tbase, t_end, len, blk;
        run.piece(it, n_tgt, tbase, t_end, len, blk);
        if (tid == 0) {
            s_lo = INT_MAX;
            s_hi = INT_MIN;
        }
        const int64_t i0 = tbase + static_cast<int64_t>(tid) * T;
        // frame origin: the middle target (else the first valid one), rounded
        // to FP32 -- unless the thread's targets spread farther from it than
        // it lies from the centre (targets that are not nodes of one fiber),
        // where the centre itself rounds no worse
        const int64_t im = i0 + T / 2 < t_end ? i0 + T / 2 : i0;
        float gx = 0.0f, gy = 0.0f, gz = 0.0f;
        if (im < t_end) {
            const double mx = tgt[3 * im + 0] - c0, my = tgt[3 * im + 1] - c1, mz = tgt[3 * im + 2] - c2;
            double spread = 0.0;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const int64_t i = i0 + t;
                if (i < t_end)
                    spread = fmax(spread, fmax(fabs(tgt[3 * i] - c0 - mx),
                                               fmax(fabs(tgt[3 * i + 1] - c1 - my), fabs(tgt[3 * i + 2] - c2 - mz))));
            }
            if (spread < fmax(fabs(mx), fmax(fabs(my), fabs(mz)))) {
                gx = static_cast<float>(mx);
                gy = static_cast<float>(my);
                gz = static_cast<float>(mz);
            }
        }
        float2 tx[NP], ty[NP], tz[NP];
        int my_lo = INT_MAX, my_hi = INT_MIN;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = i0 + t;
            double x = 0.0, y = 0.0, z = 0.0;
            if (i < t_end) {
                x = (tgt[3 * i + 0] - c0) - static_cast<double>(gx);
                y = (tgt[3 * i + 1] - c1) - static_cast<double>(gy);
                z = (tgt[3 * i + 2] - c2) - static_cast<double>(gz);
                if (excl) {
                    const int2 e = excl[i];
                    if (e.y > e.x) {
                        my_lo = min(my_lo, e.x);
                        my_hi = max(my_hi, e.y);
                    }
                }
            }
            float *px = reinterpret_cast<float *>(&tx[t / 2]) + (t & 1);
            float *py = reinterpret_cast<float *>(&ty[t / 2]) + (t & 1);
            float *pz = reinterpret_cast<float *>(&tz[t / 2]) + (t & 1);
            *px = static_cast<float>(x);
            *py = static_cast<float>(y);
            *pz = static_cast<float>(z);
#pragma unroll
            for (int v = 0; v < 6; ++v) sum_at(v, t) = 0.0f;
        }
        __syncthreads();
        if (my_hi > my_lo) {
            atomicMin(&s_lo, my_lo);
            atomicMax(&s_hi, my_hi);
        }
        __syncthreads();
        const int blo = s_lo, bhi = s_hi;

        for (int64_t q = 0; q < len; ++q, ++it) {
            const int stage = static_cast<int>(it & 1);
            const bool ok = mbar_wait(&bars[stage], static_cast<uint32_t>((it >> 1) & 1));
            if (!__syncthreads_and(ok)) {
                failed = true;
                break;
            }
            if (tid == 0 && it >= 1 && it + 1 < run.n_run) issue(it + 1);
            int64_t j0;
            int cnt;
            run.src(it, j0, cnt);
            const bool masked = bhi > blo && j0 < bhi && j0 + cnt > blo;
            float2 ax[NP], ay[NP], az[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) ax[p] = ay[p] = az[p] = make_float2(0.0f, 0.0f);
            if (masked) {
                // targets past the end (a ragged last block) carry an empty range
                int2 ex[T];
#pragma unroll
                for (int t = 0; t < T; ++t) ex[t] = (excl && i0 + t < t_end) ? excl[i0 + t] : make_int2(0, 0);
                tile_x2<T, true>(stage_ptr(stage, 0), stage_ptr(stage, 1), stage_ptr(stage, 2), cnt,
                                 static_cast<int>(j0), gx, gy, gz, tx, ty, tz, ex, ax, ay, az);
            } else {
                tile_x2<T, false>(stage_ptr(stage, 0), stage_ptr(stage, 1), stage_ptr(stage, 2), cnt,
                                  static_cast<int>(j0), gx, gy, gz, tx, ty, tz, nullptr, ax, ay, az);
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float v[6] = {ax[p].x, ax[p].y, ay[p].x, ay[p].y, az[p].x, az[p].y};
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const int t = 2 * p + (k & 1), comp = k >> 1;
                    float sv = sum_at(comp, t), cv = sum_at(3 + comp, t);
                    two_sum(sv, cv, v[k]);
                    sum_at(comp, t) = sv;
                    sum_at(3 + comp, t) = cv;
                }
            }
        }
        if (failed) break;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = i0 + t;
            if (i >= t_end) continue;
            const double ux = static_cast<double>(sum_at(0, t)) + static_cast<double>(sum_at(3, t));
            const double uy = static_cast<double>(sum_at(1, t)) + static_cast<double>(sum_at(4, t));
            const double uz = static_cast<double>(sum_at(2, t)) + static_cast<double>(sum_at(5, t));
            if (work) {
                double *o = out + 3 * i;
                o[0] = (acc ? o[0] : 0.0) + scale * ux;
                o[1] = (acc ? o[1] : 0.0) + scale * uy;
                o[2] = (acc ? o[2] : 0.0) + scale * uz;
            } else {
                double *o = part + ((static_cast<int64_t>(blockIdx.x) + blk) * TB + tid * T + t) * 3;
                o[0] = ux;
                o[1] = uy;
                o[2] = uz;
            }
        }
    } while (it < run.n_run);
    if (failed) {
        if (tid == 0) {
            atomicOr(status, DEV_ERR_TIMEOUT);
            mbar_wait(&bars[0], 0);
            mbar_wait(&bars[1], 0);
        }
    }
}

// ------------------------------------------------------------ float-float
// Stokeslet sum in float-float ("double-single") arithmetic on the FP32 pipe:
// every quantity is an unevaluated sum hi + lo of two floats, built from
// Knuth's TwoSum and the FMA-based TwoProduct; 1/sqrt(r^2) is the MUFU seed
// refined by one Newton step in float-float.  Each pair carries ~2^-44
// relative rounding (vs 2^-24 in FP32), at ~10x the FP32 instruction count --
// far cheaper than the FP64 pipe on this GPU.  Used for the right-hand side
// and the refinement residuals of the mixed-precision step.
__device__ __forceinline__ void ts(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fts(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}

template <int T, bool MASK>
__device__ __forceinline__ void tile_ff(const float4 *__restrict__ sph, const float4 *__restrict__ spl,
                                        const float4 *__restrict__ sfh, const float4 *__restrict__ sfl,
                                        int cnt, int j0, const float (&th)[T][3], const float (&tl)[T][3],
                                        const int (&elo)[T], const int (&ecnt)[T], float (&uh)[T][3],
                                        float (&ul)[T][3])
{
#pragma unroll 1
    for (int j = 0; j < cnt; ++j) {
        const float4 ph4 = sph[j], pl4 = spl[j], fh4 = sfh[j], fl4 = sfl[j];
        const float ph[3] = {ph4.x, ph4.y, ph4.z}, pl[3] = {pl4.x, pl4.y, pl4.z};
        const float fh[3] = {fh4.x, fh4.y, fh4.z}, fl[3] = {fl4.x, fl4.y, fl4.z};
#pragma unroll
        for (int t = 0; t < T; ++t) {
            float dh[3], dl[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float e;
                ts(th[t][a], -ph[a], dh[a], e);
                dl[a] = (tl[t][a] - pl[a]) + e;
            }
            // r^2 = sum (dh + dl)^2
            float p[3], pe[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                p[a] = dh[a] * dh[a];
                pe[a] = fmaf(dh[a], dh[a], -p[a]);
            }
            float S, e1, S2, e2;
            ts(p[0], p[1], S, e1);
            ts(S, p[2], S2, e2);
            float lo = (e1 + e2) + (pe[0] + pe[1] + pe[2]);
            lo = fmaf(2.0f * dh[0], dl[0], lo);
            lo = fmaf(2.0f * dh[1], dl[1], lo);
            lo = fmaf(2.0f * dh[2], dl[2], lo);
            float R, Rl;
            fts(S2, lo, R, Rl);
            bool skip = false;
            if constexpr (MASK) {
                skip = static_cast<unsigned>(j0 + j - elo[t]) < static_cast<unsigned>(ecnt[t]);
                if (skip) {
                    R = 1.0f;
                    Rl = 0.0f;
                }
            }
            // rinv = y + yl: one Newton step on the rsqrt seed, residual in float-float
            float y = rsqrtf(R);
            const float hh = y * y, hl = fmaf(y, y, -hh);
            const float qh = R * hh;
            float ql = fmaf(R, hh, -qh);
            ql = fmaf(R, hl, ql);
            ql = fmaf(Rl, hh, ql);
            const float ee = (1.0f - qh) - ql;
            float yl = 0.5f * y * ee;
            if constexpr (MASK) {
                if (skip) {
                    y = 0.0f;
                    yl = 0.0f;
                }
            }
            // rinv^2
            const float r2h = y * y;
            const float r2l = fmaf(2.0f * y, yl, fmaf(y, y, -r2h));
            // r . wf
            float q[3], qe[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                q[a] = dh[a] * fh[a];
                qe[a] = fmaf(dh[a], fh[a], -q[a]);
            }
            float F1, f1, F2, f2;
            ts(q[0], q[1], F1, f1);
            ts(F1, q[2], F2, f2);
            float flo = (f1 + f2) + (qe[0] + qe[1] + qe[2]);
#pragma unroll
            for (int a = 0; a < 3; ++a) flo = fmaf(dh[a], fl[a], fmaf(dl[a], fh[a], flo));
            float Fh, Fl;
            fts(F2, flo, Fh, Fl);
            // s = (r . wf) rinv^2
            const float sh = Fh * r2h;
            float sl = fmaf(Fh, r2h, -sh);
            sl = fmaf(Fh, r2l, sl);
            sl = fmaf(Fl, r2h, sl);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // v = wf + s r
                const float mh = sh * dh[a];
                float ml = fmaf(sh, dh[a], -mh);
                ml = fmaf(sh, dl[a], ml);
                ml = fmaf(sl, dh[a], ml);
                float vh, ve;
                ts(fh[a], mh, vh, ve);
                const float vl = (ve + fl[a]) + ml;
                // u += rinv v
                const float wh = y * vh;
                float wl = fmaf(y, vh, -wh);
                wl = fmaf(y, vl, wl);
                wl = fmaf(yl, vh, wl);
                float nh, ne;
                ts(uh[t][a], wh, nh, ne);
                ul[t][a] += ne + wl;
                uh[t][a] = nh;
            }
        }
    }
}

// Float-float stresslet: u_i += r (r . wq)(r . n) rinv^5 over the tile
// (the constant -3/(4 pi) is applied once at the end), every product and sum
// in float-float as in tile_ff.  Arrays: position hi/lo, w q hi/lo, normal hi/lo.
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float &ph, float &pl)
{
    ph = ah * bh;
    pl = fmaf(ah, bh, -ph);
    pl = fmaf(ah, bl, pl);
    pl = fmaf(al, bh, pl);
}

// (h, l) = a . b for float-float 3-vectors
__device__ __forceinline__ void ff_dot3(const float (&ah)[3], const float (&al)[3], const float (&bh)[3],
                                        const float (&bl)[3], float &h, float &l)
{
    float q[3], qe[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        q[a] = ah[a] * bh[a];
        qe[a] = fmaf(ah[a], bh[a], -q[a]);
    }
    float F1, f1, F2, f2;
    ts(q[0], q[1], F1, f1);
    ts(F1, q[2], F2, f2);
    float lo = (f1 + f2) + (qe[0] + qe[1] + qe[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) lo = fmaf(ah[a], bl[a], fmaf(al[a], bh[a], lo));
    fts(F2, lo, h, l);
}

template <int T, bool MASK>
__device__ __forceinline__ void tile_ff_stresslet(const float4 *__restrict__ sph, const float4 *__restrict__ spl,
                                                  const float4 *__restrict__ sqh, const float4 *__restrict__ sql,
                                                  const float4 *__restrict__ snh, const float4 *__restrict__ snl,
                                                  int cnt, int j0, const float (&th)[T][3],
                                                  const float (&tl)[T][3], const int (&elo)[T],
                                                  const int (&ecnt)[T], float (&uh)[T][3], float (&ul)[T][3])
{
#pragma unroll 1
    for (int j = 0; j < cnt; ++j) {
        const float4 ph4 = sph[j], pl4 = spl[j], qh4 = sqh[j], ql4 = sql[j], nh4 = snh[j], nl4 = snl[j];
        const float ph[3] = {ph4.x, ph4.y, ph4.z}, pl[3] = {pl4.x, pl4.y, pl4.z};
        const float qh[3] = {qh4.x, qh4.y, qh4.z}, ql[3] = {ql4.x, ql4.y, ql4.z};
        const float nh[3] = {nh4.x, nh4.y, nh4.z}, nl[3] = {nl4.x, nl4.y, nl4.z};
#pragma unroll
        for (int t = 0; t < T; ++t) {
            float dh[3], dl[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float e;
                ts(th[t][a], -ph[a], dh[a], e);
                dl[a] = (tl[t][a] - pl[a]) + e;
            }
            float R, Rl;
            ff_dot3(dh, dl, dh, dl, R, Rl);
            bool skip = false;
            if constexpr (MASK) {
                skip = static_cast<unsigned>(j0 + j - elo[t]) < static_cast<unsigned>(ecnt[t]);
                if (skip) {
                    R = 1.0f;
                    Rl = 0.0f;
                }
            }
            // rinv = y + yl: one Newton step on the rsqrt seed
            float y = rsqrtf(R);
            const float hh = y * y, hl = fmaf(y, y, -hh);
            const float qh2 = R * hh;
            float ql2 = fmaf(R, hh, -qh2);
            ql2 = fmaf(R, hl, ql2);
            ql2 = fmaf(Rl, hh, ql2);
            const float ee = (1.0f - qh2) - ql2;
            float yl = 0.5f * y * ee;
            if constexpr (MASK) {
                if (skip) {
                    y = 0.0f;
                    yl = 0.0f;
                }
            }
            float r2h, r2l, r4h, r4l, r5h, r5l;
            ff_mul(y, yl, y, yl, r2h, r2l);
            ff_mul(r2h, r2l, r2h, r2l, r4h, r4l);
            ff_mul(r4h, r4l, y, yl, r5h, r5l);
            float rqh, rql, rnh, rnl, ph2, pl2, sh, sl;
            ff_dot3(dh, dl, qh, ql, rqh, rql);
            ff_dot3(dh, dl, nh, nl, rnh, rnl);
            ff_mul(rqh, rql, rnh, rnl, ph2, pl2);
            ff_mul(ph2, pl2, r5h, r5l, sh, sl);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float wh, wl;
                ff_mul(sh, sl, dh[a], dl[a], wh, wl);
                float nh2, ne;
                ts(uh[t][a], wh, nh2, ne);
                ul[t][a] += ne + wl;
                uh[t][a] = nh2;
            }
        }
    }
}

template <int T, int KIND>
__global__ void __launch_bounds__(kThreads)
    k_pairsum_ff(const float4 *__restrict__ src, int64_t n_src, int64_t nt, int64_t W, int G,
                 const double *__restrict__ tgt, const int2 *__restrict__ excl, int64_t n_tgt,
                 const double *__restrict__ center, double *__restrict__ out, double *__restrict__ part,
                 double scale, int acc, int *__restrict__ status, const int4 *__restrict__ work)
{
    constexpr int NARR = KIND == PAIR_STRESSLET ? 6 : 4, TILE = kTileFF, TB = T * kThreads;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *smem = reinterpret_cast<float4 *>(smem_raw);   // [stage][array][TILE]
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_lo, s_hi;

    const int tid = threadIdx.x;
    const Run run(work, nt, W, G, n_src, TILE, TB);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto stage_ptr = [&](int stage, int arr) -> float4 * { return smem + (stage * NARR + arr) * TILE; };
    auto issue = [&](int64_t it) {
        int64_t j0;
        int cnt;
        run.src(it, j0, cnt);
        const int stage = static_cast<int>(it & 1);
        const uint32_t bytes = static_cast<uint32_t>(cnt) * 16u;
        mbar_expect_tx(&bars[stage], bytes * NARR);
#pragma unroll
        for (int a = 0; a < NARR; ++a) bulk_g2s(stage_ptr(stage, a), src + a * n_src + j0, bytes, &bars[stage]);
    };
    if (tid == 0) {
        if (run.n_run > 0) issue(0);
        if (run.n_run > 1) issue(1);
    }
    const double c[3] = {center[0], center[1], center[2]};
    bool failed = false;
    int64_t it = 0;
    do {
        int64_t tbase, t_end, len, blk;
        run.piece(it, n_tgt, tbase, t_end, len, blk);
        if (tid == 0) {
            s_lo = INT_MAX;
            s_hi = INT_MIN;
        }
        float th[T][3], tl[T][3], uh[T][3], ul[T][3];
        int elo[T], ecnt[T];
        int my_lo = INT_MAX, my_hi = INT_MIN;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = tbase + tid + static_cast<int64_t>(t) * kThreads;
            int2 e = make_int2(0, 0);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double x = i < t_end ? tgt[3 * i + a] - c[a] : 0.0;
                th[t][a] = static_cast<float>(x);
                tl[t][a] = static_cast<float>(x - static_cast<double>(th[t][a]));
                uh[t][a] = ul[t][a] = 0.0f;
            }
            if (i < t_end && excl) e = excl[i];
            elo[t] = e.x;
            ecnt[t] = e.y > e.x ? e.y - e.x : 0;
            if (e.y > e.x) {
                my_lo = min(my_lo, e.x);
                my_hi = max(my_hi, e.y);
            }
        }
        __syncthreads();
        if (my_hi > my_lo) {
            atomicMin(&s_lo, my_lo);
            atomicMax(&s_hi, my_hi);
        }
        __syncthreads();
        const int blo = s_lo, bhi = s_hi;
        for (int64_t q = 0; q < len; ++q, ++it) {
            const int stage = static_cast<int>(it & 1);
            const bool ok = mbar_wait(&bars[stage], static_cast<uint32_t>((it >> 1) & 1));
            if (!__syncthreads_and(ok)) {
                failed = true;
                break;
            }
            if (tid == 0 && it >= 1 && it + 1 < run.n_run) issue(it + 1);
            int64_t j0;
            int cnt;
            run.src(it, j0, cnt);
            const bool masked = bhi > blo && j0 < bhi && j0 + cnt > blo;
            if constexpr (KIND == PAIR_STRESSLET) {
                if (masked)
                    tile_ff_stresslet<T, true>(stage_ptr(stage, 0), stage_ptr(stage, 1), stage_ptr(stage, 2),
                                               stage_ptr(stage, 3), stage_ptr(stage, 4), stage_ptr(stage, 5), cnt,
                                               static_cast<int>(j0), th, tl, elo, ecnt, uh, ul);
                else
                    tile_ff_stresslet<T, false>(stage_ptr(stage, 0), stage_ptr(stage, 1), stage_ptr(stage, 2),
                                                stage_ptr(stage, 3), stage_ptr(stage, 4), stage_ptr(stage, 5), cnt,
                                                static_cast<int>(j0), th, tl, elo, ecnt, uh, ul);
            } else {
                if (masked)
                    tile_ff<T, true>(stage_ptr(stage, 0), stage_ptr(stage, 1), stage_ptr(stage, 2),
                                     stage_ptr(stage, 3), cnt, static_cast<int>(j0), th, tl, elo, ecnt, uh, ul);
                else
                    tile_ff<T, false>(stage_ptr(stage, 0), stage_ptr(stage, 1), stage_ptr(stage, 2),
                                      stage_ptr(stage, 3), cnt, static_cast<int>(j0), th, tl, elo, ecnt, uh, ul);
            }
#pragma unroll
            for (int t = 0; t < T; ++t)
#pragma unroll
                for (int a = 0; a < 3; ++a) fts(uh[t][a], ul[t][a], uh[t][a], ul[t][a]);
        }
        if (failed) break;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int64_t i = tbase + tid + static_cast<int64_t>(t) * kThreads;
            if (i >= t_end) continue;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double v = static_cast<double>(uh[t][a]) + static_cast<double>(ul[t][a]);
                if (work) {
                    double *o = out + 3 * i + a;
                    *o = (acc ? *o : 0.0) + scale * v;
                } else {
                    part[((static_cast<int64_t>(blockIdx.x) + blk) * TB + tid + t * kThreads) * 3 + a] = v;
                }
            }
        }
    } while (it < run.n_run);
    if (failed) {
        if (tid == 0) {
            atomicOr(status, DEV_ERR_TIMEOUT);
            mbar_wait(&bars[0], 0);
            mbar_wait(&bars[1], 0);
        }
    }
}

// Pack for the float-float kernel: [0] position hi, [1] position lo,
// [2] W f hi, [3] W f lo (positions relative to the centre).
// Stresslet (wgt and nrm given): [2], [3] w q hi/lo and [4], [5] the normal hi/lo.
__global__ void k_pack_ff(const double *__restrict__ xyz, const double *__restrict__ dens,
                          const double *__restrict__ wgt, const double *__restrict__ nrm, int64_t n,
                          const double *__restrict__ center, float4 *__restrict__ out)
{
    const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (j >= n) return;
    const double wj = wgt ? wgt[j] : 1.0;
    float h[3], l[3], fh[3], fl[3], nh[3], nl[3];
    for (int a = 0; a < 3; ++a) {
        const double x = xyz[3 * j + a] - center[a];
        h[a] = static_cast<float>(x);
        l[a] = static_cast<float>(x - static_cast<double>(h[a]));
        const double f = wj * dens[3 * j + a];
        fh[a] = static_cast<float>(f);
        fl[a] = static_cast<float>(f - static_cast<double>(fh[a]));
        const double v = nrm ? nrm[3 * j + a] : 0.0;
        nh[a] = static_cast<float>(v);
        nl[a] = static_cast<float>(v - static_cast<double>(nh[a]));
    }
    out[j] = make_float4(h[0], h[1], h[2], 0.0f);
    out[n + j] = make_float4(l[0], l[1], l[2], 0.0f);
    out[2 * n + j] = make_float4(fh[0], fh[1], fh[2], 0.0f);
    out[3 * n + j] = make_float4(fl[0], fl[1], fl[2], 0.0f);
    if (nrm) {
        out[4 * n + j] = make_float4(nh[0], nh[1], nh[2], 0.0f);
        out[5 * n + j] = make_float4(nl[0], nl[1], nl[2], 0.0f);
    }
}

// ------------------------------------------------------------------ helpers
// Midpoint of the bounding box of n points, in two passes: kBoxParts CTAs
// reduce strided slices to partial boxes part[cta][6], then one CTA combines
// them (min / max are exact, so the result does not depend on the split).
constexpr int kBoxParts = 128;

__global__ void __launch_bounds__(256) k_bbox_part(const double *__restrict__ p, int64_t n,
                                                   double *__restrict__ part)
{
    __shared__ double sm[6][8];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const double v = p[3 * i + a];
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int a = 0; a < 3; ++a) {
            sm[a][w] = lo[a];
            sm[3 + a][w] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int q = threadIdx.x;
        double v = q < 3 ? INFINITY : -INFINITY;
        for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) v = q < 3 ? fmin(v, sm[q][k]) : fmax(v, sm[q][k]);
        part[blockIdx.x * 6 + q] = v;
    }
}

__global__ void k_bbox_center(const double *__restrict__ part, int parts, int64_t n, double *__restrict__ center)
{
    const int a = threadIdx.x;
    if (a >= 3) return;
    double mn = INFINITY, mx = -INFINITY;
    for (int k = 0; k < parts; ++k) {
        mn = fmin(mn, part[k * 6 + a]);
        mx = fmax(mx, part[k * 6 + 3 + a]);
    }
    center[a] = (n > 0 && mn <= mx) ? 0.5 * (mn + mx) : 0.0;
}

// Pack sources: arrays [0] position (hi), [1] density x weight, [2] normal, [last] lo.
template <class R>
__global__ void k_pack(const double *__restrict__ xyz, const double *__restrict__ dens,
                       const double *__restrict__ wgt, const double *__restrict__ nrm, int64_t n,
                       const double *__restrict__ center, typename Vec4Of<R>::type *__restrict__ out,
                       int n_arr, int lo_slot)
{
    using V4 = typename Vec4Of<R>::type;
    const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (j >= n) return;
    const double x = xyz[3 * j] - center[0], y = xyz[3 * j + 1] - center[1],
                 z = xyz[3 * j + 2] - center[2];
    const R xh = static_cast<R>(x), yh = static_cast<R>(y), zh = static_cast<R>(z);
    V4 v;
    v.x = xh; v.y = yh; v.z = zh; v.w = R(0);
    out[j] = v;
    const double wj = wgt ? wgt[j] : 1.0;
    v.x = static_cast<R>(wj * dens[3 * j]);
    v.y = static_cast<R>(wj * dens[3 * j + 1]);
    v.z = static_cast<R>(wj * dens[3 * j + 2]);
    out[n + j] = v;
    if (nrm) {
        v.x = static_cast<R>(nrm[3 * j]);
        v.y = static_cast<R>(nrm[3 * j + 1]);
        v.z = static_cast<R>(nrm[3 * j + 2]);
        out[2 * n + j] = v;
    }
    if (lo_slot > 0 && lo_slot < n_arr) {
        v.x = static_cast<R>(x - static_cast<double>(xh));
        v.y = static_cast<R>(y - static_cast<double>(yh));
        v.z = static_cast<R>(z - static_cast<double>(zh));
        out[lo_slot * n + j] = v;
    }
}

// Sum of the stream-K partials of target i: the CTAs c_lo..c_hi whose runs
// cover target block b (the CTAs holding its first and last tile, and all
// between), in ascending order (deterministic).  CTA c holds tiles
// [floor(c W / G), floor((c + 1) W / G)); the largest c with floor(c W / G) <= t
// is ceil((t + 1) G / W) - 1.
// A CTA whose bounded wait gave up leaves its partial slots unwritten (they
// hold whatever an earlier sum left there), so when the status word carries
// DEV_ERR_TIMEOUT every output is set to NaN instead: the failure is visible
// in the result without a host synchronisation.
__global__ void k_reduce_streamk(const double *__restrict__ part, int64_t n_tgt, int tb, int64_t nt,
                                 int64_t W, int G, double scale, int acc, double *__restrict__ out,
                                 const int *__restrict__ status)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n_tgt) return;
    if (status && (*status & DEV_ERR_TIMEOUT)) {
        double *o = out + 3 * i;
        o[0] = o[1] = o[2] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    const int64_t b = i / tb, l = i - b * tb;
    const int64_t t0 = b * nt, t1 = (b + 1) * nt - 1;
    const int64_t c_lo = ((t0 + 1) * G + W - 1) / W - 1;
    const int64_t c_hi = ((t1 + 1) * G + W - 1) / W - 1;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t c = c_lo; c <= c_hi; ++c) {
        const double *q = part + ((c + b) * tb + l) * 3;
        s0 += q[0];
        s1 += q[1];
        s2 += q[2];
    }
    double *o = out + 3 * i;
    o[0] = (acc ? o[0] : 0.0) + scale * s0;
    o[1] = (acc ? o[1] : 0.0) + scale * s1;
    o[2] = (acc ? o[2] : 0.0) + scale * s2;
}

__global__ void k_excl_ids(const int32_t *__restrict__ sf, int64_t ns, const int32_t *__restrict__ tf,
                           int64_t nt, int2 *__restrict__ ex)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= nt) return;
    const int32_t id = tf[i];
    int64_t lo = 0, hi = ns;  // lower_bound
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (sf[m] < id) lo = m + 1; else hi = m;
    }
    int64_t lo2 = lo, hi2 = ns;  // upper_bound
    while (lo2 < hi2) {
        const int64_t m = (lo2 + hi2) >> 1;
        if (sf[m] <= id) lo2 = m + 1; else hi2 = m;
    }
    ex[i] = make_int2(static_cast<int>(lo), static_cast<int>(lo2));
}

}  // namespace

int num_sms()
{
    // initialised once, thread-safely (contexts may be created from several threads)
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 1;
        }
        return v;
    }();
    return n;
}

namespace {

// The FP32 Stokeslet without hi/lo targets runs in packed pairs with
// per-thread frames (k_stokeslet_x2); its sources carry the lo parts.
bool packed_x2(int kind, int prec, bool hilo)
{
    return kind == PAIR_STOKESLET && prec == FS_SUM_FP32 && !hilo;
}

// Kernel instantiation for (kind, precision, hi/lo, targets per thread).
const void *kernel_of(int kind, int prec, bool hilo, int tpt)
{
    if (packed_x2(kind, prec, hilo))
        return tpt == 2 ? reinterpret_cast<const void *>(&k_stokeslet_x2<2>)
                        : tpt == 4 ? reinterpret_cast<const void *>(&k_stokeslet_x2<4>)
                                   : reinterpret_cast<const void *>(&k_stokeslet_x2<8>);
#define FS_K(R, TT, K, HL) reinterpret_cast<const void *>(&k_pairsum<R, TT, K, HL>)
#define FS_K_T(R, K, HL) (tpt == 2 ? FS_K(R, 2, K, HL) : tpt == 8 ? FS_K(R, 8, K, HL) : FS_K(R, 4, K, HL))
#define FS_K_T64(K) (tpt == 1 ? FS_K(double, 1, K, false) : tpt == 4 ? FS_K(double, 4, K, false) \
                                                          : FS_K(double, 2, K, false))
#define FS_KF(TT, K) reinterpret_cast<const void *>(&k_pairsum_ff<TT, K>)
    if (prec == FS_SUM_FF) {
        if (kind == PAIR_STRESSLET)
            return tpt == 1 ? FS_KF(1, PAIR_STRESSLET) : (tpt == 4 ? FS_KF(4, PAIR_STRESSLET) : FS_KF(2, PAIR_STRESSLET));
        return tpt == 1 ? FS_KF(1, PAIR_STOKESLET) : (tpt == 4 ? FS_KF(4, PAIR_STOKESLET) : FS_KF(2, PAIR_STOKESLET));
    }
#undef FS_KF
    if (prec == FS_SUM_FP32) {
        if (kind == PAIR_STOKESLET) return hilo ? FS_K_T(float, PAIR_STOKESLET, true) : FS_K_T(float, PAIR_STOKESLET, false);
        return hilo ? FS_K_T(float, PAIR_STRESSLET, true) : FS_K_T(float, PAIR_STRESSLET, false);
    }
    return kind == PAIR_STOKESLET ? FS_K_T64(PAIR_STOKESLET) : FS_K_T64(PAIR_STRESSLET);
#undef FS_K_T64
#undef FS_K_T
#undef FS_K
}

// Allow a kernel `smem` bytes of dynamic shared memory: beyond 48 KB per
// CTA (static included) a launch needs the opt-in attribute.  Cached per
// kernel at the largest size set so far.
bool allow_smem(const void *k, size_t smem)
{
    static std::mutex mu;
    static std::map<const void *, size_t> set;
    std::lock_guard<std::mutex> lk(mu);
    auto it = set.find(k);
    if (it != set.end() && it->second >= smem) return true;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    set[k] = smem;
    return true;
}

// Resident CTAs per SM of a kernel at kThreads threads and `smem` dynamic
// shared memory (occupancy calculator, cached per kernel and size).
int resident_ctas(const void *k, size_t smem)
{
    allow_smem(k, smem);
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(k, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kThreads, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    cache[key] = n;
    return n;
}

}  // namespace

SumPlan plan_pairsum(int kind, int64_t n_src, int64_t n_tgt, int sum_prec, bool hilo, int shape_override,
                     int slots)
{
    const bool f32 = sum_prec == FS_SUM_FP32, ff = sum_prec == FS_SUM_FF;
    hilo = hilo && f32;
    SumPlan p;
    p.tile = f32 ? kTile32 : (ff ? kTileFF : kTile64);
    // measured on GB300 (65,536 points): FP32 8 targets per thread, float-float 4, FP64 2
    p.tpt = f32 ? 8 : (ff ? 4 : 2);
    if (shape_override > 0) {
        static const int f32_opts[] = {2, 4, 8};
        static const int f64_opts[] = {1, 2, 4};
        const int k = (shape_override - 1) % 3;
        p.tpt = f32 ? f32_opts[k] : f64_opts[k];
        if (ff) p.tpt = k == 0 ? 1 : (k == 1 ? 2 : 4);
    }
    p.threads = kThreads;
    p.tb = p.tpt * kThreads;
    p.n_arr = ff ? (kind == PAIR_STRESSLET ? 6 : 4)
                 : (kind == PAIR_STRESSLET ? 3 : 2) + ((hilo || packed_x2(kind, sum_prec, hilo)) ? 1 : 0);
    p.v4 = (f32 || ff) ? sizeof(float4) : sizeof(double4_32a);
    p.smem = static_cast<size_t>(p.n_arr) * 2 * p.tile * p.v4;
    if (packed_x2(kind, sum_prec, hilo)) p.smem += x2_sum_bytes(p.tpt);
    p.nb = (n_tgt + p.tb - 1) / p.tb;
    p.nt = (n_src + p.tile - 1) / p.tile;
    p.W = p.nb * p.nt;
    if (slots <= 0) slots = num_sms() * resident_ctas(kernel_of(kind, sum_prec, hilo, p.tpt), p.smem);
    p.grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(p.W, slots)));
    return p;
}

size_t pairsum_scratch_bytes(int kind, int64_t n_src, int64_t n_tgt, int sum_prec, int shape_override,
                             int slots)
{
    size_t most = 0;
    // FP32 sums may run with or without hi/lo coordinates: size for the larger
    for (bool hilo : {false, true}) {
        const SumPlan p = plan_pairsum(kind, n_src, n_tgt, sum_prec, hilo, shape_override, slots);
        const size_t packed = static_cast<size_t>(p.n_arr) * static_cast<size_t>(n_src) * p.v4;
        const size_t part = static_cast<size_t>(p.grid + p.nb) * static_cast<size_t>(p.tb) * 3 * sizeof(double);
        most = std::max(most, 4 * 256 + 6 * kBoxParts * sizeof(double) + packed + part + 1024);
    }
    return most;
}

fs_status exclusion_from_ids(const int32_t *src_fiber, int64_t n_src, const int32_t *tgt_fiber,
                             int64_t n_tgt, int2 *excl, cudaStream_t st)
{
    if (n_tgt == 0) return FS_OK;
    k_excl_ids<<<static_cast<unsigned>((n_tgt + 255) / 256), 256, 0, st>>>(src_fiber, n_src, tgt_fiber,
                                                                           n_tgt, excl);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

namespace {

// One work item per block of tb targets of a group, sources of that group
// only; largest source ranges first (the order schedules, the sums of an item
// do not depend on it).
std::vector<int4> work_items(const PairSumArgs &a, int tb)
{
    std::vector<int4> items;
    for (const int4 &g : *a.groups)
        for (int t0 = g.x; t0 < g.y; t0 += tb) items.push_back(make_int4(t0, std::min(tb, g.y - t0), g.z, g.w));
    std::stable_sort(items.begin(), items.end(),
                     [](const int4 &u, const int4 &v) { return (u.w - u.z) > (v.w - v.z); });
    return items;
}

}  // namespace

fs_status pairsum_work_list(const PairSumArgs &a, cudaStream_t st, int64_t *n_items)
{
    *n_items = 0;
    if (!a.groups) return FS_OK;
    const bool f32 = a.sum_prec == FS_SUM_FP32;
    const SumPlan p = plan_pairsum(a.kind, a.n_src, a.n_tgt, a.sum_prec, f32 && a.hilo, a.shape_override, 0);
    const std::vector<int4> items = work_items(a, p.tb);
    if (items.empty()) return FS_OK;
    if (static_cast<int64_t>(items.size()) > a.work_cap) {
        set_error("pairsum: %zu work items exceed the capacity %lld", items.size(),
                  static_cast<long long>(a.work_cap));
        return FS_EINVAL;
    }
    FS_CUDA(cudaMemcpyAsync(a.work_dev, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    *n_items = static_cast<int64_t>(items.size());
    return FS_OK;
}

fs_status pairsum(const PairSumArgs &a, void *scratch, size_t scratch_bytes, int *d_status,
                  cudaStream_t st)
{
    if (a.n_tgt == 0) return FS_OK;
    if (a.n_src == 0) {
        if (!a.accumulate)
            FS_CUDA(cudaMemsetAsync(a.out, 0, static_cast<size_t>(a.n_tgt) * 3 * sizeof(double), st));
        return FS_OK;
    }
    if (a.n_src >= INT_MAX || a.n_tgt >= INT_MAX) {
        set_error("pairsum: at most 2^31-2 sources and targets");
        return FS_EINVAL;
    }
    const int prec = a.sum_prec;
    const bool ff = prec == FS_SUM_FF;
    const bool f32 = prec == FS_SUM_FP32;
    const bool hilo = f32 && a.hilo;
    const SumPlan p = plan_pairsum(a.kind, a.n_src, a.n_tgt, prec, hilo, a.shape_override, 0);
    Carve cv(scratch, scratch_bytes);
    double *center = cv.take<double>(4);
    double *box = cv.take<double>(6 * kBoxParts);
    void *packed = cv.take<unsigned char>(static_cast<size_t>(p.n_arr) * a.n_src * p.v4);
    const int4 *work = nullptr;
    unsigned grid = static_cast<unsigned>(p.grid);
    double *part = nullptr;
    if (a.groups) {
        int64_t n_items = 0;
        if (a.work_uploaded)
            n_items = static_cast<int64_t>(work_items(a, p.tb).size());
        else
            FS_TRY(pairsum_work_list(a, st, &n_items));
        if (n_items == 0) return FS_OK;
        work = a.work_dev;
        grid = static_cast<unsigned>(n_items);
    } else {
        part = cv.take<double>(static_cast<size_t>(p.grid + p.nb) * p.tb * 3);
    }
    if (cv.used > scratch_bytes) {
        set_error("pairsum: scratch too small (%zu > %zu bytes)", cv.used, scratch_bytes);
        return FS_EINVAL;
    }
    if (work) {
        // independent systems: the coordinates are not centred on a box of
        // all of them, so that each system's sums do not depend on the
        // others (the kernels' frames and lo parts keep the accuracy)
        FS_CUDA(cudaMemsetAsync(center, 0, 3 * sizeof(double), st));
    } else {
        k_bbox_part<<<kBoxParts, 256, 0, st>>>(a.src_xyz, a.n_src, box);
        FS_LAUNCH_CHECK();
        k_bbox_center<<<1, 32, 0, st>>>(box, kBoxParts, a.n_src, center);
        FS_LAUNCH_CHECK();
    }
    const unsigned pb = static_cast<unsigned>((a.n_src + 255) / 256);
    const bool x2 = packed_x2(a.kind, prec, hilo);
    const int lo_slot = (hilo || x2) ? p.n_arr - 1 : 0;
    if (ff)
        k_pack_ff<<<pb, 256, 0, st>>>(a.src_xyz, a.src_dens, a.kind == PAIR_STRESSLET ? a.src_w : nullptr,
                                      a.kind == PAIR_STRESSLET ? a.src_nrm : nullptr, a.n_src, center,
                                      static_cast<float4 *>(packed));
    else if (f32)
        k_pack<float><<<pb, 256, 0, st>>>(a.src_xyz, a.src_dens, a.src_w, a.src_nrm, a.n_src, center,
                                          static_cast<float4 *>(packed), p.n_arr, lo_slot);
    else
        k_pack<double><<<pb, 256, 0, st>>>(a.src_xyz, a.src_dens, a.src_w, a.src_nrm, a.n_src, center,
                                           static_cast<double4_32a *>(packed), p.n_arr, 0);
    FS_LAUNCH_CHECK();
    const int acc = a.accumulate ? 1 : 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (a.prof) {
        ev0 = a.prof->get();
        ev1 = a.prof->get();
        if (!ev0 || !ev1) {
            set_error("pairsum: could not create profiling events");
            return FS_ECUDA;
        }
        FS_CUDA(cudaEventRecord(ev0, st));
    }
    {
        const void *src = packed;
        int64_t n_src = a.n_src, nt = p.nt, W = p.W, n_tgt = a.n_tgt;
        int G = p.grid;
        const double *tgt = a.tgt_xyz;
        const int2 *excl = a.excl;
        double *out = a.out;
        double scale = a.scale;
        int accv = acc;
        int *status = d_status;
        void *args[] = {&src, &n_src, &nt, &W, &G, &tgt, &excl, &n_tgt, &center, &out, &part, &scale, &accv,
                        &status, &work};
        const void *kern = kernel_of(a.kind, prec, hilo, p.tpt);
        if (!allow_smem(kern, p.smem)) {
            set_error("pairsum: cannot allow %zu bytes of shared memory", p.smem);
            return FS_ECUDA;
        }
        const cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(kThreads), args, p.smem, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("pairsum: launch failed: %s", cudaGetErrorString(e));
            return FS_ECUDA;
        }
    }
    FS_LAUNCH_CHECK();
    if (a.prof) {
        FS_CUDA(cudaEventRecord(ev1, st));
        const int cls = ff ? (a.kind == PAIR_STOKESLET ? 4 : 6)
                           : (f32 && !hilo && a.kind == PAIR_STOKESLET) ? 5
                                                                      : (a.kind == PAIR_STOKESLET ? 0 : 2) + (f32 ? 0 : 1);
        a.prof->recs.push_back(Profiler::Rec{cls, ev0, ev1, a.pairs});
    }
    if (!work) {
        k_reduce_streamk<<<static_cast<unsigned>((a.n_tgt + 255) / 256), 256, 0, st>>>(
            part, a.n_tgt, p.tb, p.nt, p.W, p.grid, a.scale, acc, a.out, d_status);
        FS_LAUNCH_CHECK();
    }
    return FS_OK;
}

}  // namespace fs
