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

// out (direct): out[i] = (acc ? out[i] : 0) + scale * sum;  else partial[split][i] = sum
template <class R, int T, int KIND, bool HILO>
__global__ void __launch_bounds__(kThreads)
    k_pairsum(const typename Vec4Of<R>::type *__restrict__ src, int64_t n_src, int64_t per_split,
              const double *__restrict__ tgt, const int2 *__restrict__ excl, int64_t n_tgt,
              const double *__restrict__ center, double *__restrict__ out, double scale, int direct,
              int acc, int *__restrict__ status, const int4 *__restrict__ work)
{
    using V4 = typename Vec4Of<R>::type;
    using A = Arr<KIND, HILO>;
    constexpr int TILE = sizeof(R) == 4 ? kTile32 : kTile64;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V4 *smem = reinterpret_cast<V4 *>(smem_raw);   // [stage][array][TILE]
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_lo, s_hi;

    const int tid = threadIdx.x;
    // work item (batched systems): targets [x, x + y), sources [z, w)
    int64_t tbase, t_end, j_begin, j_end;
    if (work) {
        const int4 wi = work[blockIdx.x];
        tbase = wi.x;
        t_end = static_cast<int64_t>(wi.x) + wi.y;
        j_begin = wi.z;
        j_end = wi.w;
    } else {
        tbase = static_cast<int64_t>(blockIdx.x) * (T * kThreads);
        t_end = n_tgt;
        j_begin = static_cast<int64_t>(blockIdx.y) * per_split;
        j_end = min(n_src, j_begin + per_split);
    }
    const int64_t n_tiles = j_end > j_begin ? (j_end - j_begin + TILE - 1) / TILE : 0;

    if (tid == 0) {
        s_lo = INT_MAX;
        s_hi = INT_MIN;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const double c0 = center[0], c1 = center[1], c2 = center[2];
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
    auto stage_ptr = [&](int stage, int arr) -> V4 * { return smem + (stage * A::n + arr) * TILE; };
    auto issue = [&](int64_t tile, int stage) {
        const int64_t j0 = j_begin + tile * TILE;
        const int cnt = static_cast<int>(min(static_cast<int64_t>(TILE), j_end - j0));
        const uint32_t bytes = static_cast<uint32_t>(cnt) * static_cast<uint32_t>(sizeof(V4));
        mbar_expect_tx(&bars[stage], bytes * A::n);
#pragma unroll
        for (int a = 0; a < A::n; ++a) bulk_g2s(stage_ptr(stage, a), src + a * n_src + j0, bytes, &bars[stage]);
    };
    if (tid == 0) {
        if (n_tiles > 0) issue(0, 0);
        if (n_tiles > 1) issue(1, 1);
    }
    __syncthreads();
    const int blo = s_lo, bhi = s_hi;

    // FP32: compensated cross-tile sums (s, c); FP64: plain accumulation in s
    R sx[T], sy[T], sz[T], cx[T], cy[T], cz[T];
#pragma unroll
    for (int t = 0; t < T; ++t) sx[t] = sy[t] = sz[t] = cx[t] = cy[t] = cz[t] = R(0);

    bool failed = false;
    for (int64_t it = 0; it < n_tiles; ++it) {
        const int stage = static_cast<int>(it & 1);
        const bool ok = mbar_wait(&bars[stage], static_cast<uint32_t>((it >> 1) & 1));
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        // every thread has finished tile it-1, so its stage can be refilled
        if (tid == 0 && it >= 1 && it + 1 < n_tiles) issue(it + 1, static_cast<int>((it + 1) & 1));
        const int64_t j0 = j_begin + it * TILE;
        const int cnt = static_cast<int>(min(static_cast<int64_t>(TILE), j_end - j0));
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
    if (failed) {
        if (tid == 0) {
            atomicOr(status, DEV_ERR_TIMEOUT);
            // let copies already in flight land before the CTA exits (bounded)
            mbar_wait(&bars[0], 0);
            mbar_wait(&bars[1], 0);
        }
        return;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t i = tbase + tid + static_cast<int64_t>(t) * kThreads;
        if (i >= t_end) continue;
        const double ux = static_cast<double>(sx[t]) + static_cast<double>(cx[t]);
        const double uy = static_cast<double>(sy[t]) + static_cast<double>(cy[t]);
        const double uz = static_cast<double>(sz[t]) + static_cast<double>(cz[t]);
        if (direct) {
            double *o = out + 3 * i;
            o[0] = (acc ? o[0] : 0.0) + scale * ux;
            o[1] = (acc ? o[1] : 0.0) + scale * uy;
            o[2] = (acc ? o[2] : 0.0) + scale * uz;
        } else {
            double *o = out + (static_cast<int64_t>(blockIdx.y) * n_tgt + i) * 3;
            o[0] = ux;
            o[1] = uy;
            o[2] = uz;
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

template <int T>
__global__ void __launch_bounds__(kThreads)
    k_pairsum_ff(const float4 *__restrict__ src, int64_t n_src, int64_t per_split,
                 const double *__restrict__ tgt, const int2 *__restrict__ excl, int64_t n_tgt,
                 const double *__restrict__ center, double *__restrict__ out, double scale, int direct,
                 int acc, int *__restrict__ status, const int4 *__restrict__ work)
{
    constexpr int NARR = 4, TILE = kTileFF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4 *smem = reinterpret_cast<float4 *>(smem_raw);   // [stage][array][TILE]
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_lo, s_hi;

    const int tid = threadIdx.x;
    // work item (batched systems): targets [x, x + y), sources [z, w)
    int64_t tbase, t_end, j_begin, j_end;
    if (work) {
        const int4 wi = work[blockIdx.x];
        tbase = wi.x;
        t_end = static_cast<int64_t>(wi.x) + wi.y;
        j_begin = wi.z;
        j_end = wi.w;
    } else {
        tbase = static_cast<int64_t>(blockIdx.x) * (T * kThreads);
        t_end = n_tgt;
        j_begin = static_cast<int64_t>(blockIdx.y) * per_split;
        j_end = min(n_src, j_begin + per_split);
    }
    const int64_t n_tiles = j_end > j_begin ? (j_end - j_begin + TILE - 1) / TILE : 0;
    if (tid == 0) {
        s_lo = INT_MAX;
        s_hi = INT_MIN;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const double c[3] = {center[0], center[1], center[2]};
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
    auto stage_ptr = [&](int stage, int arr) -> float4 * { return smem + (stage * NARR + arr) * TILE; };
    auto issue = [&](int64_t tile, int stage) {
        const int64_t j0 = j_begin + tile * TILE;
        const int cnt = static_cast<int>(min(static_cast<int64_t>(TILE), j_end - j0));
        const uint32_t bytes = static_cast<uint32_t>(cnt) * 16u;
        mbar_expect_tx(&bars[stage], bytes * NARR);
#pragma unroll
        for (int a = 0; a < NARR; ++a) bulk_g2s(stage_ptr(stage, a), src + a * n_src + j0, bytes, &bars[stage]);
    };
    if (tid == 0) {
        if (n_tiles > 0) issue(0, 0);
        if (n_tiles > 1) issue(1, 1);
    }
    __syncthreads();
    const int blo = s_lo, bhi = s_hi;
    bool failed = false;
    for (int64_t it = 0; it < n_tiles; ++it) {
        const int stage = static_cast<int>(it & 1);
        const bool ok = mbar_wait(&bars[stage], static_cast<uint32_t>((it >> 1) & 1));
        if (!__syncthreads_and(ok)) {
            failed = true;
            break;
        }
        if (tid == 0 && it >= 1 && it + 1 < n_tiles) issue(it + 1, static_cast<int>((it + 1) & 1));
        const int64_t j0 = j_begin + it * TILE;
        const int cnt = static_cast<int>(min(static_cast<int64_t>(TILE), j_end - j0));
        const bool masked = bhi > blo && j0 < bhi && j0 + cnt > blo;
        if (masked)
            tile_ff<T, true>(stage_ptr(stage, 0), stage_ptr(stage, 1), stage_ptr(stage, 2),
                             stage_ptr(stage, 3), cnt, static_cast<int>(j0), th, tl, elo, ecnt, uh, ul);
        else
            tile_ff<T, false>(stage_ptr(stage, 0), stage_ptr(stage, 1), stage_ptr(stage, 2),
                              stage_ptr(stage, 3), cnt, static_cast<int>(j0), th, tl, elo, ecnt, uh, ul);
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int a = 0; a < 3; ++a) fts(uh[t][a], ul[t][a], uh[t][a], ul[t][a]);
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(status, DEV_ERR_TIMEOUT);
            mbar_wait(&bars[0], 0);
            mbar_wait(&bars[1], 0);
        }
        return;
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int64_t i = tbase + tid + static_cast<int64_t>(t) * kThreads;
        if (i >= t_end) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double v = static_cast<double>(uh[t][a]) + static_cast<double>(ul[t][a]);
            if (direct) {
                double *o = out + 3 * i + a;
                *o = (acc ? *o : 0.0) + scale * v;
            } else {
                out[(static_cast<int64_t>(blockIdx.y) * n_tgt + i) * 3 + a] = v;
            }
        }
    }
}

// Pack for the float-float kernel: [0] position hi, [1] position lo,
// [2] W f hi, [3] W f lo (positions relative to the centre).
__global__ void k_pack_ff(const double *__restrict__ xyz, const double *__restrict__ dens, int64_t n,
                          const double *__restrict__ center, float4 *__restrict__ out)
{
    const int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (j >= n) return;
    float h[3], l[3], fh[3], fl[3];
    for (int a = 0; a < 3; ++a) {
        const double x = xyz[3 * j + a] - center[a];
        h[a] = static_cast<float>(x);
        l[a] = static_cast<float>(x - static_cast<double>(h[a]));
        const double f = dens[3 * j + a];
        fh[a] = static_cast<float>(f);
        fl[a] = static_cast<float>(f - static_cast<double>(fh[a]));
    }
    out[j] = make_float4(h[0], h[1], h[2], 0.0f);
    out[n + j] = make_float4(l[0], l[1], l[2], 0.0f);
    out[2 * n + j] = make_float4(fh[0], fh[1], fh[2], 0.0f);
    out[3 * n + j] = make_float4(fl[0], fl[1], fl[2], 0.0f);
}

// ------------------------------------------------------------------ helpers
// Midpoint of the bounding box of n points (one CTA).
__global__ void __launch_bounds__(512) k_bbox_center(const double *__restrict__ p, int64_t n,
                                                     double *__restrict__ center)
{
    __shared__ double smin[3][16], smax[3][16];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
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
            smin[a][w] = lo[a];
            smax[a][w] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        double mn = INFINITY, mx = -INFINITY;
        for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) {
            mn = fmin(mn, smin[a][k]);
            mx = fmax(mx, smax[a][k]);
        }
        center[a] = (n > 0 && mn <= mx) ? 0.5 * (mn + mx) : 0.0;
    }
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

__global__ void k_reduce_splits(const double *__restrict__ part, int splits, int64_t n3,
                                double scale, int acc, double *__restrict__ out)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n3) return;
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += part[k * n3 + i];
    out[i] = (acc ? out[i] : 0.0) + scale * s;
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

SumPlan plan_pairsum(int64_t n_src, int64_t n_tgt, int sum_prec, int shape_override)
{
    const int tile = sum_prec == FS_SUM_FP32 ? kTile32 : (sum_prec == FS_SUM_FF ? kTileFF : kTile64);
    int tpt = sum_prec == FS_SUM_FP32 ? 4 : 2;
    if (shape_override > 0) {
        static const int f32_opts[] = {2, 4, 8};
        static const int f64_opts[] = {1, 2, 4};
        const int k = (shape_override - 1) % 3;
        tpt = sum_prec == FS_SUM_FP32 ? f32_opts[k] : f64_opts[k];
        if (sum_prec == FS_SUM_FF) tpt = k == 0 ? 1 : 2;
    }
    const int64_t nb = (n_tgt + tpt * kThreads - 1) / (tpt * kThreads);
    const int64_t want = 4LL * num_sms();
    int64_t splits = nb > 0 ? (want + nb - 1) / nb : 1;
    const int64_t max_split = n_src / (2 * tile);
    if (splits > max_split) splits = max_split;
    if (splits < 1) splits = 1;
    int64_t per = (n_src + splits - 1) / splits;
    per = (per + tile - 1) / tile * tile;
    if (per < tile) per = tile;
    splits = (n_src + per - 1) / per;
    if (splits < 1) splits = 1;
    SumPlan p;
    p.tpt = tpt;
    p.splits = static_cast<int>(splits);
    p.per_split = per;
    p.tile = tile;
    p.threads = kThreads;
    return p;
}

size_t pairsum_scratch_bytes(int kind, int64_t n_src, int64_t n_tgt, int sum_prec, int shape_override)
{
    if (sum_prec == FS_SUM_FF && kind == PAIR_STRESSLET) sum_prec = FS_SUM_FP64;   // as in pairsum()
    const SumPlan p = plan_pairsum(n_src, n_tgt, sum_prec, shape_override);
    const size_t arrs = sum_prec == FS_SUM_FF ? 4 : (kind == PAIR_STRESSLET ? 3 : 2) + (sum_prec == FS_SUM_FP32 ? 1 : 0);
    const size_t v4 = sum_prec == FS_SUM_FP64 ? sizeof(double4_32a) : sizeof(float4);
    return 1024 + arrs * static_cast<size_t>(n_src) * v4 +
           (p.splits > 1 ? static_cast<size_t>(p.splits) * static_cast<size_t>(n_tgt) * 3 * sizeof(double) : 0) +
           1024;
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
    // the float-float path exists for the Stokeslet; stresslet sums asked for
    // in float-float run in FP64 (more, not less, precise)
    const int prec = (a.sum_prec == FS_SUM_FF && a.kind == PAIR_STRESSLET) ? FS_SUM_FP64 : a.sum_prec;
    const bool ff = prec == FS_SUM_FF;
    const bool f32 = prec == FS_SUM_FP32;
    const bool hilo = f32 && a.hilo;
    const SumPlan p = plan_pairsum(a.n_src, a.n_tgt, prec, a.shape_override);
    const int n_arr = ff ? 4 : (a.kind == PAIR_STRESSLET ? 3 : 2) + (hilo ? 1 : 0);
    const size_t v4 = (f32 || ff) ? sizeof(float4) : sizeof(double4_32a);
    Carve cv(scratch, scratch_bytes);
    double *center = cv.take<double>(4);
    void *packed = cv.take<unsigned char>(static_cast<size_t>(n_arr) * a.n_src * v4);
    int direct = p.splits == 1;
    double *part = direct ? nullptr : cv.take<double>(static_cast<size_t>(p.splits) * a.n_tgt * 3);
    if (cv.used > scratch_bytes) {
        set_error("pairsum: scratch too small (%zu > %zu bytes)", cv.used, scratch_bytes);
        return FS_EINVAL;
    }
    k_bbox_center<<<1, 512, 0, st>>>(a.src_xyz, a.n_src, center);
    FS_LAUNCH_CHECK();
    const unsigned pb = static_cast<unsigned>((a.n_src + 255) / 256);
    const int lo_slot = hilo ? n_arr - 1 : 0;
    if (ff)
        k_pack_ff<<<pb, 256, 0, st>>>(a.src_xyz, a.src_dens, a.n_src, center, static_cast<float4 *>(packed));
    else if (f32)
        k_pack<float><<<pb, 256, 0, st>>>(a.src_xyz, a.src_dens, a.src_w, a.src_nrm, a.n_src, center,
                                          static_cast<float4 *>(packed), n_arr, lo_slot);
    else
        k_pack<double><<<pb, 256, 0, st>>>(a.src_xyz, a.src_dens, a.src_w, a.src_nrm, a.n_src, center,
                                           static_cast<double4_32a *>(packed), n_arr, 0);
    FS_LAUNCH_CHECK();
    dim3 grid(static_cast<unsigned>((a.n_tgt + p.tpt * kThreads - 1) / (p.tpt * kThreads)),
              static_cast<unsigned>(p.splits));
    const size_t sm = static_cast<size_t>(n_arr) * 2 * p.tile * v4;
    const int4 *work = nullptr;
    if (a.groups) {
        // one work item per block of tpt x threads targets of a group, sources of
        // that group only; largest source ranges first
        std::vector<int4> items;
        const int chunk = p.tpt * kThreads;
        for (const int4 &g : *a.groups)
            for (int t0 = g.x; t0 < g.y; t0 += chunk)
                items.push_back(make_int4(t0, std::min(chunk, g.y - t0), g.z, g.w));
        std::stable_sort(items.begin(), items.end(),
                         [](const int4 &u, const int4 &v) { return (u.w - u.z) > (v.w - v.z); });
        if (items.empty()) return FS_OK;
        if (static_cast<int64_t>(items.size()) > a.work_cap) {
            set_error("pairsum: %zu work items exceed the capacity %lld", items.size(),
                      static_cast<long long>(a.work_cap));
            return FS_EINVAL;
        }
        FS_CUDA(cudaMemcpyAsync(a.work_dev, items.data(), items.size() * sizeof(int4),
                                cudaMemcpyHostToDevice, st));
        work = a.work_dev;
        grid = dim3(static_cast<unsigned>(items.size()), 1);
        direct = 1;
    }
    double *dst = (direct || work) ? a.out : part;
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
#define FS_LAUNCH(R, TT, K, HL)                                                                   \
    k_pairsum<R, TT, K, HL><<<grid, kThreads, sm, st>>>(                                         \
        static_cast<const Vec4Of<R>::type *>(packed), a.n_src, p.per_split, a.tgt_xyz, a.excl,   \
        a.n_tgt, center, dst, a.scale, direct, acc, d_status, work)
#define FS_BY_T(R, K, HL)                                                                         \
    do {                                                                                          \
        if (p.tpt == 2) FS_LAUNCH(R, 2, K, HL);                                                   \
        else if (p.tpt == 8) FS_LAUNCH(R, 8, K, HL);                                              \
        else FS_LAUNCH(R, 4, K, HL);                                                              \
    } while (0)
#define FS_BY_T64(K)                                                                              \
    do {                                                                                          \
        if (p.tpt == 1) FS_LAUNCH(double, 1, K, false);                                           \
        else if (p.tpt == 4) FS_LAUNCH(double, 4, K, false);                                      \
        else FS_LAUNCH(double, 2, K, false);                                                      \
    } while (0)
    if (ff) {
        if (p.tpt == 1)
            k_pairsum_ff<1><<<grid, kThreads, sm, st>>>(static_cast<const float4 *>(packed), a.n_src,
                                                        p.per_split, a.tgt_xyz, a.excl, a.n_tgt, center,
                                                        dst, a.scale, direct, acc, d_status, work);
        else
            k_pairsum_ff<2><<<grid, kThreads, sm, st>>>(static_cast<const float4 *>(packed), a.n_src,
                                                        p.per_split, a.tgt_xyz, a.excl, a.n_tgt, center,
                                                        dst, a.scale, direct, acc, d_status, work);
    } else if (f32) {
        if (a.kind == PAIR_STOKESLET) {
            if (hilo) FS_BY_T(float, PAIR_STOKESLET, true); else FS_BY_T(float, PAIR_STOKESLET, false);
        } else {
            if (hilo) FS_BY_T(float, PAIR_STRESSLET, true); else FS_BY_T(float, PAIR_STRESSLET, false);
        }
    } else {
        if (a.kind == PAIR_STOKESLET) FS_BY_T64(PAIR_STOKESLET);
        else FS_BY_T64(PAIR_STRESSLET);
    }
#undef FS_BY_T64
#undef FS_BY_T
#undef FS_LAUNCH
    FS_LAUNCH_CHECK();
    if (a.prof) {
        FS_CUDA(cudaEventRecord(ev1, st));
        const int cls = ff ? 4 : (a.kind == PAIR_STOKESLET ? 0 : 2) + (f32 ? 0 : 1);
        a.prof->recs.push_back(Profiler::Rec{cls, ev0, ev1, a.pairs});
    }
    if (!direct && !work) {
        const int64_t n3 = a.n_tgt * 3;
        k_reduce_splits<<<static_cast<unsigned>((n3 + 255) / 256), 256, 0, st>>>(part, p.splits, n3,
                                                                                 a.scale, acc, a.out);
        FS_LAUNCH_CHECK();
    }
    return FS_OK;
}

}  // namespace fs
