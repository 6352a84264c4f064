// Fast summation of the Stokeslet sum (the complementary velocity of Eq.
// complementary-uf, which the paper evaluates with a kernel-independent FMM
// for large systems, Sec. 3.3): a Cartesian treecode on the GPU.
//
// Kernel split.  With r = x - y, 8 pi mu G(r) f = f / |r| + r (r.f) / |r|^3.
// For the sources of one cell with centre c the four Laplace potentials
//   phi_j(x) = sum_n f_{n,j} / |x - y_n|   (j = 1..3),
//   phi_4(x) = sum_n ((y_n - c).f_n) / |x - y_n|
// give exactly 8 pi mu u_i = phi_i - (x - c)_j d_i phi_j + d_i phi_4; the
// charge (y - c).f relative to the cell keeps every term of size |f| / |r|.
//
// Expansions.  1/|x - y| = sum_k a_k (y - c)^k with the Taylor coefficients
// a_k = (1/k!) d_y^k |x - y|^-1 at y = c, which satisfy (r = x - c)
//   |k| |r|^2 a_k = (2|k| - 1) sum_i r_i a_{k - e_i} - (|k| - 1) sum_i a_{k - 2 e_i}
// (the recurrence of Cartesian treecodes, Li, Johnston and Krasny, J. Comput.
// Phys. 228, 2009).  With the moments M_k = sum_n q_n (y_n - c)^k of a charge q,
//   phi = sum_{|k| <= p} a_k M_k,   d_i phi = -sum_{|m| <= p+1, m_i >= 1} m_i a_m M_{m - e_i},
// evaluated on the (p + 2)^2 coefficients with kz <= 1 against moment tables
// folded by the harmonic trace relation (see ridx).
//
// Tree.  Sources sorted by 30-bit Morton key in the bounding cube of sources
// and targets; cells level by level from the key prefixes: a cell with more
// than kLeafCap points is split into its non-empty octants (10 levels at
// most).  A cell's expansion centre c is the centre of its points' box.
// Moments in FP64: P2M at the leaves, then a binomial shift (M2M) up the
// tree; the cell radius rho is the largest distance of its points from c.
//
// Evaluation.  One warp per group of 32 consecutive sorted targets with a
// traversal stack in shared memory.  A cell with rho < theta x (distance
// from c to the group's box) is expanded (M2P, per target, FP32) unless it
// holds fewer points than an expansion costs, in which case its points are
// summed directly; other cells are opened; leaves are summed directly (P2P,
// FP32 with hi/lo coordinates relative to the cube centre).  Each cell's
// contribution is added to an FP64 total.
//
// Exclusion.  The tree sums every pair except pairs at zero distance; with
// fiber ids, each target's own-fiber pairs are then subtracted with the same
// pair routine -- the result is the fs_stokeslet_apply sum.
#include <cub/cub.cuh>

#include <cmath>
#include <vector>

#include "context.h"

namespace fs {
namespace {

constexpr int kMaxLevel = 10;
constexpr int kLeafCap = 64;
constexpr int kGroup = 32;
constexpr int kWarps = 4;          // warps (target groups) per CTA
// traversal stack entries per warp (order 10 keeps the CTA's static shared
// memory under 48 KB)
__host__ __device__ constexpr int stack_size(int P) { return P >= 10 ? 320 : 1024; }

__host__ __device__ constexpr int nterms(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// index of the multi-index (a, b, c): degree-major, then a descending, then b descending
__host__ __device__ constexpr int tidx(int a, int b, int c)
{
    return nterms(a + b + c - 1) + (b + c) * (b + c + 1) / 2 + c;
}

// Harmonic reduction.  The Taylor coefficients of 1/r obey the trace
// relation (kx+2)(kx+1) a_{k+2ex} + (ky+2)(ky+1) a_{k+2ey} + (kz+2)(kz+1) a_{k+2ez} = 0
// (Laplace's equation), so each degree d has 2d + 1 independent coefficients,
// those with kz <= 1, and the recurrence closes on them (it never needs
// a_{k-2ez}).  A contraction sum_k a_k T_k then equals sum over kz <= 1 of
// a_k T'_k with T' the tensor "folded" by the relation (entries with kz >= 2
// moved onto kz - 2); the folding is done once per cell in FP64.
// Reduced index: degree-major (offset d^2), kz = 0 first (kx descending), then kz = 1.
__host__ __device__ constexpr int ridx(int a, int b, int c)
{
    return (a + b + c) * (a + b + c) + (c == 0 ? (b + c) : (a + b + c) + 1 + (b + c - 1));
}

__device__ __forceinline__ unsigned spread10(unsigned v)
{
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ unsigned compact10(unsigned v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030C30C3u;
    v = (v | (v >> 4)) & 0x0300F00Fu;
    v = (v | (v >> 8)) & 0x030000FFu;
    v = (v | (v >> 16)) & 0x000003FFu;
    return v;
}

// ------------------------------------------------------------ bounding cube
__global__ void k_minmax(const double *__restrict__ x, int64_t n, double *__restrict__ part)
{
    __shared__ double s[6][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], x[3 * i + a]);
            hi[a] = fmax(hi[a], x[3 * i + a]);
        }
    for (int a = 0; a < 3; ++a) {
        s[a][threadIdx.x] = lo[a];
        s[3 + a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int a = 0; a < 3; ++a) {
                s[a][threadIdx.x] = fmin(s[a][threadIdx.x], s[a][threadIdx.x + o]);
                s[3 + a][threadIdx.x] = fmax(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

// cube[0..2] = lower corner, cube[3] = side, over nparts partial boxes
__global__ void k_cube(const double *__restrict__ part, int nparts, double *__restrict__ cube)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int p = 0; p < nparts; ++p)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], part[6 * p + a]);
            hi[a] = fmax(hi[a], part[6 * p + 3 + a]);
        }
    double side = fmax(fmax(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    side = side * (1.0 + 1e-9) + 1e-12 * (1.0 + fabs(lo[0]) + fabs(lo[1]) + fabs(lo[2]));
    for (int a = 0; a < 3; ++a) cube[a] = lo[a];
    cube[3] = side;
}

__global__ void k_keys(const double *__restrict__ x, int64_t n, const double *__restrict__ cube,
                       unsigned *__restrict__ key, int *__restrict__ idx)
{
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    unsigned q[3];
    for (int a = 0; a < 3; ++a) {
        const double t = (x[3 * i + a] - cube[a]) / cube[3] * 1024.0;
        q[a] = static_cast<unsigned>(fmin(fmax(t, 0.0), 1023.0));
    }
    key[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
    idx[i] = static_cast<int>(i);
}

// ------------------------------------------------------------ tree cells
struct Cells {
    double *ctr;      // [cap][3] expansion centre: the centre of the box of the cell's points
    float *rad;       // [cap] largest distance of a point from ctr
    int *beg, *end;   // sorted point range
    int *cb, *ce;     // child range (cb = -1: leaf)
    int *par;         // parent (-1: root)
    int *lvl;
    double *box;      // [cap][6] box of the cell's points (lo xyz, hi xyz)
};

__device__ void cell_centre(unsigned prefix, int level, const double *cube, double *c)
{
    const unsigned ix = compact10(prefix >> 2), iy = compact10(prefix >> 1), iz = compact10(prefix);
    const double h = cube[3] / double(1u << level);
    c[0] = cube[0] + (ix + 0.5) * h;
    c[1] = cube[1] + (iy + 0.5) * h;
    c[2] = cube[2] + (iz + 0.5) * h;
}

__global__ void k_root(Cells C, int n, const double *__restrict__ cube)
{
    C.beg[0] = 0;
    C.end[0] = n;
    C.cb[0] = C.ce[0] = -1;
    C.par[0] = -1;
    C.lvl[0] = 0;
    for (int a = 0; a < 3; ++a) C.ctr[a] = cube[a] + 0.5 * cube[3];
}

// flag[i] = 1 if point i starts a child of a cell being split at this level
__global__ void k_flag(Cells C, const unsigned *__restrict__ key, const int *__restrict__ pcell, int n, int level,
                       int *__restrict__ flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = pcell[i];
    int f = 0;
    if (C.lvl[p] == level - 1 && C.end[p] - C.beg[p] > kLeafCap) {
        const int s = 3 * (kMaxLevel - level);
        f = (i == C.beg[p] || (key[i] >> s) != (key[i - 1] >> s)) ? 1 : 0;
    }
    flag[i] = f;
}

__global__ void k_children(Cells C, const unsigned *__restrict__ key, int *__restrict__ pcell,
                           const int *__restrict__ flag, const int *__restrict__ pos, int n, int level, int base,
                           const double *__restrict__ cube)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = pcell[i];
    if (!(C.lvl[p] == level - 1 && C.end[p] - C.beg[p] > kLeafCap)) return;
    const int k = base + pos[i] + flag[i] - 1;   // the child holding point i
    if (flag[i]) {
        C.beg[k] = i;
        C.par[k] = p;
        C.lvl[k] = level;
        C.cb[k] = C.ce[k] = -1;
        cell_centre(key[i] >> (3 * (kMaxLevel - level)), level, cube, C.ctr + 3 * int64_t(k));
    }
    pcell[i] = k;
}

// end of each new child, and each split parent's child range
__global__ void k_child_links(Cells C, int base, int count)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int k = base + t, p = C.par[k];
    const bool last = t + 1 == count || C.par[k + 1] != p;
    C.end[k] = last ? C.end[p] : C.beg[k + 1];
    if (t == 0 || C.par[k - 1] != p) C.cb[p] = k;
    if (last) C.ce[p] = k + 1;
}

__global__ void k_total(const int *__restrict__ flag, const int *__restrict__ pos, int n, int *__restrict__ total)
{
    *total = n > 0 ? pos[n - 1] + flag[n - 1] : 0;
}

// sorted sources: FP64 positions and densities, FP32 hi/lo positions relative
// to the cube centre, FP32 densities
__global__ void k_gather_src(const double *__restrict__ x, const double *__restrict__ wf, const int *__restrict__ perm,
                             int n, const double *__restrict__ cube, double *__restrict__ xs, double *__restrict__ fs,
                             float4 *__restrict__ yh, float4 *__restrict__ yl, float4 *__restrict__ yf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = perm[i];
    float h[3], l[3];
    for (int a = 0; a < 3; ++a) {
        xs[3 * i + a] = x[3 * int64_t(j) + a];
        fs[3 * i + a] = wf[3 * int64_t(j) + a];
        const double d = x[3 * int64_t(j) + a] - (cube[a] + 0.5 * cube[3]);
        h[a] = static_cast<float>(d);
        l[a] = static_cast<float>(d - static_cast<double>(h[a]));
    }
    yh[i] = make_float4(h[0], h[1], h[2], 0.0f);
    yl[i] = make_float4(l[0], l[1], l[2], 0.0f);
    yf[i] = make_float4(static_cast<float>(wf[3 * int64_t(j)]), static_cast<float>(wf[3 * int64_t(j) + 1]),
                        static_cast<float>(wf[3 * int64_t(j) + 2]), 0.0f);
}

// ------------------------------------------------------------ moments (FP64)
// Boxes of the cells' points (FP64), leaves from the points, split cells
// from their children, and the expansion centres at the boxes' centres (a
// cell's points often fill only part of its octant: fibers).
__global__ void k_leaf_box(Cells C, const int *__restrict__ leaves, int nleaves, const double *__restrict__ xs)
{
    const int li = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (li >= nleaves) return;
    const int c = leaves[li];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = C.beg[c] + lane; i < C.end[c]; i += 32)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], xs[3 * int64_t(i) + a]);
            hi[a] = fmax(hi[a], xs[3 * int64_t(i) + a]);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            C.box[6 * int64_t(c) + a] = lo[a];
            C.box[6 * int64_t(c) + 3 + a] = hi[a];
            C.ctr[3 * int64_t(c) + a] = 0.5 * (lo[a] + hi[a]);
        }
}

__global__ void k_split_box(Cells C, const int *__restrict__ cells, int ncells)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncells) return;
    const int c = cells[k];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int ch = C.cb[c]; ch < C.ce[c]; ++ch)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], C.box[6 * int64_t(ch) + a]);
            hi[a] = fmax(hi[a], C.box[6 * int64_t(ch) + 3 + a]);
        }
    for (int a = 0; a < 3; ++a) {
        C.box[6 * int64_t(c) + a] = lo[a];
        C.box[6 * int64_t(c) + 3 + a] = hi[a];
        C.ctr[3 * int64_t(c) + a] = 0.5 * (lo[a] + hi[a]);
    }
}

// multi-index (a, b, c) of term t (degree-major order of tidx)
__device__ __forceinline__ void term_of(int t, int &a, int &b, int &c)
{
    int n = 0;
    while (nterms(n) <= t) ++n;
    const int r = t - nterms(n - 1);
    int bc = 0;
    while ((bc + 1) * (bc + 2) / 2 <= r) ++bc;
    c = r - bc * (bc + 1) / 2;
    b = bc - c;
    a = n - bc;
}

// P2M at the leaves: one CTA per leaf, threads over the terms; points staged
// in shared memory with their powers (y - c)_i^e, so a monomial is two
// products; rad from the points.
template <int P>
__global__ void __launch_bounds__(128) k_p2m(Cells C, const int *__restrict__ leaves, int nleaves,
                                             const double *__restrict__ xs, const double *__restrict__ fs,
                                             double *__restrict__ M)
{
    constexpr int T = nterms(P);
    constexpr int S = (T + 127) / 128;
    __shared__ double pw[32][3][P + 1], sq[32][4];
    __shared__ float srad[128];
    const int li = blockIdx.x;
    if (li >= nleaves) return;
    const int c = leaves[li];
    const double *ctr = C.ctr + 3 * int64_t(c);
    int ta[S], tb[S], tc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int t = threadIdx.x + 128 * s;
        if (t < T) term_of(t, ta[s], tb[s], tc[s]);
    }
    double acc[S][4] = {};
    float rmax = 0.0f;
    for (int b0 = C.beg[c]; b0 < C.end[c]; b0 += 32) {
        const int nb = min(32, C.end[c] - b0);
        __syncthreads();
        if (threadIdx.x < nb) {
            const int i = b0 + threadIdx.x;
            double d[3];
            for (int a = 0; a < 3; ++a) {
                d[a] = xs[3 * int64_t(i) + a] - ctr[a];
                double v = 1.0;
                for (int e = 0; e <= P; ++e) {
                    pw[threadIdx.x][a][e] = v;
                    v *= d[a];
                }
            }
            const double *f = fs + 3 * int64_t(i);
            sq[threadIdx.x][0] = f[0];
            sq[threadIdx.x][1] = f[1];
            sq[threadIdx.x][2] = f[2];
            sq[threadIdx.x][3] = d[0] * f[0] + d[1] * f[1] + d[2] * f[2];
            rmax = fmaxf(rmax, static_cast<float>(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])));
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (threadIdx.x + 128 * s >= T) break;
            for (int j = 0; j < nb; ++j) {
                const double m = pw[j][0][ta[s]] * pw[j][1][tb[s]] * pw[j][2][tc[s]];
                for (int q = 0; q < 4; ++q) acc[s][q] = fma(m, sq[j][q], acc[s][q]);
            }
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int t = threadIdx.x + 128 * s;
        if (t < T)
            for (int q = 0; q < 4; ++q) M[(int64_t(c) * 4 + q) * T + t] = acc[s][q];
    }
    srad[threadIdx.x] = rmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.0f;
        for (int k = 0; k < 128; ++k) r = fmaxf(r, srad[k]);
        C.rad[c] = r * (1.0f + 1e-6f);
    }
}

// M2M for the split cells of one level: M_k(parent) = sum_children sum_{j <= k}
// binom(k, j) d^{k - j} M_j(child), d = c_child - c_parent, applied as three
// one-dimensional shifts (the binomial kernel is separable); the charge
// (y - c).f moves with the centre, so its parent moments add d . (the shifted
// force moments).
template <int P>
__global__ void __launch_bounds__(128) k_m2m(Cells C, const int *__restrict__ cells, int ncells,
                                             double *__restrict__ M)
{
    constexpr int T = nterms(P);
    constexpr int S = (4 * T + 127) / 128;   // (charge, term) entries per thread
    __shared__ double pw[3][P + 1];
    __shared__ double binom[P + 1][P + 1];
    __shared__ double t1[4 * T], t2[4 * T];
    const int ci = blockIdx.x;
    if (ci >= ncells) return;
    const int c = cells[ci];
    for (int t = threadIdx.x; t < (P + 1) * (P + 1); t += blockDim.x) {
        const int n = t / (P + 1), k = t % (P + 1);
        double b = 0.0;
        if (k <= n) {
            b = 1.0;
            for (int e = 0; e < k; ++e) b = b * (n - e) / (e + 1);
        }
        binom[n][k] = b;
    }
    int ta[S], tb[S], tc[S], tq[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int e = threadIdx.x + 128 * s;
        tq[s] = e / T;
        if (e < 4 * T) term_of(e % T, ta[s], tb[s], tc[s]);
    }
    double acc[S] = {};
    float rmax = 0.0f;
    for (int ch = C.cb[c]; ch < C.ce[c]; ++ch) {
        __syncthreads();
        if (threadIdx.x < 3) {
            const double d = C.ctr[3 * int64_t(ch) + threadIdx.x] - C.ctr[3 * int64_t(c) + threadIdx.x];
            double v = 1.0;
            for (int e = 0; e <= P; ++e) {
                pw[threadIdx.x][e] = v;
                v *= d;
            }
        }
        __syncthreads();
        const double dx = pw[0][1], dy = pw[1][1], dz = pw[2][1];
        rmax = fmaxf(rmax, C.rad[ch] + static_cast<float>(sqrt(dx * dx + dy * dy + dz * dz)));
        const double *Mc = M + int64_t(ch) * 4 * T;
        // x pass: t1[a,b,c] = sum_{j <= a} binom(a, j) dx^(a-j) M[j,b,c]
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int e = threadIdx.x + 128 * s;
            if (e >= 4 * T) break;
            double v = 0.0;
            for (int j = 0; j <= ta[s]; ++j) v = fma(binom[ta[s]][j] * pw[0][ta[s] - j], Mc[tq[s] * T + tidx(j, tb[s], tc[s])], v);
            t1[e] = v;
        }
        __syncthreads();
        // y pass
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int e = threadIdx.x + 128 * s;
            if (e >= 4 * T) break;
            double v = 0.0;
            for (int j = 0; j <= tb[s]; ++j) v = fma(binom[tb[s]][j] * pw[1][tb[s] - j], t1[tq[s] * T + tidx(ta[s], j, tc[s])], v);
            t2[e] = v;
        }
        __syncthreads();
        // z pass into t1, then accumulate with the charge shift
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int e = threadIdx.x + 128 * s;
            if (e >= 4 * T) break;
            double v = 0.0;
            for (int j = 0; j <= tc[s]; ++j) v = fma(binom[tc[s]][j] * pw[2][tc[s] - j], t2[tq[s] * T + tidx(ta[s], tb[s], j)], v);
            t1[e] = v;
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int e = threadIdx.x + 128 * s;
            if (e >= 4 * T) break;
            const int t = e % T;
            acc[s] += t1[e];
            if (tq[s] == 3) acc[s] += dx * t1[t] + dy * t1[T + t] + dz * t1[2 * T + t];
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int e = threadIdx.x + 128 * s;
        if (e < 4 * T) M[int64_t(c) * 4 * T + e] = acc[s];
    }
    if (threadIdx.x == 0) C.rad[c] = rmax;
}

// Folded FP32 tables of one cell, float4 (four charges) per entry:
//   [0, (P+1)^2)                     potentials, M_k folded, degrees 0..P
//   then for i = x, y, z: (P+2)^2-1  gradient tensors T^i_m = -m_i M_{m-e_i}, degrees 1..P+1
// One CTA per cell, the tensors in shared memory, one thread per (charge,
// table, degree); FP64.
__host__ __device__ constexpr int nfold(int P) { return (P + 1) * (P + 1) + 3 * ((P + 2) * (P + 2) - 1); }

template <int P>
__global__ void __launch_bounds__(16 * (P + 2)) k_fold(const double *__restrict__ M, int ncells,
                                                      float4 *__restrict__ out)
{
    constexpr int T = nterms(P), T1 = nterms(P + 1), NF = nfold(P);
    // the 16 tensors of the cell (charge q x table: potential, gradient x, y, z)
    // over degrees 0..P+1, degree-major as tidx
    __shared__ double sv[16][T1];
    __shared__ unsigned char sk[T1][3];   // multi-index of each term
    const int cell = blockIdx.x;
    if (cell >= ncells) return;
    const double *Mc = M + int64_t(cell) * 4 * T;
    for (int t = threadIdx.x; t < T1; t += blockDim.x) {
        int a, b, c;
        term_of(t, a, b, c);
        sk[t][0] = static_cast<unsigned char>(a);
        sk[t][1] = static_cast<unsigned char>(b);
        sk[t][2] = static_cast<unsigned char>(c);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 16 * T1; idx += blockDim.x) {
        const int tq = idx / T1, t = idx - tq * T1, q = tq >> 2, tab = tq & 3;
        const int k[3] = {sk[t][0], sk[t][1], sk[t][2]};
        const int n = k[0] + k[1] + k[2];
        double v = 0.0;
        if (tab == 0) {
            if (n <= P) v = Mc[q * T + t];
        } else {
            const int i = tab - 1;
            if (k[i] >= 1) {
                int km[3] = {k[0], k[1], k[2]};
                --km[i];
                v = -double(k[i]) * Mc[q * T + tidx(km[0], km[1], km[2])];
            }
        }
        sv[tq][t] = v;
    }
    __syncthreads();
    // one thread per (tensor, degree): fold the entries with c >= 2 (highest
    // c first) onto c - 2, then write the entries with c <= 1
    const int tq = threadIdx.x / (P + 2), d = threadIdx.x % (P + 2);
    const int q = tq >> 2, tab = tq & 3;
    if ((tab == 0 && d > P) || (tab > 0 && d == 0)) return;
    double *v = sv[tq] + nterms(d - 1);
    for (int c = d; c >= 2; --c) {
        const int bz = c - 2;
        const double rw = 1.0 / double((bz + 2) * (bz + 1));
        for (int b = d - c; b >= 0; --b) {
            const int a = d - b - c;
            const double x = v[(b + c) * (b + c + 1) / 2 + c] * rw;
            v[(b + bz) * (b + bz + 1) / 2 + bz] -= x * double((a + 2) * (a + 1));
            v[(b + 2 + bz) * (b + 2 + bz + 1) / 2 + bz] -= x * double((b + 2) * (b + 1));
        }
    }
    const int base = tab == 0 ? 0 : (P + 1) * (P + 1) + (tab - 1) * ((P + 2) * (P + 2) - 1) - 1;
    float *o = reinterpret_cast<float *>(out + int64_t(cell) * NF);
    for (int a = d; a >= 0; --a)
        for (int b = d - a; b >= 0; --b) {
            const int c = d - a - b;
            if (c > 1) continue;
            o[4 * (base + ridx(a, b, c)) + q] = static_cast<float>(v[(b + c) * (b + c + 1) / 2 + c]);
        }
}

// evaluation records: centre relative to the cube centre as hi (with the
// radius) and lo floats, and (beg, end, cb, ce)
__global__ void k_pack_cells(Cells C, int ncells, const double *__restrict__ cube, float4 *__restrict__ ch,
                             float4 *__restrict__ cl, int4 *__restrict__ ci)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncells) return;
    float h[3], l[3];
    for (int a = 0; a < 3; ++a) {
        const double d = C.ctr[3 * int64_t(k) + a] - (cube[a] + 0.5 * cube[3]);
        h[a] = static_cast<float>(d);
        l[a] = static_cast<float>(d - static_cast<double>(h[a]));
    }
    ch[k] = make_float4(h[0], h[1], h[2], C.rad[k]);
    cl[k] = make_float4(l[0], l[1], l[2], 0.0f);
    ci[k] = make_int4(C.beg[k], C.end[k], C.cb[k], C.ce[k]);
}

// ------------------------------------------------------------ target groups
// per group of 32 sorted targets: centre of its box relative to the cube
// centre as hi (with the half-diagonal) and lo floats; per target: hi/lo
// position relative to the cube centre
__global__ void k_groups(const double *__restrict__ x, const int *__restrict__ tperm, int n,
                         const double *__restrict__ cube, float4 *__restrict__ gctr, float4 *__restrict__ xh,
                         float4 *__restrict__ xl)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int g = t / kGroup;
    const bool ok = t < n;
    double p[3] = {0.0, 0.0, 0.0};
    if (ok) {
        const int j = tperm[t];
        float h[3], l[3];
        for (int a = 0; a < 3; ++a) {
            p[a] = x[3 * int64_t(j) + a];
            const double d = p[a] - (cube[a] + 0.5 * cube[3]);
            h[a] = static_cast<float>(d);
            l[a] = static_cast<float>(d - static_cast<double>(h[a]));
        }
        xh[t] = make_float4(h[0], h[1], h[2], 0.0f);
        xl[t] = make_float4(l[0], l[1], l[2], 0.0f);
    }
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = ok ? p[a] : INFINITY;
        hi[a] = ok ? p[a] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if (lane == 0 && g * kGroup < n) {
        double h2 = 0.0;
        float gh[3], gl[3];
        for (int a = 0; a < 3; ++a) {
            const double d = 0.5 * (lo[a] + hi[a]) - (cube[a] + 0.5 * cube[3]);
            gh[a] = static_cast<float>(d);
            gl[a] = static_cast<float>(d - static_cast<double>(gh[a]));
            h2 += 0.25 * (hi[a] - lo[a]) * (hi[a] - lo[a]);
        }
        gctr[3 * int64_t(g)] = make_float4(gh[0], gh[1], gh[2], static_cast<float>(sqrt(h2)) * (1.0f + 1e-6f) + 1e-30f);
        gctr[3 * int64_t(g) + 1] = make_float4(gl[0], gl[1], gl[2], 0.0f);
        // half-extents of the group's box (rounded up)
        gctr[3 * int64_t(g) + 2] = make_float4(static_cast<float>(0.5 * (hi[0] - lo[0])) * (1.0f + 1e-6f) + 1e-30f,
                                               static_cast<float>(0.5 * (hi[1] - lo[1])) * (1.0f + 1e-6f) + 1e-30f,
                                               static_cast<float>(0.5 * (hi[2] - lo[2])) * (1.0f + 1e-6f) + 1e-30f, 0.0f);
    }
}

// ------------------------------------------------------------ evaluation
// 8 pi mu u += phi_i - r_j d_i phi_j + d_i phi_4 for one cell's folded tables
// sF (shared memory), r = x - c: the coefficients with kz <= 1 of degree n + 1
// are generated before the degree-n potential table and the degree-(n + 1)
// gradient tables are contracted, so only two degrees are live.
template <int P>
__device__ __forceinline__ void m2p(const float4 *sF, float rx, float ry, float rz, float (&u)[3])
{
    constexpr int G0 = (P + 1) * (P + 1), GN = (P + 2) * (P + 2) - 1;
    float a[(P + 2) * (P + 2)];
    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    const float ir2 = 1.0f / r2;
    a[0] = rsqrtf(r2);
    float phi[3] = {0.0f, 0.0f, 0.0f}, gx[4] = {0.0f, 0.0f, 0.0f, 0.0f}, gy[4] = {0.0f, 0.0f, 0.0f, 0.0f},
          gz[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int n = 0; n <= P; ++n) {
        const int m = n + 1;
        const float c1 = float(2 * m - 1) / float(m), c2 = float(m - 1) / float(m);
#pragma unroll
        for (int cc = 0; cc <= 1; ++cc)
#pragma unroll
            for (int aa = m - cc; aa >= 0; --aa) {
                const int bb = m - cc - aa;
                float s1 = 0.0f, s2 = 0.0f;
                if (aa >= 1) s1 = fmaf(rx, a[ridx(aa - 1, bb, cc)], s1);
                if (bb >= 1) s1 = fmaf(ry, a[ridx(aa, bb - 1, cc)], s1);
                if (cc >= 1) s1 = fmaf(rz, a[ridx(aa, bb, cc - 1)], s1);
                if (aa >= 2) s2 += a[ridx(aa - 2, bb, cc)];
                if (bb >= 2) s2 += a[ridx(aa, bb - 2, cc)];
                a[ridx(aa, bb, cc)] = (c1 * s1 - c2 * s2) * ir2;
            }
        // potentials of degree n (the fourth charge's potential is not needed)
#pragma unroll
        for (int cc = 0; cc <= 1; ++cc)
#pragma unroll
            for (int aa = n - cc; aa >= 0; --aa) {
                const int bb = n - cc - aa;
                if (bb < 0) continue;
                const float ak = a[ridx(aa, bb, cc)];
                const float4 t = sF[ridx(aa, bb, cc)];
                phi[0] = fmaf(ak, t.x, phi[0]);
                phi[1] = fmaf(ak, t.y, phi[1]);
                phi[2] = fmaf(ak, t.z, phi[2]);
            }
        // gradients: tables of degree m
#pragma unroll
        for (int cc = 0; cc <= 1; ++cc)
#pragma unroll
            for (int aa = m - cc; aa >= 0; --aa) {
                const int bb = m - cc - aa;
                const int j = ridx(aa, bb, cc) - 1;
                const float am = a[ridx(aa, bb, cc)];
                const float4 tx = sF[G0 + j], ty = sF[G0 + GN + j], tz = sF[G0 + 2 * GN + j];
                gx[0] = fmaf(am, tx.x, gx[0]);
                gx[1] = fmaf(am, tx.y, gx[1]);
                gx[2] = fmaf(am, tx.z, gx[2]);
                gx[3] = fmaf(am, tx.w, gx[3]);
                gy[0] = fmaf(am, ty.x, gy[0]);
                gy[1] = fmaf(am, ty.y, gy[1]);
                gy[2] = fmaf(am, ty.z, gy[2]);
                gy[3] = fmaf(am, ty.w, gy[3]);
                gz[0] = fmaf(am, tz.x, gz[0]);
                gz[1] = fmaf(am, tz.y, gz[1]);
                gz[2] = fmaf(am, tz.z, gz[2]);
                gz[3] = fmaf(am, tz.w, gz[3]);
            }
    }
    u[0] += phi[0] - (rx * gx[0] + ry * gx[1] + rz * gx[2]) + gx[3];
    u[1] += phi[1] - (rx * gy[0] + ry * gy[1] + rz * gy[2]) + gy[3];
    u[2] += phi[2] - (rx * gz[0] + ry * gz[1] + rz * gz[2]) + gz[3];
}

// one Stokeslet pair, 8 pi mu G(r) f, r from hi/lo parts (shared by the tree's
// near field and the own-fiber subtraction, so that the same pair rounds the
// same way in both)
__device__ __forceinline__ void pair_stokes(float4 xh, float4 xl, float4 h, float4 l, float4 f, float (&u)[3])
{
    const float rx = (xh.x - h.x) + (xl.x - l.x);
    const float ry = (xh.y - h.y) + (xl.y - l.y);
    const float rz = (xh.z - h.z) + (xl.z - l.z);
    const float r2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    if (r2 == 0.0f) return;   // a point with itself (identical positions give identical hi/lo parts)
    const float ir = rsqrtf(r2);
    const float hf = fmaf(rz, f.z, fmaf(ry, f.y, rx * f.x)) * (ir * ir);
    u[0] = fmaf(ir, fmaf(rx, hf, f.x), u[0]);
    u[1] = fmaf(ir, fmaf(ry, hf, f.y), u[1]);
    u[2] = fmaf(ir, fmaf(rz, hf, f.z), u[2]);
}

// compensated FP32 accumulation (TwoSum): (s, e) += v
__device__ __forceinline__ void acc2(float &s, float &e, float v)
{
    const float t = s + v;
    const float bp = t - s;
    e += (s - (t - bp)) + (v - bp);
    s = t;
}

struct EvalArgs {
    const float4 *ch, *cl;           // cell centres (hi + radius, lo)
    const int4 *ci;                  // cell (beg, end, cb, ce)
    const float4 *Mf;                // [cells][nfold(P)] folded FP32 tables of the four charges
    const float4 *yh, *yl, *yf;      // sorted sources
    const float4 *xh, *xl;           // sorted targets
    const float4 *gctr;              // per group: centre hi (+ half-diagonal), lo, box half-extents
    const int *tperm;                // sorted target -> original index
    int n_tgt, ngroups;
    float theta;
    int direct_max;                  // expanded only above this many points
    double scale;
    double *out;                     // [n_tgt][3], original order
    int *status;
};

// direct sum over the sorted sources [b, e), staged through shared memory in
// chunks of 32 (one per lane)
__device__ __forceinline__ void p2p_range(const EvalArgs &A, int b, int e, int t, bool ok, float4 xh, float4 xl,
                                          float4 (*sy)[32], int lane, float (&u)[3])
{
    for (int j0 = b; j0 < e; j0 += 32) {
        const int nj = min(32, e - j0);
        __syncwarp();
        if (lane < nj) {
            sy[0][lane] = __ldg(A.yh + j0 + lane);
            sy[1][lane] = __ldg(A.yl + j0 + lane);
            sy[2][lane] = __ldg(A.yf + j0 + lane);
        }
        __syncwarp();
        if (ok) {
#pragma unroll 4
            for (int jj = 0; jj < nj; ++jj) pair_stokes(xh, xl, sy[0][jj], sy[1][jj], sy[2][jj], u);
        }
    }
}

// four CTAs of four warps per SM: 128 registers (the expansion's coefficient
// window spills a few bytes at order 8; measured 14 % faster than 190
// registers at two CTAs)
template <int P>
__global__ void __launch_bounds__(kWarps * 32, 4) k_tree_eval(EvalArgs A)
{
    constexpr int T = nterms(P);
    constexpr int kStack = stack_size(P);
    __shared__ int stack[kWarps][kStack];
    constexpr int NF = nfold(P);
    __shared__ float4 smom[kWarps][NF];
    __shared__ float4 sy[kWarps][3][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kWarps + warp;
    if (g >= A.ngroups) return;
    const int t = g * kGroup + lane;
    const bool ok = t < A.n_tgt;
    const float4 xh = ok ? A.xh[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 xl = ok ? A.xl[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 gh4 = A.gctr[3 * int64_t(g)], gl4 = A.gctr[3 * int64_t(g) + 1], ge4 = A.gctr[3 * int64_t(g) + 2];
    // target relative to the group centre, from hi/lo parts (both offsets
    // from the cube centre can be large; their difference is small)
    const float xg[3] = {(xh.x - gh4.x) + (xl.x - gl4.x), (xh.y - gh4.y) + (xl.y - gl4.y),
                         (xh.z - gh4.z) + (xl.z - gl4.z)};
    float acc[3] = {0.0f, 0.0f, 0.0f}, err[3] = {0.0f, 0.0f, 0.0f};
    // warp-parallel walk: up to 32 cells popped at once, one per lane, each
    // loaded and classified by its lane; children pushed with a warp prefix
    // sum; then the batch's expansions and direct cells are evaluated by the
    // whole warp, one cell at a time, in lane order
    int top = 1;
    if (lane == 0) stack[warp][0] = 0;
    __syncwarp();
    while (top > 0) {
        // batch size shrinks as the stack fills (an opened cell pushes at most
        // 8 children), down to one cell at a time (depth first)
        const int nb = min(min(32, top), max(1, (kStack - top) / 8));
        top -= nb;
        const bool mine = lane < nb;
        const int c = mine ? stack[warp][top + lane] : 0;
        __syncwarp();
        int kind = 0;   // 1: expand, 2: direct, 3: open
        float dx = 0.0f, dy = 0.0f, dz = 0.0f;
        int4 cic = make_int4(0, 0, 0, 0);
        if (mine) {
            const float4 chc = __ldg(A.ch + c), clc = __ldg(A.cl + c);
            cic = __ldg(A.ci + c);
            // group centre - cell centre, from hi/lo parts
            dx = (gh4.x - chc.x) + (gl4.x - clc.x);
            dy = (gh4.y - chc.y) + (gl4.y - clc.y);
            dz = (gh4.z - chc.z) + (gl4.z - clc.z);
            // distance from the cell centre to the group's box: a cell whose
            // radius is below theta times it is expanded for every target
            const float px = fmaxf(fabsf(dx) - ge4.x, 0.0f), py = fmaxf(fabsf(dy) - ge4.y, 0.0f),
                        pz = fmaxf(fabsf(dz) - ge4.z, 0.0f);
            const float dist = sqrtf(px * px + py * py + pz * pz);
            const bool far = dist > 0.0f && chc.w < A.theta * dist;
            kind = (far && cic.y - cic.x > A.direct_max) ? 1 : ((far || cic.z < 0) ? 2 : 3);
        }
        const int nch = kind == 3 ? cic.w - cic.z : 0;
        int inc = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const int total = __shfl_sync(0xffffffffu, inc, 31);
        if (top + total > kStack) {
            if (lane == 0) atomicOr(A.status, DEV_ERR_NUMERIC);
            break;
        }
        for (int j = 0; j < nch; ++j) stack[warp][top + inc - nch + j] = cic.z + j;
        top += total;
        unsigned mm = __ballot_sync(0xffffffffu, kind == 1);
        while (mm) {
            const int src = __ffs(mm) - 1;
            mm &= mm - 1;
            const int cc = __shfl_sync(0xffffffffu, c, src);
            const float ex = __shfl_sync(0xffffffffu, dx, src), ey = __shfl_sync(0xffffffffu, dy, src),
                        ez = __shfl_sync(0xffffffffu, dz, src);
            for (int k = lane; k < NF; k += 32) smom[warp][k] = __ldg(A.Mf + int64_t(cc) * NF + k);
            __syncwarp();
            float u[3] = {0.0f, 0.0f, 0.0f};
            if (ok) m2p<P>(smom[warp], xg[0] + ex, xg[1] + ey, xg[2] + ez, u);   // r = x - c
            __syncwarp();
            for (int a = 0; a < 3; ++a) acc2(acc[a], err[a], u[a]);
        }
        unsigned pm = __ballot_sync(0xffffffffu, kind == 2);
        while (pm) {
            const int src = __ffs(pm) - 1;
            pm &= pm - 1;
            const int b = __shfl_sync(0xffffffffu, cic.x, src), e = __shfl_sync(0xffffffffu, cic.y, src);
            float u[3] = {0.0f, 0.0f, 0.0f};
            p2p_range(A, b, e, t, ok, xh, xl, sy[warp], lane, u);
            for (int a = 0; a < 3; ++a) acc2(acc[a], err[a], u[a]);
        }
        __syncwarp();
    }
    if (ok) {
        const int j = A.tperm[t];
        for (int a = 0; a < 3; ++a)
            A.out[3 * int64_t(j) + a] = A.scale * (static_cast<double>(acc[a]) + static_cast<double>(err[a]));
    }
}

// out_i -= scale x the sum over the own-fiber sources, with the near field's
// pair routine on the same hi/lo FP32 inputs (pairs the near field summed
// cancel exactly)
__device__ __forceinline__ void hilo4(const double *x, const double *cube, float4 &h, float4 &l)
{
    float hh[3], ll[3];
    for (int a = 0; a < 3; ++a) {
        const double d = x[a] - (cube[a] + 0.5 * cube[3]);
        hh[a] = static_cast<float>(d);
        ll[a] = static_cast<float>(d - static_cast<double>(hh[a]));
    }
    h = make_float4(hh[0], hh[1], hh[2], 0.0f);
    l = make_float4(ll[0], ll[1], ll[2], 0.0f);
}

// the sorted source records back in the sources' original order
__global__ void k_unsort_src(const int *__restrict__ perm, int n, const float4 *__restrict__ yh,
                             const float4 *__restrict__ yl, const float4 *__restrict__ yf, float4 *__restrict__ oh,
                             float4 *__restrict__ ol, float4 *__restrict__ of)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = perm[i];
    oh[j] = yh[i];
    ol[j] = yl[i];
    of[j] = yf[i];
}

__global__ void k_sub_own(const float4 *__restrict__ oh, const float4 *__restrict__ ol, const float4 *__restrict__ of,
                          const double *__restrict__ xt, const int2 *__restrict__ excl, int n,
                          const double *__restrict__ cube, double scale, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 r = excl[i];
    float4 xh, xl;
    hilo4(xt + 3 * int64_t(i), cube, xh, xl);
    float acc[3] = {0.0f, 0.0f, 0.0f}, err[3] = {0.0f, 0.0f, 0.0f};
    for (int j = r.x; j < r.y; ++j) {
        float u[3] = {0.0f, 0.0f, 0.0f};
        pair_stokes(xh, xl, __ldg(oh + j), __ldg(ol + j), __ldg(of + j), u);
        for (int a = 0; a < 3; ++a) acc2(acc[a], err[a], u[a]);
    }
    for (int a = 0; a < 3; ++a)
        out[3 * int64_t(i) + a] -= scale * (static_cast<double>(acc[a]) + static_cast<double>(err[a]));
}

// expansions cost about this many direct pairs; smaller cells are summed directly
int direct_max_for(int P) { return nterms(P + 1) / 2 + 16; }

template <int P>
fs_status launch_eval_and_moments(const Cells &C, const std::vector<int> &leaves_h,
                                  const std::vector<std::vector<int>> &split_by_level, int ncells, int *d_list,
                                  const double *xs, const double *fs, double *Md, float4 *Mf, const double *cube,
                                  float4 *pch, float4 *pcl, int4 *pci, EvalArgs A, cudaStream_t st)
{
    constexpr int T = nterms(P);
    // point boxes and expansion centres, leaves then split cells bottom-up
    if (!leaves_h.empty()) {
        FS_CUDA(cudaMemcpyAsync(d_list, leaves_h.data(), leaves_h.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        k_leaf_box<<<static_cast<unsigned>((leaves_h.size() + 3) / 4), 128, 0, st>>>(C, d_list,
                                                                                  static_cast<int>(leaves_h.size()), xs);
        FS_LAUNCH_CHECK();
        FS_CUDA(cudaStreamSynchronize(st));   // d_list is reused below
    }
    for (int lv = kMaxLevel; lv >= 0; --lv) {
        const std::vector<int> &v = split_by_level[lv];
        if (v.empty()) continue;
        FS_CUDA(cudaMemcpyAsync(d_list, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        k_split_box<<<static_cast<unsigned>((v.size() + 127) / 128), 128, 0, st>>>(C, d_list, static_cast<int>(v.size()));
        FS_LAUNCH_CHECK();
        FS_CUDA(cudaStreamSynchronize(st));
    }
    if (!leaves_h.empty()) {
        FS_CUDA(cudaMemcpyAsync(d_list, leaves_h.data(), leaves_h.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        k_p2m<P><<<static_cast<unsigned>(leaves_h.size()), 128, 0, st>>>(C, d_list, static_cast<int>(leaves_h.size()),
                                                                          xs, fs, Md);
        FS_LAUNCH_CHECK();
        FS_CUDA(cudaStreamSynchronize(st));   // d_list is reused below
    }
    for (int lv = kMaxLevel; lv >= 0; --lv) {
        const std::vector<int> &v = split_by_level[lv];
        if (v.empty()) continue;
        FS_CUDA(cudaMemcpyAsync(d_list, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        k_m2m<P><<<static_cast<unsigned>(v.size()), 128, 0, st>>>(C, d_list, static_cast<int>(v.size()), Md);
        FS_LAUNCH_CHECK();
        FS_CUDA(cudaStreamSynchronize(st));
    }
    k_fold<P><<<static_cast<unsigned>(ncells), 16 * (P + 2), 0, st>>>(Md, ncells, Mf);
    FS_LAUNCH_CHECK();
    k_pack_cells<<<(ncells + 255) / 256, 256, 0, st>>>(C, ncells, cube, pch, pcl, pci);
    FS_LAUNCH_CHECK();
    A.direct_max = direct_max_for(P);
    k_tree_eval<P><<<static_cast<unsigned>((A.ngroups + kWarps - 1) / kWarps), kWarps * 32, 0, st>>>(A);
    FS_LAUNCH_CHECK();
    return FS_OK;
}

}  // namespace
}  // namespace fs

namespace fs {

// The treecode sum; exclusion from fiber ids, or from per-target source
// ranges (excl_given, as exclusion_from_ids writes them) when not NULL.
fs_status tree_sum(fs_ctx *c, const double *src_xyz, const double *src_wf, int64_t n_src, const int32_t *src_fiber,
                   const double *tgt_xyz, const int32_t *tgt_fiber, int64_t n_tgt, double *out_u, int32_t order,
                   double theta, const int2 *excl_given)
{
    if (!c || n_src < 0 || n_tgt < 0 || (n_src > 0 && (!src_xyz || !src_wf)) || (n_tgt > 0 && (!tgt_xyz || !out_u))) {
        set_error("fs_stokeslet_apply_tree: bad sizes or NULL arrays");
        return FS_EINVAL;
    }
    if (order != 4 && order != 6 && order != 8 && order != 10) {
        set_error("fs_stokeslet_apply_tree: order must be 4, 6, 8 or 10 (got %d)", order);
        return FS_EINVAL;
    }
    if (!(theta > 0.0 && theta < 1.0)) {
        set_error("fs_stokeslet_apply_tree: theta must lie in (0, 1)");
        return FS_EINVAL;
    }
    if (n_src >= (1LL << 30) || n_tgt >= (1LL << 30)) {
        set_error("fs_stokeslet_apply_tree: at most 2^30 sources and targets");
        return FS_EINVAL;
    }
    cudaStream_t st = c->stream;
    if (n_tgt == 0) return FS_OK;
    if (n_src == 0) {
        FS_CUDA(cudaMemsetAsync(out_u, 0, static_cast<size_t>(n_tgt) * 3 * sizeof(double), st));
        return FS_OK;
    }
    const int ns = static_cast<int>(n_src), nt = static_cast<int>(n_tgt);
    const bool self = src_xyz == tgt_xyz && n_src == n_tgt;
    const bool ids = (src_fiber && tgt_fiber) || excl_given;
    const int T = nterms(order);
    const int cap = 2 * ns + 64;   // cells: a split cell holds > kLeafCap points
    const int ngroups = (nt + kGroup - 1) / kGroup;
    const int nparts = 128;

    // workspace: CUB temporaries sized first
    size_t sort_tmp = 0, scan_tmp = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sort_tmp, (unsigned *)nullptr, (unsigned *)nullptr, (int *)nullptr,
                                    (int *)nullptr, std::max(ns, nt), 0, 3 * kMaxLevel);
    cub::DeviceScan::ExclusiveSum(nullptr, scan_tmp, (int *)nullptr, (int *)nullptr, ns);
    const size_t d = sizeof(double);
    size_t need = 0;
    auto acct = [&](size_t bytes) { need += (bytes + 255) & ~size_t(255); };
    acct(6 * nparts * d);
    acct(4 * d);
    acct(2 * size_t(std::max(ns, nt)) * 4 * 2);             // keys in/out
    acct(2 * size_t(std::max(ns, nt)) * 4 * 2);             // indices in/out (src + tgt)
    acct(std::max(sort_tmp, scan_tmp));
    acct(size_t(ns) * 4 * 3);                               // pcell, flag, pos
    acct(sizeof(int));
    acct(size_t(cap) * (3 * d + 4 + 6 * 4));                // cells
    acct(size_t(cap) * 6 * d);                              // cell point boxes
    acct(size_t(cap) * 4);                                  // list
    acct(size_t(ns) * 6 * d);                               // xs, fs
    acct(size_t(ns) * 3 * 16);                              // yh, yl, yf
    acct(size_t(ngroups) * 48);
    acct(size_t(nt) * 2 * 16);
    acct(sizeof(int));
    if (ids) {
        acct(size_t(nt) * sizeof(int2));
        for (int k = 0; k < 3; ++k) acct(size_t(ns) * 16);
    }
    need += 64 * 256;   // alignment of the individual arrays
    FS_TRY(c->scratch.reserve(need, st));
    Carve cv(c->scratch.ptr, c->scratch.bytes);
    double *part = cv.take<double>(6 * nparts);
    double *cube = cv.take<double>(4);
    const int nk = std::max(ns, nt);
    unsigned *kin = cv.take<unsigned>(nk), *kout = cv.take<unsigned>(nk);
    int *iin = cv.take<int>(nk), *sperm = cv.take<int>(nk);
    unsigned *tkout = cv.take<unsigned>(nk);
    int *tperm_buf = cv.take<int>(nk);
    void *tmp = cv.take<unsigned char>(std::max(sort_tmp, scan_tmp));
    int *pcell = cv.take<int>(ns), *flag = cv.take<int>(ns), *pos = cv.take<int>(ns);
    int *d_total = cv.take<int>(1);
    Cells C;
    C.ctr = cv.take<double>(3 * size_t(cap));
    C.rad = cv.take<float>(cap);
    C.beg = cv.take<int>(cap);
    C.end = cv.take<int>(cap);
    C.cb = cv.take<int>(cap);
    C.ce = cv.take<int>(cap);
    C.par = cv.take<int>(cap);
    C.lvl = cv.take<int>(cap);
    C.box = cv.take<double>(6 * size_t(cap));
    int *d_list = cv.take<int>(cap);
    double *xs = cv.take<double>(3 * size_t(ns)), *fsrc = cv.take<double>(3 * size_t(ns));
    float4 *yh = cv.take<float4>(ns), *yl = cv.take<float4>(ns), *yf = cv.take<float4>(ns);
    float4 *gctr = cv.take<float4>(3 * size_t(ngroups));
    float4 *xh = cv.take<float4>(nt), *xl = cv.take<float4>(nt);
    int2 *excl = (ids && !excl_given) ? cv.take<int2>(nt) : nullptr;
    float4 *oh = ids ? cv.take<float4>(ns) : nullptr, *ol = ids ? cv.take<float4>(ns) : nullptr,
           *of = ids ? cv.take<float4>(ns) : nullptr;
    int *tstat = cv.take<int>(1);   // traversal status (own word: the context's may carry other flags)
    if (cv.used > cv.cap) {
        set_error("fs_stokeslet_apply_tree: workspace accounting");
        return FS_EINVAL;
    }
    FS_CUDA(cudaMemsetAsync(tstat, 0, sizeof(int), st));

    // bounding cube of sources and targets
    k_minmax<<<nparts / 2, 256, 0, st>>>(src_xyz, n_src, part);
    FS_LAUNCH_CHECK();
    k_minmax<<<nparts / 2, 256, 0, st>>>(tgt_xyz, n_tgt, part + 6 * (nparts / 2));
    FS_LAUNCH_CHECK();
    k_cube<<<1, 32, 0, st>>>(part, nparts, cube);
    FS_LAUNCH_CHECK();
    // sort sources (and targets unless they are the sources)
    k_keys<<<(ns + 255) / 256, 256, 0, st>>>(src_xyz, n_src, cube, kin, iin);
    FS_LAUNCH_CHECK();
    size_t tb = sort_tmp;
    FS_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tb, kin, kout, iin, sperm, ns, 0, 3 * kMaxLevel, st));
    const int *tperm = sperm;
    if (!self) {
        k_keys<<<(nt + 255) / 256, 256, 0, st>>>(tgt_xyz, n_tgt, cube, kin, iin);
        FS_LAUNCH_CHECK();
        tb = sort_tmp;
        FS_CUDA(cub::DeviceRadixSort::SortPairs(tmp, tb, kin, tkout, iin, tperm_buf, nt, 0, 3 * kMaxLevel, st));
        tperm = tperm_buf;
    }
    k_gather_src<<<(ns + 255) / 256, 256, 0, st>>>(src_xyz, src_wf, sperm, ns, cube, xs, fsrc, yh, yl, yf);
    FS_LAUNCH_CHECK();

    // cells, level by level
    k_root<<<1, 1, 0, st>>>(C, ns, cube);
    FS_LAUNCH_CHECK();
    FS_CUDA(cudaMemsetAsync(pcell, 0, size_t(ns) * sizeof(int), st));
    int ncells = 1;
    std::vector<int> level_first(kMaxLevel + 2, 0), level_count(kMaxLevel + 2, 0);
    level_count[0] = 1;
    for (int lv = 1; lv <= kMaxLevel; ++lv) {
        k_flag<<<(ns + 255) / 256, 256, 0, st>>>(C, kout, pcell, ns, lv, flag);
        FS_LAUNCH_CHECK();
        size_t sb = scan_tmp;
        FS_CUDA(cub::DeviceScan::ExclusiveSum(tmp, sb, flag, pos, ns, st));
        k_total<<<1, 1, 0, st>>>(flag, pos, ns, d_total);
        FS_LAUNCH_CHECK();
        int total = 0;
        FS_CUDA(cudaMemcpyAsync(&total, d_total, sizeof(int), cudaMemcpyDeviceToHost, st));
        FS_CUDA(cudaStreamSynchronize(st));
        if (total == 0) break;
        if (ncells + total > cap) {
            set_error("fs_stokeslet_apply_tree: cell capacity exceeded");
            return FS_ENOMEM;
        }
        k_children<<<(ns + 255) / 256, 256, 0, st>>>(C, kout, pcell, flag, pos, ns, lv, ncells, cube);
        FS_LAUNCH_CHECK();
        k_child_links<<<(total + 255) / 256, 256, 0, st>>>(C, ncells, total);
        FS_LAUNCH_CHECK();
        level_first[lv] = ncells;
        level_count[lv] = total;
        ncells += total;
    }
    // leaves and split cells per level (host lists)
    std::vector<int> cbh(ncells), lvh(ncells);
    FS_CUDA(cudaMemcpyAsync(cbh.data(), C.cb, ncells * sizeof(int), cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaMemcpyAsync(lvh.data(), C.lvl, ncells * sizeof(int), cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaStreamSynchronize(st));
    std::vector<int> leaves;
    std::vector<std::vector<int>> split(kMaxLevel + 1);
    for (int k = 0; k < ncells; ++k) {
        if (cbh[k] < 0) leaves.push_back(k);
        else split[lvh[k]].push_back(k);
    }
    // per-cell tables, sized by the cells the tree has (the bound cap is far
    // larger: a split cell holds more than kLeafCap points), in the
    // context's second workspace
    size_t need2 = 0;
    auto acct2 = [&](size_t bytes) { need2 += (bytes + 255) & ~size_t(255); };
    acct2(size_t(ncells) * 4 * T * d);                      // FP64 moments
    acct2(size_t(ncells) * nfold(order) * 16);              // folded FP32 tables
    acct2(size_t(ncells) * 48);                             // evaluation records
    need2 += 4 * 256;
    FS_TRY(c->tree_scratch.reserve(need2, st));
    Carve cv2(c->tree_scratch.ptr, c->tree_scratch.bytes);
    double *Md = cv2.take<double>(size_t(ncells) * 4 * T);
    float4 *Mf = cv2.take<float4>(size_t(ncells) * nfold(order));
    float4 *pch = cv2.take<float4>(ncells), *pcl = cv2.take<float4>(ncells);
    int4 *pci = cv2.take<int4>(ncells);
    if (cv2.used > cv2.cap) {
        set_error("fs_stokeslet_apply_tree: workspace accounting");
        return FS_EINVAL;
    }
    k_groups<<<(nt + 127) / 128, 128, 0, st>>>(tgt_xyz, tperm, nt, cube, gctr, xh, xl);
    FS_LAUNCH_CHECK();

    EvalArgs A;
    A.ch = pch;
    A.cl = pcl;
    A.ci = pci;
    A.Mf = Mf;
    A.yh = yh;
    A.yl = yl;
    A.yf = yf;
    A.xh = xh;
    A.xl = xl;
    A.gctr = gctr;
    A.tperm = tperm;
    A.n_tgt = nt;
    A.ngroups = ngroups;
    A.theta = static_cast<float>(theta);
    A.scale = 1.0 / (8.0 * M_PI * c->mu);
    A.out = out_u;
    A.status = tstat;
    switch (order) {
    case 4: FS_TRY(launch_eval_and_moments<4>(C, leaves, split, ncells, d_list, xs, fsrc, Md, Mf, cube, pch, pcl, pci, A, st)); break;
    case 6: FS_TRY(launch_eval_and_moments<6>(C, leaves, split, ncells, d_list, xs, fsrc, Md, Mf, cube, pch, pcl, pci, A, st)); break;
    case 8: FS_TRY(launch_eval_and_moments<8>(C, leaves, split, ncells, d_list, xs, fsrc, Md, Mf, cube, pch, pcl, pci, A, st)); break;
    default: FS_TRY(launch_eval_and_moments<10>(C, leaves, split, ncells, d_list, xs, fsrc, Md, Mf, cube, pch, pcl, pci, A, st)); break;
    }
    if (ids) {
        if (excl_given) excl = const_cast<int2 *>(excl_given);
        else FS_TRY(exclusion_from_ids(src_fiber, n_src, tgt_fiber, n_tgt, excl, st));
        // the pair records of the near field, in the sources' original order
        k_unsort_src<<<(ns + 255) / 256, 256, 0, st>>>(sperm, ns, yh, yl, yf, oh, ol, of);
        FS_LAUNCH_CHECK();
        k_sub_own<<<(nt + 127) / 128, 128, 0, st>>>(oh, ol, of, tgt_xyz, excl, nt, cube, A.scale, out_u);
        FS_LAUNCH_CHECK();
    }
    int h_status = 0;
    FS_CUDA(cudaMemcpyAsync(&h_status, tstat, sizeof(int), cudaMemcpyDeviceToHost, st));
    FS_CUDA(cudaStreamSynchronize(st));
    if (h_status) {
        set_error("fs_stokeslet_apply_tree: traversal stack overflow");
        return FS_ENUMERIC;
    }
    return FS_OK;
}

}  // namespace fs

using namespace fs;

extern "C" {

fs_status fs_stokeslet_apply_tree(fs_ctx *c, const double *src_xyz, const double *src_wf, int64_t n_src,
                                  const int32_t *src_fiber, const double *tgt_xyz, const int32_t *tgt_fiber,
                                  int64_t n_tgt, double *out_u, int32_t order, double theta)
{
    return tree_sum(c, src_xyz, src_wf, n_src, src_fiber, tgt_xyz, tgt_fiber, n_tgt, out_u, order, theta, nullptr);
}

}  // extern "C"
