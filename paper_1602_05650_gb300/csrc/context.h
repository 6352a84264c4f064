// The fs_ctx object and the internal interfaces of the implicit step.
#pragma once

#include <map>

#include <cuda_bf16.h>

#include "internal.h"

namespace fs {

// Offsets (in doubles) of the per-N operator matrices inside one op set; all
// matrices row-major.  Built on the host in long double by chebops.cu and
// rounded to double (geometry matrices kept as double-double pairs).
struct OpsLayout {
    int N;
    int64_t alpha, omega, Vy, V2, V3, Sig, Tn, Vn, D1, D2, D3, D4, Py, Dz, total;
    // geometry matrices as double-double (hi, lo) pairs: first derivative at
    // the nodes (G1) and at the tension points (Gz), 2nd / 3rd derivative at
    // alpha = +1, -1 (G2, G3), 4th derivative at the nodes (G4)
    int64_t G1h, G1l, Gzh, Gzl, G2h, G2l, G3h, G3l, G4h, G4l;
    int64_t Vgy;   // (y_i + 1) x alpha-derivative of the velocity basis at y_i (growth)
    int64_t V1;    // alpha-derivative of the velocity basis at alpha = +1, -1 (clamped end)
    __host__ __device__ explicit OpsLayout(int n) : N(n)
    {
        int64_t o = 0;
        alpha = o; o += N;
        omega = o; o += N;
        Vy = o; o += int64_t(N - 4) * N;
        V2 = o; o += 2 * N;
        V3 = o; o += 2 * N;
        Sig = o; o += int64_t(N) * N;
        Tn = o; o += int64_t(N) * N;
        Vn = o; o += int64_t(N) * N;
        D1 = o; o += int64_t(N) * N;
        D2 = o; o += int64_t(N) * N;
        D3 = o; o += int64_t(N) * N;
        D4 = o; o += int64_t(N) * N;
        Py = o; o += int64_t(N - 4) * N;
        Dz = o; o += int64_t(N - 2) * N;
        G1h = o; o += int64_t(N) * N;
        G1l = o; o += int64_t(N) * N;
        Gzh = o; o += int64_t(N - 2) * N;
        Gzl = o; o += int64_t(N - 2) * N;
        G2h = o; o += 2 * N;
        G2l = o; o += 2 * N;
        G3h = o; o += 2 * N;
        G3l = o; o += 2 * N;
        G4h = o; o += int64_t(N) * N;
        G4l = o; o += int64_t(N) * N;
        Vgy = o; o += int64_t(N - 4) * N;
        V1 = o; o += 2 * N;
        total = (o + 3) & ~int64_t(3);
    }
};

// Digit-plane sizes of the tensor-core block build for fibers of at most N
// points: left operands S (3N rows) and Rw (three components' N - 4 velocity
// rows and N - 2 tension rows, each group padded to 64), right operands F and
// W (4N columns), inner dimension 3N; rows padded to 64, k to 16.
struct OzDims {
    int r1, r2, ry, kp;
    __host__ __device__ explicit OzDims(int N)
        : r1((3 * N + 63) / 64 * 64), r2(3 * ((N - 4 + 63) / 64 * 64) + (N - 2 + 63) / 64 * 64),
          ry((4 * N + 63) / 64 * 64),
          kp((3 * N + 15) / 16 * 16)
    {
    }
    static constexpr int digits = 9;
    // bytes per fiber: the bf16 digit planes and the exponents of both operands
    __host__ __device__ int64_t bytes_per_fiber() const
    {
        const int64_t rx = r1 > r2 ? r1 : r2;
        return (digits * (rx + ry) * int64_t(kp)) * 2 + (rx + ry) * 4 + 512;
    }
};

// Digit planes of the LU's tensor-core trailing updates for fibers of at most
// N points: per fiber and operand, nine planes of rows (4 N padded to 64) x 32
// bf16 and one exponent per row; the LU runs on the tensor cores while one
// CTA holds a fiber's panel rows one per thread (4 N <= 512).
struct LuTcDims {
    int rows, kp = 32;
    __host__ __device__ explicit LuTcDims(int N) : rows((4 * N + 63) / 64 * 64) {}
    __host__ __device__ static bool fits(int N) { return 4 * N <= 512; }
    __host__ __device__ int64_t plane_elems() const { return int64_t(9) * rows * kp; }
};

struct OzPlan {
    int oz_chunk = 0, lu_chunk = 0;
    int64_t x = 0, y = 0, xe = 0, ye = 0;
};
OzPlan oz_plan(int M, int maxN, const fs_options &o);

// Host construction of one op set (FP64): returns `total` doubles.
std::vector<double> build_ops(int N);

// Device pointers describing all fibers (passed by value to kernels).
struct FiberTable {
    int M;
    const int *N;              // [M] points per fiber
    const int64_t *node_ptr;   // [M+1]
    const int64_t *unk_ptr;    // [M+1] fiber unknown offsets (4N each)
    const int64_t *blk_ptr;    // [M+1] offsets of the (4N)^2 blocks
    const int64_t *kp_ptr;     // [M+1] offsets of the N^2 self-pair records
    const int64_t *z_ptr;      // [M+1] offsets of the N-2 tension points
    const int64_t *ops_off;    // [M]   op-set offset of each fiber
    const double *ops;         // op sets
    const double *L;           // [M]
    double mu, eps, E, dt, delta_over_L;
    int lsb;
    // geometry, written by k_geometry each step
    double *t;       // [N_tot][3] X_s at nodes
    double *tz;      // [sum(N-2)][3] X_s at the tension points
    double *fknown;  // [N_tot][3] f^E - E g^4 X_aaaa
    double *W;       // [N_tot] Clenshaw-Curtis source weights
    double *mloc;    // [N_tot][2] local operator coefficients (see k_geometry)
    double *bc;      // [M][12] free-end data X''(+-1)/dt, X'''(+-1)/dt
    double *kp;      // [sum N^2][4] K_delta pair records (a_kj, rhat)
    // block-build scratch (offsets from blk_ptr: 16 N^2 per fiber)
    double *ftau;    // [3 N^2] per fiber: force of each tension column, [a][l][j]
    double *wsc;     // [12 N^2] per fiber: w = (M + K_delta) f of each column, [col][b N + k]
    const double *Ldot;  // [M] plus-end growth rates (nullptr: fixed lengths)
    int growth_implicit; // 0: growth term at the current time (Eq. discrete-rhs); 1: at the new time
    const int *attach;   // [M] minus-end condition FS_END_* (nullptr: all free)
};

// Surface nodes of the periphery (first n_per) and of the rigid body (the
// next n - n_per), one source set for the double-layer sums.
struct Surface {
    int n = 0;
    int n_per = 0;
    double *y = nullptr, *nrm = nullptr, *w = nullptr;  // [n][3], [n][3], [n]
    double *diag = nullptr;                             // [n][3] Jacobi entries
    double *A = nullptr;                                // [n][9] subtraction matrices
    double *tmp = nullptr;                              // [n][3] work
    double *flux = nullptr;                             // [1] sum w n.q
    int2 *excl = nullptr;                               // [n] own-node exclusion
};

// The rigid body (Sec. 2.2): device record rb[kRb*] and the attached fibers.
enum : int {
    kRbCenter = 0,   // [3] X^P
    kRbF = 3,        // [3] Stokeslet strength F of the current evaluation
    kRbL = 6,        // [3] rotlet strength L
    kRbFext = 9,     // [3] external force
    kRbLext = 12,    // [3] external torque
    kRbArea = 15,    // surface area (sum of the weights)
    kRbU = 16,       // [3] U of the last step
    kRbOm = 19,      // [3] Omega of the last step
    kRbSize = 24
};

// An instantiated GMRES cycle graph (opt.use_graph) and its launch shape.
struct CycleGraph {
    int prec = 0;
    bool hilo = false;
    int nch = 0, nsch = 0, max_iter = 0;
    int64_t items = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t body_launches = 0;   // kernels of one loop iteration
};

struct Body {
    bool on = false;
    int n = 0;                    // surface nodes (inside Surface, after the periphery)
    double radius = 0.0;
    double *rb = nullptr;         // [kRbSize]
    int *attach = nullptr;        // [M] FS_END_*
    int *att_list = nullptr;      // [n_att] attached fiber indices
    int n_att = 0;
};

}  // namespace fs

struct fs_ctx {
    cudaStream_t stream = nullptr;
    double mu = 1, eps = 1e-3, E = 1, dt = 1e-3;
    fs_options opt{};
    int M = 0;
    int64_t n_tot = 0, n_fib_unk = 0, n_unk = 0, n_blk = 0, n_kp = 0, n_z = 0;
    std::vector<int> Nm;
    std::vector<int64_t> node_ptr, unk_ptr, blk_ptr;
    std::map<int, int64_t> ops_offset;  // N -> offset in d_ops
    int max_N = 0;
    // independent systems (fs_create_batch): consecutive fiber ranges
    int S = 1;
    std::vector<int> sys_fib_ptr;
    std::vector<int64_t> sys_node_ptr, sys_unk_ptr;
    std::vector<double> sys_self_pairs;
    std::vector<int> all_sys;
    std::vector<int> sys_iters, sys_outer, sys_conv;
    std::vector<double> sys_resid;
    int64_t chunk_cap = 0, work_cap = 0;
    int4 *d_work = nullptr;
    int4 *d_ich = nullptr, *d_isch = nullptr, *d_och = nullptr, *d_osch = nullptr;
    int *d_ikk = nullptr, *d_okk = nullptr;

    // device
    int *d_status = nullptr;
    int *d_N = nullptr;
    int64_t *d_node_ptr = nullptr, *d_unk_ptr = nullptr, *d_blk_ptr = nullptr, *d_kp_ptr = nullptr,
            *d_z_ptr = nullptr, *d_ops_off = nullptr;
    double *d_ops = nullptr;
    int2 *d_excl = nullptr;       // per node: its own fiber's node range
    double *d_X = nullptr, *d_L = nullptr, *d_fext = nullptr;
    double *d_t = nullptr, *d_tz = nullptr, *d_fknown = nullptr, *d_W = nullptr, *d_mloc = nullptr,
           *d_bc = nullptr, *d_kp = nullptr;
    double *d_B = nullptr;        // column-major blocks, LU factors after build
    double *d_Ldot = nullptr;     // [M] plus-end growth rates (fs_set_growth)
    bool growth = false;          // some rate is non-zero
    double *d_ftau = nullptr;     // block-build scratch: tension-column forces (3 N^2 per fiber)
    double *d_wsc = nullptr;      // block-build scratch: w of every column (12 N^2 per fiber)
    int *d_piv = nullptr;
    double *d_dinv = nullptr;     // 1 / U_ii of the block LU factors
    double *d_V = nullptr, *d_T = nullptr;
    double *d_f = nullptr, *d_wf = nullptr, *d_ubar = nullptr;
    // Krylov workspace
    int kdim = 0;
    double *d_basis = nullptr, *d_b = nullptr, *d_x = nullptr, *d_r = nullptr, *d_w = nullptr,
           *d_e = nullptr, *d_pb = nullptr, *d_h = nullptr,
           *d_part = nullptr;
    double *h_pinned = nullptr;
    // outer (flexible) Krylov space of the mixed-precision solve
    int okdim = 0;
    double *d_obasis = nullptr, *d_oz = nullptr, *d_oh = nullptr, *d_opart = nullptr, *d_ow = nullptr,
           *d_or = nullptr, *oh_pinned = nullptr;
    fs::Surface surf;
    fs::Body body;
    int64_t n_surf_unk = 0;       // 3 x surface nodes (+ 6 rigid-body unknowns)
    double *d_usurf = nullptr;    // fiber Stokeslets at the surface nodes [n_s][3]
    bool have_state = false, precond_ok = false, geometry_ok = false;
    fs::Scratch scratch;          // far-field scratch (grown on demand)
    fs::Scratch tree_scratch;     // treecode per-cell tables (grown on demand)
    fs::Profiler prof;            // CUDA-event records (opt.profile)
    int64_t pairs_last = 0;
    size_t dev_bytes = 0;         // device memory allocated by the context (without scratch)
    // GMRES cycles as CUDA graphs (opt.use_graph): device Givens state of the
    // inner Krylov space ([S][R][R+1], [S][R] x 2, [S][R+1], [S][4] x 2),
    // the iteration index, per-system start values, the current basis vector,
    // host mirrors, and the instantiated graphs
    double *d_gH = nullptr, *d_gcs = nullptr, *d_gsn = nullptr, *d_gg = nullptr, *d_gsc = nullptr,
           *d_ginit = nullptr, *d_vcur = nullptr;
    int *d_gst = nullptr, *d_gj = nullptr;
    double *h_ginit = nullptr, *h_gsc = nullptr;
    int *h_gst = nullptr, *h_gj = nullptr;
    double *h_gbuf = nullptr;     // pinned block behind the host mirrors
    bool capturing = false;       // kernels are being captured into a graph
    // autotuned far-field shapes, [2 sum precision + hi/lo] (0: not tuned)
    int tuned[8] = {};
    cudaStream_t cap_stream = nullptr;   // the stream graphs are captured on
    std::vector<fs::CycleGraph> graphs;
    // tensor-core block build (opt.tc_blocks): digit planes of a chunk of
    // oz_chunk fibers (0: the FP64 CUDA-core build)
    int oz_chunk = 0;
    // fibers per chunk of the LU with tensor-core trailing updates (0: k_lu);
    // its digit planes live in d_ozx / d_ozy, its exponents in d_ozxe / d_ozye
    int lu_chunk = 0;
    __nv_bfloat16 *d_ozx = nullptr, *d_ozy = nullptr;
    int *d_ozxe = nullptr, *d_ozye = nullptr;
    fs::Pool *pool = nullptr;     // preallocated region for every buffer (serving), or nullptr
    bool worklist = false;        // far fields always per system (work-list mode), also for one system
    bool partial_ok = false;      // batch step: update every system, report convergence per system

    fs::FiberTable table() const;
};

namespace fs {
fs_status context_init(fs_ctx *c, int S, const int32_t *fibers_per_system, int M, const int32_t *ppf,
                       const fs_boundary *b, const fs_body *body = nullptr, const int32_t *minus_end = nullptr);
void context_free(fs_ctx *c);
// A context for a serving batch: n_systems independent systems (or one with a
// boundary), every buffer carved from `pool`, far fields per system even for
// one system (a request's arithmetic does not depend on the batch it runs
// in), and a step that updates every system whatever the others do.
fs_status create_serving(fs_ctx **out, int32_t n_systems, const int32_t *fps, int32_t n_fibers, const int32_t *ppf,
                         double mu, double eps, double E, double dt, const fs_boundary *boundary,
                         const fs_options *opt, void *cuda_stream, Pool *pool);
size_t estimate_bytes(int M, const int32_t *ppf, int n_surf, const fs_options &opt);
// FS_EINVAL (with the message prefixed by `who`) unless every field of the
// options is in its documented range
fs_status check_options(const fs_options &o, const char *who, int n_systems);

// fiber.cu
fs_status launch_geometry(fs_ctx *c);
// f (and W f) at the nodes from the unknowns u (or f_known when u == nullptr)
fs_status launch_force(fs_ctx *c, const double *u, double *f, double *wf, bool add_known = false);
// rows of the fiber equations; mode 0: out = B u + Rw(ubar); 1: right-hand side
// b = -(rows of the known force and free-end data + Rw(ubar)); 2: out = Rw(ubar)
enum : int { ROWS_FULL = 0, ROWS_RHS = 1, ROWS_COUPLING = 2 };
fs_status launch_rows(fs_ctx *c, const double *u, const double *f, const double *ubar, double *out,
                      int mode);
fs_status launch_block_build(fs_ctx *c);
fs_status launch_lu_factor(fs_ctx *c);
fs_status launch_lu_solve(fs_ctx *c, const double *in, double *out);
fs_status launch_update(fs_ctx *c, const double *u);

// surface.cu
fs_status surface_couplings(fs_ctx *c, const double *q, double *ubar_fibers, int sum_prec,
                            bool hilo);
fs_status surface_rows(fs_ctx *c, const double *q, const double *usurf, double *out, bool rhs,
                       int sum_prec, bool hilo);
fs_status surface_diag(fs_ctx *c);
fs_status surface_precond(fs_ctx *c, const double *in, double *out);

// tree.cu: the treecode sum (fs_stokeslet_apply_tree), exclusion from ids or
// from per-target source ranges excl_given
fs_status tree_sum(fs_ctx *c, const double *src_xyz, const double *src_wf, int64_t n_src, const int32_t *src_fiber,
                   const double *tgt_xyz, const int32_t *tgt_fiber, int64_t n_tgt, double *out_u, int32_t order,
                   double theta, const int2 *excl_given);

// body.cu
// Stokeslet and rotlet strengths of the body from the attached ends: mode
// LOAD_KNOWN (external load + ends' known part), LOAD_LIN (part linear in the
// unknowns u), LOAD_BOTH (their sum).
enum : int { LOAD_KNOWN = 0, LOAD_LIN = 1, LOAD_BOTH = 2 };
fs_status body_load(fs_ctx *c, const double *u, int mode);
// out[i] += G(x_i - X^P) F + R(x_i - X^P) L at n points
fs_status body_point_flow(fs_ctx *c, const double *x, int64_t n, double *out);
// fiber rows += sign x (terms of the attached-end rows in U, Omega of v)
fs_status body_rigid_rows(fs_ctx *c, const double *v, double *rows, double sign);
// out[0..6) = constraint rows: mean of w q1 - U, mean of w (y - X^P) x q1 - Omega
fs_status body_constraints(fs_ctx *c, const double *q1, const double *rigid, double *out);
// X^P, body nodes += dt U; record U, Omega
fs_status body_update(fs_ctx *c, const double *rigid);
}  // namespace fs
