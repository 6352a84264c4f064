/*
 * fibersolve: the implicit time step of nonlocal slender-body fibers in Stokes
 * flow (Nazockdast, Rahimian, Zorin, Shelley, "A fast platform for simulating
 * flexible fiber suspensions applied to cell mechanics"), as a C-ABI library
 * running on one sm_103a GPU.
 *
 * Conventions for every entry point:
 *  - Return value is an fs_status; on failure fs_last_error() returns a
 *    thread-local message describing the first error of the failing call.
 *  - Arrays are plain C arrays of double (or int32) in the layout stated at
 *    each argument.  "device" pointers are CUDA device addresses (e.g. a torch
 *    tensor's data_ptr()) that are only borrowed for the duration of the call
 *    (the work they feed is enqueued on the context's stream, so the caller
 *    must keep them alive until that stream reaches the enqueued work);
 *    "host" pointers are copied before the call returns unless stated.
 *  - All GPU work of a context runs in the CUDA stream given to fs_create
 *    (NULL = the legacy default stream).  Calls that return results to host
 *    memory synchronise that stream.
 *  - No call throws; no call falls back to the CPU.  A missing GPU or a CUDA
 *    error returns FS_ECUDA.
 *  - A context is not thread-safe: serialise calls on one context.
 */
#ifndef FIBERSOLVE_H
#define FIBERSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FS_OK = 0,
    FS_EINVAL = 1,     /* invalid argument or state */
    FS_ENOMEM = 2,     /* device allocation failed or exceeds the memory budget */
    FS_ECUDA = 3,      /* CUDA runtime / launch error */
    FS_ENOTCONV = 4,   /* GMRES / refinement did not reach the tolerance */
    FS_ENUMERIC = 5,   /* NaN / Inf found in inputs or results, or a singular block */
    FS_EAGAIN = 6,     /* serving: result not ready yet */
    FS_EBUSY = 7,      /* serving: no free slot / memory */
    FS_ETIMEOUT = 8    /* a bounded device-side wait gave up */
} fs_status;

typedef enum {
    FS_FP64 = 0,   /* everything in FP64 (the plain FP64 GPU path) */
    FS_MIXED = 1   /* GMRES-based refinement: flexible GMRES on the operator whose far
                      field is float-float (FP64-grade, on the FP32 pipe), each
                      direction preconditioned by a GMRES solve with the FP32 far
                      field; FP64 everywhere else; same stopping test as FS_FP64 */
} fs_precision;

typedef enum {
    FS_SUM_FP64 = 0, /* direct sums in FP64 arithmetic */
    FS_SUM_FP32 = 1, /* FP32 arithmetic: hi/lo-split coordinates, FP32 tile sums,
                        compensated (TwoSum) accumulation across tiles, FP64 output */
    FS_SUM_FF = 2,   /* float-float ("double-single") arithmetic on the FP32 pipe,
                        ~2^-44 relative rounding per pair */
    FS_SUM_FP32_PLAIN = 3 /* Stokeslet: FP32 in packed two-target instructions,
                        each thread's consecutive targets in a frame at its middle
                        target (sources moved into it from their hi/lo parts): on
                        fiber nodes the pair differences round relative to the
                        fiber's extent (hi/lo accuracy) at ~20% less cost; targets
                        that are not spatially grouped round like coordinates
                        centred on the sources' bounding box (2^-24 of its extent);
                        Stokeslet sums only */
} fs_sum_precision;

/* Spherical no-slip periphery (Sec. 2.1, Eq. main-cortex-density) discretised
 * by Gauss-Legendre patch quadrature (Sec. 3.1.1, Eq. patch-gl-quad): node
 * positions, outward unit normals and quadrature weights (GL weight x surface
 * Jacobian), all host arrays, copied at fs_create.  NULL = free space. */
typedef struct {
    double R;
    int32_t n_nodes;
    const double *nodes;    /* [n_nodes][3] */
    const double *normals;  /* [n_nodes][3] */
    const double *weights;  /* [n_nodes]    */
} fs_boundary;

/* A rigid sphere immersed in the suspension (Sec. 2.2, Eqs.
 * main-nsb-second-kind, main-nsb-rgbt, main-nsb-rgbr): the fluid outside it
 * sees its completed double layer T[q1] + G(x - center) F + R(x - center) L,
 * its surface moves rigidly with the unknown velocities U, Omega, and F, L are
 * the external force and torque below plus those of the attached fibers
 * (Eqs. f-ext, t-ext).  Surface quadrature as for fs_boundary: node positions
 * (absolute), outward unit normals, weights; host arrays, copied at creation. */
typedef struct {
    double center[3];
    double radius;
    int32_t n_nodes;
    const double *nodes;    /* [n_nodes][3] */
    const double *normals;  /* [n_nodes][3] */
    const double *weights;  /* [n_nodes]    */
    double force[3];        /* external force on the body */
    double torque[3];       /* external torque on the body, about center */
} fs_body;

/* Minus-end (s = 0, alpha = -1) condition of a fiber (Sec. 2.3): free
 * (Eq. bc-free), clamped to the body (Eqs. BC2-1, BC2-2, BC2-T: the end moves
 * with the body and its tangent turns with it) or hinged (Eqs. BC2-1, BC2-T
 * and X_ss = 0: the end moves with the body, no torque at the hinge). */
enum { FS_END_FREE = 0, FS_END_CLAMPED = 1, FS_END_HINGED = 2 };

typedef struct {
    int32_t prec;           /* fs_precision (default FS_MIXED) */
    double tol;             /* preconditioned relative residual target (default 1e-8):
                               ||P^-1 (b - A u)|| <= tol ||P^-1 b|| */
    int32_t max_iter;       /* GMRES iterations per solve (default 200) */
    int32_t restart;        /* GMRES restart length (default 60; 1..250, 1 acts as 2) */
    int32_t max_refine;     /* FS_MIXED, free space, relax = 1: at most this many float-float
                               true residuals per step (default 6; normally one is used) */
    double inner_tol;       /* FS_MIXED: relative tolerance of the FP32-far-field GMRES
                               solves (the first stage of the free-space step, the inner
                               solves of the flexible GMRES) (default 1e-6) */
    double delta_over_L;    /* regularisation delta of K_delta as a fraction of L (default 0.01) */
    int32_t lsb;            /* 1 = local slender-body theory: drop K_delta (default 0) */
    int32_t use_graph;      /* 1 = every restart cycle of the (inner) GMRES runs as ONE CUDA
                               graph launch: a conditional WHILE node whose body is one
                               iteration (operator, CGS2, norm, the Givens rotations of every
                               system on the device, which also set the loop condition), so
                               the host synchronises once per cycle instead of once per
                               iteration; graphs are instantiated once per launch shape and
                               reused.  Applies with the direct far field and profile = 0;
                               the flexible outer GMRES (relax = 0) keeps the host path.
                               Same arithmetic as 0 (default 0) */
    int32_t tile_override;  /* direct-sum launch shape: 0 = the shape measured fastest on
                               GB300 for each precision (targets per thread: FP32 8,
                               float-float 4, FP64 2; grid from the occupancy
                               calculator); 1, 2, 3 = 2, 4, 8 targets per thread in FP32
                               and 1, 2, 4 in float-float and FP64 (default 0) */
    int32_t profile;        /* 1 = bracket every direct-sum kernel with CUDA events on the
                               context's stream (read with fs_kernel_stats) (default 0) */
    int32_t relax;          /* FS_MIXED: 1 = evaluate the far fields in float-float only
                               where the residual needs it (default 1): GMRES on the
                               FP32-far-field operator with an FP32 right-hand side to
                               inner_tol, ONE float-float true residual r (one set of far
                               fields of the known force plus the solution's force and of
                               the periphery density), then GMRES on the plain FP32 operator
                               for the correction until |r - P^-1 A d| <= tol |P^-1 b| (its
                               operator error, relative ~3e-6 and at most 1e-4, acts on a
                               correction of size |r|); a residual with 1e-4 |r| > tol
                               |P^-1 b| / 20 is only reduced 1e3-fold before the next true
                               residual.
                               0 = flexible GMRES with every outer direction in float-float,
                               each preconditioned by an FP32-far-field GMRES solve */
    int32_t tree_order;     /* 0 = direct far field (default); 4, 6, 8 or 10 = every
                               fiber-fiber far field of the step (every precision) is the
                               treecode of fs_stokeslet_apply_tree at this order: the
                               operator is then the treecode's, and tol applies to it (as
                               with the paper's fast summation); single-system contexts */
    double tree_theta;      /* opening angle of the treecode (default 0.5) */
    int32_t growth_implicit;/* growing or shrinking fibers (fs_set_growth): 0 = the
                               reparametrisation term (alpha + 1)(Ldot / L) X_alpha at the
                               current time, on the right-hand side (Sec. 3.2, Eq.
                               discrete-rhs) (default); 1 = the same term at the new time,
                               (alpha + 1) kappa X+_alpha with kappa = Ldot / (L + dt Ldot):
                               its dt V_alpha part enters the self block.  The explicit
                               term is forward Euler on an advection in alpha and goes
                               unstable for fast-shrinking fibers (dt |Ldot| / L of a few
                               percent); the implicit one stays stable there */
    int32_t tc_blocks;      /* 1 = the two large products of the self-block build (W = S F
                               and the w rows Rw W, Eq. prec) on the bf16 tensor cores by
                               operand splitting: each row / column scaled by a power of
                               two and rounded to a 62-bit integer split into nine 7-bit
                               digits, the digit products summed exactly in FP32 per
                               diagonal, the diagonals summed as integers and rounded once
                               to FP64, an FP64-grade result (error below the FP64
                               product's bound); 0 = FP64 CUDA cores (default 1) */
    int32_t tc_lu;          /* 1 = the block LU's trailing updates A22 -= L21 U12 (panels
                               of 32 columns) on the bf16 tensor cores by the same split,
                               the panels (pivoting) on the FP64 pipe; used while one CTA
                               holds a fiber's panel rows one per thread (4N <= 512, i.e.
                               N <= 128), else the FP64 LU; 0 = FP64 LU (default 1) */
    int32_t autotune;       /* 1 = the fiber far field's launch shape (targets per thread,
                               tile_override's ids 1..3) chosen per precision class by
                               timing: the first sum of each class (outside a graph
                               capture) runs every shape once untimed and once timed on
                               the context's stream and keeps the fastest for the
                               context's life (fs_get_tuned_shapes).  Results then depend
                               on that choice through the summation order, so contexts
                               tuned differently agree to the sums' accuracy, not bit for
                               bit; ignored when tile_override > 0; refused with
                               use_graph (a captured cycle keeps its capture's shapes).
                               0 = the measured default shapes (default 0) */
} fs_options;

/* Direct-sum kernel classes reported by fs_kernel_stats. */
typedef enum {
    FS_KS_STOKESLET_FP32 = 0,
    FS_KS_STOKESLET_FP64 = 1,
    FS_KS_STRESSLET_FP32 = 2,
    FS_KS_STRESSLET_FP64 = 3,
    FS_KS_STOKESLET_FF = 4,
    FS_KS_STOKESLET_FP32_PLAIN = 5,
    FS_KS_STRESSLET_FF = 6,
    FS_KS_COUNT = 8
} fs_kernel_class;

typedef struct {
    int64_t launches;   /* kernel launches recorded */
    double total_ms;    /* summed CUDA-event durations of those launches */
    double pairs;       /* pair interactions they evaluated */
} fs_kernel_stat;

typedef struct {
    int32_t iters;          /* GMRES iterations: FS_FP64 all; FS_MIXED the inner (FP32
                               far field) iterations summed over the outer steps */
    int32_t refine_sweeps;  /* FS_MIXED: outer (flexible GMRES) steps, each applying the
                               accurate operator once; FS_FP64: 1 */
    double resid;           /* final preconditioned relative residual estimate of the
                               (outer) GMRES recurrence, accurate operator */
    double t_ms[8];         /* host wall-clock ms: [0] right-hand side [1] geometry and
                               preconditioner build [2] solve [3] update [4] total;
                               serving only: [5] queued [6] submit to done [7] requests
                               in the batch; (filled when info is requested) */
    int64_t pairs;          /* Stokeslet pairs evaluated */
} fs_step_info;

typedef struct fs_ctx fs_ctx;

/* Default options (values listed in fs_options). */
fs_status fs_options_default(fs_options *opt);

/* Create a context for n_fibers fibers with points_per_fiber[m] >= 6
 * Chebyshev points each (host array, copied), viscosity mu, slenderness eps,
 * bending modulus E and time step dt (Sec. 2.3-2.4, 3.2).  n_fibers = 0 gives a
 * context usable only for the direct-sum entry points.  cuda_stream is a
 * cudaStream_t or NULL.  Allocates the context's device memory.  opt NULL =
 * the defaults; FS_EINVAL (before any CUDA call) when a size or parameter is
 * out of range or a field of opt is outside its documented values (prec not
 * FS_FP64/FS_MIXED, tol or inner_tol outside (0, 1), max_iter or max_refine
 * < 1, restart outside 1..250, delta_over_L negative, lsb/relax/profile not
 * 0 or 1, use_graph not 0 or 1, tile_override outside 0..3, bad tree options). */
fs_status fs_create(fs_ctx **out, int32_t n_fibers, const int32_t *points_per_fiber,
                    double mu, double eps, double E, double dt,
                    const fs_boundary *boundary, const fs_options *opt, void *cuda_stream);

/* fs_create with a rigid body (body != NULL) and per-fiber minus-end
 * conditions minus_end[n_fibers] (FS_END_*; host array, copied; NULL = all
 * free).  Fibers clamped or hinged to the body should start with their last
 * node (alpha = -1) on its surface.  The unknown vector (fs_get_unknowns)
 * then ends with the body's density [n_nodes][3], U [3] and Omega [3], after
 * the periphery density.  Every fs_step moves the body's center and nodes by
 * dt U.  Errors: FS_EINVAL for an incomplete body, a non-positive radius, an
 * unknown end code, or an attached end without a body. */
fs_status fs_create_with_body(fs_ctx **out, int32_t n_fibers, const int32_t *points_per_fiber,
                              const int32_t *minus_end, double mu, double eps, double E, double dt,
                              const fs_boundary *boundary, const fs_body *body, const fs_options *opt,
                              void *cuda_stream);

/* The body's current center, and U, Omega of the last step (host arrays of
 * 3, any may be NULL).  Synchronises the context's stream.  FS_EINVAL
 * without a body. */
fs_status fs_get_body(fs_ctx *ctx, double *center, double *U, double *Omega);

/* Replace the external force and torque on the body (host arrays of 3). */
fs_status fs_set_body_load(fs_ctx *ctx, const double *force, const double *torque);

/* A context holding n_systems independent free-space suspensions (fibers
 * 0..fibers_per_system[0]-1 form system 0, and so on; points_per_fiber lists all
 * fibers, system-major), sharing mu, eps, E and dt.  Every kernel launch of a
 * step covers all systems (the far field of a target block sums only its own
 * system's sources); GMRES runs per system (own Krylov space, own convergence)
 * in lockstep.  State arrays of fs_set_state / fs_get_state cover all fibers.
 * fs_step fails with FS_ENOTCONV (no update) if any system does not converge. */
fs_status fs_create_batch(fs_ctx **out, int32_t n_systems, const int32_t *fibers_per_system,
                          const int32_t *points_per_fiber, double mu, double eps, double E, double dt,
                          const fs_options *opt, void *cuda_stream);

/* Per-system results of the last fs_step of a batch context (arrays of
 * n_systems, any may be NULL): GMRES iterations (inner iterations for
 * FS_MIXED), outer steps, final relative residual estimate, converged flag. */
fs_status fs_batch_info(const fs_ctx *ctx, int32_t *iters, int32_t *outer, double *resid,
                        int32_t *converged);

/* Synchronise the context's stream, then free everything the context holds
 * (device arrays, scratch, pinned host buffers).  NULL is a no-op; the caller's
 * stream itself is not destroyed. */
void fs_destroy(fs_ctx *ctx);

/* Set the fiber state: node positions X [N_tot][3] (fiber-major, node k of
 * fiber m is alpha_k = cos(k pi/(N_m-1)), k = 0 at alpha = +1), lengths
 * [n_fibers] and external force per unit length f_ext [N_tot][3] (NULL = 0).
 * ptr_is_device selects device or host pointers.  Invalidates the
 * preconditioner. */
fs_status fs_set_state(fs_ctx *ctx, const double *X, const double *lengths,
                       const double *f_ext, int32_t ptr_is_device);

/* Read the state after the last step: positions X [N_tot][3], tension T
 * [N_tot] and velocity V [N_tot][3] at the nodes (any may be NULL).
 * Synchronises the context's stream. */
fs_status fs_get_state(fs_ctx *ctx, double *X, double *T, double *V, int32_t ptr_is_device);

/* Direct Stokeslet sum (Eqs. oseen, single-layer; Eq. complementary-uf when
 * fiber ids are given):
 *   out_u[i] = sum_j G(tgt_i - src_j) src_wf[j],  G(r) = (I + rhat rhat)/(8 pi mu |r|)
 * over all j, skipping pairs with tgt_fiber[i] == src_fiber[j] when both id
 * arrays are non-NULL (then src_fiber must be non-decreasing, i.e. sources
 * grouped by fiber).  Without ids every pair counts and a target that
 * coincides with a source gives a non-finite result.
 * src_xyz [n_src][3], src_wf [n_src][3] (force times quadrature weight),
 * tgt_xyz [n_tgt][3], out_u [n_tgt][3]: DEVICE arrays of double; ids int32.
 * mu comes from the context.  Enqueued on the context's stream; uses the
 * context's scratch memory (grown on demand).  Returns without synchronising,
 * so a bounded device-side wait that gives up (not expected in normal
 * operation) shows in the result: every out_u entry is NaN, in this and
 * every later sum of the context, until the context's next fs_step returns
 * FS_ETIMEOUT and clears the flag. */
fs_status fs_stokeslet_apply(fs_ctx *ctx, const double *src_xyz, const double *src_wf,
                             int64_t n_src, const int32_t *src_fiber,
                             const double *tgt_xyz, const int32_t *tgt_fiber, int64_t n_tgt,
                             double *out_u, int32_t sum_precision);

/* Same sum as fs_stokeslet_apply, for callers that cannot let the library
 * allocate device memory: applications whose own allocator owns or has
 * reserved all of the GPU's memory (a cudaMalloc here could fail or fragment
 * their pool), and latency-bound loops that cannot absorb the device-wide
 * synchronisation of cudaMalloc / cudaFree.  (No counterpart in the paper: an
 * interface addition of this library.)
 *  - Needs no context: mu and the CUDA stream (cudaStream_t or NULL) are
 *    arguments; arrays as in fs_stokeslet_apply (DEVICE arrays, fiber ids
 *    optional and then non-decreasing over the sources).
 *  - Allocates nothing: its scratch is a fixed 32 MiB array in device memory
 *    that every GPU which loads this library holds until the process exits.
 *    A call needs the packed sources (32-64 bytes each), one partial sum per
 *    target per resident CTA wave ((SMs x resident CTAs + target blocks) x
 *    targets per block x 24 bytes) and, with ids, 8 bytes per target; on a
 *    152-SM GB300 that admits 65,536 sources and targets in every precision.
 *    Larger requests return FS_EINVAL with the size in fs_last_error().
 *  - The first call on a device looks up that array's device address (no
 *    allocation); make that first call before any stream capture.
 *  - All calls share the one array and it keeps the previous call's
 *    contents; calls that overlap on the GPU (different streams or threads
 *    without ordering between them) race on it and give wrong results.
 *  - Enqueued on `cuda_stream`; returns without synchronising.  A bounded
 *    device-side wait that gives up (not expected in normal operation) is
 *    reported only in the result: every out_u entry is NaN. */
fs_status fs_stokeslet_apply_noalloc(const double *src_xyz, const double *src_wf, int64_t n_src,
                                     const int32_t *src_fiber, const double *tgt_xyz,
                                     const int32_t *tgt_fiber, int64_t n_tgt, double *out_u,
                                     double mu, int32_t sum_precision, void *cuda_stream);

/* Fast summation of the sum of fs_stokeslet_apply (same arguments, same
 * exclusion of same-fiber pairs when both id arrays are given): a Cartesian
 * treecode (the paper evaluates this far field with a fast multipole method
 * for large systems, Sec. 3.3).  The Stokeslet is split into four Laplace
 * potentials; a source cell of radius rho (largest distance of its points
 * from its centre) is replaced by its Taylor expansion of the given order
 * (4, 6, 8 or 10) for a group of 32 targets whose box lies farther than
 * rho / theta from the centre (theta in (0, 1)), nearer cells are opened and
 * leaves summed directly.  FP32 arithmetic (hi/lo coordinates in the direct
 * part), FP64 moments and totals; the error falls with order and theta (see
 * the tests).  Pairs at zero distance (a point with itself) are skipped.
 * Uses the context's scratch (grown as needed); synchronises
 * the context's stream.  FS_EINVAL for a bad order or theta, FS_ENUMERIC if
 * a traversal exceeded its stack (the output is then incomplete). */
fs_status fs_stokeslet_apply_tree(fs_ctx *ctx, const double *src_xyz, const double *src_wf, int64_t n_src,
                                  const int32_t *src_fiber, const double *tgt_xyz, const int32_t *tgt_fiber,
                                  int64_t n_tgt, double *out_u, int32_t order, double theta);

/* Direct double-layer (stresslet) sum (Eqs. stresslet, double-layer,
 * cortex-vel) at targets off the surface:
 *   out_u[i] = sum_j w_j T(tgt_i - y_j) : (q_j n_j),
 *   T_abc(r) = -(3/4 pi) rhat_a rhat_b rhat_c / |r|^2  (no 1/mu factor),
 * src_xyz, src_nrm (outward unit normals), src_q: [n_src][3]; src_w [n_src];
 * tgt_xyz, out_u [n_tgt][3]; all DEVICE arrays of double.  A target on a
 * source point gives a non-finite result.  Enqueued on the context's stream. */
fs_status fs_stresslet_apply(fs_ctx *ctx, const double *src_xyz, const double *src_nrm,
                             const double *src_w, const double *src_q, int64_t n_src,
                             const double *tgt_xyz, int64_t n_tgt, double *out_u,
                             int32_t sum_precision);

/* Periphery operator of the context's boundary on a density q (Eq.
 * main-cortex-density, fluid-side limit, singularity subtraction of Sec.
 * 3.1.2, rank completion N):
 *   out_i = sum_{j != i} w_j T(y_i - y_j):((q_j - q_i) n_j) + q_i + n_i sum_j w_j n_j.q_j
 * q, out: DEVICE [n_nodes][3].  FS_EINVAL if the context has no boundary.
 * With a rigid body (fs_create_with_body) q and out span all surface
 * unknowns: the periphery's then the body's nodes [n][3], then U, Omega; body
 * nodes give the rows of Eq. main-nsb-second-kind without the fibers' flow,
 * followed by the six constraint rows (Eqs. main-nsb-rgbt, main-nsb-rgbr). */
fs_status fs_surface_apply(fs_ctx *ctx, const double *q, double *out, int32_t sum_precision);

/* Assemble the per-fiber self blocks (Eq. prec: fiber rows with the
 * complementary velocity removed, Sec. 3.3) for the current state and LU-factor
 * them with partial pivoting: FP64 panels, and the trailing updates on the
 * tensor cores by split operands (FP64-grade) with fs_options.tc_lu, else on
 * the FP64 pipe.  Called by fs_step when needed. */
fs_status fs_build_precond(fs_ctx *ctx);

/* The assembled self block B_m of one fiber (Eq. prec; before its LU
 * factorisation), column-major (4N)^2 doubles into the HOST array out, in the
 * unknown order of the fiber (sigma_x, sigma_y, sigma_z with their p columns,
 * then tau, q0, q1).  Assembles all blocks for the current state (so the next
 * fs_step factors them again) and synchronises the stream.  For tests and
 * diagnostics: with fs_options.tc_blocks it shows the tensor-core build. */
fs_status fs_get_self_block(fs_ctx *ctx, int32_t fiber, double *out);

/* The LU factors of one fiber's self block (Eq. prec, factored with partial
 * pivoting by fs_build_precond, which this calls first when the factors are
 * not current): lu receives the column-major (4N)^2 doubles of L (unit lower,
 * below the diagonal) and U (upper) in one array, piv the 4N row indices
 * with P B = L U, row i of P B being row piv[i] of B; both HOST arrays.
 * Synchronises the stream.  For tests and diagnostics: with fs_options.tc_lu
 * it shows the LU with tensor-core trailing updates. */
fs_status fs_get_block_lu(fs_ctx *ctx, int32_t fiber, double *lu, int32_t *piv);

/* The fiber far field's launch shapes chosen by fs_options.autotune: out[2 p
 * + h] for sum precision p (fs_sum_precision) with (h = 1) or without (h = 0)
 * hi/lo coordinates, a tile_override id 1..3, or 0 where that class has not
 * been tuned (yet, or autotune is off).  out: HOST array of 8 int32. */
fs_status fs_get_tuned_shapes(const fs_ctx *ctx, int32_t *out);

/* One implicit backward-Euler step (Sec. 3.2, set:time-stepping): solve
 * P^-1 A u = P^-1 b by GMRES with the block-Jacobi preconditioner P of Eq. prec
 * (Sec. 3.3), then X <- X + dt V.  The preconditioned operator is applied as
 * v + P^-1 (A - P) v on the fiber unknowns (P is their exact self block).
 * info may be NULL; when given it is filled (and the stream synchronised).
 * FS_ENOTCONV leaves the state unchanged. */
fs_status fs_step(fs_ctx *ctx, fs_step_info *info);

/* Per-class totals of the direct-sum kernels recorded since the last reset
 * (requires opt.profile = 1; otherwise all zero).  out: [FS_KS_COUNT].
 * Synchronises the context's stream.  reset != 0 clears the records. */
fs_status fs_kernel_stats(fs_ctx *ctx, fs_kernel_stat *out, int32_t reset);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t fs_kernel_launches(void);

/* Measured arithmetic throughput of the current device's CUDA cores: a
 * register-resident FMA loop over all SMs (precision 0 = FP64, 1 = FP32),
 * timed with CUDA events; *flops_per_s receives 2 x FMAs / s.  Used as the
 * roofline peak of the pipe-bound direct sums.  Synchronises the device. */
fs_status fs_probe_fma(int32_t precision, double *flops_per_s);

/* Plus-end growth rates dL/dt per fiber [n_fibers] for the following steps
 * (fiber (de)polymerization, Sec. 2.4 kinetics; 0 = fixed length, the
 * default).  The nodes stay at alpha_k in alpha = 2 s / L - 1 (minus end at
 * alpha = -1 fixed), so each step moves them by dt (w + R) -- w the material
 * velocity of Eq. main-sb-local, R the reparametrisation term of Eq.
 * chain-rule with the sign that advances the plus end: R = (alpha + 1)
 * (Ldot / L) X_alpha at the current time (Eq. discrete-rhs; the default) or,
 * with fs_options.growth_implicit = 1, R = (alpha + 1) kappa X+_alpha, X+ =
 * X + dt V, kappa = Ldot / (L + dt Ldot) -- and sets L <- L + dt Ldot.  fs_get_state's V is then (X+ - X)/dt,
 * the nodes' rate.  FS_EINVAL if some L + dt Ldot would not stay positive.
 * Synchronises the context's stream. */
fs_status fs_set_growth(fs_ctx *ctx, const double *Ldot, int32_t ptr_is_device);

/* The unknown vector of the last step's solve [n_unknowns] (fs_sizes): per
 * fiber the coefficients [c_x, c_y, c_z, d] (N each) of V_a = sum_j c_a,j
 * phi_j, phi = I^4 T_0 .. I^4 T_{N-5}, T_0 .. T_3, and T = sum_j d_j psi_j,
 * psi = I^2 T_0 .. I^2 T_{N-3}, T_0, T_1 (Eq. cheb-basis, integrated form;
 * I^m the m-fold integral from alpha = -1), then the periphery density
 * [n_nodes][3], then (with a body) its density [n_nodes][3], U and Omega.
 * Synchronises the context's stream. */
fs_status fs_get_unknowns(fs_ctx *ctx, double *u, int32_t ptr_is_device);

/* Current fiber lengths [n_fibers] (after growth).  Synchronises the stream. */
fs_status fs_get_lengths(fs_ctx *ctx, double *lengths, int32_t ptr_is_device);

/* Two-state dynamic instability (Sec. 5 kinetics: catastrophe and rescue of
 * growing and shrinking plus ends).  Host arrays; no CUDA call.  For each of
 * the n fibers, with one uniform random number u[i] in [0, 1) supplied by
 * the caller: a growing fiber (state 1) switches to shrinking (0) if
 * u < 1 - exp(-f_cat dt), a shrinking one to growing if u < 1 - exp(-f_res
 * dt); a shrinking fiber that would pass below L_min grows instead, a growing
 * one that would pass L_max (if L_max > 0) shrinks; then Ldot[i] = v_grow or
 * -v_shrink (pass Ldot to fs_set_growth).  state is updated in place.
 * FS_EINVAL: NULL arrays, dt not finite and > 0, a speed or rate negative or
 * not finite, L_min or L_max not finite. */
typedef struct {
    double v_grow, v_shrink;   /* plus-end speeds (length / time) */
    double f_cat, f_res;       /* catastrophe and rescue rates (1 / time) */
    double L_min, L_max;       /* rescue length; capping length (<= 0: none) */
} fs_kinetics;

fs_status fs_dynamic_instability(int32_t n, const fs_kinetics *kinetics, double dt, const double *lengths,
                                 const double *u, int32_t *state, double *Ldot);

/* Device bytes a context for this problem allocates (fs_create with these
 * fibers, a boundary of n_surface_nodes nodes or 0, and these options) plus
 * the largest direct-sum scratch one step reserves.  An upper bound of what
 * fs_device_bytes reports after a step; 0 for invalid arguments (including
 * options fs_create would refuse).  Host-only:
 * no CUDA call.  (No counterpart in the paper: sizing for admission control.) */
size_t fs_estimate_bytes(int32_t n_fibers, const int32_t *points_per_fiber, int32_t n_surface_nodes,
                         const fs_options *options);

/* Device bytes the context holds now (its arrays and its scratch). */
fs_status fs_device_bytes(const fs_ctx *ctx, size_t *bytes);

/* Serving (continuous batching): independent step requests submitted at any
 * time.  The server allocates its HBM budget ONCE at creation and runs two
 * engines, each with its own CUDA stream.  A free engine takes the queue head
 * and every queued request that can share a step with it -- same mu, eps, E,
 * dt, precision and tolerance, free space, at most max_slots requests, as long
 * as the batch's memory estimate fits the largest free piece of the budget --
 * and runs ONE batched implicit step for them (every launch covers all of the
 * batch's systems, each system with its own GMRES; fs_create_batch).
 * Requests that arrive meanwhile join the next batch, so the two engines'
 * batches overlap on the GPU.  No request allocates device memory: its batch
 * context carves its buffers from the budget, and the piece goes back when
 * the step ends.  A request with a boundary runs in a batch of its own.  A
 * request's arithmetic does not depend on its batch (far fields per system,
 * per-system reductions), so it gives the same bits alone and in any mix;
 * they agree with fs_step on the same input within the solve tolerance
 * (fs_step sums one system's far field in another order). */
typedef struct fs_server fs_server;

typedef struct fs_request {
    int32_t n_fibers;
    const int32_t *points_per_fiber;   /* [n_fibers], each in [6, 256] */
    const double *X;                   /* [N_tot][3] node positions, as fs_set_state */
    const double *lengths;             /* [n_fibers] */
    const double *f_ext;               /* [N_tot][3] or NULL (= 0) */
    const fs_boundary *boundary;       /* NULL: free space */
    double mu, eps, E, dt;             /* as fs_create */
    int32_t prec;                      /* fs_precision */
    double tol;                        /* GMRES tolerance; <= 0: the default */
    double *out_X;                     /* [N_tot][3] positions after the step, or NULL */
    double *out_V;                     /* [N_tot][3] velocity (required) */
    double *out_T;                     /* [N_tot] tension, or NULL */
} fs_request;

/* Start a server on `device`: allocates hbm_budget_bytes of device memory
 * (FS_ENOMEM if it cannot) and starts two engine threads; max_slots in
 * [1, 4096] is the largest number of requests one batched step admits. */
fs_status fs_server_create(fs_server **out, size_t hbm_budget_bytes, int32_t max_slots, int32_t device);

/* Queue a request.  All its input arrays are copied before the call returns;
 * the output arrays must stay valid until the ticket completes (fs_poll /
 * fs_server_wait returns anything but FS_EAGAIN / FS_ETIMEOUT).  FS_EBUSY: the
 * request alone needs more than the whole budget; FS_EINVAL: bad request. */
fs_status fs_submit(fs_server *sv, const fs_request *request, uint64_t *ticket);

/* Non-blocking completion check: FS_EAGAIN while queued or running;
 * otherwise the request's own status (FS_OK, or the error of fs_create /
 * fs_step with its message in fs_last_error()) and the ticket is released.
 * info (may be NULL) receives the batch step's info with the request's own
 * iterations, sweeps and residual, t_ms[5] = time queued and t_ms[6] =
 * submit-to-done latency in milliseconds, t_ms[7] = requests in its batch.
 * A request whose system did not converge reports FS_ENOTCONV (its outputs
 * still hold the last iterate's step); the others of its batch are not
 * affected. */
fs_status fs_poll(fs_server *sv, uint64_t ticket, fs_step_info *info);

/* Blocking form of fs_poll: waits up to timeout_s seconds; FS_ETIMEOUT if the
 * request is still queued or running then (the ticket stays valid). */
fs_status fs_server_wait(fs_server *sv, uint64_t ticket, fs_step_info *info, double timeout_s);

/* Snapshot of the queue: requests waiting, running, bytes of the budget in
 * use, and requests completed since creation (any may be NULL). */
fs_status fs_server_stats(fs_server *sv, int32_t *pending, int32_t *running, size_t *bytes_in_use,
                          int64_t *completed);

/* Batched steps the server has started since creation. */
fs_status fs_server_batches(fs_server *sv, int64_t *batches);

/* Finish the running batches, drop the queued requests (their tickets
 * become invalid), join the engines and free the budget's memory.  Running requests still write their output
 * arrays before this returns.  No other call on sv may be in progress or
 * follow it (a thread blocked in fs_server_wait on sv must return first). */
void fs_server_destroy(fs_server *sv);

/* Number of points N_tot and unknowns of the context. */
fs_status fs_sizes(const fs_ctx *ctx, int64_t *n_points, int64_t *n_unknowns);

/* Message of the last failed call on this thread (thread-local, static storage;
 * empty if none failed). */
const char *fs_last_error(void);
/* Name of a status code ("FS_OK", "FS_EINVAL", ...; "FS_UNKNOWN" otherwise). */
const char *fs_status_str(int32_t status);

#ifdef __cplusplus
}
#endif
#endif /* FIBERSOLVE_H */
