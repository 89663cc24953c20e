/*
 * sf.h — C ABI of the batched Safety-Filter (SF) solver for B300 (sm_103a).
 *
 * The SF projects candidate multi-robot trajectories, given as polynomial
 * coefficients, onto the constraint set of the paper's projection problem
 * (Sec. IV-B, eqs. proj_cost..proj_robot): boundary equalities A xi = b,
 * workspace box G xi <= h, and inter-robot / robot-obstacle separation written
 * in spherical form (Appendix, eqs. inter_robot_polar, workspace_polar).  It
 * runs the fixed-point operator T of eq. fixed_point — the alternating
 * minimisation of the augmented Lagrangian (eq. aug_lag) in the order alpha,
 * beta, d, s, lambda, xi_bar (eqs. alpha_step..xi_step) — for many independent
 * instances at once, and differentiates through it.
 *
 * Conventions shared by every call
 *  - Coefficients are axis-major per instance, [n_d][n][n_xi] (Sec. III-A,
 *    coefficient stacking); the trajectory basis is Bernstein of degree n_xi-1
 *    sampled at tau_k = k/(H-1), k = 0..H-1, so coefficient 0 is the start and
 *    coefficient n_xi-1 the goal.
 *  - Per-instance arrays are packed back to back in instance order; the packing
 *    offsets are returned by sf_layout().
 *  - Element type T of every floating-point array argument: double when the
 *    handle's precision is SF_FP64, float otherwise.
 *  - Array arguments of sf_solve / sf_solve_backward are DEVICE pointers owned
 *    by the caller; the library never frees them.  The library owns its factor
 *    and workspace memory (allocated in sf_create, freed in sf_destroy).
 *  - All calls return an sf_status; SF_OK is 0.  No call aborts, traps or exits.
 *  - sf_solve and sf_solve_backward are asynchronous on the given stream
 *    (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *    Device-side failures (non-finite values, bounded waits that ran out) are
 *    reported per instance by sf_get_status() after the stream is synchronised.
 *  - A handle is not thread-safe; calls on one handle must be serialised.
 */
#ifndef SF_H
#define SF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
enum {
    SF_OK = 0,
    SF_EINVAL = 1,      /* invalid argument (NULL pointer, size or value out of range)   */
    SF_ESHAPE = 2,      /* inconsistent shapes (e.g. backward after a solve with other sizes) */
    SF_ECUDA = 3,       /* a CUDA runtime call failed                                     */
    SF_ENOMEM = 4,      /* device or host allocation failed                               */
    SF_ETIMEOUT = 5,    /* a bounded device-side wait ran out (reported per instance)     */
    SF_ENONFINITE = 6,  /* NaN/Inf met in an iterate (reported per instance)              */
    SF_ESTATE = 7,      /* call order violated (e.g. backward without checkpoints)        */
    SF_EUNSUPPORTED = 8, /* option not built into this library                            */
    SF_ETOOBIG = 9,      /* sizes beyond the fixed limits of sf_solve_noalloc                  */
    SF_EBOUNDS = 10      /* a device-side bounds check failed (per instance; only libraries
                            built with SF_BOUNDS_CHECK run the checks)                        */
};

/* ---- precision of the iteration ------------------------------------------ */
enum {
    SF_FP64 = 0,       /* everything in FP64 (plain reference path on the GPU)            */
    SF_FP32 = 1,       /* FP32 elementwise steps, FP32 SIMT projection                    */
    SF_TF32 = 2,       /* FP32 elementwise, projection on tensor cores in TF32, FP32 acc  */
    SF_BF16X3 = 3,     /* FP32 elementwise, projection as three BF16 tensor-core products
                          (hi*hi + hi*lo + lo*hi of a two-term BF16 split), FP32 acc      */
    SF_BF16 = 4        /* FP32 elementwise, projection in one BF16 tensor-core product    */
};

/* ---- projection operator (step xi_bar, eq. batch_comp) -------------------- */
enum {
    SF_PROJ_DENSE = 0,      /* dense P_eta (N x N per shape), as in eq. batch_comp          */
    SF_PROJ_STRUCTURED = 1  /* same operator through its Kronecker form (n_xi x n_xi blocks) */
};

/* Cost of the xi_bar step (the constraints and the iteration are the same) */
enum {
    SF_COST_PROJECTION = 0, /* the Safety Filter: 1/2 ||xi_bar - xi||^2 to the candidate xi
                               (eq. proj_cost)                                              */
    SF_COST_SMOOTHNESS = 1  /* the trajectory optimiser of eq. eq::form: 1/2 sum over robots
                               and timesteps of ||p''||^2 (eq. cost), p'' in time
                               t = tau (H - 1) dt; xi_cand then serves only as the default
                               initial iterate and receives no gradient                   */
};

/* ---- per-instance shape ---------------------------------------------------- */
/* sf_create accepts n <= 256, n_obs <= 4096, H <= 4096; an instance must also fit the
 * per-CTA shared-memory budget (227 KB) at some cluster size: each CTA keeps its share of
 * the horizon's basis rows, the instance's iterate, multipliers and obstacle records, and
 * a chunk of positions.  For example H = 4096 fits in FP32 and FP64, n_obs = 4096 in FP32
 * only, n = 256 robots in the 2-D FP32 forward only (no checkpoints); sizes that fit
 * nowhere return SF_EUNSUPPORTED. */
typedef struct sf_shape {
    int32_t n;          /* robots, >= 1                                                    */
    int32_t n_obs;      /* obstacles, >= 0                                                 */
    int32_t H;          /* timesteps K+1 of the planning period, >= 2                      */
    int32_t dyn_obs;    /* 0: static centres [n_obs][n_d]; 1: per timestep [n_obs][H][n_d] */
    double a, b;        /* robot spheroid: M_r = diag(a, a, b) (Sec. III-A); centre
                           distance >= a between spherical robots of radius a/2             */
    double p_min[3];    /* workspace box (eq. workspace_con), already inset by the robot   */
    double p_max[3];
} sf_shape;

/* ---- solver description --------------------------------------------------- */
typedef struct sf_desc {
    int32_t n_d;        /* workspace dimension, 2 or 3                                     */
    int32_t n_xi;       /* Bernstein coefficients per robot per axis, 4..32                */
    double rho;         /* augmented-Lagrangian penalty (eq. aug_lag), > 0                 */
    int32_t precision;  /* SF_FP64 .. SF_BF16                                              */
    int32_t proj;       /* SF_PROJ_DENSE or SF_PROJ_STRUCTURED                             */
    int32_t n_refine;   /* refinement passes of the tensor-core projection (SF_TF32,
                           SF_BF16X3, SF_BF16; ignored otherwise; 0 .. 8): each pass adds P~(v - H d)
                           to the projected d, the residual taken in FP32 through the
                           Kronecker-structured Hessian of eq. batch_comp.  With P~ the
                           rounded projector the error shrinks by ||I - P~H|| per pass.  On
                           the benchmark workloads one pass brings SF_BF16X3 within 1e-4 m
                           of FP64, two or three SF_TF32, and five SF_BF16                 */
    int32_t max_iters;  /* upper bound on `iters` of sf_solve (sizes checkpoint storage)    */
    int32_t ckpt_every; /* > 0: sf_solve keeps (xi_bar, lambda) every ckpt_every iterations
                           so sf_solve_backward can run, and every launch plan leaves room
                           for the adjoint kernel; 1: the adjoint recomputes nothing;
                           0: no backward                                                  */
    double tol;         /* residual threshold in metres for iterations-to-tolerance        */
    int32_t n_inst;     /* number of instances, >= 1                                       */
    const sf_shape *shapes; /* host array [n_inst], copied by sf_create                    */
    void *stream;       /* cudaStream_t on which sf_create runs the factorisations         */
    int32_t cost;       /* SF_COST_PROJECTION (0) or SF_COST_SMOOTHNESS                    */
    double dt;          /* time step in seconds of the smoothness cost and of the velocity
                           rows (> 0 when either is used): t = tau (H - 1) dt               */
    int32_t n_bc;       /* boundary rows of A per robot and axis (eq. boundary_con): 2 (or 0)
                           start and goal; 3 adds the initial velocity p'(t = 0) = v_0, the
                           planner conditioned on the robots' current velocities (Sec. V,
                           hardware experiments); needs dt > 0 and n_xi >= 5.  For the
                           Bernstein basis the rows fix coefficients 0, n_xi - 1 and, with
                           the velocity row, 1 (xi_1 = start + v_0 (H - 1) dt / (n_xi - 1)) */
} sf_desc;

typedef struct sf_handle sf_handle;

/* ---- instance data (device pointers, element type T) ---------------------- */
typedef struct sf_instance_data {
    const void *bnd;    /* [n_d][n][n_bc] start, goal [, initial velocity in m/s] per axis
                           and robot (eq. boundary_con)                                     */
    const void *obs_c;  /* obstacle centres, static [n_obs][n_d] or dynamic [n_obs][H][n_d]  */
    const void *obs_ab; /* [n_obs][2] obstacle axes (a_o, b_o), inflated by the robot size  */
} sf_instance_data;

/* Layout kinds for sf_layout */
enum { SF_LAYOUT_XI = 0, SF_LAYOUT_BND = 1, SF_LAYOUT_OBS = 2, SF_LAYOUT_OBS_AB = 3 };

/* Per-instance outputs of sf_solve in resid_out (double, device, [n_inst][SF_NRES]) */
enum {
    SF_RES_RP = 0,      /* ||r_p||_2 of the returned xi_bar, FP64 (eq. primal_residual)      */
    SF_RES_MAX = 1,     /* max constraint residual of the returned xi_bar in metres, FP64:
                           max over rows of ||r_1 row|| (penetration) and of r_2 entries   */
    SF_RES_FP = 2,      /* ||z^L - z^(L-1)||_2, last fixed-point step (eq. fixed_point_residual) */
    SF_RES_ITERS = 3,   /* first l whose iterate met max residual <= tol, or -1            */
    SF_RES_FPSUM = 4,   /* sum over the iterations of ||z^{l+1} - z^l||_2^2, z = (xi_bar, lambda):
                           the fixed-point term of the self-supervised loss (eq. NN_loss)    */
    SF_NRES = 5
};

/*
 * sf_create — validate `desc`, build every distinct (n, n_obs, H) shape's basis W
 * and the xi_bar-step operators, and factor them in FP64 on the GPU (eq. xi_step:
 * Cholesky of H = I + rho F'F + rho G'G, Schur complement of A; the factorisation
 * is independent of the candidate and is stored, as the Appendix notes, and only
 * changes with rho or the horizon).  Runs on desc->stream and synchronises it.
 * On success *out owns all device memory of the solver.
 * Errors: SF_EINVAL (bad sizes/values, NULL), SF_ENOMEM, SF_ECUDA, SF_EUNSUPPORTED.
 * On any error every allocation made so far is freed and *out is NULL.  For tests of
 * that unwinding, the environment variable SF_TEST_FAIL_ALLOC = k (k >= 0) makes the
 * (k+1)-th device allocation of this call fail as out of memory (SF_ENOMEM).
 */
int sf_create(const sf_desc *desc, sf_handle **out);

/* sf_destroy — free the handle and its device memory (synchronises its streams). */
int sf_destroy(sf_handle *h);

/*
 * sf_layout — packing offsets (in elements of T) of one per-instance array kind:
 * offsets[i] = start of instance i, offsets[n_inst] = total length.
 * `offsets` is a host array of n_inst + 1 entries.
 */
int sf_layout(const sf_handle *h, int32_t kind, int64_t *offsets);

/*
 * sf_solve — run `iters` applications of T (eq. fixed_point) on every instance.
 *  data            instance data (device, T), see sf_instance_data
 *  xi_cand         candidate coefficients xi (SF_LAYOUT_XI packing)
 *  xi0, lam0       initial (xi_bar^0, lambda^0); NULL means xi_bar^0 = xi_cand, lambda^0 = 0
 *  iters           0 <= iters <= desc->max_iters
 *  xi_out, lam_out (xi_bar^L, lambda^L); lam_out may be NULL
 *  resid_out       device double [n_inst][SF_NRES] or NULL
 *  iters_to_tol    device int32 [n_inst] or NULL (same value as resid_out[SF_RES_ITERS])
 *  stream          cudaStream_t
 * When desc->ckpt_every > 0 the call also records what sf_solve_backward needs; the
 * caller must keep data, xi_cand, xi0, lam0 unchanged until that backward call.
 * Errors: SF_EINVAL, SF_ECUDA.
 */
int sf_solve(sf_handle *h, const sf_instance_data *data, const void *xi_cand, const void *xi0,
             const void *lam0, int32_t iters, void *xi_out, void *lam_out, double *resid_out,
             int32_t *iters_to_tol, void *stream);

/*
 * sf_solve_backward — vector-Jacobian product through the iterations of the last
 * sf_solve on this handle (the unrolled chain of T, Fig. unroll_learning), by a
 * hand-written adjoint that recomputes each checkpoint segment.
 *  g_xi_out, g_lam_out  seeds dL/dxi_bar^L, dL/dlambda^L (either may be NULL = 0)
 *  g_rp2                device double [n_inst] or NULL: dL/d||r_p(xi_bar^L)||^2
 *  g_fp                 device double [n_inst] or NULL: dL/dS with S = sum over the
 *                       iterations l = 0..L-1 of ||z^{l+1} - z^l||^2, z = (xi_bar, lambda)
 *                       (resid_out[SF_RES_FPSUM] of the solve): the fixed-point term of the
 *                       self-supervised loss that trains an initialisation network through
 *                       the solver (eq. NN_loss, Sec. IV-B); its second term
 *                       ||xi_bar^L - xi||^2 is an ordinary g_xi_out seed
 *  g_xi_cand            out: dL/dxi_cand (through eta in every iteration; when that
 *                       solve had xi0 = NULL, also through xi_bar^0 = xi_cand)
 *  g_xi0, g_lam0        out: dL/dxi_bar^0, dL/dlambda^0 (either may be NULL)
 * Errors: SF_ESTATE (no preceding solve with checkpoints), SF_EINVAL, SF_ECUDA.
 */
int sf_solve_backward(sf_handle *h, const void *g_xi_out, const void *g_lam_out,
                      const double *g_rp2, const double *g_fp, void *g_xi_cand, void *g_xi0,
                      void *g_lam0, void *stream);

/*
 * sf_get_status — copy the per-instance device status words (SF_OK, SF_ENONFINITE,
 * SF_ETIMEOUT) of the last solve/backward into the host array [n_inst] and
 * clear them.  Synchronises the handle's last stream.
 */
int sf_get_status(sf_handle *h, int32_t *per_instance_status);

/*
 * sf_shape_operator — diagnostic copy of the FP64 operators of instance `inst`'s shape
 * to host memory `host_out`:
 *   which = 0: basis W [H][n_xi]
 *   which = 1: P_eta [N][N]            (N = n * n_xi)
 *   which = 2: P_b [N][n_bc n]         (columns robot-major: start, goal[, velocity])
 *   which = 3: Kronecker blocks P_dev [n_xi][n_xi], P_mean [n_xi][n_xi],
 *              B_dev [n_xi][n_bc], B_mean [n_xi][n_bc], then the per-robot cost block
 *              [n_xi][n_xi] (the identity, or Wdd' Wdd of the smoothness cost with Wdd
 *              the basis' second time derivative), back to back
 * Synchronises the device.  Errors: SF_EINVAL, SF_ECUDA.
 */
int sf_shape_operator(const sf_handle *h, int32_t inst, int32_t which, double *host_out);

/*
 * sf_set_launch — override the launch geometry of this handle's kernels:
 *  cluster   CTAs that share one instance (a thread-block cluster, each CTA taking a
 *            contiguous share of the timesteps), 1..8, or 0 for the automatic choice
 *            (enough clusters to cover the SMs)
 *  threads   threads per CTA, a multiple of 32 in 64..512 (SF_FP64) or 64..1024 (the
 *            FP32-based precisions), or 0 for 512
 * Results do not depend on the geometry beyond rounding order.  Errors: SF_EINVAL,
 * SF_EUNSUPPORTED (an instance does not fit in shared memory with this geometry).
 */
int sf_set_launch(sf_handle *h, int32_t cluster, int32_t threads);

/*
 * sf_autotune — time each candidate launch geometry (cluster 1, 2, 4, 8 x threads
 * 128, 256, 512, 1024 that fit) on this handle's own batch with `iters` iterations of
 * sf_solve, followed by sf_solve_backward when the handle keeps checkpoints (CUDA
 * events on `stream`, best of `reps` runs), keep the fastest and return it.  Allocates and frees temporary output buffers; results of later solves
 * do not depend on the choice beyond rounding order.  The choice is also remembered
 * for the batch's shape signature, and sf_create of a later handle with the same
 * signature starts from it.
 *  best_cluster, best_threads, best_ms  host outputs (any may be NULL)
 * Errors: SF_EINVAL, SF_ENOMEM, SF_ECUDA.
 */
int sf_autotune(sf_handle *h, const sf_instance_data *data, const void *xi_cand, int32_t iters, int32_t reps,
                void *stream, int32_t *best_cluster, int32_t *best_threads, float *best_ms);

/* sf_get_launch — the geometry in use: cluster, threads, staged projection rows. */
int sf_get_launch(const sf_handle *h, int32_t *cluster, int32_t *threads, int32_t *p_rows);

/* Options of sf_set_option / sf_get_option */
enum {
    SF_OPT_CULL = 1,  /* row culling: 1 (default) loops, per chunk of timesteps, over the
                         partners and obstacles whose bounding boxes come within the
                         activity threshold of the robot's box (steps alpha..d of the
                         iteration, and their adjoint); 0 loops over all of them.  The
                         two give identical bits: a culled row is inactive throughout
                         the chunk and contributes nothing.  Culling is dropped silently
                         when its lists do not fit in shared memory.                   */
    SF_OPT_TEST_TIMEOUT = 2, /* tests of the failure path only: 1 gives the tensor-core
                         projection's pipeline waits a zero polling budget, so the first
                         wait of each CTA gives up at once, no MMA is issued, the copies
                         in flight are still drained before the CTA exits, and every
                         instance reports SF_ETIMEOUT; 0 (default) restores the budget */
    SF_OPT_TC_RESIDENT = 3, /* read-only: 1 when the plan keeps each CTA's tensor-core
                         projector rows resident in shared memory (loaded once per solve),
                         0 when they stream through a two-stage ring every projection   */
    SF_OPT_TC_BATCH = 4, /* the batched tensor-core projection of eq. batch_comp: 1 (default)
                         lets the plan run G instances of one shape in one thread-block
                         cluster of G x (CTAs per instance) <= 16 CTAs, when the precision
                         is SF_BF16 or SF_BF16X3 with SF_PROJ_DENSE, every instance has the
                         same shape and G divides the batch: each CTA keeps its rows of
                         P_eta in tensor memory (BF16; with SF_BF16X3 the low parts beneath
                         the high ones) and one tcgen05.mma chain multiplies them by the
                         right-hand sides of all G instances (G n_d <= 16 columns); 0 keeps
                         one instance per cluster.  sf_get_option gives G (0: not used).
                         Results agree with the per-instance product to rounding order   */
    SF_OPT_EARLY_EXIT = 5 /* 1: an instance stops iterating after the iteration whose iterate
                         first met max residual <= tol (SF_RES_ITERS); its outputs are the
                         iterate that iteration produced, and the other instances run on,
                         so a batch where some instances converge frees their SMs early.
                         Handles without checkpoints only (SF_EUNSUPPORTED otherwise: the
                         adjoint differentiates a fixed iteration count); not applied while
                         instances share clusters (SF_OPT_TC_BATCH, whose instances share
                         barriers: sf_get_option then reads 0).  0 (default): every
                         instance runs `iters` iterations                                 */
};

/*
 * sf_set_option — set an option (SF_OPT_*) and re-plan the launch with the current
 * geometry (synchronises the device).  Errors: SF_EINVAL (unknown or read-only
 * option, bad value),
 * SF_EUNSUPPORTED (the re-plan does not fit).
 * sf_get_option — the option's effective value in the current plan (for SF_OPT_CULL,
 * 0 when culling was requested but does not fit).
 */
int sf_set_option(sf_handle *h, int32_t option, int32_t value);
int sf_get_option(const sf_handle *h, int32_t option, int32_t *value);

/* Kernel timing slots of sf_kernel_times */
enum { SF_KT_FORWARD = 0, SF_KT_RESIDUAL = 1, SF_KT_BACKWARD = 2, SF_NKT = 3 };

/*
 * sf_profile — enable (1) or disable (0) CUDA-event timing of each kernel that
 * sf_solve / sf_solve_backward launch on this handle (events are recorded on the
 * call's stream around the launch).  Off by default.
 */
int sf_profile(sf_handle *h, int32_t enable);

/*
 * sf_kernel_times — durations in milliseconds of the kernels of the most recent
 * profiled calls, into host ms_out[SF_NKT] (0 for a kernel that did not run).
 * Synchronises on the recorded events.  Errors: SF_EINVAL, SF_ESTATE (profiling off).
 */
int sf_kernel_times(sf_handle *h, float *ms_out);

/*
 * sf_solve_noalloc — the same SF solve as sf_create + sf_solve with SF_FP32 and
 * SF_PROJ_STRUCTURED, for a batch whose instances all share one shape, in one call
 * that allocates no memory at all.  The paper has no counterpart to this call.
 *
 * Who needs it: code that must not allocate device memory once it is running — a
 * robot's control loop with a fixed memory budget set at start-up, or a plug-in
 * running inside a host framework that owns every device allocation and forbids its
 * plug-ins to call cudaMalloc — cannot use sf_create, which allocates the factor and
 * workspace memory of a handle.  This call instead keeps its working memory (instance
 * table, basis, the projection's Kronecker blocks, status words) in one fixed array
 * of about 450 KB compiled into the library, which every GPU that loads the library
 * holds until the process exits.
 *
 *  n_d, n_xi, rho  as in sf_desc (2 or 3, 4..32, > 0)
 *  shape           host pointer to the one sf_shape every instance has
 *  n_inst          1 .. SF_NOALLOC_MAX_INST instances
 *  bnd, obs_c, obs_ab, xi_cand   device float arrays packed as sf_layout would pack
 *                  n_inst copies of `shape` (instance k's coefficients start at
 *                  k * n_d * n * n_xi, and so on)
 *  iters           >= 0
 *  xi_out, lam_out device float [n_inst * n_d * n * n_xi]; lam_out may be NULL
 *  resid_out       device double [n_inst][SF_NRES] or NULL (iterations-to-tolerance
 *                  uses tol = 1e-3 m)
 *  stream          cudaStream_t
 * Limits: n_inst <= SF_NOALLOC_MAX_INST, H <= SF_NOALLOC_MAX_H, n_xi <= 32; larger
 * sizes return SF_ETOOBIG before anything is launched.  Other bad arguments return
 * SF_EINVAL; CUDA failures SF_ECUDA.
 * Set-up: the first call on each device looks up the device address of the fixed
 * array (with that device current, under a mutex); make that first call before any
 * stream capture.  Every call then hands its sizes to its own set-up kernel by value,
 * which writes the instance table, basis and operators into the array; no host memory
 * is read after the call returns.
 * Sharing: every call on one device, on every stream, uses that device's array, which
 * keeps the last call's contents (each call rewrites what it reads and clears its status
 * words), so calls whose work overlaps on one GPU race with each other: serialise them.
 * Calls on different devices use different copies and are independent.
 * Per-instance status words are not reported; a non-finite iterate, or a singular
 * boundary system (then every output is NaN), shows as a non-finite entry of resid_out.
 * Only the two boundary rows (start, goal) are supported: bnd is [n_d][n][2].
 */
#define SF_NOALLOC_MAX_INST 256
#define SF_NOALLOC_MAX_H 1024
int sf_solve_noalloc(int32_t n_d, int32_t n_xi, double rho, const sf_shape *shape, int32_t n_inst,
                     const float *bnd, const float *obs_c, const float *obs_ab, const float *xi_cand,
                     int32_t iters, float *xi_out, float *lam_out, double *resid_out, void *stream);

/*
 * sf_alu_peaks — measured throughput of the arithmetic pipes the solver's row kernels run
 * on, for their roofline (a diagnostic; the paper has no counterpart): out[0] FP32 FMA
 * (flop/s, 2 per FMA), out[1] FP64 FMA (flop/s), out[2] MUFU reciprocal square roots per
 * second.  Each is a kernel that keeps every SM of the current device busy with
 * independent dependency chains, timed with CUDA events (best of three launches of about
 * seconds / 3 each, after a warm-up).  Allocates and frees 64 bytes of device memory and
 * synchronises `stream`.  seconds in (0, 60].  Errors: SF_EINVAL, SF_ENOMEM, SF_ECUDA.
 */
int sf_alu_peaks(double seconds, double *out, void *stream);

/* sf_strerror — static description of a status code. */
/*
 * sf_fit_positions — least-squares Bernstein coefficients of sampled trajectories, with
 * the end coefficients pinned to the first and last sample (eq. poly, p = W xi; the
 * boundary rows A xi = b fix coefficients 0 and n_xi - 1, which the basis interpolates).
 * For every instance, robot and axis, xi minimises ||W xi - p||^2 subject to
 * xi_0 = p_0 and xi_{n_xi-1} = p_{H-1}.  A helper for building candidates from sampled
 * positions; not part of the solve.
 *  n_d, n_xi      2..3, 3..32
 *  n_inst         instances; n[k], H[k] (HOST arrays): robots and timesteps of
 *                 instance k, with n_xi <= H[k] <= 2^20
 *  pos            DEVICE, FP64, instance after instance, [n_d][n][H]
 *  xi_out         DEVICE, FP64, instance after instance, [n_d][n][n_xi] (the packing of
 *                 SF_LAYOUT_XI)
 * Allocates and frees its scratch on `stream` and synchronises it before returning.
 * Errors: SF_EINVAL (bad sizes, singular fit), SF_ENOMEM, SF_ECUDA.
 */
int sf_fit_positions(int32_t n_d, int32_t n_xi, int32_t n_inst, const int32_t *n, const int32_t *H,
                     const double *pos, double *xi_out, void *stream);

/*
 * sf_metrics — per instance of the handle, in FP64 from the coefficients `xi` (DEVICE,
 * packed like sf_solve's arrays, the handle's precision) and the instance data:
 *   out[k][0] = ||r_p||_2 and out[k][1] = the max residual in metres (as SF_RES_RP,
 *               SF_RES_MAX; eq. primal_residual),
 *   out[k][2] = smoothness cost, sum over timesteps of ||p''||^2 averaged across robots,
 *   out[k][3] = path length, the polygon length of the H positions averaged across robots
 *               (the paper's trajectory-quality metrics, Sec. V "Metrics"),
 * with p'' in time t = tau (H - 1) dt, dt from sf_desc (the handle must have dt > 0).
 * out: DEVICE, double, [n_inst][4].  Asynchronous on `stream`.
 * Errors: SF_EINVAL, SF_ECUDA.
 */
int sf_metrics(sf_handle *h, const sf_instance_data *data, const void *xi, double *out, void *stream);

/*
 * sf_select — per group of candidates, the indices of the k best, in order (the ranking
 * stages of the paper's pipeline: keep the candidates of least constraint violation
 * before the SF; return the feasible one of least smoothness cost after it).
 * A candidate is feasible when primary <= threshold.  Feasible candidates come first,
 * ordered by `secondary` (or by `primary` when secondary is NULL); then the others,
 * ordered by `primary`; NaN scores last; ties to the lower index.
 *  n_groups, group_size  HOST: groups of consecutive candidates, each 0..4096
 *  primary, secondary    DEVICE, double, one score per candidate (secondary may be NULL)
 *  threshold             e.g. -INFINITY to rank every candidate by `primary`
 *  k                     1..4096
 *  out_idx               DEVICE, int32, [n_groups][k]: indices within the group, -1 past
 *                        the group's size
 * Asynchronous on `stream` (its small scratch is stream-ordered).
 * Errors: SF_EINVAL, SF_ENOMEM, SF_ECUDA.
 */
int sf_select(int32_t n_groups, const int32_t *group_size, const double *primary, const double *secondary,
              double threshold, int32_t k, int32_t *out_idx, void *stream);

const char *sf_strerror(int32_t code);

/* sf_version — library version as an integer (major * 10000 + minor * 100 + patch). */
int32_t sf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SF_H */
