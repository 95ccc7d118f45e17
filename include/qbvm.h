/*
 * qbvm.h -- C ABI of the GB300 (sm_103a) solver for the parallel-in-time
 * quasi-boundary value methods PinT-QBVM and PinT-MQBVM of
 * J. Liu, "Fast Parallel-in-Time Quasi-Boundary Value Methods for Backward
 * Heat Conduction Problems" (arXiv 2107.06381).
 *
 * The problem (Section 1, eq. 1.1): recover z(., 0) from a measurement g_delta
 * of z(., T) for z_t = Laplace(z) on (0, L)^d with z = 0 on the boundary.
 * The library solves the regularised all-at-once system of Section 3
 *
 *     A y = f,   A = (1/tau) C_omega (x) I_x - I_t (x) Delta_h      (Section 3.3)
 *
 * where Delta_h is the Dirichlet 3/5/7-point Laplacian on the (M-1)^d interior
 * nodes (Section 2), tau = T/N, C_omega is the N_t x N_t matrix with unit
 * diagonal, -1 on the subdiagonal and -omega in the top-right corner, and
 *   PinT-QBVM  (Section 3.1, eq. 3.3): omega = -1/alpha,   f^0 = g/(tau alpha)
 *   PinT-MQBVM (Section 3.2, eq. 3.6): omega = -tau/alpha, f^0 = g/alpha
 * (in both cases f^0 = -omega g / tau and f^n = 0 for n >= 1), by the
 * diagonalisation C_omega = V D V^{-1}, V = Gamma_omega^{-1} F* of Section 3.3:
 * omega-scaling and an FFT along time, N_t decoupled complex-shifted spatial
 * solves, an inverse FFT and the omega-unscaling (eq. 3.8).
 *
 * Conventions shared by every entry point
 *  - nt is the number of time levels N_t = N + 1 (Section 2); tau = T/(nt - 1).
 *  - Arrays are FP64, row-major [nt][n_z][n_y][n_x] with x fastest, n_d = m[d]-1;
 *    this is the paper's ordering y_h = (y^0; y^1; ...; y^N).  A "g" array is
 *    one time level [n_z][n_y][n_x].
 *  - Array arguments may be device pointers or host pointers (pageable or
 *    pinned).  Device pointers: the call only enqueues work on `stream` and
 *    returns.  Host pointers: the call stages through device buffers owned by
 *    the plan and returns after the result has been copied back (it
 *    synchronises `stream`).  Input and output may not be a mix of the two,
 *    and device pointers must be memory of the device the plan was made on
 *    (or managed memory): another GPU's memory is BAD_ARG.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  A plan may be
 *    used by one stream at a time; calls on one plan must not overlap.
 *  - The caller owns every array it passes; the plan owns its device tables
 *    and workspace and frees them in qbvm_destroy.  Every *_destroy accepts
 *    NULL (and returns QBVM_OK), as free() does.
 *  - Every entry point returns QBVM_OK (0) or a negative QBVM_ERR_* code; on an
 *    error nothing has been enqueued unless the code is QBVM_ERR_CUDA.
 */
#ifndef QBVM_H
#define QBVM_H

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define QBVM_OK               0
#define QBVM_ERR_BAD_ARG     -1   /* invalid descriptor or argument            */
#define QBVM_ERR_OOM         -2   /* device or host allocation failed          */
#define QBVM_ERR_NONFINITE   -3   /* NaN/Inf in the input or the result        */
#define QBVM_ERR_DIVERGED    -4   /* FP32 refinement stalled above 1e-10 or hit
                                     its iteration cap above the tolerance     */
#define QBVM_ERR_TIMEOUT     -5   /* a bounded device wait gave up             */
#define QBVM_ERR_CUDA        -6   /* a CUDA runtime call failed                */
#define QBVM_ERR_UNSUPPORTED -7   /* size outside what the kernels implement   */

/* ------------------------------------------------------------ enumerations */
#define QBVM_FORM_PQ 0            /* PinT-QBVM,  Section 3.1                    */
#define QBVM_FORM_PM 1            /* PinT-MQBVM, Section 3.2                    */

#define QBVM_FP64        0        /* every stage in FP64                        */
#define QBVM_FP32_REFINE 1        /* FP32 transforms (tables computed in FP64 and
                                     rounded once), double-float residual and
                                     iterate: iterative refinement.  Needs the
                                     space-first order. */

#define QBVM_RHS_DELTA   0        /* input is g (one level): f^0 = -omega g/tau */
#define QBVM_RHS_GENERAL 1        /* input is a full right-hand side F [nt][..] */

/* ------------------------------------------------------------ descriptor
 * dim     space dimension d = 1, 2 or 3.
 * m[3]    intervals per axis (x, y, z); m[d] >= 2; entries beyond dim ignored.
 *         Supported: any m in [2, 2048] on every axis (space-first order:
 *         the DST-I of length m-1 runs as a radix-4/2 FFT of length m when m
 *         is a power of two in [4, 1024], else as a mixed-radix FFT -- radix
 *         4, 2, 3, 5 passes and a direct DFT for any other prime factor, so
 *         its cost per element grows with m's largest prime factor); in 1D
 *         with the time-first order any m with m-1 <= 2^20.
 * L       side length of the domain (0, L)^d; h = L/m[d].
 * T       final time, > 0.
 * nt      time levels N_t: a power of two in [2, 1024] (half-length time
 *         transforms), or any other nt in [3, 2048] (Bluestein time DFTs over
 *         every frequency, FP64 or FP32; the paper's meshes have N_t = N + 1).
 * form    QBVM_FORM_PQ or QBVM_FORM_PM.
 * alpha   regularisation parameter > 0, or <= 0 for the a-priori rule of
 *         Section 5 from `delta`: alpha = delta (PQ), alpha = tau*delta (PM).
 * delta   noise level (only read when alpha <= 0; must then be > 0).
 * precision  QBVM_FP64 or QBVM_FP32_REFINE.
 * rhs_kind   QBVM_RHS_DELTA or QBVM_RHS_GENERAL.
 * refine_tol       FP32_REFINE: stop when ||f - A y||/||f|| <= refine_tol
 *                  (<= 0 selects 1e-13).
 * refine_max_iters FP32_REFINE: iteration cap (<= 0 selects 10).
 * order   QBVM_ORDER_*: how the factors of eq. 3.8 are applied.  Space-first
 *         (DST-I along every axis, one scalar omega-circulant time solve per
 *         spatial mode, inverse DST) is the only order in 2D/3D.  In 1D the
 *         time-first order of Section 3.3 (omega-scaled time DFT, one complex
 *         tridiagonal solve per frequency, inverse DFT) is also available;
 *         it is the paper's order but loses accuracy when |omega| is large and
 *         the data are smooth (the spatial systems of the low frequencies are
 *         nearly singular): 2e-10 to 1e-9 against the exact solution on the
 *         paper's 1D meshes at noise 1e-4, where space-first gives 1e-12.
 *         AUTO takes space-first whenever m allows it.
 */
#define QBVM_ORDER_AUTO        0
#define QBVM_ORDER_TIME_FIRST  1
#define QBVM_ORDER_SPACE_FIRST 2
typedef struct qbvm_desc {
    int    dim;
    int    m[3];
    double L;
    double T;
    int    nt;
    int    form;
    double alpha;
    double delta;
    int    precision;
    int    rhs_kind;
    double refine_tol;
    int    refine_max_iters;
    int    order;
} qbvm_desc;

/* Read-only facts about a plan (qbvm_plan_info). */
typedef struct qbvm_info {
    double alpha;            /* alpha in use (after the a-priori rule)         */
    double omega;            /* omega of eq. 3.3 / 3.6                         */
    double tau;              /* T / (nt - 1)                                   */
    long long unknowns;      /* N_x * N_t                                      */
    long long workspace_bytes;  /* device bytes the plan holds                 */
    int    last_refine_iters;   /* refinement steps of the last FP32_REFINE solve */
    double last_rel_residual;   /* ||f - A y||/||f|| after that solve           */
    int    kernels_per_solve;   /* kernel launches of one solve (device pointers) */
} qbvm_info;

typedef struct qbvm_plan qbvm_plan_t;

/* qbvm_plan -- validate `desc`, derive tau, alpha, omega (Sections 3.1/3.2, 5)
 * and build the FP64 tables of the diagonalisation (Section 3.3: the powers
 * omega^{k/N_t} of Gamma_omega with the principal root, the eigenvalues
 * d_k = 1 - omega^{1/N_t} theta^k of C_omega, the FFT roots of unity and the
 * Dirichlet eigenvalues (4/h^2) sin^2(k pi/(2m))), then allocate the device
 * workspace on the current device.
 * On success *out receives a plan that the caller frees with qbvm_destroy.
 * Errors: BAD_ARG (dim, m, nt, T, L, alpha/delta, form, precision, rhs_kind
 * out of range; the check needs no GPU), UNSUPPORTED (valid but not a size
 * the kernels implement), OOM, CUDA. */
int qbvm_plan(const qbvm_desc* desc, qbvm_plan_t** out);

/* qbvm_solve -- solve A y = f (eq. 3.3 or 3.6) with the three steps of
 * eq. 3.8.  `g_or_F` is g (one level, rhs_kind DELTA) or F (nt levels,
 * rhs_kind GENERAL); `y` receives all nt levels, or only y^0 (the first
 * level, n_z*n_y*n_x values) when n0_only != 0.  In and out may alias for
 * rhs_kind GENERAL (FP32_REFINE then copies F into plan memory first, since
 * the refinement re-reads it).  FP32_REFINE solves data whose root-mean-square
 * magnitude lies outside [1e-18, 1e28] (where FP32 cannot carry the residuals)
 * with the FP64 pipeline; last_refine_iters is then 0, and so it does data
 * FP32 cannot hold at all (finite values beyond its range, or so small that
 * every one flushes to zero).  Non-finite input: the FP64 solve is
 * asynchronous and carries NaN / Inf through by IEEE arithmetic (qbvm_residual
 * then reports NONFINITE); the FP32_REFINE solve, which synchronises, returns
 * NONFINITE for NaN or Inf in g_or_F.  Errors: BAD_ARG (NULL arguments, mixed
 * host/device), DIVERGED (FP32_REFINE only; y holds the last iterate),
 * NONFINITE, CUDA. */
int qbvm_solve(qbvm_plan_t* plan, const double* g_or_F, double* y, int n0_only, void* stream);

/* qbvm_residual -- the relative all-at-once residual ||f - A y||_2 / ||f||_2
 * in FP64 (A applied as the stencil of eq. 3.3/3.6 without assembling it),
 * for y with all nt levels and f built from `g_or_F` as in qbvm_solve.
 * Synchronises `stream` and writes the scalar to *rel_norm_out (host).
 * Errors: BAD_ARG, NONFINITE (NaN or Inf in y or f: a sum of squares is not
 * finite), CUDA. */
int qbvm_residual(qbvm_plan_t* plan, const double* y, const double* g_or_F,
                  double* rel_norm_out, void* stream);

/* qbvm_plan_info -- copy the plan's derived values into *out. */
int qbvm_plan_info(const qbvm_plan_t* plan, qbvm_info* out);

/* Per-kernel timing (tracing).  While profiling is on, every kernel a plan
 * launches is bracketed by a pair of CUDA events recorded on the launching
 * stream; qbvm_profile_read synchronises on those events and returns, per
 * kernel name, the number of launches and their summed device time.
 * qbvm_profile_enable(plan, 1) turns it on and clears the record,
 * qbvm_profile_enable(plan, 0) turns it off.  capacity = entries of `out`;
 * *count receives the number filled.  Reading clears the record.
 * Errors: BAD_ARG, CUDA. */
typedef struct qbvm_kernel_stat {
    char      name[32];
    long long launches;
    double    total_ms;
} qbvm_kernel_stat;

int qbvm_profile_enable(qbvm_plan_t* plan, int on);
int qbvm_profile_read(qbvm_plan_t* plan, qbvm_kernel_stat* out, int capacity, int* count);

/* ------------------------------------------------------------------------
 * qbvm_measure_peak -- the fused multiply-add throughput of the current GPU,
 * measured: the ALU roofline against which the FP64 kernels of the solve are
 * rated (on GB300 they are bound by the FP64 pipe, not by HBM: the time
 * solve and the DST-I passes of Section 3.3 need tens of FP64 operations per
 * 16 bytes moved).  The paper has no counterpart; it reports no hardware
 * rates.
 * kind  QBVM_PEAK_FP64_FMA (DFMA) or QBVM_PEAK_FP32_FMA (FFMA).
 * A kernel of independent FMA chains (8 per thread, 32 warps per SM, every
 * SM) is launched six times on `stream`; the first launch is a warm-up and
 * the best of the other five, timed with CUDA events, is written to
 * *fma_per_s_out in FMA instructions per second (flops = 2x).  About 25 ms of
 * GPU time.  The call synchronises `stream`.  Allocates nothing but two
 * events.  Errors: BAD_ARG (unknown kind, NULL output), CUDA. */
#define QBVM_PEAK_FP64_FMA 0
#define QBVM_PEAK_FP32_FMA 1
int qbvm_measure_peak(int kind, double* fma_per_s_out, void* stream);

/* qbvm_residual_noalloc -- the value qbvm_residual returns, ||f - A y||_2 /
 * ||f||_2 in FP64, for callers that cannot allocate device memory: no plan is
 * needed and the call makes no cudaMalloc/cudaFree or other allocating call
 * (but see "Module loading" below for the first use of the library).
 * Such callers include code whose device memory is entirely reserved by
 * another allocator or memory pool (a framework's caching allocator holding
 * the HBM), and monitoring or real-time loops that must not change the
 * device-memory footprint or pay for cudaMalloc/cudaFree, which may
 * synchronise the device.  The paper has no counterpart to this entry point.
 *
 * `desc` is validated as in qbvm_plan (BAD_ARG / UNSUPPORTED alike); y and
 * g_or_F must be DEVICE pointers laid out as for qbvm_residual (host pointers
 * would need staging memory: BAD_ARG).  The result is written to
 * *rel_norm_out after `stream` has been synchronised.
 *
 * Scratch: a static device array of 8194 doubles (64 KiB) that every GPU
 * loading this library holds until the process exits: partial sums for at
 * most 4096 residual blocks plus two totals.  The residual kernel strides over
 * the unknowns, so the scratch need does not grow with the problem; a launch
 * that would need more than 4096 blocks is rejected with UNSUPPORTED.  All
 * calls on a device share the array and each call overwrites what it reads,
 * so nothing carries over between calls -- but calls that overlap on the GPU
 * (other streams, other host threads) race on it and must be serialised by
 * the caller.  Every call looks up the array's device address
 * (cudaGetSymbolAddress, with the caller's device current); the lookup
 * allocates nothing.  Module loading: under CUDA's default lazy loading the
 * library's device code, this array included, is loaded into a context the
 * first time one of its kernels or symbols is used there, and that load
 * reserves device memory for the code and the 64 KiB array.  A caller that
 * must not see that happen later should make the first call (on every
 * device, before any stream capture) at set-up, or run the process with
 * CUDA_MODULE_LOADING=EAGER so that the load happens when the context is
 * created.
 * y and g_or_F must be memory of the current device (or managed memory);
 * another GPU's pointer is BAD_ARG.
 * Errors: BAD_ARG, UNSUPPORTED, NONFINITE, CUDA. */
int qbvm_residual_noalloc(const qbvm_desc* desc, const double* y, const double* g_or_F,
                          double* rel_norm_out, void* stream);

/* ------------------------------------------------------------------------
 * Batched solve: `count` instances of ONE shape, each with its own alpha.
 * `desc` fixes everything but alpha (dim, m, L, T, nt, form, rhs_kind,
 * order, precision, refine_tol, refine_max_iters); `alphas` is a host array of `count`
 * values (NULL: desc's alpha, or its a-priori rule, for every instance), and
 * each alpha gives its instance's omega (-1/alpha for PinT-QBVM, -tau/alpha
 * for PinT-MQBVM, eqs. 3.3 / 3.6).  The instances are stored back to back in
 * device memory: g_or_F is [count][Nx] (delta right-hand side) or
 * [count][nt][Nx]; y is [count][nt][Nx], or [count][Nx] with n0_only.  Every
 * stage of Section 3.3 runs once over the whole batch -- the DST-I passes
 * over count*nt levels, the time solve over every (instance, mode tile) with
 * the instance's own omega tables -- so a batch costs the launches of one
 * solve, whatever `count` is.  Asynchronous on `stream`.
 * Supported: space-first order (2D/3D; 1D with m <= 2048), nt a power
 * of two <= 1024.  Device pointers (asynchronous), or host pointers (staged
 * through batch-owned device copies; the call then synchronises `stream`).
 * precision QBVM_FP32_REFINE: the refinement of the single plan over the
 * whole batch -- FP32 DST passes over count*nt levels, the FP32 time solve
 * with each instance's omega, one batched double-float residual with
 * per-instance norms per step -- until the LARGEST relative residual of the
 * batch is <= refine_tol (DIVERGED as for the single plan); the call then
 * synchronises `stream` after every residual.  Needs (m-1)^d * nt divisible
 * by 4.  Data FP32 cannot hold (root mean square of some instance's f outside
 * [1e-18, 1e28]) or NaN / Inf send the batch to the FP64 pipeline (NaN / Inf:
 * QBVM_ERR_NONFINITE after it).  qbvm_batch_refine_info reports the steps
 * and the largest relative residual of the last solve.
 * The batch owns its tables ([count][nt/2] omega factors and [count][nt/2][Nx]
 * Step (b) reciprocals; FP32_REFINE: their FP32 roundings, the FP32 work
 * array [count][nt][Nx] and per-instance norms) and a base plan.  Errors: BAD_ARG (count < 1, an
 * alpha not finite and positive, one host and one device pointer, memory of
 * a GPU other than the one the batch was planned on),
 * UNSUPPORTED, OOM, CUDA. */
typedef struct qbvm_batch qbvm_batch_t;
int qbvm_batch_plan(const qbvm_desc* desc, int count, const double* alphas, qbvm_batch_t** out);
int qbvm_solve_batched(qbvm_batch_t* batch, const double* g_or_F, double* y, int n0_only, void* stream);
/* alphas: host [count] (may be NULL); unknowns_per_instance = nt * Nx (may be NULL). */
int qbvm_batch_info(const qbvm_batch_t* batch, double* alphas, long long* unknowns_per_instance);
/* FP32_REFINE batches: refinement steps and the largest relative residual
 * ||f_b - A_b y_b|| / ||f_b|| over the instances after the last solve (NaN
 * after an FP64 fallback).  Either output may be NULL. */
int qbvm_batch_refine_info(const qbvm_batch_t* batch, int* iters, double* max_rel_residual);
/* FP32_REFINE batches: *fused = 1 when the batch runs the whole refinement
 * in one launch, 0 when it runs the staged passes above.  The one-launch
 * form takes 1D space-first batches with (m, nt) in {(64, 32), (64, 64),
 * (64, 128), (128, 32), (128, 64), (256, 32)}: one CTA per instance keeps the
 * instance's double-float iterate and FP32 work array in shared memory for
 * every step, and each instance stops on its own relative residual
 * (<= refine_tol, or DIVERGED as above);
 * refine_info then reports the most steps any instance took and the largest
 * final residual.  The call synchronises `stream` once, after the launch. */
int qbvm_batch_refine_fused(const qbvm_batch_t* batch, int* fused);
int qbvm_batch_destroy(qbvm_batch_t* batch);

/* ------------------------------------------------------------------------
 * Uneven batch of full solves: `count` instances of DIFFERENT shapes (dim,
 * m, nt), each with its own form, alpha, right-hand-side kind and arrays,
 * solved for every time level in ONE persistent kernel launch replayed from
 * a CUDA graph captured on the first run.  Each instance is planned as an
 * ordinary FP64 space-first plan (its tables of Section 3.3); the kernel then
 * runs the three steps of eq. 3.8 of every instance -- forward DST-I along
 * each axis, the time solve per tile of spatial modes (Steps (a)-(c)), the
 * inverse DST-I -- as one queue of tiles in which a stage of an instance
 * waits (bounded) for all tiles of the instance's previous stage.  Results
 * equal the single plans' (the same tiles).
 * Supported: FP64, space-first, nt a power of two in [2, 1024], every m a
 * power of two in [4, 2048].  g_or_F ([Nx] for the delta right-hand side,
 * else [nt][Nx]) and y ([nt][Nx]) are caller-owned DEVICE arrays of the
 * current device that must stay valid while the plan is used.
 * qbvm_multi_run enqueues one solve of every instance on `stream`
 * (asynchronous); qbvm_multi_check synchronises `stream` and returns
 * QBVM_ERR_TIMEOUT if a bounded wait inside the kernel gave up (then no
 * result is valid).  Errors: BAD_ARG, UNSUPPORTED, OOM, CUDA. */
typedef struct qbvm_multi_instance {
    qbvm_desc desc;              /* shape, form, alpha (or delta), rhs_kind; precision QBVM_FP64 */
    const double* g_or_F;        /* device input */
    double* y;                   /* device output [nt][Nx] */
} qbvm_multi_instance;
typedef struct qbvm_multi qbvm_multi_t;
int qbvm_multi_plan(const qbvm_multi_instance* inst, int count, qbvm_multi_t** out);
int qbvm_multi_run(qbvm_multi_t* multi, void* stream);
int qbvm_multi_check(qbvm_multi_t* multi, void* stream);
/* total unknowns (sum of nt * Nx), queue length and persistent grid; NULL outputs allowed */
int qbvm_multi_info(const qbvm_multi_t* multi, long long* unknowns, int* work_items, int* grid);
int qbvm_multi_destroy(qbvm_multi_t* multi);

/* ------------------------------------------------------------------------
 * Batched regularisation-parameter sweep.  Many PinT-QBVM / PinT-MQBVM
 * instances of uneven size (1D or 2D, delta right-hand side f^0 = -omega g/tau),
 * each solved for n_alpha values of alpha log-spaced around the a-priori rule
 * of Section 5 (alpha_rule = delta for PQ, tau*delta for PM) or around a
 * caller-given alpha_base:
 *     alpha_i = base * 10^(log10_lo + (log10_hi - log10_lo) i/(n_alpha-1)).
 * For every (instance, alpha) the sweep forms y^0 in the sine basis by the
 * three steps of eq. 3.8 (Step (c) evaluated at t = 0), the discrepancy
 * ||y^N - g||, which the first block row of eq. 3.3/3.6 gives as
 * alpha ||(I - tau Lap) y^0|| (PQ) or (alpha/tau) ||(I - tau Lap) y^0|| (PM),
 * and, when z0 is given, the error ||y^0 - z0|| (grid-weighted L2 norms).
 * It then picks alpha by the discrepancy principle -- the largest alpha with
 * ||y^N - g|| <= tau_dp * delta, else the one with the smallest discrepancy --
 * and writes y^0 at that alpha (FP64) to `y0` when given.
 * All of it runs as ONE persistent kernel launch, captured once into a CUDA
 * graph and replayed by every qbvm_sweep_run; its launch shape (modes per
 * thread, CTAs per SM) is picked by qbvm_sweep_autotune.
 * Supported: dim 1 or 2; m a power of two in [4, 2048]; nt a power of two in
 * [2, 1024]; n_alpha in [1, 64].  precision:
 *   QBVM_FP64: the DSTs in FP64; the spectral sums over the even frequencies
 *     (of the scan and of y^0 at the pick) in double-float arithmetic on the
 *     FP32 pipes, since this GPU's FP64 pipe issues under 2 operations per
 *     SM per clock against 128 FP32 ones: a mode's sum to about 6e-14 of the
 *     sum of its terms' magnitudes (FP64 summation: about 1e-16), so sums
 *     whose terms cancel keep fewer digits than in FP64; the discrepancies
 *     were within 3e-12 of the oracle's on 512 mixed instances.  Instances
 *     with |Re d_{2m}| above 2^30, or |Im d_{2m}| or tau Lambda outside
 *     [2^-30, 2^30], sum in FP64, each 1/|d_{2m} + tau Lambda_l|^2 from an
 *     FP32 seed and one third-order FP64 step x (1 + e + e^2), e = 1 - d x
 *     (a few units in the last place; qbvm_selftest_newton_rcp).
 *   QBVM_FP32_REFINE: the alpha scan in FP32; the picked alpha's y^0 summed in
 *     double-float, about 2^-44 per term; the DSTs in FP64.
 * The sweep holds device copies of its tables; g, z0 and y0 are caller-owned
 * device arrays that must stay valid while the sweep is used. */
typedef struct qbvm_sweep_instance {
    int    dim;
    int    m[3];
    double L;
    double T;
    int    nt;
    int    form;
    double delta;          /* noise level of g (bound of the discrepancy principle) */
    double alpha_base;     /* > 0: replaces the a-priori alpha_rule as the centre of the scan */
    const double* g;       /* device: g_delta, one level */
    const double* z0;      /* device, optional: true z(., 0) for the error report */
    double* y0;            /* device, optional: receives y^0 at the picked alpha */
} qbvm_sweep_instance;

typedef struct qbvm_sweep_desc {
    int    count;                       /* instances */
    const qbvm_sweep_instance* inst;    /* host array of `count` entries */
    int    n_alpha;
    double log10_lo, log10_hi;
    double tau_dp;                      /* e.g. 1.1 */
    int    precision;
} qbvm_sweep_desc;

typedef struct qbvm_sweep_config {
    int   modes_per_thread;   /* 1, 2 or 4 modes per thread in the alpha scan */
    int   ctas_per_sm;        /* 0 = every resident slot */
    int   grid;               /* resulting persistent grid (read only) */
    float ms;                 /* time of one run measured by the autotuner */
} qbvm_sweep_config;

typedef struct qbvm_sweep qbvm_sweep_t;

/* Validate and build a sweep (tables in FP64 on the host).  Errors: BAD_ARG,
 * UNSUPPORTED, OOM, CUDA. */
int qbvm_sweep_plan(const qbvm_sweep_desc* desc, qbvm_sweep_t** out);
/* Enqueue one run on `stream` (first call captures the CUDA graph). */
int qbvm_sweep_run(qbvm_sweep_t* sweep, void* stream);
/* Synchronise `stream` and copy results to host arrays (any may be NULL):
 * alphas, discrepancy, error: [count][n_alpha]; pick: [count][2] = (discrepancy
 * pick, smallest-error alpha; the latter only meaningful with z0).
 * TIMEOUT if a bounded wait inside the persistent kernel gave up. */
int qbvm_sweep_read(qbvm_sweep_t* sweep, double* alphas, double* discrepancy, double* error, int* pick,
                    void* stream);
/* Time every candidate launch shape `repeats` times on the actual batch and
 * keep the fastest; *best receives it (NULL accepted). */
int qbvm_sweep_autotune(qbvm_sweep_t* sweep, int repeats, qbvm_sweep_config* best, void* stream);
/* Set or read the launch shape (e.g. one cached from an earlier autotune). */
int qbvm_sweep_set_config(qbvm_sweep_t* sweep, const qbvm_sweep_config* cfg);
int qbvm_sweep_get_config(const qbvm_sweep_t* sweep, qbvm_sweep_config* cfg);
int qbvm_sweep_destroy(qbvm_sweep_t* sweep);
/* Diagnostic of the failure path above: `ctas` CTAs (1..64) of one kernel run
 * the sweep's bounded wait on a counter that nothing advances.  The wait gives
 * up after its spin limit (about half a second), raises the error flag, the
 * other CTAs see the flag and leave, and the kernel returns.  Returns
 * QBVM_ERR_TIMEOUT (what qbvm_sweep_read reports in that case) when every CTA
 * gave up and the flag was raised, QBVM_OK if a wait wrongly succeeded;
 * *seconds (may be NULL) receives the kernel's duration.  The context stays
 * usable afterwards. */
int qbvm_selftest_bounded_wait(int ctas, double* seconds, void* stream);
/* Diagnostic of the FP64 scan's reciprocal: for n positive FP64 values d
 * (device array), the largest relative difference between the reciprocal
 * the FP64 sweep uses (an FP32 seed and one third-order FP64 step) and the
 * IEEE quotient 1/d.  Synchronises `stream`. */
int qbvm_selftest_newton_rcp(const double* d, long long n, double* max_rel_diff, void* stream);

/* ------------------------------------------------------------------------
 * Learned regularisation parameter.  The paper picks alpha a priori
 * (Section 5); this network predicts t = log10(alpha / alpha_rule) from
 * spectrum features of g_delta and is trained on solves of the method itself
 * (labels: the alpha with the smallest reconstruction error in a sweep).
 *
 * Features (qbvm_features_*): for a 2D instance on (0,L)^2 with m intervals
 * per axis, 67 FP32 values: 64 bins of the radial sine spectrum of g_delta
 * (bin b = floor(64 |k| / (sqrt(2) m)) over modes k = (k_x, k_y), value
 * log10 of the mean squared sine-series coefficient in the bin), then
 * log10 delta, T and log2 nt; the bin values are log10(mean square +
 * 1e-30).  The FP32 spectrum is taken of g 2^k, 2^k the power of two nearest
 * 1/delta, and the bins corrected by the exact 2^-2k, so data of any magnitude
 * FP64 holds gives its own features.  g is a device array [B][m-1][m-1]
 * (FP64), delta a host array of B values, feats a device array [B][67].
 *
 * Network (qbvm_mlp_*): x -> relu(W1 x' + b1) -> relu(W2 h1 + b2) -> w3.h2 + b3,
 * x' = (x - mean)/sd (qbvm_mlp_set_norm), bfloat16 weights in the products,
 * FP32 accumulation and FP32 master weights; loss (1/2B) sum (y - t)^2;
 * Adam (beta 0.9/0.999, eps 1e-8).  Flat parameter order: W1 [width][in],
 * b1 [width], W2 [width][width], b2 [width], w3 [width], b3 [1].
 * x, t, y are device FP32 arrays; grads (qbvm_mlp_gradients) a host array of
 * qbvm_mlp_num_params values, loss_out a host double. */
typedef struct qbvm_mlp qbvm_mlp_t;
typedef struct qbvm_features qbvm_features_t;

int qbvm_mlp_create(int in_dim, int width, int max_batch, unsigned long long seed, qbvm_mlp_t** out);
long long qbvm_mlp_num_params(const qbvm_mlp_t* mlp);
int qbvm_mlp_set_norm(qbvm_mlp_t* mlp, const float* mean, const float* sd);
int qbvm_mlp_get_params(const qbvm_mlp_t* mlp, float* params, float* adam_m, float* adam_v, long long* step);
int qbvm_mlp_set_params(qbvm_mlp_t* mlp, const float* params, const float* adam_m, const float* adam_v,
                        long long step);
int qbvm_mlp_forward(qbvm_mlp_t* mlp, const float* x, int batch, float* y, void* stream);
int qbvm_mlp_gradients(qbvm_mlp_t* mlp, const float* x, const float* t, int batch, float* grads,
                       double* loss_out, void* stream);
int qbvm_mlp_train_step(qbvm_mlp_t* mlp, const float* x, const float* t, int batch, float lr, void* stream);
int qbvm_mlp_last_loss(qbvm_mlp_t* mlp, double* loss, void* stream);
int qbvm_mlp_destroy(qbvm_mlp_t* mlp);

int qbvm_features_plan(int m, double T, int nt, int max_batch, qbvm_features_t** out);
int qbvm_features_run(qbvm_features_t* feats_plan, const double* g, const double* delta_host, int batch,
                      float* feats, void* stream);
int qbvm_features_destroy(qbvm_features_t* feats_plan);

/* ------------------------------------------------------------------------
 * The original QBVM / MQBVM systems (Section 2) by Krylov iteration with the
 * PinT solve as preconditioner.  The paper solves them only by sparse direct
 * LU and proposes the diagonalization-based PinT direct solver as a
 * preconditioner for Krylov methods (Sections 2 and 6); this is that use.
 *
 * The systems (f = (g, 0, ..., 0), backward Euler rows for n >= 1 as in the
 * PinT systems, first block row):
 *   QBVM_ORIGINAL_QBVM  (A_h, eq. 2.3):  alpha y^0 + y^N = g;
 *   QBVM_ORIGINAL_MQBVM (B_h, eq. 2.6):  (alpha/tau)(y^0 - y^1) + y^N = g.
 * With the first block row of the PinT system scaled by tau*alpha (PQ) or
 * alpha (PM) it reads alpha (I - tau Delta_h) y^0 + y^N = g or
 * alpha (I/tau - Delta_h) y^0 + y^N = g, so the PinT operator differs from
 * A_h / B_h in one block row only.  The iteration is flexible
 * right-preconditioned GMRES(restart): each preconditioner application scales
 * block 0 by 1/(tau alpha) (QBVM) or 1/alpha (MQBVM) and calls qbvm_solve;
 * orthogonalisation is classical Gram-Schmidt applied twice.
 *
 * qbvm_gmres_create -- `plan` must be FP64, rhs_kind GENERAL and of the form
 *   matching `method` (PQ for QBVM, PM for MQBVM); the handle borrows it (keep
 *   it alive) and allocates (2 restart + 4) vectors of nt*N_x doubles.
 *   restart in [1, 64].  Errors: BAD_ARG, UNSUPPORTED, OOM.
 * qbvm_gmres_solve -- device pointers g (N_x values) and y (nt*N_x values,
 *   output; the initial guess is zero).  Stops when ||f - A y||/||f|| <= tol
 *   (the true residual, recomputed at the end) or after max_iters inner
 *   iterations, or when a whole restart cycle lowers the true residual by less
 *   than 10 % (its FP64 floor lies above tol: the original systems are far
 *   worse conditioned than the PinT ones); *iters and *rel_residual report
 *   (either may be NULL).
 *   Synchronises `stream` once per iteration (the Hessenberg update runs on
 *   the host).  Errors: BAD_ARG, DIVERGED (max_iters reached above tol; y holds
 *   the last iterate), NONFINITE, CUDA. */
#define QBVM_ORIGINAL_QBVM  0
#define QBVM_ORIGINAL_MQBVM 1
typedef struct qbvm_gmres qbvm_gmres_t;
int qbvm_gmres_create(qbvm_plan_t* plan, int method, int restart, qbvm_gmres_t** out);
int qbvm_gmres_solve(qbvm_gmres_t* gm, const double* g, double* y, double tol, int max_iters, int* iters,
                     double* rel_residual, void* stream);
int qbvm_gmres_destroy(qbvm_gmres_t* gm);

/* qbvm_destroy -- free the plan and everything it owns (NULL is accepted). */
int qbvm_destroy(qbvm_plan_t* plan);

/* qbvm_strerror -- a static message for a status code. */
const char* qbvm_strerror(int code);

/* qbvm_version -- ABI version of this header (major*100 + minor). */
int qbvm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QBVM_H */
