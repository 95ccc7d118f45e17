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
 *    synchronises `stream`).  Input and output may not be a mix of the two.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  A plan may be
 *    used by one stream at a time; calls on one plan must not overlap.
 *  - The caller owns every array it passes; the plan owns its device tables
 *    and workspace and frees them in qbvm_destroy.
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
#define QBVM_ERR_DIVERGED    -4   /* FP32 refinement did not contract          */
#define QBVM_ERR_TIMEOUT     -5   /* a bounded device wait gave up             */
#define QBVM_ERR_CUDA        -6   /* a CUDA runtime call failed                */
#define QBVM_ERR_UNSUPPORTED -7   /* size outside what the kernels implement   */

/* ------------------------------------------------------------ enumerations */
#define QBVM_FORM_PQ 0            /* PinT-QBVM,  Section 3.1                    */
#define QBVM_FORM_PM 1            /* PinT-MQBVM, Section 3.2                    */

#define QBVM_FP64        0        /* every stage in FP64                        */
#define QBVM_FP32_REFINE 1        /* FP32 transforms, FP64 scaling tables, FP64
                                     residual and update: iterative refinement */

#define QBVM_RHS_DELTA   0        /* input is g (one level): f^0 = -omega g/tau */
#define QBVM_RHS_GENERAL 1        /* input is a full right-hand side F [nt][..] */

/* ------------------------------------------------------------ descriptor
 * dim     space dimension d = 1, 2 or 3.
 * m[3]    intervals per axis (x, y, z); m[d] >= 2; entries beyond dim ignored.
 *         Supported: 1D any m with m-1 <= 2^20; 2D/3D m a power of two in
 *         [4, 1024] (the DST-I length m-1 is then 2^k - 1).
 * L       side length of the domain (0, L)^d; h = L/m[d].
 * T       final time, > 0.
 * nt      time levels N_t, a power of two in [2, 1024].
 * form    QBVM_FORM_PQ or QBVM_FORM_PM.
 * alpha   regularisation parameter > 0, or <= 0 for the a-priori rule of
 *         Section 5 from `delta`: alpha = delta (PQ), alpha = tau*delta (PM).
 * delta   noise level (only read when alpha <= 0; must then be > 0).
 * precision  QBVM_FP64 or QBVM_FP32_REFINE.
 * rhs_kind   QBVM_RHS_DELTA or QBVM_RHS_GENERAL.
 * refine_tol       FP32_REFINE: stop when ||f - A y||/||f|| <= refine_tol
 *                  (<= 0 selects 1e-12).
 * refine_max_iters FP32_REFINE: iteration cap (<= 0 selects 10).
 */
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
 * rhs_kind GENERAL.  Errors: BAD_ARG (NULL arguments, mixed host/device),
 * DIVERGED (FP32_REFINE only; y holds the last iterate), CUDA. */
int qbvm_solve(qbvm_plan_t* plan, const double* g_or_F, double* y, int n0_only, void* stream);

/* qbvm_residual -- the relative all-at-once residual ||f - A y||_2 / ||f||_2
 * in FP64 (A applied as the stencil of eq. 3.3/3.6 without assembling it),
 * for y with all nt levels and f built from `g_or_F` as in qbvm_solve.
 * Synchronises `stream` and writes the scalar to *rel_norm_out (host).
 * Errors: BAD_ARG, CUDA. */
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

/* qbvm_residual_noalloc -- the value qbvm_residual returns, ||f - A y||_2 /
 * ||f||_2 in FP64, for callers that cannot allocate device memory: no plan is
 * needed and the call makes no cudaMalloc/cudaFree or other allocating call.
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
 * the caller.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current) and caches it;
 * make that first call before any stream capture.
 * Errors: BAD_ARG, UNSUPPORTED, NONFINITE, CUDA. */
int qbvm_residual_noalloc(const qbvm_desc* desc, const double* y, const double* g_or_F,
                          double* rel_norm_out, void* stream);

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
