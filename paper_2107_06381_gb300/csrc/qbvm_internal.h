// qbvm_internal.h -- host-side declarations shared by the plan code and the
// kernel translation units (launch wrappers; no CUDA types beyond streams).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace qbvm {

// Columns of one shared-memory tile: TILE_ELEMS complex values per CTA.
constexpr int TILE_ELEMS = 4096;
constexpr int TILE_THREADS = 256;

// Device tables of a plan (all FP64; FP32 copies where a kernel reads them in FP32).
struct Tables {
    int nt = 0, lnt = 0;             // time levels, log2
    int dim = 0;
    int sf = 0;                      // space-first order (DST, per-mode time solve, inverse DST)
    int n[3] = {1, 1, 1};            // interior points per axis (x, y, z)
    int lpd[3] = {0, 0, 0};          // log2(M_d) = log2(n_d + 1), the DST FFT length
    long long Nx = 0;                // spatial unknowns per level
    double tau = 0, omega = 0;
    double rho_h = 1, rho_hinv = 1;  // |omega|^{1/2} = rho^{nt/2} and its inverse
    double2* tw_t = nullptr;         // exp(-2 pi i m / H), m < H = nt/2
    float2*  tw_t32 = nullptr;
    double2* tw_s[3] = {nullptr, nullptr, nullptr};   // exp(-2 pi i m / M_d), m < M_d
    float2*  tw_s32[3] = {nullptr, nullptr, nullptr};
    double*  sn_s[3] = {nullptr, nullptr, nullptr};   // sin(j pi / M_d), j = 0..M_d/2
    float*   sn_s32[3] = {nullptr, nullptr, nullptr};
    double2* gpow = nullptr;         // scale * gamma^t (t < H), gamma = omega^{1/nt} principal
    double2* gipw = nullptr;         // 2 gamma^{-t} (t < H)
    double2* gpowr = nullptr;        // i rho^H gpow[t]: the second half's scaling, folded
    double2* gipr = nullptr;         // rho^{-H} gipw[t]: the second half's unscaling, folded
    double2* ak = nullptr;           // d_{2m} = 1 - gamma theta^{2m}, m < H (eigenvalues of C_omega)
    double*  lamtau = nullptr;       // tau * Lambda_l for every spatial mode (2D/3D)
    float2*  gpow32 = nullptr;       // FP32 roundings of gpow, gipw, ak, lamtau
    float2*  gipw32 = nullptr;
    float2*  gpowr32 = nullptr;
    float2*  gipr32 = nullptr;
    float2*  ak32 = nullptr;
    float*   lamtau32 = nullptr;
    double2* bk = nullptr;           // 1D Thomas diagonal for frequency 2m: h^2 d_{2m} / tau + 2
    double2* qinv = nullptr;         // FP64 2D/3D: cnorm / (d_{2m} + tau Lambda_l), [H][Nx]
    double*  y0fac = nullptr;        // FP64 delta rhs: y^0_l = y0fac[l] * (DST g)_l (Step (c) at t = 0)
    // general nt (not a power of two): Bluestein tables, every frequency k < nt
    int gen = 0;                     // 1: the time DFTs use k_bluestein
    int lL = 0;                      // log2 L, L >= 2 nt - 1
    double2* tw_L = nullptr;         // exp(-2 pi i m / L), m < L
    double2* chirp = nullptr;        // exp(i pi m^2 / nt), m < nt
    double2* bs_fwd = nullptr;       // FFT_L of conj(chirp) wrapped, / L (for the +theta transform)
    double2* bs_inv = nullptr;       // FFT_L of chirp wrapped, / L (for the -theta transform)
    double2* gpw_full = nullptr;     // scale * gamma^t, t < nt
    double2* gip_full = nullptr;     // gamma^{-t}, t < nt
    double2* dk_full = nullptr;      // d_k = 1 - gamma theta^k, k < nt
    float2 *tw_L32 = nullptr, *chirp32 = nullptr, *bs_fwd32 = nullptr, *bs_inv32 = nullptr;   // FP32 roundings
    float2 *gpw_full32 = nullptr, *gip_full32 = nullptr, *dk_full32 = nullptr;
};

// DST-I (unnormalised, S_{jk} = sin(pi j k /(n+1))) along one axis of an
// array viewed as [outer][n][inner], in place allowed (in == out).
// lm = log2(n + 1); tw = roots of length n+1, sn = sin(j pi/(n+1)) tables of
// precision R.  TIN: element type read.  OMODE: 0 store R, 1 accumulate into
// a double-float (float2 hi, lo) array, 2 store into a double-float array.
// X4: the output is 4 times the DST (two operations fewer per element).
template <typename R, typename TIN, int OMODE, bool X4 = false>
cudaError_t launch_dst(const TIN* in, void* out, int n, int lm, long long outer, long long inner,
                       const void* tw, const void* sn, cudaStream_t s);

// Space-first time solve: per spatial mode l (column), scale by gamma^t, FFT
// (theta^{+kt}), divide by (d_k + tau Lambda_l)/cnorm, inverse FFT, unscale by
// gamma^{-t}, real part.  in/out are [nt][Nx]; delta_rhs reads only level 0.
template <typename R>
cudaError_t launch_time_solve(const R* in, R* out, const Tables& tb, double cnorm, int delta_rhs,
                              int n0_only, cudaStream_t s);

// The FP64 time solve of `count` same-shape instances stored back to back
// (instance b: in + b in_stride -> out + b out_stride), each with its own
// omega tables gpow, gipw, gpowr, gipr ([count][nt/2]) and Step (b)
// reciprocals qinv ([count][nt/2][Nx], the constant cnorm folded in); the
// shape tables (time roots, Nx, nt) are tb's.  Power-of-two nt.
cudaError_t launch_time_solve_batched(const double* in, double* out, const Tables& tb, long long count,
                                      long long in_stride, long long out_stride, const double2* gpow,
                                      const double2* gipw, const double2* gpowr, const double2* gipr,
                                      const double2* qinv, int delta_rhs, int n0_only, cudaStream_t s);

// y0fac[l] = Re sum over the formed frequencies of cnorm / (d_k + tau Lambda_l)
// (x2 for the half spectrum of a power-of-two nt): with the delta right-hand
// side the forward time transform is the constant f^0, so Step (c) at t = 0
// is this factor times the mode's coefficient.  Power-of-two nt: from tb.qinv;
// other nt: direct FP64 divisions over every frequency.
cudaError_t launch_make_y0fac(const Tables& tb, double cnorm, double* out, cudaStream_t s);
// Per-instance FP32 omega tables of a batch: gpow, gipw, gpowr, gipr, ak are
// [count][H] (the FP64 tables rounded once), cnorm, rho_h = |omega|^{1/2},
// rho_hinv [count].
struct BatchTables32 {
    const float2 *gpow = nullptr, *gipw = nullptr, *gpowr = nullptr, *gipr = nullptr, *ak = nullptr;
    const float *cnorm = nullptr, *rho_h = nullptr, *rho_hinv = nullptr;
};
// The FP32 time solve of `count` instances (Step (a)-(c) in the sine basis,
// each with its own omega); instance b reads in + b in_stride, writes
// out + b out_stride.
cudaError_t launch_time_solve_batched32(const float* in, float* out, const Tables& tb, long long count,
                                        long long in_stride, long long out_stride, const BatchTables32& bt,
                                        int delta_rhs, int n0_only, cudaStream_t s);
// Double-float residual of `count` instances stored back to back ([count][nt][Nx]
// y and r, f [count][nt][Nx] or [count][Nx] for the delta right-hand side),
// instance b with omega_b as a double-float pair omega_df[b] and in FP64
// omega64[b]; sums[2 b], sums[2 b + 1] receive ||r_b||^2 and (fnorm) ||f_b||^2.
// partials: 2 * count * bpi doubles, bpi <= residual_blocks_per_instance(tb).
// Requires nt * Nx divisible by 4 and 16-byte aligned y, r (and f, general).
cudaError_t launch_residual_df_batched(const void* y_df, const double* f, int delta_rhs, const Tables& tb,
                                       const double h2inv[3], long long count, const float2* omega_df,
                                       const double* omega64, float* r_out, double* partials, double* sums,
                                       int fnorm, int bpi, cudaStream_t s);
int residual_blocks_per_instance(const Tables& tb);

// FP32 + double-float refinement of `count` 1D instances of one shape in one
// launch (qbvm_refine1d.cu): one CTA per instance holds its iterate and work
// array in shared memory for the whole loop and stops on its own residual.
// f: [count][n] (delta: g) or [count][nt][n]; y: [count][nt][n] or
// [count][n] (n0_only).  Per-instance tables as BatchTables32 (the general
// cnorm), omega as a double-float pair and in FP64; ct = 1/tau and
// cx = 1/h^2 as double-float pairs.  Outputs per instance: refinement steps,
// final relative residual and a status (0 ok, 1 NaN / Inf in f, 2 f outside
// the FP32 range, 3 no contraction above 1e-10 or the step cap, 4 NaN / Inf
// residual); instances with status 1 or 2 write no y.
enum Refine1dStatus : int { R1_OK = 0, R1_NONFINITE_IN = 1, R1_RANGE = 2, R1_DIVERGED = 3, R1_NONFINITE = 4 };
struct Refine1dArgs {
    const double* f = nullptr;
    double* y = nullptr;
    int delta = 0, n0_only = 0;
    const float2* tws = nullptr;   // DST roots exp(-2 pi i m / M), m < M
    const float* sns = nullptr;    // sin(j pi / M), j <= M/2
    const float2* twt = nullptr;   // time roots exp(-2 pi i m / H), m < H
    const float* lamtau = nullptr; // tau Lambda_l, l < n
    const float2 *gpow = nullptr, *gipw = nullptr, *ak = nullptr;       // [count][H]
    const float *cnorm = nullptr, *rho_h = nullptr, *rho_hinv = nullptr; // [count]
    const float2* omega_df = nullptr;
    const double* omega64 = nullptr;
    float2 ct{}, cx{};
    double inv_tau = 0, tol = 0;
    int maxit = 0;
    int* iters = nullptr;
    double* rel = nullptr;
    int* status = nullptr;
};
// 1 when the fused kernel takes tb's shape (1D space-first, power-of-two nt,
// (m, nt) in {(64, 32), (64, 64), (64, 128), (128, 32), (128, 64), (256, 32)}, within
// the device's shared memory).
int refine1d_supported(const Tables& tb);
cudaError_t launch_refine1d(const Tables& tb, long long count, const Refine1dArgs& a, cudaStream_t s);
// y[l] = fac[l] * x[l], l < n
cudaError_t launch_mul_modes(const double* x, const double* fac, double* y, long long n, cudaStream_t s);

// Time DFTs of length nt for a general nt (tb.gen): mode 0 = Step (a) + the
// divide of Step (b) (real [nt][N] in, complex out), 1 = Step (a) only (1D),
// 2 = Step (c) (complex in, real out).  N columns, in place not allowed.
cudaError_t launch_bluestein(int mode, const void* in, void* out, long long N, const Tables& tb, double cnorm,
                             int delta_rhs, int n0_only, cudaStream_t s);
// The same three modes in FP32 (the FP32 roundings of the tables; in and out
// FP32 / complex FP32): the FP32 solve of the refinement for nt not a power of two.
cudaError_t launch_bluestein32(int mode, const void* in, void* out, long long N, const Tables& tb, float cnorm,
                               int delta_rhs, int n0_only, cudaStream_t s);
cudaError_t launch_thomas_1d_n(double2* wk, double2* cp, int nsys, const Tables& tb, cudaStream_t s);

// tb.qinv[m][l] = cnorm / (d_{2m} + tau Lambda_l) (IEEE FP64 division), built
// once per plan so that Step (b) of the FP64 time solve is one complex product.
cudaError_t launch_make_qinv(const Tables& tb, double cnorm, double2* q, cudaStream_t s);

// 1D time-first path (Section 3.3 order): forward time transform to complex
// workspace, Thomas per frequency, inverse transform.
cudaError_t launch_time_fwd_1d(const double* in, double2* wk, const Tables& tb, int delta_rhs, double in_scale,
                               cudaStream_t s);
cudaError_t launch_thomas_1d(double2* wk, double2* cp, const Tables& tb, cudaStream_t s);
cudaError_t launch_time_inv_1d(const double2* wk, double* out, const Tables& tb, int n0_only, cudaStream_t s);

// FP64 residual r = f - A y (eq. 3.3/3.6 stencil); per-block partial sums of
// r^2 and f^2 into partials[2*blocks], then reduced into sums[2].
// Optionally writes r (FP64) to r_out.
cudaError_t launch_residual(const double* y, const double* f, int delta_rhs, const Tables& tb,
                            const double h2inv[3], double* partials, int nblocks, double* sums,
                            double* r_out, cudaStream_t s);
int residual_blocks(const Tables& tb);
// flags[0] = 1 if x[0..n) holds a NaN or an infinity, flags[1] = 1 if any
// value is nonzero (two device ints).
cudaError_t launch_classify(const double* x, long long n, int* flags, cudaStream_t s);

// Double-float residual of the refinement: y_df is a (hi, lo) float2 array,
// f FP64 (F, or g for the delta right-hand side); writes r.hi (FP32) to r_out
// and sums[2] = (||r||^2, ||f||^2).
// fnorm: also sum ||f||^2 (sums[1]); otherwise sums[1] is not meaningful.
// rscale > 0 (with fnorm 0; 2D / 3D): ||r||^2 summed as an FP32 sum of
// (r rscale)^2, rscale a power of two near 1 / rms(f) (+Inf when that sum
// overflows, i.e. r beyond ~1e19 rms(f)).
cudaError_t launch_residual_df(const void* y_df, const double* f, int delta_rhs, const Tables& tb,
                               const double h2inv[3], float* r_out, double* partials, int nblocks, double* sums,
                               int fnorm, cudaStream_t s, float rscale = 0.f);
// In place: double-float (float2) array of n values -> FP64 array.
cudaError_t launch_df_to_double(void* buf, long long n, cudaStream_t s);

}  // namespace qbvm

namespace qbvm {
// Shared-memory bytes of one DST tile of length M = 2^lm in precision R, and
// the tile width log2(W) (2W real columns per tile).
template <typename R>
size_t dst_smem_bytes(int lm);
int dst_tile_lw(int lm);
}  // namespace qbvm

struct qbvm_desc;
struct qbvm_plan;
namespace qbvm {
// The descriptor checks of qbvm_plan (status code; needs no GPU).
int validate_desc(const qbvm_desc* d);
// The FP64 space-first time-solve constant without its right-hand-side
// factor: prod_d 2/(n_d + 1) (inverse DST-I) / nt (inverse DFT) / 4^dim per
// forward-inverse DST pair (the 4x transform).
double time_cn(const Tables& tb);
// Read access to a plan's descriptor and tables for the other translation
// units (the plan type itself is private to qbvm_plan.cu).
struct PlanView {
    const Tables* tb;
    int form, precision, rhs_kind, dim;
    int dev;                       // the device the plan was made on (its tables live there)
    double alpha, tau, h2inv[3];
    double* ghat;                  // FP64 space-first plans: one level of workspace (the DST of g)
};
int plan_view(const struct ::qbvm_plan* p, PlanView* out);

}  // namespace qbvm
