// qbvm_sweep.cu -- batched regularisation-parameter sweep: many PinT-QBVM /
// PinT-MQBVM instances of uneven size, each solved for a set of alpha values,
// in ONE persistent kernel launch replayed from a captured CUDA graph.
//
// Per instance (delta right-hand side f^0 = -omega g/tau, Sections 3.1/3.2):
//   A  forward DST-I of g (and of z0 when given) along each axis, FP64;
//   B  for every alpha and every spatial mode l, the t = 0 output of the
//      three steps of eq. 3.8 in the sine basis: the forward time transform of
//      a delta is constant over the even frequencies 2m, Step (b) divides by
//      d_{2m} + tau Lambda_l, and Step (c) at t = 0 sums over them:
//          yhat0_l = 2 cnorm ghat_l  sum_m Re 1/(d_{2m} + tau Lambda_l);
//      the discrepancy ||y^N - g|| follows from the first block row of
//      eq. 3.3/3.6, y^N - g = -c_alpha (I - tau Lap) y^0 with c = alpha (PQ) or
//      alpha/tau (PM), and ||S v|| = prod(M/2)^{1/2} ||v|| (Parseval for DST-I);
//   C  pick alpha by the discrepancy principle: the largest alpha with
//      ||y^N - g|| <= tau_dp * delta (else the smallest discrepancy);
//   D-F  y^0 at the picked alpha in FP64: the spectral values, then the
//      inverse DST along y and x.
// Stage B runs in FP32 for the FP32 sweep; for the FP64 sweep its sums, and
// those of stage D, run in double-float on the FP32 pipes (FP64 where the
// instance's tables leave FP32's comfortable range); A and E-F in FP64.
//
// Work items are queued in topological order and claimed with an atomic
// ticket; an item whose inputs come from earlier stages waits on per-instance
// counters.  Every CTA of the grid is resident (the grid is sized from the
// occupancy calculator), so every item a CTA waits for is held by a running
// CTA; the waits are bounded anyway and give up with an error flag.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "qbvm.h"
#include "qbvm_dfsum.cuh"
#include "qbvm_dst.cuh"
#include "qbvm_internal.h"

namespace {

using qbvm::cplx;

enum Stage { ST_GX = 0, ST_GY, ST_ZX, ST_ZY, ST_SPEC, ST_PICK, ST_FIN, ST_IY, ST_IX, NSTAGE };

constexpr int SW_THREADS = qbvm::TILE_THREADS;
constexpr long long SPIN_LIMIT = 1ll << 22;      // bounded waits (~0.5 s with the back-off)

struct SwInst {
    int dim, nx, ny, H, lmx, lmy, n_alpha, form;
    long long Nx;
    int tiles_gx, tiles_gy, tiles_spec, tiles_fin, tiles_iy, tiles_ix;
    int has_z0, has_y0;
    int df_sums;                 // FP64 sweep: the spectral sums of stages B and D in
                                 // double-float (tables inside [2^-30, 2^30]), else FP64
    double delta, tau_dp, tau, wnorm, zscale;
    double sscale, sinv;         // 2^-floor(log2 delta) and its inverse: the scan runs on
                                 // g, z0 scaled so that delta ~ 1 (exact; any data scale)
    const double* g;
    const double* z0;
    double* y0;
    double* ghat;
    double* zhat;
    double* yhat;
    const double* lamx;          // tau * lambda_x (nx)
    const double* lamy;          // tau * lambda_y (ny), 2D
    const double2* dtab;         // n_alpha x H: d_{2m}(alpha)
    const float2* dtab32;
    const float4* dtabdf;        // the same as double-float pairs (re.hi, re.lo, im.hi, im.lo)
    const double* cn;            // n_alpha: 2 * cnorm(alpha)
    const double* coef;          // n_alpha: alpha (PQ) or alpha / tau (PM)
    const double* alphas;        // n_alpha
    const double2* twx;
    const double2* twy;
    const double* snx;
    const double* sny;
    double* stats;               // n_alpha x 2: sum ((1 + tau Lambda) yhat)^2, sum (yhat - zhat)^2
    double* disc;                // n_alpha outputs
    double* err;                 // n_alpha outputs (when z0 is given)
    int* pick;                   // [0] discrepancy pick, [1] smallest-error alpha
};

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Thread 0 waits until counters[c] >= target; all threads learn the outcome.
__device__ bool wait_for(const int* counter, int target, int* errflag) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        long long it = 0;
        int good = 1;
        while (ld_volatile(counter) < target) {
            if (ld_volatile(errflag) != 0 || ++it > SPIN_LIMIT) {
                good = 0;
                atomicCAS(errflag, 0, 1);
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    int r = ok;
    __syncthreads();
    return r != 0;
}

__device__ double block_sum_d(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (threadIdx.x < (blockDim.x >> 5)) v = sh[threadIdx.x];
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// 1/d for a positive normal FP64 d, from an FP32 seed and one third-order
// FP64 step of the Newton-type iteration for f(x) = 1/x - d: with
// e = 1 - d x, x' = x (1 + e + e^2) has 1 - d x' = e^3 (the Newton step
// x (1 + e) squares e; one more term of the series cubes it).  The seed is the
// approximate FP32 reciprocal of d truncated to FP32 -- the exponent rebased
// and the top 23 significand bits kept, on the integer pipes -- widened back
// to FP64 exactly from its bits: relative error below 2^-21, so the step leaves
// the rounding of its last fused multiply-adds (a few units in the last
// place).  Three FP64 operations instead of a division (two Newton steps took
// four); d outside FP32's normal range (never for the scan's
// |d_{2m} + tau Lambda|^2) takes the division.
__device__ __forceinline__ double rcp_newton(double d) {
    const unsigned int H = (unsigned int)__double2hiint(d);
    const int fe = (int)((H >> 20) & 0x7FFu) - 1023 + 127;
    if (fe < 2 || fe > 252 || (H >> 31)) return 1.0 / d;
    const float f = __uint_as_float(((unsigned int)fe << 23) | ((H & 0xFFFFFu) << 3) |
                                    ((unsigned int)__double2loint(d) >> 29));
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));
    const unsigned int rb = __float_as_uint(r);
    double x = __hiloint2double((int)((((rb >> 23) & 0xFFu) + 896u) << 20 | ((rb & 0x7FFFFFu) >> 3)), (int)(rb << 29));
    // one third-order step: with e = 1 - d x, x (1 + e + e^2) leaves 1 - d x' = e^3
    // (below 2^-63) and the roundings of the last two fused multiply-adds
    const double e = fma(-d, x, 1.0);
    return fma(x, fma(e, e, e), x);
}

// Diagnostic: the largest relative difference of rcp_newton from the IEEE
// quotient 1/d over n values (one FP64 atomic max through its bits: the
// values are positive).
__global__ void k_rcp_check(const double* d, long long n, unsigned long long* maxbits) {
    double worst = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double q = __drcp_rn(d[i]);
        const double a = rcp_newton(d[i]);
        worst = fmax(worst, fabs(a - q) / fabs(q));
    }
    atomicMax(maxbits, (unsigned long long)__double_as_longlong(worst));
}

// Stage B: one tile of SW_THREADS * MPT modes, every alpha, precision R.
template <typename R, int MPT>
__device__ void spectral_tile(const SwInst& I, int tile, unsigned char* smem) {
    using C = cplx<R>;
    __shared__ double sh[32];
    C* sd = reinterpret_cast<C*>(smem);
    const C* dt = reinterpret_cast<const C*>(std::is_same<R, double>::value ? (const void*)I.dtab
                                                                           : (const void*)I.dtab32);
    R lam[MPT], gh[MPT], zh[MPT];
    bool valid[MPT];
#pragma unroll
    for (int q = 0; q < MPT; ++q) {
        long long l = (long long)tile * SW_THREADS * MPT + q * SW_THREADS + threadIdx.x;
        valid[q] = l < I.Nx;
        lam[q] = gh[q] = zh[q] = R(0);
        if (valid[q]) {
            int lx = (int)(l % I.nx), ly = (int)(l / I.nx);
            double lt = __ldcg(I.lamx + lx) + (I.dim == 2 ? __ldcg(I.lamy + ly) : 0.0);
            lam[q] = R(lt);
            gh[q] = R(__ldcg(I.ghat + l) * I.sscale);
            if (I.has_z0) zh[q] = R(__ldcg(I.zhat + l) * I.zscale * I.sscale);
        }
    }
    for (int a = 0; a < I.n_alpha; ++a) {
        __syncthreads();
        for (int m = threadIdx.x; m < I.H; m += blockDim.x) sd[m] = dt[(long long)a * I.H + m];
        __syncthreads();
        R s[MPT];
#pragma unroll
        for (int q = 0; q < MPT; ++q) s[q] = R(0);
        for (int m = 0; m < I.H; ++m) {
            C d = sd[m];
#pragma unroll
            for (int q = 0; q < MPT; ++q) {
                R zr = d.x + lam[q];
                if (std::is_same<R, float>::value)      // the FP32 scan: the 2-ulp fast division
                    s[q] += __fdividef((float)zr, fmaf((float)zr, (float)zr, (float)(d.y * d.y)));
                else                                    // FP64: third-order reciprocal (3 FP64 operations)
                    s[q] = fma((double)zr, rcp_newton(fma((double)zr, (double)zr, (double)(d.y * d.y))), (double)s[q]);
            }
        }
        const R cna = R(I.cn[a]);
        // the thread's squares in its own precision (the FP32 scan's values are of
        // the data scaled to about 1/delta), widened once for the block sum: FP64
        // conversions and adds per term had kept the FP64 pipe a third busy in the
        // FP32 scan
        R ds = R(0), es = R(0);
#pragma unroll
        for (int q = 0; q < MPT; ++q) {
            if (!valid[q]) continue;
            R y = cna * gh[q] * s[q];
            R dv = (R(1) + lam[q]) * y;
            ds = fma(dv, dv, ds);
            if (I.has_z0) {
                R e = y - zh[q];
                es = fma(e, e, es);
            }
        }
        double dsum = (double)ds, esum = (double)es;
        dsum = block_sum_d(dsum, sh);
        esum = block_sum_d(esum, sh);
        if (threadIdx.x == 0) {
            atomicAdd(I.stats + 2 * a, dsum);
            if (I.has_z0) atomicAdd(I.stats + 2 * a + 1, esum);
        }
    }
}

// Stage B of the FP64 sweep in double-float on the FP32 pipes: on GB300 the
// FP64 pipe issues under two operations per SM per clock against 128 FP32
// ones, so the six FP64 operations per term of spectral_tile<double> cost as
// much as ~450 FP32 ones.  Each term Re 1/(d_{2m} + tau Lambda_l) is
// df_scan_term (qbvm_dfsum.cuh: about 35 FP32 operations and one approximate
// reciprocal, about 2^-44 of the term's scale), the thread's accumulators folded every
// four frequencies.  The squares of the discrepancy and error sums are FP64,
// as in spectral_tile<double>.
template <int MPT>
__device__ void spectral_tile_df(const SwInst& I, int tile, unsigned char* smem) {
    __shared__ double sh[32];
    float4* sd = reinterpret_cast<float4*>(smem);
    qbvm::dfloat lam[MPT];
    double w[MPT], gh[MPT], zh[MPT];
    bool valid[MPT];
#pragma unroll
    for (int q = 0; q < MPT; ++q) {
        const long long l = (long long)tile * SW_THREADS * MPT + q * SW_THREADS + threadIdx.x;
        valid[q] = l < I.Nx;
        lam[q] = {0.f, 0.f};
        w[q] = gh[q] = zh[q] = 0.0;
        if (valid[q]) {
            const int lx = (int)(l % I.nx), ly = (int)(l / I.nx);
            const double lt = __ldcg(I.lamx + lx) + (I.dim == 2 ? __ldcg(I.lamy + ly) : 0.0);
            lam[q] = qbvm::df_from_double(lt);
            gh[q] = __ldcg(I.ghat + l) * I.sscale;
            w[q] = (1.0 + lt) * gh[q];
            if (I.has_z0) zh[q] = __ldcg(I.zhat + l) * I.zscale * I.sscale;
        }
    }
    for (int a = 0; a < I.n_alpha; ++a) {
        __syncthreads();
        for (int m = threadIdx.x; m < I.H; m += blockDim.x) sd[m] = I.dtabdf[(long long)a * I.H + m];
        __syncthreads();
        float shi[MPT], slo[MPT];
#pragma unroll
        for (int q = 0; q < MPT; ++q) shi[q] = slo[q] = 0.f;
        for (int m0 = 0; m0 < I.H; m0 += 4) {
            const int m1 = min(m0 + 4, I.H);
            for (int m = m0; m < m1; ++m) {
                const float4 d = sd[m];                         // (Re.hi, Re.lo, Im.hi, Im.lo)
                const qbvm::DfSq im2 = qbvm::df_scan_im2(d.z, d.w);
#pragma unroll
                for (int q = 0; q < MPT; ++q) qbvm::df_scan_term(d.x, d.y, im2, lam[q].hi, lam[q].lo, shi[q], slo[q]);
            }
            // fold the low word into the high one every four terms: a low word
            // left to grow over all H terms rounds at its own, growing size
#pragma unroll
            for (int q = 0; q < MPT; ++q) qbvm::df_scan_fold(shi[q], slo[q]);
        }
        const double cna = I.cn[a];
        double ds = 0.0, es = 0.0;
#pragma unroll
        for (int q = 0; q < MPT; ++q) {
            if (!valid[q]) continue;
            const double sq = qbvm::qbvm_join_df_dadd(shi[q], slo[q]);
            const double dv = w[q] * sq;                        // (1 + tau Lambda) yhat / cna
            ds = fma(dv, dv, ds);
            if (I.has_z0) {
                const double e = fma(cna * gh[q], sq, -zh[q]);
                es = fma(e, e, es);
            }
        }
        double dsum = block_sum_d(cna * cna * ds, sh);
        double esum = block_sum_d(es, sh);
        if (threadIdx.x == 0) {
            atomicAdd(I.stats + 2 * a, dsum);
            if (I.has_z0) atomicAdd(I.stats + 2 * a + 1, esum);
        }
    }
}

// Stage C: discrepancy principle on one instance (single thread).
__device__ void pick_alpha(const SwInst& I) {
    if (threadIdx.x != 0) return;
    int pick = -1, best = 0, closest = 0;
    double bestv = INFINITY, closev = INFINITY;
    for (int a = 0; a < I.n_alpha; ++a) {
        // stats are of the scaled data: compare and rank scaled, report unscaled
        double d2 = __ldcg(I.stats + 2 * a), e2 = __ldcg(I.stats + 2 * a + 1);
        double dsc = I.coef[a] * sqrt(I.wnorm * d2);
        I.disc[a] = dsc * I.sinv;
        if (I.has_z0) {
            double ev = sqrt(I.wnorm * e2);
            I.err[a] = ev * I.sinv;
            if (ev < bestv) {
                bestv = ev;
                best = a;
            }
        }
        if (dsc <= I.tau_dp * (I.delta * I.sscale) && (pick < 0 || I.alphas[a] > I.alphas[pick])) pick = a;
        if (dsc < closev) {
            closev = dsc;
            closest = a;
        }
    }
    I.pick[0] = pick >= 0 ? pick : closest;
    I.pick[1] = best;
    __threadfence();
}

// Stage D: FP64 spectral y^0 at the picked alpha for one tile of modes.
// Stage D: y^0 in the sine basis at the picked alpha, Step (c) at t = 0:
// sum over the even frequencies of Re 1/(d_{2m} + tau Lambda_l).  FP64 for the
// FP64 sweep; for the FP32 sweep in double-float on the FP32 pipes (each term
// to about 2^-44: |z|^2 in double-float, one fast division and one correction
// step), since FP64 sums cost the FP64 pipe ~16 operations per term.
template <typename R>
__device__ void final_tile(const SwInst& I, int tile) {
    const int a = __ldcg(I.pick);
    const long long l = (long long)tile * SW_THREADS + threadIdx.x;
    if (l >= I.Nx) return;
    const int lx = (int)(l % I.nx), ly = (int)(l / I.nx);
    const double lt = I.lamx[lx] + (I.dim == 2 ? I.lamy[ly] : 0.0);
    double s = 0.0;
    if (std::is_same<R, double>::value) {
        const double2* dt = I.dtab + (long long)a * I.H;
        for (int m = 0; m < I.H; ++m) {
            double2 d = dt[m];
            double zr = d.x + lt;
            s = fma(zr, rcp_newton(fma(zr, zr, d.y * d.y)), s);
        }
    } else {
        const float4* dt = I.dtabdf + (long long)a * I.H;
        const qbvm::dfloat ltd = qbvm::df_from_double(lt);
        qbvm::dfloat acc = {0.f, 0.f};
        for (int m = 0; m < I.H; ++m) {
            const float4 d = dt[m];
            const qbvm::dfloat zr = qbvm::df_add_sloppy(qbvm::dfloat{d.x, d.y}, ltd), zi = {d.z, d.w};
            const qbvm::dfloat den = qbvm::df_add_sloppy(qbvm::df_mul(zr, zr), qbvm::df_mul(zi, zi));
            const float q1 = __fdividef(zr.hi, den.hi);
            const qbvm::dfloat r = qbvm::df_add_sloppy(zr, qbvm::df_neg(qbvm::df_mul(den, qbvm::dfloat{q1, 0.f})));
            const float q2 = __fdividef(r.hi, den.hi);
            acc = qbvm::df_add_sloppy(acc, qbvm::df_fast_two_sum(q1, q2));
        }
        s = qbvm::df_to_double(acc);
    }
    I.yhat[l] = I.cn[a] * __ldcg(I.ghat + l) * s;
}

// Each stage out of line: the persistent kernel's register budget is then set
// per stage rather than by the union of all of them inlined into one body.
template <bool LDCG>
__device__ __noinline__ void dst_stage(const double* in, double* out, int n, int lm, long long outer,
                                       long long inner, long long tile, const double2* tw, const double* sn,
                                       unsigned char* smem) {
    qbvm::dst_tile<double, double, 0, qbvm::DST_TILE / 4 / SW_THREADS, LDCG>(in, out, n, lm, qbvm::dst_lw(lm), outer,
                                                                            inner, tile, tw, sn, smem);
}
template <typename R, int MPT>
__device__ __noinline__ void spectral_stage(const SwInst& I, int tile, unsigned char* smem) {
    if (std::is_same<R, double>::value && I.df_sums)
        spectral_tile_df<MPT>(I, tile, smem);
    else
        spectral_tile<R, MPT>(I, tile, smem);
}
template <typename R>
__device__ __noinline__ void final_stage(const SwInst& I, int tile) {
    if (std::is_same<R, double>::value && I.df_sums)
        final_tile<float>(I, tile);              // y^0 summed in double-float
    else
        final_tile<R>(I, tile);
}

struct SwRun {
    const SwInst* inst;
    const int4* items;
    int nitems;
    int* counters;       // count x NSTAGE
    int* next;
    int* errflag;
};

template <typename R, int MPT>
__global__ void __launch_bounds__(SW_THREADS, 2) k_sweep(SwRun run) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ SwInst I;
    for (;;) {
        if (threadIdx.x == 0) s_item = ld_volatile(run.errflag) ? run.nitems : atomicAdd(run.next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= run.nitems) return;
        const int4 w = run.items[it];
        if (threadIdx.x == 0) I = run.inst[w.y];
        __syncthreads();
        int* cnt = run.counters + (long long)w.y * NSTAGE;
        bool ok = true;
        switch (w.x) {
            case ST_GY: ok = wait_for(cnt + ST_GX, I.tiles_gx, run.errflag); break;
            case ST_ZY: ok = wait_for(cnt + ST_ZX, I.tiles_gx, run.errflag); break;
            case ST_SPEC:
                ok = wait_for(cnt + (I.dim == 2 ? ST_GY : ST_GX), I.dim == 2 ? I.tiles_gy : I.tiles_gx, run.errflag);
                if (ok && I.has_z0)
                    ok = wait_for(cnt + (I.dim == 2 ? ST_ZY : ST_ZX), I.dim == 2 ? I.tiles_gy : I.tiles_gx, run.errflag);
                break;
            case ST_PICK: ok = wait_for(cnt + ST_SPEC, I.tiles_spec, run.errflag); break;
            case ST_FIN: ok = wait_for(cnt + ST_PICK, 1, run.errflag); break;
            case ST_IY: ok = wait_for(cnt + ST_FIN, I.tiles_fin, run.errflag); break;
            case ST_IX:
                ok = I.dim == 2 ? wait_for(cnt + ST_IY, I.tiles_iy, run.errflag)
                                : wait_for(cnt + ST_FIN, I.tiles_fin, run.errflag);
                break;
            default: break;
        }
        if (!ok) return;
        switch (w.x) {
            case ST_GX:       // x-DST of g, one level: rows = ny
                dst_stage<false>(I.g, I.ghat, I.nx, I.lmx, I.ny, 1, w.z, I.twx, I.snx, smem);
                break;
            case ST_GY:
                dst_stage<true>(I.ghat, I.ghat, I.ny, I.lmy, 1, I.nx, w.z, I.twy, I.sny, smem);
                break;
            case ST_ZX:
                dst_stage<false>(I.z0, I.zhat, I.nx, I.lmx, I.ny, 1, w.z, I.twx, I.snx, smem);
                break;
            case ST_ZY:
                dst_stage<true>(I.zhat, I.zhat, I.ny, I.lmy, 1, I.nx, w.z, I.twy, I.sny, smem);
                break;
            case ST_SPEC: spectral_stage<R, MPT>(I, w.z, smem); break;
            case ST_PICK: pick_alpha(I); break;
            case ST_FIN: final_stage<R>(I, w.z); break;
            case ST_IY:
                dst_stage<true>(I.yhat, I.yhat, I.ny, I.lmy, 1, I.nx, w.z, I.twy, I.sny, smem);
                break;
            case ST_IX:
                dst_stage<true>(I.yhat, I.y0, I.nx, I.lmx, I.ny, 1, w.z, I.twx, I.snx, smem);
                break;
            default: break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(cnt + w.x, 1);
        }
    }
}

// (The shared-memory attribute is set by max_resident in configure(), outside
// any stream capture.)
template <typename R, int MPT>
cudaError_t launch_sweep(const SwRun& run, int grid, size_t smem, cudaStream_t s) {
    k_sweep<R, MPT><<<grid, SW_THREADS, smem, s>>>(run);
    return cudaGetLastError();
}

template <typename R, int MPT>
int max_resident(size_t smem) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto kern = k_sweep<R, MPT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SW_THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

}  // namespace

struct qbvm_sweep {
    int count = 0, n_alpha = 0, precision = 0;
    std::vector<SwInst> host_inst;
    std::vector<void*> allocs;
    SwInst* d_inst = nullptr;
    int4* d_items = nullptr;
    int nitems = 0;
    int* d_counters = nullptr;
    int* d_next = nullptr;
    int* d_err = nullptr;
    double* d_stats = nullptr;
    double* d_disc = nullptr;
    double* d_err_out = nullptr;
    double* d_alphas = nullptr;
    int* d_pick = nullptr;
    size_t stats_bytes = 0;
    size_t smem = 0;
    // launch configuration (autotuned): modes per thread in stage B, CTAs per SM
    int mpt = 1, ctas_per_sm = 0;
    int grid = 0;
    int spec_tiles_total = 0;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    bool graph_valid = false;
    float last_ms = 0.f;
    int last_error = 0;
};

namespace {

template <typename T>
int sw_alloc(qbvm_sweep_t* p, T** ptr, size_t count) {
    *ptr = nullptr;
    if (!count) return QBVM_OK;
    void* v = nullptr;
    if (cudaMalloc(&v, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_OOM;
    }
    p->allocs.push_back(v);
    *ptr = static_cast<T*>(v);
    return QBVM_OK;
}

template <typename T>
int sw_upload(qbvm_sweep_t* p, T** ptr, const std::vector<T>& h) {
    int rc = sw_alloc(p, ptr, h.size());
    if (rc) return rc;
    return cudaMemcpy(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess ? QBVM_OK
                                                                                                   : QBVM_ERR_CUDA;
}

void sw_destroy(qbvm_sweep_t* p) {
    if (!p) return;
    if (p->graph) cudaGraphExecDestroy(p->graph);
    for (void* v : p->allocs) cudaFree(v);
    delete p;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int lg2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

int configure(qbvm_sweep_t* p, int mpt, int ctas_per_sm) {
    // spectral tiles depend on the modes per tile
    std::vector<int4> items;
    int total_spec = 0;
    for (int i = 0; i < p->count; ++i) {
        SwInst& I = p->host_inst[i];
        I.tiles_spec = (int)((I.Nx + (long long)SW_THREADS * mpt - 1) / ((long long)SW_THREADS * mpt));
        total_spec += I.tiles_spec;
    }
    // the final stage (one alpha, FP64) uses one mode per thread
    for (int i = 0; i < p->count; ++i)
        p->host_inst[i].tiles_fin = (int)((p->host_inst[i].Nx + SW_THREADS - 1) / SW_THREADS);
    for (int st = 0; st < NSTAGE; ++st) {
        for (int i = 0; i < p->count; ++i) {
            const SwInst& I = p->host_inst[i];
            int n = 0;
            switch (st) {
                case ST_GX: n = I.tiles_gx; break;
                case ST_GY: n = I.dim == 2 ? I.tiles_gy : 0; break;
                case ST_ZX: n = I.has_z0 ? I.tiles_gx : 0; break;
                case ST_ZY: n = (I.has_z0 && I.dim == 2) ? I.tiles_gy : 0; break;
                case ST_SPEC: n = I.tiles_spec; break;
                case ST_PICK: n = 1; break;
                case ST_FIN: n = I.has_y0 ? I.tiles_fin : 0; break;
                case ST_IY: n = (I.has_y0 && I.dim == 2) ? I.tiles_iy : 0; break;
                case ST_IX: n = I.has_y0 ? I.tiles_ix : 0; break;
            }
            for (int t = 0; t < n; ++t) items.push_back(make_int4(st, i, t, 0));
        }
    }
    p->nitems = (int)items.size();
    p->spec_tiles_total = total_spec;
    if (p->d_items) {
        cudaFree(p->d_items);
        p->allocs.erase(std::find(p->allocs.begin(), p->allocs.end(), (void*)p->d_items));
        p->d_items = nullptr;
    }
    int rc = sw_upload(p, &p->d_items, items);
    if (rc) return rc;
    if (cudaMemcpy(p->d_inst, p->host_inst.data(), sizeof(SwInst) * p->count, cudaMemcpyHostToDevice) != cudaSuccess)
        return QBVM_ERR_CUDA;
    // resident grid
    int maxres = 0;
    if (p->precision == QBVM_FP64) {
        maxres = mpt == 1 ? max_resident<double, 1>(p->smem) : mpt == 2 ? max_resident<double, 2>(p->smem)
                                                                         : max_resident<double, 4>(p->smem);
    } else {
        maxres = mpt == 1 ? max_resident<float, 1>(p->smem) : mpt == 2 ? max_resident<float, 2>(p->smem)
                                                                        : max_resident<float, 4>(p->smem);
    }
    if (maxres <= 0) return QBVM_ERR_UNSUPPORTED;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int want = ctas_per_sm > 0 ? ctas_per_sm * sms : maxres;
    p->grid = std::min(want, maxres);
    p->mpt = mpt;
    p->ctas_per_sm = ctas_per_sm;
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    p->graph_valid = false;
    return QBVM_OK;
}

int enqueue(qbvm_sweep_t* p, cudaStream_t s) {
    const size_t cnt_bytes = sizeof(int) * ((size_t)p->count * NSTAGE + 2);
    if (cudaMemsetAsync(p->d_counters, 0, cnt_bytes, s) != cudaSuccess) return QBVM_ERR_CUDA;
    if (cudaMemsetAsync(p->d_stats, 0, p->stats_bytes, s) != cudaSuccess) return QBVM_ERR_CUDA;
    SwRun run{p->d_inst, p->d_items, p->nitems, p->d_counters, p->d_next, p->d_err};
    cudaError_t e;
    if (p->precision == QBVM_FP64) {
        e = p->mpt == 1 ? launch_sweep<double, 1>(run, p->grid, p->smem, s)
            : p->mpt == 2 ? launch_sweep<double, 2>(run, p->grid, p->smem, s)
                          : launch_sweep<double, 4>(run, p->grid, p->smem, s);
    } else {
        e = p->mpt == 1 ? launch_sweep<float, 1>(run, p->grid, p->smem, s)
            : p->mpt == 2 ? launch_sweep<float, 2>(run, p->grid, p->smem, s)
                          : launch_sweep<float, 4>(run, p->grid, p->smem, s);
    }
    return e == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

// Capture the run (counter reset + persistent launch) into a graph once.
int run_graph(qbvm_sweep_t* p, cudaStream_t s) {
    if (!p->graph_valid || p->graph_stream != s) {
        if (p->graph) {
            cudaGraphExecDestroy(p->graph);
            p->graph = nullptr;
        }
        cudaStream_t cs = s;
        bool own = false;
        if (cs == nullptr) {        // the legacy default stream cannot be captured: use a private one
            if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return QBVM_ERR_CUDA;
            own = true;
        }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return QBVM_ERR_CUDA;
        int rc = enqueue(p, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (own) cudaStreamDestroy(cs);
            cudaGetLastError();
            return rc ? rc : QBVM_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&p->graph, g, 0);
        cudaGraphDestroy(g);
        if (own) cudaStreamDestroy(cs);
        if (e != cudaSuccess) return QBVM_ERR_CUDA;
        p->graph_valid = true;
        p->graph_stream = s;
    }
    return cudaGraphLaunch(p->graph, s) == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

}  // namespace

// Diagnostic: every CTA runs the persistent kernel's bounded wait on a
// counter that nothing advances.  The first CTA to exhaust SPIN_LIMIT raises
// the error flag; the others see it and leave.  out[b] = 1 if CTA b's wait
// succeeded (it never should).
__global__ void k_wait_selftest(const int* counter, int* errflag, int* out) {
    const bool ok = wait_for(counter, 1, errflag);
    if (threadIdx.x == 0) out[blockIdx.x] = ok ? 1 : 0;
}

extern "C" {

int qbvm_sweep_plan(const qbvm_sweep_desc* d, qbvm_sweep_t** out) {
    if (!out) return QBVM_ERR_BAD_ARG;
    *out = nullptr;
    if (!d || d->count < 1 || !d->inst || d->n_alpha < 1 || d->n_alpha > 64) return QBVM_ERR_BAD_ARG;
    if (d->precision != QBVM_FP64 && d->precision != QBVM_FP32_REFINE) return QBVM_ERR_BAD_ARG;
    if (!(d->tau_dp > 0) || !std::isfinite(d->log10_lo) || !std::isfinite(d->log10_hi)) return QBVM_ERR_BAD_ARG;
    for (int i = 0; i < d->count; ++i) {
        const qbvm_sweep_instance& in = d->inst[i];
        if (in.dim < 1 || in.dim > 2 || !in.g) return QBVM_ERR_BAD_ARG;
        if (!(in.T > 0) || !(in.L > 0) || !(in.delta > 0) || in.nt < 2) return QBVM_ERR_BAD_ARG;
        if (in.form != QBVM_FORM_PQ && in.form != QBVM_FORM_PM) return QBVM_ERR_BAD_ARG;
        if (!pow2(in.nt) || in.nt > 1024) return QBVM_ERR_UNSUPPORTED;
        for (int a = 0; a < in.dim; ++a)
            if (!pow2(in.m[a]) || in.m[a] < 4 || in.m[a] > 2048) return QBVM_ERR_UNSUPPORTED;
    }
    qbvm_sweep_t* p = new (std::nothrow) qbvm_sweep();
    if (!p) return QBVM_ERR_OOM;
    p->count = d->count;
    p->n_alpha = d->n_alpha;
    p->precision = d->precision;
    p->host_inst.resize(d->count);
    int rc = QBVM_OK;
    const int na = d->n_alpha;
    rc = sw_alloc(p, &p->d_stats, (size_t)d->count * na * 2);
    p->stats_bytes = sizeof(double) * (size_t)d->count * na * 2;
    if (!rc) rc = sw_alloc(p, &p->d_disc, (size_t)d->count * na);
    if (!rc) rc = sw_alloc(p, &p->d_err_out, (size_t)d->count * na);
    if (!rc) rc = sw_alloc(p, &p->d_pick, (size_t)d->count * 2);
    if (!rc) rc = sw_alloc(p, &p->d_counters, (size_t)d->count * NSTAGE + 2);
    if (!rc) {
        p->d_next = p->d_counters + (size_t)d->count * NSTAGE;
        p->d_err = p->d_next + 1;
    }
    if (!rc) rc = sw_alloc(p, &p->d_inst, (size_t)d->count);
    std::vector<double> alphas_all((size_t)d->count * na);
    size_t smem = 0;
    // All per-instance tables go into one host arena uploaded in one copy; the
    // per-instance device scratch (DST of g, z0 and y^0) into a second arena.
    // DST-I tables are shared by every instance with the same length.
    std::vector<unsigned char> arena;
    auto put = [&](const void* src, size_t bytes) {
        size_t off = (arena.size() + 255) & ~(size_t)255;
        arena.resize(off + bytes);
        std::memcpy(arena.data() + off, src, bytes);
        return off;
    };
    struct Offs { size_t lamx, lamy, dtab, dtab32, dtabdf, cn, coef, al, twx, twy, snx, sny, gh, zh, yh; };
    std::vector<Offs> offs(d->count);
    std::vector<std::pair<int, std::pair<size_t, size_t>>> dst_cache;   // M -> (tw, sn) offsets
    auto dst_tables = [&](int M) {
        for (auto& c : dst_cache)
            if (c.first == M) return c.second;
        std::vector<double2> w(M);
        std::vector<double> sv(M / 2 + 2, 0.0);
        for (int m = 0; m < M; ++m) {
            double a = M_PI * (2.0 * m / M);
            w[m] = make_double2(std::cos(a), -std::sin(a));
        }
        for (int j = 0; j <= M / 2; ++j) sv[j] = std::sin(M_PI * j / M);
        std::pair<size_t, size_t> r(put(w.data(), w.size() * sizeof(double2)), put(sv.data(), sv.size() * sizeof(double)));
        dst_cache.push_back({M, r});
        return r;
    };
    size_t scratch = 0;
    auto take = [&](size_t bytes) {
        size_t off = (scratch + 255) & ~(size_t)255;
        scratch = off + bytes;
        return off;
    };
    for (int i = 0; i < d->count; ++i) {
        const qbvm_sweep_instance& in = d->inst[i];
        SwInst& I = p->host_inst[i];
        std::memset(&I, 0, sizeof(I));
        I.dim = in.dim;
        I.form = in.form;
        I.nx = in.m[0] - 1;
        I.ny = in.dim == 2 ? in.m[1] - 1 : 1;
        I.lmx = lg2(in.m[0]);
        I.lmy = in.dim == 2 ? lg2(in.m[1]) : 0;
        I.Nx = (long long)I.nx * I.ny;
        I.H = in.nt / 2;
        I.n_alpha = na;
        I.delta = in.delta;
        {
            int e = -std::ilogb(in.delta);
            e = e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
            I.sscale = std::ldexp(1.0, e);
            I.sinv = std::ldexp(1.0, -e);
        }
        I.tau_dp = d->tau_dp;
        I.tau = in.T / (in.nt - 1);
        const double hx = in.L / in.m[0], hy = in.dim == 2 ? in.L / in.m[1] : 1.0;
        // ||S v||^2 = prod(M/2) ||v||^2, times the grid weight prod(h)
        I.wnorm = (in.L / 2.0) * (in.dim == 2 ? in.L / 2.0 : 1.0);
        I.zscale = (2.0 / in.m[0]) * (in.dim == 2 ? 2.0 / in.m[1] : 1.0);
        I.g = in.g;
        I.z0 = in.z0;
        I.y0 = in.y0;
        I.has_z0 = in.z0 != nullptr;
        I.has_y0 = in.y0 != nullptr;
        const int lwx = qbvm::dst_lw(I.lmx), lwy = in.dim == 2 ? qbvm::dst_lw(I.lmy) : 0;
        I.tiles_gx = (int)((I.ny + 2 * (1 << lwx) - 1) / (2 * (1 << lwx)));
        I.tiles_ix = I.tiles_gx;
        I.tiles_gy = in.dim == 2 ? (int)((I.nx + 2 * (1 << lwy) - 1) / (2 * (1 << lwy))) : 0;
        I.tiles_iy = I.tiles_gy;
        smem = std::max(smem, qbvm::dst_smem<double>(I.lmx));
        if (in.dim == 2) smem = std::max(smem, qbvm::dst_smem<double>(I.lmy));
        smem = std::max(smem, sizeof(double2) * (size_t)I.H);
        std::vector<double> lx(I.nx), ly(I.ny, 0.0);
        for (int k = 1; k <= I.nx; ++k) {
            double sk = std::sin(M_PI * k / (2.0 * in.m[0]));
            lx[k - 1] = I.tau * 4.0 / (hx * hx) * sk * sk;
        }
        if (in.dim == 2)
            for (int k = 1; k <= I.ny; ++k) {
                double sk = std::sin(M_PI * k / (2.0 * in.m[1]));
                ly[k - 1] = I.tau * 4.0 / (hy * hy) * sk * sk;
            }
        std::vector<double2> dtab((size_t)na * I.H);
        std::vector<float2> dtab32((size_t)na * I.H);
        std::vector<float4> dtabdf((size_t)na * I.H);
        std::vector<double> cn(na), coef(na), al(na);
        const double rule = in.alpha_base > 0 ? in.alpha_base
                                              : (in.form == QBVM_FORM_PQ ? in.delta : I.tau * in.delta);   // Section 5
        for (int a = 0; a < na; ++a) {
            double ex = na > 1 ? d->log10_lo + (d->log10_hi - d->log10_lo) * a / (na - 1) : d->log10_lo;
            double alpha = rule * std::pow(10.0, ex);
            al[a] = alpha;
            alphas_all[(size_t)i * na + a] = alpha;
            double omega = in.form == QBVM_FORM_PQ ? -1.0 / alpha : -I.tau / alpha;
            double g1 = std::pow(std::fabs(omega), 1.0 / in.nt);
            for (int m = 0; m < I.H; ++m) {
                double ang = M_PI * ((4.0 * m + 1.0) / in.nt);
                double2 v = make_double2(1.0 - g1 * std::cos(ang), -g1 * std::sin(ang));
                dtab[(size_t)a * I.H + m] = v;
                dtab32[(size_t)a * I.H + m] = make_float2((float)v.x, (float)v.y);
                // on the host the plain casts (the device uses an integer split of the same value)
                const float rh = (float)v.x, ih = (float)v.y;
                dtabdf[(size_t)a * I.H + m] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
            }
            // 2 cnorm with cnorm = -omega * prod(2/M) / nt (the delta right-hand side)
            cn[a] = 2.0 * (-omega) * I.zscale / in.nt;
            coef[a] = in.form == QBVM_FORM_PQ ? alpha : alpha / I.tau;
        }
        {
            // the FP64 sweep sums in double-float where |Re d|, |Im d| and
            // tau Lambda stay inside [2^-30, 2^30] (|Im d| and tau Lambda away
            // from zero): squares, products and low words then stay normal FP32
            const double lo = std::ldexp(1.0, -30), hi = std::ldexp(1.0, 30);
            double lmin = *std::min_element(lx.begin(), lx.end()), lmax = *std::max_element(lx.begin(), lx.end());
            if (in.dim == 2) {
                lmin += *std::min_element(ly.begin(), ly.end());
                lmax += *std::max_element(ly.begin(), ly.end());
            }
            bool ok = p->precision == QBVM_FP64 && lmin >= lo && lmax <= hi;
            for (const double2& v : dtab)
                ok = ok && std::fabs(v.x) <= hi && std::fabs(v.y) >= lo && std::fabs(v.y) <= hi;
            I.df_sums = ok ? 1 : 0;
        }
        Offs& o = offs[i];
        o.lamx = put(lx.data(), lx.size() * sizeof(double));
        o.lamy = put(ly.data(), ly.size() * sizeof(double));
        o.dtab = put(dtab.data(), dtab.size() * sizeof(double2));
        o.dtab32 = put(dtab32.data(), dtab32.size() * sizeof(float2));
        o.dtabdf = put(dtabdf.data(), dtabdf.size() * sizeof(float4));
        o.cn = put(cn.data(), cn.size() * sizeof(double));
        o.coef = put(coef.data(), coef.size() * sizeof(double));
        o.al = put(al.data(), al.size() * sizeof(double));
        auto tx = dst_tables(in.m[0]);
        o.twx = tx.first;
        o.snx = tx.second;
        auto ty = in.dim == 2 ? dst_tables(in.m[1]) : tx;
        o.twy = ty.first;
        o.sny = ty.second;
        o.gh = take(sizeof(double) * (size_t)I.Nx);
        o.zh = I.has_z0 ? take(sizeof(double) * (size_t)I.Nx) : 0;
        o.yh = I.has_y0 ? take(sizeof(double) * (size_t)I.Nx) : 0;
    }
    unsigned char *tab = nullptr, *scr = nullptr;
    if (!rc) rc = sw_upload(p, &tab, arena);
    if (!rc) rc = sw_alloc(p, &scr, scratch);
    for (int i = 0; i < d->count && !rc; ++i) {
        SwInst& I = p->host_inst[i];
        const Offs& o = offs[i];
        I.lamx = reinterpret_cast<const double*>(tab + o.lamx);
        I.lamy = reinterpret_cast<const double*>(tab + o.lamy);
        I.dtab = reinterpret_cast<const double2*>(tab + o.dtab);
        I.dtab32 = reinterpret_cast<const float2*>(tab + o.dtab32);
        I.dtabdf = reinterpret_cast<const float4*>(tab + o.dtabdf);
        I.cn = reinterpret_cast<const double*>(tab + o.cn);
        I.coef = reinterpret_cast<const double*>(tab + o.coef);
        I.alphas = reinterpret_cast<const double*>(tab + o.al);
        I.twx = reinterpret_cast<const double2*>(tab + o.twx);
        I.twy = reinterpret_cast<const double2*>(tab + o.twy);
        I.snx = reinterpret_cast<const double*>(tab + o.snx);
        I.sny = reinterpret_cast<const double*>(tab + o.sny);
        I.ghat = reinterpret_cast<double*>(scr + o.gh);
        I.zhat = I.has_z0 ? reinterpret_cast<double*>(scr + o.zh) : nullptr;
        I.yhat = I.has_y0 ? reinterpret_cast<double*>(scr + o.yh) : nullptr;
        I.stats = p->d_stats + (size_t)i * na * 2;
        I.disc = p->d_disc + (size_t)i * na;
        I.err = p->d_err_out + (size_t)i * na;
        I.pick = p->d_pick + (size_t)i * 2;
    }
    if (!rc) rc = sw_upload(p, &p->d_alphas, alphas_all);
    p->smem = smem;
    if (!rc) rc = configure(p, 1, 0);
    if (rc) {
        sw_destroy(p);
        return rc;
    }
    *out = p;
    return QBVM_OK;
}

int qbvm_sweep_run(qbvm_sweep_t* p, void* stream) {
    if (!p) return QBVM_ERR_BAD_ARG;
    return run_graph(p, static_cast<cudaStream_t>(stream));
}

int qbvm_sweep_read(qbvm_sweep_t* p, double* alphas, double* discrepancy, double* error, int* pick, void* stream) {
    if (!p) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)p->count * p->n_alpha;
    int errflag = 0;
    if (cudaMemcpyAsync(&errflag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (alphas && cudaMemcpyAsync(alphas, p->d_alphas, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (discrepancy && cudaMemcpyAsync(discrepancy, p->d_disc, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (error && cudaMemcpyAsync(error, p->d_err_out, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (pick && cudaMemcpyAsync(pick, p->d_pick, 2 * p->count * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return QBVM_ERR_CUDA;
    return errflag ? QBVM_ERR_TIMEOUT : QBVM_OK;
}

int qbvm_sweep_autotune(qbvm_sweep_t* p, int repeats, qbvm_sweep_config* best_out, void* stream) {
    if (!p || repeats < 1) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mpts[3] = {1, 2, 4};
    const int ctas[3] = {0, 1, 2};       // 0 = every resident slot
    float best = INFINITY;
    int bm = 1, bc = 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return QBVM_ERR_CUDA;
    int rc = QBVM_OK;
    for (int mi = 0; mi < 3 && !rc; ++mi)
        for (int ci = 0; ci < 3 && !rc; ++ci) {
            rc = configure(p, mpts[mi], ctas[ci]);
            if (rc) break;
            rc = run_graph(p, s);                         // warm-up + capture
            if (rc) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < repeats && !rc; ++r) rc = run_graph(p, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = QBVM_ERR_CUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            int errflag = 0;
            cudaMemcpy(&errflag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
            if (errflag) rc = QBVM_ERR_TIMEOUT;
            if (!rc && ms / repeats < best) {
                best = ms / repeats;
                bm = mpts[mi];
                bc = ctas[ci];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    rc = configure(p, bm, bc);
    if (rc) return rc;
    p->last_ms = best;
    if (best_out) {
        best_out->modes_per_thread = bm;
        best_out->ctas_per_sm = bc;
        best_out->grid = p->grid;
        best_out->ms = best;
    }
    return QBVM_OK;
}

int qbvm_sweep_set_config(qbvm_sweep_t* p, const qbvm_sweep_config* cfg) {
    if (!p || !cfg) return QBVM_ERR_BAD_ARG;
    if (cfg->modes_per_thread != 1 && cfg->modes_per_thread != 2 && cfg->modes_per_thread != 4) return QBVM_ERR_BAD_ARG;
    if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 32) return QBVM_ERR_BAD_ARG;
    return configure(p, cfg->modes_per_thread, cfg->ctas_per_sm);
}

int qbvm_sweep_get_config(const qbvm_sweep_t* p, qbvm_sweep_config* cfg) {
    if (!p || !cfg) return QBVM_ERR_BAD_ARG;
    cfg->modes_per_thread = p->mpt;
    cfg->ctas_per_sm = p->ctas_per_sm;
    cfg->grid = p->grid;
    cfg->ms = p->last_ms;
    return QBVM_OK;
}

int qbvm_sweep_destroy(qbvm_sweep_t* p) {
    sw_destroy(p);
    return QBVM_OK;
}

int qbvm_selftest_newton_rcp(const double* d, long long n, double* max_rel_diff, void* stream) {
    if (!d || n < 1 || !max_rel_diff) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_OOM;
    }
    unsigned long long h = 0;
    int rc = QBVM_OK;
    if (cudaMemsetAsync(buf, 0, sizeof(h), s) != cudaSuccess) rc = QBVM_ERR_CUDA;
    if (!rc) {
        long long blocks = (n + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        k_rcp_check<<<(unsigned)blocks, 256, 0, s>>>(d, n, buf);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&h, buf, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = QBVM_ERR_CUDA;
    }
    cudaFree(buf);
    if (rc) {
        cudaGetLastError();
        return rc;
    }
    double v;
    std::memcpy(&v, &h, sizeof(v));
    *max_rel_diff = v;
    return QBVM_OK;
}

int qbvm_selftest_bounded_wait(int ctas, double* seconds, void* stream) {
    if (ctas < 1 || ctas > 64) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* buf = nullptr;                       // [0] counter, [1] error flag, [2..] per-CTA outcome
    if (cudaMalloc(&buf, sizeof(int) * (size_t)(2 + ctas)) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_OOM;
    }
    std::vector<int> h((size_t)(2 + ctas), -1);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = QBVM_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(buf, 0, sizeof(int) * (size_t)(2 + ctas), s) != cudaSuccess ||
        cudaEventRecord(e0, s) != cudaSuccess) {
        rc = QBVM_ERR_CUDA;
    } else {
        k_wait_selftest<<<ctas, 32, 0, s>>>(buf, buf + 1, buf + 2);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaMemcpyAsync(h.data(), buf, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = QBVM_ERR_CUDA;
    }
    if (!rc && seconds) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *seconds = ms * 1e-3;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc) {
        cudaGetLastError();
        return rc;
    }
    bool any_ok = false;
    for (int b = 0; b < ctas; ++b) any_ok = any_ok || h[(size_t)(2 + b)] != 0;
    return (h[1] != 0 && !any_ok) ? QBVM_ERR_TIMEOUT : QBVM_OK;
}

}  // extern "C"
