// qbvm_timesolve.cuh -- the FP64/FP32 shared-memory time-solve tile (Steps
// (a)-(c) of eq. 3.8 in the sine basis for W spatial modes), shared by the
// per-pass kernels, the batch kernel and the persistent multi-instance kernel.
#pragma once
#include "qbvm_dst.cuh"
#include "qbvm_fft.cuh"

namespace qbvm {

// --------------------------------------------------------- time solve (2D/3D)
//
// Column l (spatial mode) of the [nt][Nx] array solves the real scalar
// omega-circulant system of eq. 3.8 in the sine basis.  With P = nt,
// gamma = omega^{1/P} = rho e^{i pi/P} and H = P/2:
//   Step (a): u^_k = sum_t theta^{kt} gamma^t f_t.  For real f the sequence is
//     conjugate-symmetric, u^_{P-1-k} = conj(u^_k), and the even frequencies are
//     one length-H DFT:  u^_{2m} = sum_{t<H} theta_H^{mt} gamma^t (f_t + i rho^H f_{t+H}).
//   Step (b): w^_{2m} = cnorm u^_{2m} / (d_{2m} + tau Lambda_l), d_k = 1 - gamma theta^k.
//   Step (c): with q_t = sum_m theta_H^{-mt} w^_{2m} and v_t = 2 gamma^{-t} q_t,
//     y_t = Re v_t and y_{t+H} = rho^{-H} Im v_t (the odd frequencies are the
//     conjugates of the even ones, so they never need to be formed).
// cnorm carries tau, 1/nt and the inverse-DST normalisation.
// The scaling, divide and unscaling use tables of the transform's precision
// (the FP32 tables are the FP64 ones rounded once on the host).
// gpowr = i rho^H gpow and gipr = rho^{-H} gipw fold the second half's factors
// into the tables (one operation fewer per element on each side).
template <typename R, int MAXB4, bool LDCG = false, bool PDL = true>
__device__ __forceinline__ void time_solve_tile(const R* in, R* out, long long Nx, int lh, int lw,
                                                const cplx<R>* __restrict__ tw, const cplx<R>* __restrict__ gpow,
                                                const cplx<R>* __restrict__ gipw, const cplx<R>* __restrict__ ak,
                                                const R* __restrict__ lamtau, R cnorm,
                                                const cplx<R>* __restrict__ gpowr, const cplx<R>* __restrict__ gipr,
                                                const cplx<R>* __restrict__ qinv, int delta_rhs, int n0_only,
                                                long long tile, unsigned char* smem_raw) {
    using C = cplx<R>;
    const int H = 1 << lh, W = 1 << lw;
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* stw = buf + (H << lw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const long long l0 = tile * W;

    if (PDL) pdl_trigger();
    for (int i = tid; i < H; i += nth) stw[i] = tw[i];
    if (PDL) pdl_wait();                                 // the input is a predecessor's output
    if (delta_rhs) {
        // f = f^0 e_0: Step (a) of a single level-0 value is that value (times
        // gamma^0) at every frequency, so the forward transform is not computed
        const C g = gpow[0];
        for (int e = tid; e < (H << lw); e += nth) {
            const long long l = l0 + (e & (W - 1));
            const R f0 = l < Nx ? ldin<LDCG>(in + l) : R(0);
            buf[e] = mkc(g.x * f0, g.y * f0);
        }
        __syncthreads();
    } else {
        for (int e = tid; e < (H << lw); e += nth) {
            int t = e >> lw, c = e & (W - 1);
            long long l = l0 + c;
            R f0 = R(0), f1 = R(0);
            if (l < Nx) {
                f0 = ldin<LDCG>(in + (long long)t * Nx + l);
                f1 = ldin<LDCG>(in + (long long)(t + H) * Nx + l);
            }
            const C g = gpow[t], gr = gpowr[t];      // gamma^t f0 + i rho^H gamma^t f1
            buf[e] = mkc(rfma(g.x, f0, gr.x * f1), rfma(g.y, f0, gr.y * f1));
        }
        __syncthreads();
        fft_tile<+1, MAXB4>(buf, stw, lh, lw);
    }

    if (qinv) {                                          // the plan's table of cnorm / (d_{2m} + tau Lambda_l)
        for (int e = tid; e < (H << lw); e += nth) {
            int k = e >> lw, c = e & (W - 1);
            long long l = l0 + c;
            if (l < Nx) buf[e] = cmul(buf[e], qinv[(long long)k * Nx + l]);
        }
    } else {
        for (int e = tid; e < (H << lw); e += nth) {
            int k = e >> lw, c = e & (W - 1);
            long long l = l0 + c;
            R lt = l < Nx ? lamtau[l] : R(0);
            C a = ak[k];
            R zr = a.x + lt, zi = a.y;
            R inv = cnorm / (zr * zr + zi * zi);
            C u = buf[e];
            buf[e] = mkc((u.x * zr + u.y * zi) * inv, (u.y * zr - u.x * zi) * inv);
        }
    }
    __syncthreads();
    fft_tile<-1, MAXB4>(buf, stw, lh, lw);

    const int tmax = n0_only ? 1 : H;
    for (int e = tid; e < (tmax << lw); e += nth) {
        int t = e >> lw, c = e & (W - 1);
        long long l = l0 + c;
        if (l < Nx) {
            const C w = buf[e];
            const C gi = gipw[t];
            out[(long long)t * Nx + l] = rfma(gi.x, w.x, -gi.y * w.y);
            if (!n0_only) {
                const C gr = gipr[t];
                out[(long long)(t + H) * Nx + l] = rfma(gr.x, w.y, gr.y * w.x);
            }
        }
    }
}

}  // namespace qbvm
