// qbvm_dfsum.cuh -- one term of the FP64 alpha sweep's spectral sums in
// double-float arithmetic: Re 1/z for z = d_{2m} + tau Lambda_l (Step (b) of
// Section 3.3 divides by it, Step (c) at t = 0 sums it over the even
// frequencies 2m), added to a double-float accumulator.  Host-and-device code:
// the kernels call it, and a host build checks it against long double
// (tests/native/df_scan_sum_check.cu).
//
// Per term:
//   z_r   two-sum of the high words, the low words added, renormalised (its
//         absolute error ~2^-48 (|Re d| + tau Lambda), as FP64's rounding of
//         the same sum is 2^-53 of it);
//   den   z_r^2 + |Im d|^2, the products' errors recovered by fused
//         multiply-adds (|Im d|^2 once per frequency: df_scan_im2);
//   q1    z_r.hi / den.hi through the approximate FP32 reciprocal r;
//   c     the remainder z_r - den q1 -- about 2^-22 |z_r|, which fused
//         multiply-adds give to about 2^-46 |z_r| -- times r;
//   sum   q1 two-summed into the high word, its rounding error and c added to
//         the low word; df_scan_fold moves the low word into the high one
//         (every few terms: a low word left to grow rounds at its own size).
// Each term to about 2^-44 of its scale: its magnitude, or (|Re d| + tau
// Lambda) / |z|^2 where Re d + tau Lambda cancels (FP64 rounds that sum at
// 2^-53 of the same).  A sum of H terms to about 6e-14 of the sum of their
// magnitudes, against about 1e-16 for FP64 summation, so a sum whose terms
// cancel keeps fewer digits than FP64 would (over the 512-instance sweep
// workload's ranges the host check finds up to 1.5e-9 of a mode's sum, where
// FP64 keeps 7e-11).
#pragma once

#include <cmath>

#include "qbvm_fft.cuh"

namespace qbvm {

// |Im d|^2 of one frequency as an unnormalised pair (p, e): p the rounded
// square of the high word, e its error plus 2 hi lo.
struct DfSq {
    float p, e;
};
QBVM_HD DfSq df_scan_im2(float ih, float il) {
    const float p = ih * ih;
    return {p, fmaf(ih + ih, il, fmaf(ih, ih, -p))};
}

// The approximate FP32 reciprocal (about 1 ulp) on the device; the quotient
// on the host.
QBVM_HD float df_scan_rcp(float x) {
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
#else
    return 1.0f / x;
#endif
}

// (shi, slo) += Re 1 / ((dxh + dxl) + (lh + ll) + i Im d), |Im d|^2 = im2.
QBVM_HD void df_scan_term(float dxh, float dxl, DfSq im2, float lh, float ll, float& shi, float& slo) {
    const float s = dxh + lh, sb = s - dxh;
    const float se = ((dxh - (s - sb)) + (lh - sb)) + (dxl + ll);
    const float zh = s + se, zl = se - (zh - s);
    const float rp = zh * zh;
    const float re = fmaf(zh + zh, zl, fmaf(zh, zh, -rp));
    const float dh = rp + im2.p, db = dh - rp;
    const float dl = ((rp - (dh - db)) + (im2.p - db)) + (re + im2.e);
    const float r = df_scan_rcp(dh);
    const float q1 = zh * r;
    const float t = fmaf(-dl, q1, fmaf(-dh, q1, zh) + zl);
    const float u = shi + q1, ub = u - shi;
    const float ue = (shi - (u - ub)) + (q1 - ub);
    shi = u;
    slo += fmaf(t, r, ue);
}

QBVM_HD void df_scan_fold(float& shi, float& slo) {
    const float s = shi + slo;
    slo = slo - (s - shi);
    shi = s;
}

}  // namespace qbvm
