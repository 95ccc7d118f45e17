// qbvm_df.cuh -- double-float helpers shared by the refinement residuals
// (the staged kernels of qbvm_kernels.cu and the fused small-instance
// refinement of qbvm_refine1d.cu): unnormalised pair arithmetic, the
// truncating FP64 -> pair split, a scaled sum of squares and a block sum.
#pragma once
#include <cuda_runtime.h>

#include "qbvm_fft.cuh"

namespace qbvm {

__device__ __forceinline__ double block_sum(double v, double* sh) {
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

// Sum of squares in FP32 with a power-of-two scale that follows the largest
// magnitude seen (sum = ssq * 4^e, every term scaled by 2^-e first), so that
// neither tiny nor huge data underflow or overflow; rescaling is exact.
struct ScaledSsq {
    float ssq = 0.f, inv = 0x1p100f, lim = 0x1p-99f;
    int e = -100;
    // 2^k as an FP32 for -126 <= k <= 127
    static __device__ __forceinline__ float p2(int k) { return __uint_as_float((unsigned)(127 + k) << 23); }
    __device__ __forceinline__ void add(float x) {
        const float a = fabsf(x);
        if (a >= lim) {                                   // a is normal: lim >= 2^-99
            const int ne = (int)((__float_as_uint(a) >> 23) & 0xFF) - 127;
            const int d = 2 * (e - ne);                  // < 0
            ssq = d >= -126 ? ssq * p2(d) : 0.f;         // terms below 2^-126 of the new scale vanish
            e = ne;
            inv = ne <= 126 ? p2(-ne) : 0x1p-127f;
            lim = ne <= 126 ? p2(ne + 1) : __uint_as_float(0x7F800000u);
        }
        const float xs = x * inv;
        ssq = fmaf(xs, xs, ssq);
    }
    __device__ __forceinline__ double value() const {
        return (double)ssq * __longlong_as_double((long long)(1023 + 2 * e) << 52);
    }
};

// FP64 -> double-float by truncation on the integer pipes: hi keeps the top 24
// significand bits of x, lo the next 23 (as 2^K(1 + m) - 2^K, one exact FP32
// subtraction).  |x - (hi + lo)| < 2^-46 |x|: the size of the double-float
// iterate's own representation error, which is all the residual needs (the
// round-to-nearest split, qbvm_split_d, costs about three times as many
// instructions).  Values whose hi or lo would leave the normal FP32 range take
// qbvm_split_d.
__device__ __forceinline__ dfloat df_from_double_trunc(double x) {
    const unsigned int H = (unsigned int)__double2hiint(x), L = (unsigned int)__double2loint(x);
    const int fe = (int)((H >> 20) & 0x7FFu) - 1023 + 127;
    if (fe < 30 || fe > 253) return df_from_double(x);
    const unsigned int sg = H & 0x80000000u;
    const float hi = __uint_as_float(sg | ((unsigned int)fe << 23) | ((H & 0xFFFFFu) << 3) | (L >> 29));
    const unsigned int kb = sg | ((unsigned int)(fe - 23) << 23);
    const float lo = __uint_as_float(kb | ((L & 0x1FFFFFFFu) >> 6)) - __uint_as_float(kb);
    return {hi, lo};
}

// (a.hi + a.lo) * (c.hi + c.lo) as an unnormalised pair (the c.lo * a.lo term,
// 2^-48 relative, dropped): 4 operations.
__device__ __forceinline__ dfloat df_mul_un(dfloat c, dfloat a) {
    const float p = c.hi * a.hi;
    float e = fmaf(c.hi, a.hi, -p);
    e = fmaf(c.hi, a.lo, e);
    e = fmaf(c.lo, a.hi, e);
    return {p, e};
}
// a - b as an unnormalised pair: exact two-sum of the high parts, low parts
// and the rounding error summed in FP32 (error O(u^2 (|a| + |b|))).
__device__ __forceinline__ dfloat df_sub_un(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, -b.hi);
    return {s.hi, s.lo + (a.lo - b.lo)};
}
__device__ __forceinline__ dfloat df_add_un(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return {s.hi, s.lo + (a.lo + b.lo)};
}

}  // namespace qbvm
