// qbvm_fft.cuh -- complex arithmetic and a shared-memory FFT engine for the
// time transforms (Section 3.3, steps (a) and (c) of eq. 3.8) and for the
// DST-I diagonalisation of the Dirichlet Laplacian (Step (b) in 2D/3D).
//
// Tile model: a CTA holds W columns of one power-of-two length P in shared
// memory, element (t, c) at index t * W + c (column index fastest, so that a
// warp touching consecutive columns of one row is bank-conflict free).  All
// threads of the CTA cooperate on every pass.
//
// FFT: Stockham autosort (decimation in time; Govindaraju et al., "High
// performance discrete Fourier transforms on graphics processors", SC 2008),
// radix 4 with one radix-2 pass when log2 P is odd, natural-order output.
// Each pass reads its butterfly inputs into registers, synchronises, and
// writes the outputs back in place, so one buffer suffices.  Twiddles come
// from a table tw[m] = exp(-2 pi i m / P) (m < P) built in FP64 on the host;
// the sign template argument S selects exp(S * 2 pi i jk / P).
#pragma once
#include <cuda_runtime.h>

namespace qbvm {

template <typename R> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float>  { using type = float2;  };
template <typename R> using cplx = typename C2<R>::type;

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialisation may start while the kernel before it in the stream finishes:
// it signals at entry that its own successor may be scheduled
// (pdl_trigger), loads its constant tables, and waits (pdl_wait) until the
// predecessor has completed and its writes are visible before it touches any
// buffer a predecessor writes.  In a kernel launched the ordinary way both are
// no-ops.
__device__ __forceinline__ void pdl_trigger() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2  mkc(float a, float b)   { return make_float2(a, b); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2  cadd(float2 a, float2 b)   { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2  csub(float2 a, float2 b)   { return make_float2(a.x - b.x, a.y - b.y); }
// a * b
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by S*i (S = +1 or -1)
template <int S, typename C> __device__ __forceinline__ C cmul_si(C a) {
    return S > 0 ? mkc(-a.y, a.x) : mkc(a.y, -a.x);
}
// twiddle exp(S * 2 pi i m / P) from the table of exp(-2 pi i m / P)
template <int S, typename C> __device__ __forceinline__ C twiddle(const C* tw, int m) {
    C w = tw[m];
    if (S > 0) w.y = -w.y;
    return w;
}

__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }

// a + w b and a - w b with fused multiply-adds (the difference as 2a - (a + w b)):
// 6 operations instead of the 8 of a complex product and two complex sums.
__device__ __forceinline__ void fma_bfly(double2 a, double2 b, double2 w, double2& p, double2& m) {
    p = make_double2(fma(w.x, b.x, fma(-w.y, b.y, a.x)), fma(w.x, b.y, fma(w.y, b.x, a.y)));
    m = make_double2(fma(2.0, a.x, -p.x), fma(2.0, a.y, -p.y));
}
__device__ __forceinline__ void fma_bfly(float2 a, float2 b, float2 w, float2& p, float2& m) {
    p = make_float2(fmaf(w.x, b.x, fmaf(-w.y, b.y, a.x)), fmaf(w.x, b.y, fmaf(w.y, b.x, a.y)));
    m = make_float2(fmaf(2.f, a.x, -p.x), fmaf(2.f, a.y, -p.y));
}

// Radix-4 DFT with kernel exp(S * 2 pi i / 4) in registers.
template <int S, typename C> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
    C a0 = cadd(v0, v2), a1 = csub(v0, v2);
    C a2 = cadd(v1, v3), a3 = cmul_si<S>(csub(v1, v3));
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = cadd(a1, a3);
    v3 = csub(a1, a3);
}

// In-place FFT of W = 2^lw columns of length P = 2^lp held at buf[t * W + c].
// Requires: P >= 2 and W * P / 4 <= MAXB4 * blockDim.x (each thread keeps at
// most MAXB4 radix-4 butterflies, or 2*MAXB4 radix-2 ones, in registers).
// Ends with __syncthreads().
template <int S, int MAXB4, typename C>
__device__ __forceinline__ void fft_tile(C* buf, const C* tw, int lp, int lw) {
    const int P = 1 << lp, W = 1 << lw;
    const int nth = blockDim.x;
    const int tid = threadIdx.x;
    int Ns = 1;
    // radix-4 passes
    const int nb4 = W * (P >> 2);
    while (Ns * 4 <= P) {
        C v[MAXB4][4];
        int cnt = 0;
        const int q = P >> 2;
#pragma unroll
        for (int i = 0; i < MAXB4; ++i) {
            int b = tid + i * nth;
            if (b < nb4) {
                int c = b & (W - 1), j = b >> lw;
#pragma unroll
                for (int r = 0; r < 4; ++r) v[i][r] = buf[(j + r * q) * W + c];
                cnt = i + 1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < MAXB4; ++i) {
            if (i < cnt) {
                int b = tid + i * nth;
                int c = b & (W - 1), j = b >> lw;
                int k = j & (Ns - 1);
                if (Ns > 1) {
                    // twiddled radix-4 with w3 = w1 w2 factored out:
                    //   x0 +- w2 x2,  x1 +- w2 x3,  then (a0 +- w1 b0), (a1 +- S i w1 b1)
                    int step = P / (Ns * 4);        // exp(S 2 pi i k r/(4 Ns)) = tw^(k r step)
                    const C w1 = twiddle<S>(tw, k * step), w2 = twiddle<S>(tw, 2 * k * step);
                    C a0, a1, b0, b1;
                    fma_bfly(v[i][0], v[i][2], w2, a0, a1);
                    fma_bfly(v[i][1], v[i][3], w2, b0, b1);
                    fma_bfly(a0, b0, w1, v[i][0], v[i][2]);
                    fma_bfly(a1, b1, cmul_si<S>(w1), v[i][1], v[i][3]);
                } else {
                    dft4<S>(v[i][0], v[i][1], v[i][2], v[i][3]);
                }
                int d = (j - k) * 4 + k;
#pragma unroll
                for (int r = 0; r < 4; ++r) buf[(d + r * Ns) * W + c] = v[i][r];
            }
        }
        __syncthreads();
        Ns *= 4;
    }
    if (Ns < P) {   // one radix-2 pass (log2 P odd)
        const int nb2 = W * (P >> 1);
        const int q = P >> 1;
        C v[2 * MAXB4][2];
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < 2 * MAXB4; ++i) {
            int b = tid + i * nth;
            if (b < nb2) {
                int c = b & (W - 1), j = b >> lw;
                v[i][0] = buf[j * W + c];
                v[i][1] = buf[(j + q) * W + c];
                cnt = i + 1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 2 * MAXB4; ++i) {
            if (i < cnt) {
                int b = tid + i * nth;
                int c = b & (W - 1), j = b >> lw;
                int k = j & (Ns - 1);
                int d = (j - k) * 2 + k;
                C y0, y1;
                if (Ns > 1) {
                    fma_bfly(v[i][0], v[i][1], twiddle<S>(tw, k * (P / (Ns * 2))), y0, y1);
                } else {
                    y0 = cadd(v[i][0], v[i][1]);
                    y1 = csub(v[i][0], v[i][1]);
                }
                buf[d * W + c] = y0;
                buf[(d + Ns) * W + c] = y1;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)/2), about 48 significand bits, computed entirely on
// the FP32 pipes.  Error-free transformations: Knuth's two-sum for additions,
// Dekker's product with the error term recovered by one fused multiply-add.
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {   // requires |a| >= |b|
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    dfloat s = df_two_sum(a.hi, b.hi);
    dfloat t = df_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return df_fast_two_sum(s.hi, s.lo);
}
// Double-float sum with one two-sum of the high parts: the absolute error is
// O(u^2 (|a| + |b|)) (u = 2^-24) rather than O(u^2 |a + b|) -- the bound a
// residual needs, since its inputs carry representation errors of that size.
__device__ __forceinline__ dfloat df_add_sloppy(dfloat a, dfloat b) {
    dfloat s = df_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfloat df_add_f(dfloat a, float b) {
    dfloat s = df_two_sum(a.hi, b);
    s.lo += a.lo;
    return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
// ---------------------------------------------------------------------------
// FP64 <-> FP32 conversions on the integer pipes.  On GB300 the hardware
// conversions issue on the FP64 pipe (2 per clock per SM), which made them the
// bottleneck of the FP32 refinement path; these bit manipulations give the
// same results for every finite value in the normal FP32 range and fall back
// to the hardware instructions outside it.
#ifdef __CUDACC__
#define QBVM_HD __host__ __device__ __forceinline__
#else
#define QBVM_HD inline
#endif

QBVM_HD unsigned long long qbvm_dbits(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long u;
    __builtin_memcpy(&u, &x, 8);
    return u;
#endif
}
QBVM_HD double qbvm_bitsd(unsigned long long u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    __builtin_memcpy(&x, &u, 8);
    return x;
#endif
}
QBVM_HD unsigned int qbvm_fbits(float x) {
#ifdef __CUDA_ARCH__
    return (unsigned int)__float_as_uint(x);
#else
    unsigned int u;
    __builtin_memcpy(&u, &x, 4);
    return u;
#endif
}
QBVM_HD int qbvm_clzll(unsigned long long a) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)a);
#else
    return __builtin_clzll(a);
#endif
}
QBVM_HD int qbvm_clz(unsigned int a) {
#ifdef __CUDA_ARCH__
    return __clz((int)a);
#else
    return __builtin_clz(a);
#endif
}
QBVM_HD float qbvm_bitsf(unsigned int u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    __builtin_memcpy(&x, &u, 4);
    return x;
#endif
}

// The hardware conversions for the rare operands outside the integer paths
// range.  Out of line on the device, so that the compiler cannot evaluate them
// speculatively (as a predicated select) for every element.
#ifdef __CUDA_ARCH__
static __device__ __noinline__ float qbvm_rem_hw(double x, float h) { return (float)(x - (double)h); }
static __device__ __noinline__ float qbvm_f_hw(double x) { return (float)x; }
static __device__ __noinline__ double qbvm_join_hw(float hi, float lo) { return (double)hi + (double)lo; }
#else
inline float qbvm_rem_hw(double x, float h) { return (float)(x - (double)h); }
inline float qbvm_f_hw(double x) { return (float)x; }
inline double qbvm_join_hw(float hi, float lo) { return (double)hi + (double)lo; }
#endif

// High and low 32-bit words of a double.  On the device these are register
// moves the compiler cannot see through: tests on the bits of the reinterpreted
// 64-bit value were turned into FP64 compares (FP64-pipe instructions).
QBVM_HD unsigned int qbvm_dhi(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned int)__double2hiint(x);
#else
    return (unsigned int)(qbvm_dbits(x) >> 32);
#endif
}
QBVM_HD unsigned int qbvm_dlo(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned int)__double2loint(x);
#else
    return (unsigned int)qbvm_dbits(x);
#endif
}

// Round-to-nearest-even FP64 -> FP32 of x, and the exact remainder x - hi as
// an FP32 (rounded to nearest; the remainder has at most 29 significant bits).
// 32-bit integer arithmetic on the two words of x.
QBVM_HD void qbvm_split_d(double x, float* hi, float* lo) {
    const unsigned int H = qbvm_dhi(x), L = qbvm_dlo(x);
    if (((H << 1) | L) == 0) {                            // +-0: exact, integer path
        *hi = qbvm_bitsf(H);
        *lo = 0.0f;
        return;
    }
    const int e = (int)((H >> 20) & 0x7FF);
    const int fe = e - 1023 + 127;                       // FP32 biased exponent of hi
    if (fe < 30 || fe > 253) {                           // tiny, huge, Inf, NaN: hardware path
        float h = qbvm_f_hw(x);
        *hi = h;
        *lo = qbvm_rem_hw(x, h);
        return;
    }
    const unsigned int sign = H & 0x80000000u;
    // 53-bit significand = [1 | 20 bits of H | 32 bits of L]; its top 24 bits:
    unsigned int q = (((H & 0xFFFFFu) | 0x100000u) << 3) | (L >> 29);
    const unsigned int rem = L & 0x1FFFFFFFu;            // the 29 bits below
    int r;                                                // remainder in units of 2^(e - 1075), |r| <= 2^28
    if (rem > 0x10000000u || (rem == 0x10000000u && (q & 1))) {
        ++q;
        r = (int)rem - 0x20000000;
    } else {
        r = (int)rem;
    }
    int he = fe;
    if (q == 0x1000000u) {                                // rounding carried into a new binade
        q >>= 1;
        ++he;
    }
    *hi = qbvm_bitsf(sign | ((unsigned int)he << 23) | (q & 0x7FFFFFu));
    if (r == 0) {
        *lo = 0.0f;
        return;
    }
    // lo = sign * r * 2^(e - 1075): normalise |r| (<= 29 bits) to 24 bits, RNE
    const unsigned int a = (unsigned int)(r < 0 ? -r : r);
    const unsigned int lsign = sign ^ (r < 0 ? 0x80000000u : 0u);
    const int top = 31 - qbvm_clz(a);                    // position of the leading bit (0..28)
    int le = (e - 1075) + top + 127;                      // FP32 biased exponent of lo
    unsigned int lq;
    if (top > 23) {
        const int sh = top - 23;
        lq = a >> sh;
        const unsigned int lr = a & ((1u << sh) - 1), half = 1u << (sh - 1);
        if (lr > half || (lr == half && (lq & 1))) ++lq;
        if (lq == 0x1000000u) {
            lq >>= 1;
            ++le;
        }
    } else {
        lq = a << (23 - top);
    }
    if (le < 1) {                                         // below the FP32 normal range: hardware path
        *lo = qbvm_rem_hw(x, *hi);
        return;
    }
    *lo = qbvm_bitsf(lsign | ((unsigned int)le << 23) | (lq & 0x7FFFFFu));
}

// (double)hi + (double)lo, correctly rounded, for a pair with |lo| <= |hi|
// (hi's significand is placed 39 bits up; lo is aligned below it with a sticky
// bit for whatever falls off, then the sum is rounded to 53 bits, ties to even).
QBVM_HD double qbvm_join_df(float hi, float lo) {
    const unsigned int hb = qbvm_fbits(hi), lb = qbvm_fbits(lo);
    const int e1 = (int)((hb >> 23) & 0xFF), e2 = (int)((lb >> 23) & 0xFF);
    if ((hb << 1) == 0 && (lb << 1) == 0)                 // 0 + 0 (sign as the hardware sum gives)
        return qbvm_bitsd((unsigned long long)(hb & lb & 0x80000000u) << 32);
    if ((hb << 1) == 0 && e2 != 0 && e2 != 255)           // 0 + normal lo: lo widened exactly
        return qbvm_bitsd(((unsigned long long)(lb & 0x80000000u) << 32) |
                          ((unsigned long long)(e2 - 127 + 1023) << 52) |
                          ((unsigned long long)(lb & 0x7FFFFFu) << 29));
    if (e1 == 0 || e1 == 255 || e2 == 255 || (e2 == 0 && (lb & 0x7FFFFFu)) || e2 > e1)
        return qbvm_join_hw(hi, lo);                      // zero/denormal/Inf/NaN/unnormalised: hardware
    if (((hb ^ lb) & 0x80000000u) && e2 != 0 && e1 - e2 <= 1)
        return qbvm_join_hw(hi, lo);                      // opposite signs within a binade: the sum may cancel
    const unsigned long long sign = (unsigned long long)(hb & 0x80000000u) << 32;
    long long S = (long long)((unsigned long long)((hb & 0x7FFFFFu) | 0x800000u) << 39);   // < 2^63
    if (e2 != 0) {
        const unsigned long long M2 = (lb & 0x7FFFFFu) | 0x800000u;
        const int d = e1 - e2;
        long long B;
        if (d <= 39) {
            B = (long long)(M2 << (39 - d));
        } else if (d - 39 < 40) {
            const int sh = d - 39;
            B = (long long)(M2 >> sh) | (long long)((M2 & ((1ull << sh) - 1)) != 0);
        } else {
            B = 1;                                        // only the sticky bit survives
        }
        if ((hb ^ lb) & 0x80000000u) S -= B;
        else S += B;
    }
    // S in (2^61, 2^63): leading bit p, round to 53 bits
    const int p = 63 - qbvm_clzll((unsigned long long)S);
    const int sh = p - 52;
    unsigned long long q = (unsigned long long)S >> sh;
    const unsigned long long rem = (unsigned long long)S & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    int de = (e1 - 127) + (p - 62) + 1023;               // hi's leading bit sits at position 62
    if (rem > half || (rem == half && (q & 1))) ++q;
    if (q == (1ull << 53)) {
        q >>= 1;
        ++de;
    }
    return qbvm_bitsd(sign | ((unsigned long long)de << 52) | (q & 0xFFFFFFFFFFFFFull));
}

// FP64 -> double-float and back, on the integer pipes.
__device__ __forceinline__ dfloat df_from_double(double x) {
    dfloat r;
    qbvm_split_d(x, &r.hi, &r.lo);
    return r;
}
__device__ __forceinline__ double df_to_double(dfloat a) { return qbvm_join_df(a.hi, a.lo); }

// The same join where the integer pipes are the bottleneck: for normal hi and
// lo (or lo = +-0) the exact widenings to FP64 are built from the bits (sign,
// exponent rebased by 1023 - 127, significand shifted by 29) and summed by one
// FP64 add, which rounds to nearest even exactly as qbvm_join_df does; any
// other operand takes qbvm_join_df.  One FP64-pipe operation per value.
__device__ __forceinline__ double qbvm_widen_normal(unsigned int b) {
    const unsigned int w = (b & 0x80000000u) | ((((b >> 23) & 0xFFu) + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)w, (int)(b << 29));
}
__device__ __forceinline__ double qbvm_join_df_dadd(float hi, float lo) {
    const unsigned int hb = __float_as_uint(hi), lb = __float_as_uint(lo);
    const unsigned int e1 = (hb >> 23) & 0xFFu, e2 = (lb >> 23) & 0xFFu;
    if (e1 - 1u < 254u) {                                 // hi normal
        const double dh = qbvm_widen_normal(hb);
        if ((lb << 1) == 0) return dh;                    // lo = +-0
        if (e2 - 1u < 254u) return __dadd_rn(dh, qbvm_widen_normal(lb));
    }
    return qbvm_join_df(hi, lo);
}
__device__ __forceinline__ float d2f_int(double x) {
    float h, l;
    qbvm_split_d(x, &h, &l);
    return h;
}

}  // namespace qbvm
