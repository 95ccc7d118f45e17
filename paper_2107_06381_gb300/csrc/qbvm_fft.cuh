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
                    int step = P / (Ns * 4);        // exp(S 2 pi i k r/(4 Ns)) = tw^(k r step)
                    v[i][1] = cmul(v[i][1], twiddle<S>(tw, k * step));
                    v[i][2] = cmul(v[i][2], twiddle<S>(tw, 2 * k * step));
                    v[i][3] = cmul(v[i][3], twiddle<S>(tw, 3 * k * step));
                }
                dft4<S>(v[i][0], v[i][1], v[i][2], v[i][3]);
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
                C t = v[i][1];
                if (Ns > 1) t = cmul(t, twiddle<S>(tw, k * (P / (Ns * 2))));
                int d = (j - k) * 2 + k;
                buf[d * W + c] = cadd(v[i][0], t);
                buf[(d + Ns) * W + c] = csub(v[i][0], t);
            }
        }
        __syncthreads();
    }
}

}  // namespace qbvm
