// qbvm_dst.cuh -- the DST-I tile (Step (b) in 2D/3D: diagonalisation of the
// Dirichlet Laplacian), shared by the per-pass kernels and the persistent
// batch kernel.
#pragma once
#include <cstdint>
#include <type_traits>

#include "qbvm_fft.cuh"
#include "qbvm_internal.h"

namespace qbvm {

// ------------------------------------------------------------------ DST-I
//
// y_k = sum_{j=1}^{n} x_j sin(pi j k / M), n = M - 1, with one complex FFT of
// length M for two real columns.  With x_0 = x_M = 0 and s_j = sin(j pi/M),
//     w_j = s_j (x_j + x_{M-j}) + (x_j - x_{M-j}) / 2,   j = 0..M-1,
// the DFT W_k = sum_j w_j exp(-2 pi i jk/M) satisfies
//     y_{2k} = -Im W_k,   y_{2k+1} - y_{2k-1} = Re W_k   (y_{-1} = -y_1),
// (the symmetric part of w carries the cosine sums, the antisymmetric part the
// sine sums), so the even outputs are read off and the odd ones are a prefix
// sum.  Columns a and b are packed as w^a + i w^b and separated with
// W^a_k = (Z_k + conj Z_{M-k})/2, W^b_k = (Z_k - conj Z_{M-k})/(2i).
//
// TIN is the element type read (FP64 input to an FP32 transform is rounded on
// load); OMODE selects the store: 0 = R values, 1 = accumulate into a
// double-float array (out += v, exact two-sum), 2 = double-float array
// (out = v), 3 = FP64 array.
// Value of precision R from an input element (FP64 -> FP32 on the integer pipes).
template <typename R, typename TIN>
__device__ __forceinline__ R to_r(TIN v) {
    if (std::is_same<R, float>::value && std::is_same<TIN, double>::value) return (R)d2f_int((double)v);
    return (R)v;
}

template <typename R, typename TIN, int OMODE, int MAXB4>
__device__ __forceinline__ void dst_store(void* out, long long idx, R v) {
    if (OMODE == 0) {
        reinterpret_cast<R*>(out)[idx] = v;
    } else if (OMODE == 1) {
        float2* o = reinterpret_cast<float2*>(out) + idx;
        float2 c = *o;
        dfloat r = df_add_f(dfloat{c.x, c.y}, (float)v);
        *o = make_float2(r.hi, r.lo);
    } else if (OMODE == 2) {
        reinterpret_cast<float2*>(out)[idx] = make_float2((float)v, 0.f);
    } else {
        reinterpret_cast<double*>(out)[idx] = (double)v;
    }
}

// Load of an input element; LDCG reads through L2 only (data written earlier
// in the same launch by other CTAs, as in the persistent batch kernel).
template <bool LDCG, typename T>
__device__ __forceinline__ T ldin(const T* p) {
    if (LDCG) return __ldcg(p);
    return *p;
}

constexpr int DST_TILE = 2048;     // complex elements per (full-width) DST tile

// One DST tile (`tile` selects 2W real columns) on a CTA of TILE_THREADS
// threads with dynamic shared memory `smem_raw` of dst_smem bytes.
// X4: produce 4 times the DST.  The factors 1/2 of the pre-processing and of
// the column separation then drop out (w'_j = 2 s_j (x_j + x_{M-j}) +
// (x_j - x_{M-j}) is one fused multiply-add), 2 operations fewer per element;
// the caller folds the exact power of two into its normalisation.
// PDL: programmatic dependent launch (tables before the wait; the kernels of
// the solve pipelines set it, the persistent sweep does not).
template <typename R, typename TIN, int OMODE, int MAXB4, bool LDCG, bool X4 = false, bool PDL = false>
__device__ __forceinline__ void dst_tile(const TIN* in, void* out, int n, int lm, int lw, long long outer,
                                         long long inner, long long tile, const cplx<R>* __restrict__ tw,
                                         const R* __restrict__ sn, unsigned char* smem_raw) {
    using C = cplx<R>;
    const int M = 1 << lm, W = 1 << lw, H = M >> 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int ncol = 2 * W;                          // real columns in this tile
    C* buf = reinterpret_cast<C*>(smem_raw);         // M x W complex
    R* obuf = reinterpret_cast<R*>(buf + (M << lw)); // M x 2W real (outputs y_1..y_n at rows 0..n-1)
    C* stw = reinterpret_cast<C*>(obuf + ((size_t)M << (lw + 1)));
    R* ssn = reinterpret_cast<R*>(stw + M);          // sin(j pi / M), j = 0..H
    R* seg = ssn + (H + 2);                          // prefix-sum segment totals
    R* bufr = reinterpret_cast<R*>(buf);

    if (PDL) pdl_trigger();
    for (int i = tid; i < M; i += nth) stw[i] = tw[i];
    for (int i = tid; i <= H; i += nth) ssn[i] = X4 ? R(2) * sn[i] : sn[i];
    for (int p = tid; p < W; p += nth) buf[p] = mkc(R(0), R(0));
    if (PDL) pdl_wait();

    long long base_row = 0, o = 0, i0 = 0;
    int rows_here = ncol;
    if (inner == 1) {
        // rows are contiguous: stage the tile [rows][n] linearly (coalesced, 16-byte
        // vectors when aligned), then scatter into the column layout; the raw
        // stride n is odd, so the transposing reads are bank-conflict free
        base_row = tile * ncol;
        rows_here = (int)min((long long)ncol, outer - base_row);
        const int count = rows_here * n;
        const TIN* src = in + base_row * n;
        R* raw = obuf;
        constexpr int VEC = 16 / sizeof(TIN);
        if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (count % VEC) == 0) {
            using V = typename std::conditional<sizeof(TIN) == 8, double2, float4>::type;
            const V* sv = reinterpret_cast<const V*>(src);
            for (int i = tid; i < count / VEC; i += nth) {
                V v = ldin<LDCG>(sv + i);
                const TIN* pv = reinterpret_cast<const TIN*>(&v);
#pragma unroll
                for (int q = 0; q < VEC; ++q) raw[i * VEC + q] = to_r<R, TIN>(pv[q]);
            }
        } else {
            for (int i = tid; i < count; i += nth) raw[i] = to_r<R, TIN>(ldin<LDCG>(src + i));
        }
        __syncthreads();
        for (int e = tid; e < ncol * n; e += nth) {
            int j = e >> (lw + 1), r = e & (ncol - 1);
            R v = r < rows_here ? raw[r * n + j] : R(0);
            bufr[((j + 1) << (lw + 1)) + r] = v;
        }
    } else {
        long long tiles_per_outer = (inner + ncol - 1) / ncol;
        o = tile / tiles_per_outer;
        i0 = (tile - o * tiles_per_outer) * ncol;
        const TIN* src = in + o * (long long)n * inner;
        for (int e = tid; e < ncol * n; e += nth) {
            int j = e >> (lw + 1), r = e & (ncol - 1);
            long long ii = i0 + r;
            R v = ii < inner ? to_r<R, TIN>(ldin<LDCG>(src + (long long)j * inner + ii)) : R(0);
            bufr[((j + 1) << (lw + 1)) + r] = v;
        }
    }
    __syncthreads();
    // w_j and w_{M-j} from the pair (x_j, x_{M-j}), j = 1..H
    for (int e = tid; e < (H << lw); e += nth) {
        int j = (e >> lw) + 1, p = e & (W - 1);
        C a = buf[(j << lw) + p], b = buf[((M - j) << lw) + p];
        R sj = ssn[j];
        C S = mkc(a.x + b.x, a.y + b.y);
        C D = X4 ? mkc(a.x - b.x, a.y - b.y) : mkc(R(0.5) * (a.x - b.x), R(0.5) * (a.y - b.y));
        buf[(j << lw) + p] = mkc(rfma(sj, S.x, D.x), rfma(sj, S.y, D.y));
        if (j != H) buf[((M - j) << lw) + p] = mkc(rfma(sj, S.x, -D.x), rfma(sj, S.y, -D.y));
    }
    __syncthreads();
    fft_tile<-1, MAXB4>(buf, stw, lm, lw);

    // separate the packed columns; even outputs and odd increments into obuf
    for (int e = tid; e < (H << lw); e += nth) {
        int k = e >> lw, p = e & (W - 1);
        C zk = buf[(k << lw) + p], zm = buf[(((M - k) & (M - 1)) << lw) + p];
        const R hf = X4 ? R(1) : R(0.5);
        R ra = hf * (zk.x + zm.x), rb = hf * (zk.y + zm.y);
        if (k == 0) {
            ra *= R(0.5);
            rb *= R(0.5);
        } else {
            C* ev = reinterpret_cast<C*>(obuf + ((size_t)(2 * k - 1) << (lw + 1)));
            ev[p] = mkc(hf * (zm.y - zk.y), hf * (zk.x - zm.x));
        }
        C* od = reinterpret_cast<C*>(obuf + ((size_t)(2 * k) << (lw + 1)));
        od[p] = mkc(ra, rb);
    }
    __syncthreads();
    // y_{2k+1} = sum_{kappa <= k} (odd increments): segmented prefix sum per real column
    // the segment count of the full-width tile whatever this tile's width, so
    // that the prefix sums (and their rounding) do not depend on the width
    const int wfull = (DST_TILE >> lm) > 0 ? (DST_TILE >> lm) : 1;
    const int segs = nth >= 2 * wfull ? nth / (2 * wfull) : 1;
    const int L = (H + segs - 1) / segs;
    for (int task = tid; task < ncol * segs; task += nth) {
        int c = task % ncol, sg = task / ncol;
        int k0 = sg * L, k1 = min(H, k0 + L);
        R acc = R(0);
        for (int k = k0; k < k1; ++k) {
            R* v = obuf + ((size_t)(2 * k) << (lw + 1)) + c;
            acc += *v;
            *v = acc;
        }
        seg[sg * ncol + c] = acc;
    }
    __syncthreads();
    if (segs > 1) {
        for (int task = tid; task < ncol * segs; task += nth) {
            int c = task % ncol, sg = task / ncol;
            if (sg == 0) continue;
            R off = R(0);
            for (int s2 = 0; s2 < sg; ++s2) off += seg[s2 * ncol + c];
            int k0 = sg * L, k1 = min(H, k0 + L);
            for (int k = k0; k < k1; ++k) obuf[((size_t)(2 * k) << (lw + 1)) + c] += off;
        }
        __syncthreads();
    }
    if (inner == 1) {
        // transpose obuf [j][column] -> raw [column][j] (odd stride n), then store linearly
        R* raw = bufr;
        for (int e = tid; e < ncol * n; e += nth) {
            int j = e >> (lw + 1), r = e & (ncol - 1);
            raw[r * n + j] = obuf[e];
        }
        __syncthreads();
        const int count = rows_here * n;
        const long long start = base_row * n;
        for (int i = tid; i < count; i += nth) dst_store<R, TIN, OMODE, MAXB4>(out, start + i, raw[i]);
    } else {
        const long long base = o * (long long)n * inner;
        for (int e = tid; e < ncol * n; e += nth) {
            int j = e >> (lw + 1), r = e & (ncol - 1);
            long long ii = i0 + r;
            if (ii < inner) dst_store<R, TIN, OMODE, MAXB4>(out, base + (long long)j * inner + ii, obuf[e]);
        }
    }
}

__host__ __device__ inline int dst_lw(int lm) {
    int lw = 0;
    while (((1 << lm) << (lw + 1)) <= DST_TILE) ++lw;
    return lw;
}

template <typename R>
inline size_t dst_smem(int lm, int lw) {
    const int M = 1 << lm, W = 1 << lw, H = M >> 1;
    const int ncol = 2 * W;
    size_t seg = (size_t)(TILE_THREADS >= ncol ? TILE_THREADS : ncol);
    return sizeof(cplx<R>) * ((size_t)M * W + M) + sizeof(R) * ((size_t)M * 2 * W + H + 2 + seg);
}
template <typename R>
inline size_t dst_smem(int lm) { return dst_smem<R>(lm, dst_lw(lm)); }

}  // namespace qbvm
