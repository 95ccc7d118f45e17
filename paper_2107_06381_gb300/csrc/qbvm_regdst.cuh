// qbvm_regdst.cuh -- register-resident DST-I tile for the FP32 transforms of
// the refinement path (Step (b) in 2D/3D), lengths M = 64, 128, 256.
//
// Same algorithm as dst_tile (qbvm_dst.cuh): two real columns packed into one
// complex DFT of length M of w_j = s_j (x_j + x_{M-j}) + (x_j - x_{M-j})/2,
// even outputs y_{2k} read off, odd outputs a prefix sum of the increments.
// What differs is where the DFT runs.  M = N1 * N2 is split Cooley-Tukey
// style (n = N2 n1 + n2, k = k1 + N1 k2):
//     X[k1 + N1 k2] = sum_{n2} W_{N2}^{n2 k2} W_M^{n2 k1} sum_{n1} x[N2 n1 + n2] W_{N1}^{n1 k1},
// and T = N2 threads of one warp own one DFT: thread n2 does the length-N1 DFT
// over n1 in registers, multiplies by W_M^{n2 k1}, and after one padded
// shared-memory transpose each thread does the length-N2 DFTs of its k1 in
// registers.  Between the CTA-wide load and store phases only warp-level
// synchronisation is needed: a DFT touches nothing but its own two columns.
//
// Layouts (all padded so that the access patterns below are bank-conflict free):
//   XAX (rows of the tile are contiguous in memory, the x pass): staging
//     element (column c, j' = j - 1) at c * CS + j' + (j' >> LPAD);
//   YAX (the tile is 32 consecutive inner indices, the y / z passes): staging
//     element at (j' + (j' >> LPAD)) * RS + c, read and written as float2 pairs;
//   per-DFT buffer of FB complex: transpose [k1][n2] with row stride BS, then
//     the spectrum X[k] at k + (k >> ZP).
#pragma once
#include "qbvm_dst.cuh"
#include "qbvm_fft.cuh"

namespace qbvm {
namespace rd {

template <int LM> struct Cfg;
template <> struct Cfg<8> {
    static constexpr int N1 = 16, N2 = 16, CS = 280, RS = 34, LPAD = 4, BS = 17, ZP = 4, FB = 272;
};
template <> struct Cfg<7> {
    static constexpr int N1 = 16, N2 = 8, CS = 148, RS = 36, LPAD = 4, BS = 9, ZP = 3, FB = 152;
};
template <> struct Cfg<6> {
    static constexpr int N1 = 8, N2 = 8, CS = 84, RS = 36, LPAD = 3, BS = 9, ZP = 3, FB = 72;
};
constexpr int NFFT = 16;          // DFTs (column pairs) per CTA
constexpr int NCOL = 2 * NFFT;    // real columns per CTA

template <int LM> __host__ __device__ constexpr int threads() { return NFFT * Cfg<LM>::N2; }

__host__ __device__ constexpr int brev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// v * exp(S 2 pi i m / 16), m in [0, 8) a compile-time constant after unrolling
template <int S>
__device__ __forceinline__ float2 w16mul(float2 v, int m) {
    constexpr float R2 = 0.70710678118654752440f;
    if (m == 0) return v;
    if (m == 4) return S > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    if (m == 2) {       // (1 + S i) / sqrt 2
        return S > 0 ? make_float2(R2 * (v.x - v.y), R2 * (v.y + v.x))
                     : make_float2(R2 * (v.x + v.y), R2 * (v.y - v.x));
    }
    if (m == 6) {       // (-1 + S i) / sqrt 2
        return S > 0 ? make_float2(-R2 * (v.x + v.y), R2 * (v.x - v.y))
                     : make_float2(R2 * (v.y - v.x), -R2 * (v.x + v.y));
    }
    float c, s;         // cos, sin of 2 pi m / 16 for m = 1, 3, 5, 7
    switch (m) {
        case 1: c = 0.92387953251128675613f; s = 0.38268343236508977173f; break;
        case 3: c = 0.38268343236508977173f; s = 0.92387953251128675613f; break;
        case 5: c = -0.38268343236508977173f; s = 0.92387953251128675613f; break;
        default: c = -0.92387953251128675613f; s = 0.38268343236508977173f; break;
    }
    const float si = S > 0 ? s : -s;
    return make_float2(fmaf(v.x, c, -v.y * si), fmaf(v.x, si, v.y * c));
}

// In-register DFT of length N (2..16): a[k] <- sum_n a[n] exp(S 2 pi i nk / N).
// Radix-2 decimation in time on the bit-reversed copy; natural order out.
template <int N, int S>
__device__ __forceinline__ void rdft(float2 (&a)[N]) {
    constexpr int B = ilog2(N);
    float2 b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) b[brev(i, B)] = a[i];
#pragma unroll
    for (int half = 1; half < N; half *= 2) {
#pragma unroll
        for (int blk = 0; blk < N; blk += 2 * half) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                float2 u = b[blk + j];
                float2 v = w16mul<S>(b[blk + j + half], j * (8 / half));
                b[blk + j] = make_float2(u.x + v.x, u.y + v.y);
                b[blk + j + half] = make_float2(u.x - v.x, u.y - v.y);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = b[i];
}

template <int LM, bool XAX>
__host__ __device__ constexpr int staging_floats() {
    return XAX ? NCOL * Cfg<LM>::CS
               : ((1 << LM) - 1 + (((1 << LM) - 2) >> Cfg<LM>::LPAD) + 1) * Cfg<LM>::RS;
}
// The staging tile and the per-DFT buffers share one region: the tile is free
// between the first reads and the output writes (CTA barriers at both ends).
template <int LM, bool XAX>
__host__ __device__ constexpr size_t region_bytes() {
    return (size_t)staging_floats<LM, XAX>() * 4 > (size_t)NFFT * Cfg<LM>::FB * 8
               ? (size_t)staging_floats<LM, XAX>() * 4
               : (size_t)NFFT * Cfg<LM>::FB * 8;
}
// Dynamic shared memory of one CTA: the region, twiddles, sines.
template <int LM, bool XAX>
__host__ __device__ constexpr size_t smem_bytes() {
    return region_bytes<LM, XAX>() + (size_t)(1 << LM) * 8 + (size_t)(((1 << (LM - 1)) + 1 + 3) & ~3) * 4;
}

// Staging offset of element (column c, j' = j - 1) and of the pair (c, c+1) in YAX.
template <int LM, bool XAX>
__device__ __forceinline__ int spos(int c, int jp) {
    using G = Cfg<LM>;
    return XAX ? c * G::CS + jp + (jp >> G::LPAD) : (jp + (jp >> G::LPAD)) * G::RS + c;
}

// One tile: NCOL real columns of length n = M - 1.
//   XAX: rows tile*NCOL ... of an [outer][n] array (inner == 1);
//   YAX: inner indices i0 .. i0+NCOL-1 of block o of an [outer][n][inner] array.
template <typename TIN, int OMODE, int LM, bool XAX>
__device__ __forceinline__ void tile(const TIN* in, void* out, long long outer, long long inner, long long tile_id,
                                     const float2* __restrict__ tw, const float* __restrict__ sn,
                                     unsigned char* smem_raw) {
    using G = Cfg<LM>;
    constexpr int M = 1 << LM, n = M - 1, H = M / 2;
    constexpr int N1 = G::N1, N2 = G::N2, T = N2, NTH = threads<LM>();
    constexpr int KP = H / T;                        // spectrum entries per thread in the blocked phase
    float* st = reinterpret_cast<float*>(smem_raw);
    float2* fb = reinterpret_cast<float2*>(smem_raw);                  // aliases the staging tile
    float2* stw = reinterpret_cast<float2*>(smem_raw + region_bytes<LM, XAX>());
    float* ssn = reinterpret_cast<float*>(stw + M);
    const int tid = threadIdx.x;

    pdl_trigger();
    for (int i = tid; i < M; i += NTH) stw[i] = tw[i];
    for (int i = tid; i <= H; i += NTH) ssn[i] = sn[i];
    pdl_wait();                                      // the input is a predecessor's output

    // ---- load phase (CTA-wide): each thread issues a batch of global loads
    // before it scatters them into the staging area
    long long base_row = 0, o = 0, i0 = 0;
    int rows_here = NCOL;
    if (XAX) {
        base_row = tile_id * NCOL;
        rows_here = (int)min((long long)NCOL, outer - base_row);
        const int count = rows_here * n;
        const TIN* src = in + base_row * n;
        constexpr int VEC = 16 / sizeof(TIN);
        if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (count % VEC) == 0) {
            using V = typename std::conditional<sizeof(TIN) == 8, double2, float4>::type;
            constexpr int BATCH = 8;
            const V* sv = reinterpret_cast<const V*>(src);
            const int nvec = count / VEC;
            for (int i0v = 0; i0v < nvec; i0v += BATCH * NTH) {
                V vv[BATCH];
#pragma unroll
                for (int q = 0; q < BATCH; ++q) {
                    const int i = i0v + q * NTH + tid;
                    if (i < nvec) vv[q] = sv[i];
                }
#pragma unroll
                for (int q = 0; q < BATCH; ++q) {
                    const int i = i0v + q * NTH + tid;
                    if (i < nvec) {
                        int r = (i * VEC) / n, jp = i * VEC - r * n;
                        const TIN* pv = reinterpret_cast<const TIN*>(&vv[q]);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) {
                            if (jp == n) {
                                jp = 0;
                                ++r;
                            }
                            st[spos<LM, true>(r, jp)] = to_r<float, TIN>(pv[e]);
                            ++jp;
                        }
                    }
                }
            }
        } else {
            for (int e = tid; e < count; e += NTH) {
                int r = e / n, jp = e - r * n;
                st[spos<LM, true>(r, jp)] = to_r<float, TIN>(src[e]);
            }
        }
        for (int e = count + tid; e < NCOL * n; e += NTH) {
            int r = e / n, jp = e - r * n;
            st[spos<LM, true>(r, jp)] = 0.f;
        }
    } else {
        const long long tiles_per_outer = (inner + NCOL - 1) / NCOL;
        o = tile_id / tiles_per_outer;
        i0 = (tile_id - o * tiles_per_outer) * NCOL;
        constexpr int RSTEP = NTH / NCOL, BATCH = 16;
        const int c = tid & (NCOL - 1), r0 = tid / NCOL;
        const bool colok = i0 + c < inner;
        const TIN* src = in + o * (long long)n * inner + i0 + c;
        for (int jb = r0; jb < n; jb += RSTEP * BATCH) {
            TIN vv[BATCH];
#pragma unroll
            for (int q = 0; q < BATCH; ++q) {
                const int jp = jb + q * RSTEP;
                vv[q] = (jp < n && colok) ? src[(long long)jp * inner] : TIN(0);
            }
#pragma unroll
            for (int q = 0; q < BATCH; ++q) {
                const int jp = jb + q * RSTEP;
                if (jp < n) st[spos<LM, false>(c, jp)] = to_r<float, TIN>(vv[q]);
            }
        }
    }
    __syncthreads();

    // ---- one DFT per T threads (one warp segment)
    const int f = tid / T, t = tid % T;
    const int ca = 2 * f;                         // columns ca, ca + 1
    float2* buf = fb + f * G::FB;

    auto ld2 = [&](int j) -> float2 {             // (x_j of column ca, x_j of column ca+1), j = 1..n
        const int p = spos<LM, XAX>(ca, j - 1);
        if (XAX) return make_float2(st[p], st[p + G::CS]);
        return *reinterpret_cast<const float2*>(st + p);
    };

    float2 v[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
        const int j = N2 * n1 + t;
        if (j == 0) {
            v[n1] = make_float2(0.f, 0.f);
        } else {
            const int jm = M - j;
            float2 x = ld2(j), m = ld2(jm);
            float s = ssn[j < jm ? j : jm];
            v[n1] = make_float2(fmaf(s, x.x + m.x, 0.5f * (x.x - m.x)), fmaf(s, x.y + m.y, 0.5f * (x.y - m.y)));
        }
    }
    __syncthreads();                              // every column read: the tile becomes the buffers
    rdft<N1, -1>(v);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) {
        if (t) v[k1] = cmul(v[k1], stw[t * k1]);
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) buf[k1 * G::BS + t] = v[k1];
    __syncwarp();
    constexpr int Q = N1 / T;                    // length-N2 DFTs per thread
    float2 u[Q][N2];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k1 = t + T * q;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[q][n2] = buf[k1 * G::BS + n2];
        rdft<N2, -1>(u[q]);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k1 = t + T * q;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int k = k1 + N1 * k2;
            buf[k + (k >> G::ZP)] = u[q][k2];
        }
    }
    __syncwarp();

    // ---- separate the columns, blocked prefix sum, outputs into the staging area
    float ra[KP], rb[KP], ea[KP], eb[KP];
    float pa = 0.f, pb = 0.f;
#pragma unroll
    for (int i = 0; i < KP; ++i) {
        const int k = KP * t + i, km = (M - k) & (M - 1);
        const float2 zk = buf[k + (k >> G::ZP)], zm = buf[km + (km >> G::ZP)];
        float a = 0.5f * (zk.x + zm.x), b = 0.5f * (zk.y + zm.y);
        if (k == 0) {
            a *= 0.5f;
            b *= 0.5f;
        }
        ea[i] = 0.5f * (zm.y - zk.y);
        eb[i] = 0.5f * (zk.x - zm.x);
        pa += a;
        pb += b;
        ra[i] = pa;
        rb[i] = pb;
    }
    float sa = pa, sb = pb;                       // inclusive scan of the thread totals over the T threads
#pragma unroll
    for (int d = 1; d < T; d <<= 1) {
        const float ya = __shfl_up_sync(0xffffffffu, sa, d, T), yb = __shfl_up_sync(0xffffffffu, sb, d, T);
        if (t >= d) {
            sa += ya;
            sb += yb;
        }
    }
    const float oa = sa - pa, ob = sb - pb;
    __syncthreads();                              // every spectrum read: the region is the tile again
    auto st2 = [&](int jp, float a, float b) {
        const int p = spos<LM, XAX>(ca, jp);
        if (XAX) {
            st[p] = a;
            st[p + G::CS] = b;
        } else {
            *reinterpret_cast<float2*>(st + p) = make_float2(a, b);
        }
    };
#pragma unroll
    for (int i = 0; i < KP; ++i) {
        const int k = KP * t + i;
        if (k > 0) st2(2 * k - 1, ea[i], eb[i]);  // y_{2k}
        st2(2 * k, ra[i] + oa, rb[i] + ob);      // y_{2k+1}
    }
    __syncthreads();

    // ---- store phase (CTA-wide)
    if (XAX) {
        const int count = rows_here * n;
        const long long start = base_row * n;
        constexpr int EV = OMODE == 0 ? 4 : 2;          // values per 16-byte vector
        constexpr int ESZ = OMODE == 0 ? 4 : 8;
        char* ob = reinterpret_cast<char*>(out) + start * ESZ;
        if ((reinterpret_cast<uintptr_t>(ob) & 15) == 0 && (count % EV) == 0) {
            constexpr int BATCH = 4;
            const int nvec = count / EV;
            float4* ov = reinterpret_cast<float4*>(ob);
            for (int i0v = 0; i0v < nvec; i0v += BATCH * NTH) {
                float4 acc[BATCH];
                if (OMODE == 1) {
#pragma unroll
                    for (int q = 0; q < BATCH; ++q) {
                        const int i = i0v + q * NTH + tid;
                        if (i < nvec) acc[q] = ov[i];
                    }
                }
#pragma unroll
                for (int q = 0; q < BATCH; ++q) {
                    const int i = i0v + q * NTH + tid;
                    if (i < nvec) {
                        float vals[EV];
                        int r = (i * EV) / n, jp = i * EV - r * n;
#pragma unroll
                        for (int e = 0; e < EV; ++e) {
                            if (jp == n) {
                                jp = 0;
                                ++r;
                            }
                            vals[e] = st[spos<LM, true>(r, jp)];
                            ++jp;
                        }
                        float4 w;
                        if (OMODE == 0) {
                            w = make_float4(vals[0], vals[EV > 1 ? 1 : 0], vals[EV > 2 ? 2 : 0], vals[EV > 3 ? 3 : 0]);
                        } else if (OMODE == 2) {
                            w = make_float4(vals[0], 0.f, vals[1], 0.f);
                        } else {
                            dfloat d0 = df_add_f(dfloat{acc[q].x, acc[q].y}, vals[0]);
                            dfloat d1 = df_add_f(dfloat{acc[q].z, acc[q].w}, vals[1]);
                            w = make_float4(d0.hi, d0.lo, d1.hi, d1.lo);
                        }
                        ov[i] = w;
                    }
                }
            }
        } else {
            for (int e = tid; e < count; e += NTH) {
                int r = e / n, jp = e - r * n;
                dst_store<float, TIN, OMODE, 1>(out, start + e, st[spos<LM, true>(r, jp)]);
            }
        }
    } else {
        constexpr int RSTEP = NTH / NCOL;
        const int c = tid & (NCOL - 1), r0 = tid / NCOL;
        if (i0 + c < inner) {
            const long long base = o * (long long)n * inner + i0 + c;
            for (int jp = r0; jp < n; jp += RSTEP)
                dst_store<float, TIN, OMODE, 1>(out, base + (long long)jp * inner, st[spos<LM, false>(c, jp)]);
        }
    }
}

}  // namespace rd
}  // namespace qbvm
