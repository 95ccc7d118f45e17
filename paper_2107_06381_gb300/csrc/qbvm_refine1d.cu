// qbvm_refine1d.cu -- FP32 transforms + double-float refinement of a batch of
// small 1D instances, one CTA per instance, the whole refinement inside
// shared memory.
//
// The method is that of the staged batch refinement: y_0 = A32^{-1} f, then
// r = f - A y in double-float arithmetic and y += A32^{-1} r until
// ||r|| / ||f|| <= tol (Section 3.3 for the FP32 solve A32^{-1}: the DST-I of
// Step (b) along x, the omega-circulant time solve of steps (a)-(c) per sine
// mode, the inverse DST; the residual is the all-at-once system of eq. 3.3 /
// 3.6).  What differs is where it runs.  An instance of m - 1 interior
// points and nt levels (63 x 64 unknowns for the paper's 1D mesh) fits in
// shared memory, so one CTA holds its double-float iterate (8 B per unknown)
// and its FP32 work array (4 B) for the whole loop: the only HBM traffic is
// the right-hand side read once and the FP64 solution written once, against
// the ~140 B per unknown the staged passes move for two refinement steps.
// Each instance stops on its own residual (the staged batch stops on the
// largest), and no step returns to the host.
//
// Phases of one solve, separated by CTA barriers, all on the work array W
// ([nt][WS] floats, row t = level t, column j' = j - 1 at a padded offset):
//   x-DST of every level (rows paired into complex DFTs of length M, split
//     N1 x N2 over T = N2 threads as in the register DST tile of the staged
//     path: qbvm_regdst.cuh);
//   time solve of every sine mode (column), the half-length DFT split
//     N1 x N2 over T = N2 threads;
//   inverse x-DST, whose outputs are added to the iterate y in double-float.
// Then the residual overwrites W with r rounded to FP32 (each thread walking
// one column down a chunk of levels, the backward difference from registers),
// and a block sum of ||r||^2 decides, in one thread, whether to go on.  The
// first solve of a delta right-hand side has one nonzero level, whose DST is
// taken by its definition over the whole CTA.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "qbvm.h"
#include "qbvm_df.cuh"
#include "qbvm_fft.cuh"
#include "qbvm_internal.h"
#include "qbvm_regdst.cuh"

namespace qbvm {
namespace r1 {

constexpr int NTH = 256;            // threads per CTA (one instance)

// Time-solve split of the half-length DFT H = 2^LH = N1 * N2 (T = N2 threads
// per mode, transpose row stride BS; FB complex per mode: the stride between
// modes' buffers that makes the transposes bank-conflict free).
template <int LH> struct TCfg;
template <> struct TCfg<4> { static constexpr int N1 = 4, N2 = 4, BS = 5, FB = 52; };
template <> struct TCfg<5> { static constexpr int N1 = 8, N2 = 4, BS = 5, FB = 52; };
template <> struct TCfg<6> { static constexpr int N1 = 8, N2 = 8, BS = 9, FB = 72; };

// Padded rows of the work array W (floats) and of the iterate Y (float2):
// column j' sits at j' + (j' >> PS), 2^PS = M / N2 being the run of outputs
// one thread of the DST phase writes, so that the T runs of a pair start on
// different banks; row strides WS = 4 mod 16 and YS = 4 mod 8 then place the
// rows of a warp's four pairs so that the paired-row float accesses and the
// float2 half-warp accesses are conflict free.
template <int LM>
struct Pad {
    static constexpr int M = 1 << LM, n = M - 1;
    static constexpr int PS = LM - rd::ilog2(rd::Cfg<LM>::N2);
    static constexpr int span = n + ((n - 1) >> PS) + 1;       // padded row length
    static constexpr int WS = ((span - 4 + 15) / 16) * 16 + 4;
    static constexpr int YS = ((span - 4 + 7) / 8) * 8 + 4;
    static __device__ __forceinline__ int col(int jp) { return jp + (jp >> PS); }
};

template <int LM, int LH>
struct Layout {
    static constexpr int M = 1 << LM, n = M - 1, H = 1 << LH, NT = 2 * H, WS = Pad<LM>::WS, YS = Pad<LM>::YS;
    static constexpr int GD = NTH / rd::Cfg<LM>::N2;            // DST row pairs per wave
    static constexpr int GT = NTH / TCfg<LH>::N2;               // time-solve modes per wave
    static constexpr int BUF = (GD * rd::Cfg<LM>::FB > GT * TCfg<LH>::FB ? GD * rd::Cfg<LM>::FB
                                                                          : GT * TCfg<LH>::FB);
    // byte offsets (every region 16-byte aligned)
    static constexpr size_t oY = 0;                                               // float2 [NT][YS]
    static constexpr size_t oW = oY + (size_t)NT * YS * 8;                        // float [NT][WS]
    static constexpr size_t oB = oW + (size_t)NT * WS * 4;                        // float2 [BUF]
    static constexpr size_t oTS = oB + (size_t)BUF * 8;                           // float2 [M] DST roots
    static constexpr size_t oTT = oTS + (size_t)M * 8;                            // float2 [H] time roots
    static constexpr size_t oGP = oTT + (size_t)H * 8;                            // float2 [H] gamma^t
    static constexpr size_t oGI = oGP + (size_t)H * 8;                            // float2 [H] 2 gamma^-t
    static constexpr size_t oAK = oGI + (size_t)H * 8;                            // float2 [H] d_2k
    static constexpr size_t oF0 = oAK + (size_t)H * 8;                            // float2 [n] f^0 (delta)
    static constexpr size_t oLT = oF0 + (((size_t)n * 8 + 15) & ~(size_t)15);      // float [n] tau Lambda
    static constexpr size_t oSN = oLT + (((size_t)n * 4 + 15) & ~(size_t)15);      // float [M/2 + 1] sines
    static constexpr size_t oSF = oSN + (((size_t)(M / 2 + 1) * 4 + 15) & ~(size_t)15);   // float [2M] sin(pi m / M)
    static constexpr size_t bytes = oSF + (size_t)2 * M * 4;
};

// DST-I (unnormalised, y_k = sum_j x_j sin(pi j k / M)) of rows 0 .. rows-1
// of W, in place.  Rows 2p and 2p+1 are the real and imaginary parts of one
// complex DFT of length M of w_j = s_j (x_j + x_{M-j}) + (x_j - x_{M-j})/2;
// the even outputs are read off the spectrum and the odd ones are a prefix
// sum of its increments (the algorithm of qbvm_dst.cuh).  T threads of one
// warp own one pair; a wave takes NTH / T pairs.  OUT 0 writes the transform
// back into W; OUT 1 stores it into the double-float iterate Y ([rows][M-1])
// as (v, 0), OUT 2 adds it to Y (the update y += z of the refinement).
template <int LM, int OUT>
__device__ __forceinline__ void dst_rows(float* W, int rows, float2* bufs, const float2* tws, const float* sns,
                                         float2* Y) {
    using G = rd::Cfg<LM>;
    constexpr int M = 1 << LM, H = M / 2, N1 = G::N1, N2 = G::N2, T = N2, KP = H / T, Q = N1 / T;
    constexpr int GW = NTH / T, WS = Pad<LM>::WS, YS = Pad<LM>::YS;
    auto P = [](int jp) { return Pad<LM>::col(jp); };
    const int tid = threadIdx.x, g = tid / T, t = tid % T;
    float2* buf = bufs + g * G::FB;
    const int pairs = rows / 2;
    for (int p0 = 0; p0 < pairs; p0 += GW) {
        const int p = p0 + g;
        const bool act = p < pairs;
        const float* wa = W + (act ? 2 * p : 0) * WS;            // inactive groups read row pair 0
        const float* wb = wa + WS;
        float2 v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            // j = N2 n1 + t (t < N2) and M - j in the padded layout, in closed form:
            // P(N2 n1 + t - 1) = P(N2 n1) + t - 1 for t >= 1 and
            // P(M - 1 - N2 n1 - t) = P(M - 1 - N2 n1) - t (no run boundary is crossed)
            const int c0 = N2 * n1, cm = M - 1 - N2 * n1;
            const int pj = t ? Pad<LM>::col(c0) + t - 1 : (n1 ? Pad<LM>::col(c0 - 1) : 0);
            const int pm = Pad<LM>::col(cm) - t;
            const int si = 2 * n1 < N1 ? c0 + t : M - c0 - t;          // min(j, M - j)
            if (n1 == 0 && t == 0) {
                v[n1] = make_float2(0.f, 0.f);
            } else {
                const float xa = wa[pj], xb = wb[pj], ma = wa[pm], mb = wb[pm];
                const float s = sns[si];
                v[n1] = make_float2(fmaf(s, xa + ma, 0.5f * (xa - ma)), fmaf(s, xb + mb, 0.5f * (xb - mb)));
            }
        }
        rd::rdft<N1, -1>(v);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1)
            if (t) v[k1] = cmul(v[k1], tws[t * k1]);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) buf[k1 * G::BS + t] = v[k1];
        __syncwarp();
        float2 u[Q][N2];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k1 = t + T * q;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) u[q][n2] = buf[k1 * G::BS + n2];
            rd::rdft<N2, -1>(u[q]);
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
        float sa = pa, sb = pb;                   // inclusive scan of the thread totals over the T threads
#pragma unroll
        for (int d = 1; d < T; d <<= 1) {
            const float ya = __shfl_up_sync(0xffffffffu, sa, d, T), yb = __shfl_up_sync(0xffffffffu, sb, d, T);
            if (t >= d) {
                sa += ya;
                sb += yb;
            }
        }
        const float oa = sa - pa, ob = sb - pb;
        if (act) {
            // outputs 2k - 1 and 2k, k = KP t + i, in the padded layout:
            // P(2k) = (2 KP + 1) t + 2i, P(2k - 1) = (2 KP + 1) t + 2i - 1 (i > 0)
            // or (2 KP + 1) t - 2 (i = 0)
            const int ob0 = (2 * KP + 1) * t;
            if (OUT == 0) {
                float* oa_row = W + 2 * p * WS;
                float* ob_row = oa_row + WS;
#pragma unroll
                for (int i = 0; i < KP; ++i) {
                    if (i > 0 || t > 0) {             // y_{2k}
                        const int q = ob0 + (i ? 2 * i - 1 : -2);
                        oa_row[q] = ea[i];
                        ob_row[q] = eb[i];
                    }
                    oa_row[ob0 + 2 * i] = ra[i] + oa; // y_{2k+1}
                    ob_row[ob0 + 2 * i] = rb[i] + ob;
                }
            } else {
                float2* ya = Y + 2 * p * YS;
                float2* yb = ya + YS;
                auto put = [&](float2* row, int q, float v) {
                    if (OUT == 1) {
                        row[q] = make_float2(v, 0.f);
                    } else {
                        const float2 o = row[q];
                        const dfloat r = df_add_f(dfloat{o.x, o.y}, v);
                        row[q] = make_float2(r.hi, r.lo);
                    }
                };
#pragma unroll
                for (int i = 0; i < KP; ++i) {
                    if (i > 0 || t > 0) {
                        const int q = ob0 + (i ? 2 * i - 1 : -2);
                        put(ya, q, ea[i]);
                        put(yb, q, eb[i]);
                    }
                    put(ya, ob0 + 2 * i, ra[i] + oa);
                    put(yb, ob0 + 2 * i, rb[i] + ob);
                }
            }
        }
        __syncwarp();                             // the group's buffer is free for the next wave
    }
}

// DST-I of row 0 alone (the first solve of a delta right-hand side, whose
// other levels are zero), by its definition y_k = sum_j x_j sin(pi j k / M):
// NTH / M consecutive threads share one output, each summing every
// (NTH / M)-th term, so that the whole CTA works on the one row.
template <int LM>
__device__ __forceinline__ void dst_row0_direct(float* W, const float* sfull) {
    constexpr int M = 1 << LM, n = M - 1, PARTS = NTH / M;
    const int k = threadIdx.x / PARTS + 1, part = threadIdx.x % PARTS;
    float acc = 0.f;
    if (k <= n)
        for (int j = 1 + part; j <= n; j += PARTS) acc = fmaf(W[Pad<LM>::col(j - 1)], sfull[(j * k) & (2 * M - 1)], acc);
#pragma unroll
    for (int o = PARTS / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, PARTS);
    __syncthreads();                              // every thread has read row 0
    if (k <= n && part == 0) W[Pad<LM>::col(k - 1)] = acc;
}

// Time solve of sine modes 0 .. nmodes-1 (columns of W), in place: per mode l,
// v_t = gamma^t (w_t + i rho^H w_{t+H}) (t < H), the length-H DFT
// (theta^{+kt}), Step (b) -- multiply by cnorm / (d_{2k} + tau Lambda_l) --
// the inverse DFT and the unscaling by 2 gamma^{-t} (Section 3.3 in the
// half-length form of the staged FP32 time solve).  With first_delta only
// w_0 is nonzero and the forward DFT is the constant w_0.
template <int LM, int LH>
__device__ __forceinline__ void time_modes(float* W, int WS, int nmodes, float2* bufs, const float2* twt,
                                           const float2* gp, const float2* gi, const float2* ak,
                                           const float* lamtau, float cnorm, float rho_h, float rho_hinv,
                                           bool first_delta) {
    using G = TCfg<LH>;
    constexpr int H = 1 << LH, N1 = G::N1, N2 = G::N2, T = N2, Q = N1 / T, GW = NTH / T;
    const int tid = threadIdx.x, c = tid / T, n2 = tid % T;
    float2* buf = bufs + c * G::FB;
    for (int l0 = 0; l0 < nmodes; l0 += GW) {
        const int l = l0 + c;
        const bool ok = l < nmodes;
        float* col = W + Pad<LM>::col(ok ? l : 0);
        float2 X[Q][N2];
        if (first_delta) {
            const float f0 = col[0];
#pragma unroll
            for (int q = 0; q < Q; ++q)
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) X[q][k2] = make_float2(f0, 0.f);
        } else {
            float2 v[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const int t = N2 * n1 + n2;
                const float2 g = gp[t];
                const float fa = col[t * WS], f1 = rho_h * col[(t + H) * WS];
                v[n1] = make_float2(fmaf(g.x, fa, -g.y * f1), fmaf(g.y, fa, g.x * f1));
            }
            rd::rdft<N1, +1>(v);
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1)
                if (n2) v[k1] = cmulc(v[k1], twt[n2 * k1]);     // exp(+2 pi i n2 k1 / H)
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) buf[k1 * G::BS + n2] = v[k1];
            __syncwarp();
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int k1 = n2 + T * q;
#pragma unroll
                for (int j = 0; j < N2; ++j) X[q][j] = buf[k1 * G::BS + j];
                rd::rdft<N2, +1>(X[q]);
            }
            __syncwarp();
        }
        const float lt = ok ? lamtau[l] : 0.f;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k1 = n2 + T * q;
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const float2 a = ak[k1 + N1 * k2];
                const float zr = a.x + lt, zi = a.y;
                // |d + tau Lambda|^2 lies far inside the fast division's range
                // (2 ulp); this solve is a correction step of the refinement
                const float inv = __fdividef(cnorm, fmaf(zr, zr, zi * zi));
                const float2 u = X[q][k2];
                X[q][k2] = make_float2(fmaf(u.x, zr, u.y * zi) * inv, fmaf(u.y, zr, -u.x * zi) * inv);
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k1 = n2 + T * q;
            rd::rdft<N2, -1>(X[q]);
#pragma unroll
            for (int j = 1; j < N2; ++j)
                if (k1) X[q][j] = cmul(X[q][j], twt[j * k1]);   // exp(-2 pi i j k1 / H)
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k1 = n2 + T * q;
#pragma unroll
            for (int j = 0; j < N2; ++j) buf[k1 * G::BS + j] = X[q][j];
        }
        __syncwarp();
        float2 w[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) w[k1] = buf[k1 * G::BS + n2];
        rd::rdft<N1, -1>(w);
        if (ok) {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
                const int t = N2 * n1 + n2;
                const float2 g = gi[t], qv = w[n1];
                col[t * WS] = fmaf(g.x, qv.x, -g.y * qv.y);
                col[(t + H) * WS] = rho_hinv * fmaf(g.x, qv.y, g.y * qv.x);
            }
        }
        __syncwarp();                             // the buffer is free for the next wave
    }
}

// Per-instance status written by the kernel (Refine1dStatus; the host maps it
// to the batch's).
constexpr int ST_OK = R1_OK, ST_NONFINITE_IN = R1_NONFINITE_IN, ST_RANGE = R1_RANGE, ST_DIVERGED = R1_DIVERGED,
              ST_NONFINITE = R1_NONFINITE;

// FP32 sum over the CTA, returned in thread 0 (warp shuffles, then one thread
// over the warps' sums).
__device__ __forceinline__ float fsum0(float v, float* shf) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) shf[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < NTH / 32; ++i) s += shf[i];
    return s;
}

// Sum of the CTA's ScaledSsq partials, returned in thread 0: within a warp the
// partials are rescaled to the warp's largest exponent and added in FP32 (a
// stopping test needs no more), the warps' sums are combined in FP64 by one
// thread.  No FP64 instruction runs on the other threads: the FP64 pipe is a
// small fraction of the FP32 pipes and would stall the whole CTA.
__device__ __forceinline__ double ssq_sum0(const ScaledSsq& q, float* shf, int* she) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int em = q.e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
    const int d = 2 * (q.e - em);                 // <= 0: this lane's scale against the warp's
    float v = d >= -126 ? q.ssq * ScaledSsq::p2(d) : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
        shf[w] = v;
        she[w] = em;
    }
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NTH / 32; ++i) s += (double)shf[i] * __longlong_as_double((long long)(1023 + 2 * she[i]) << 52);
    return s;
}

template <int LM, int LH>
__global__ void __launch_bounds__(NTH, 2) k_refine1d(Refine1dArgs a) {
    using Lo = Layout<LM, LH>;
    constexpr int M = Lo::M, n = Lo::n, H = Lo::H, NT = Lo::NT, WS = Lo::WS, YS = Lo::YS, NU = NT * n;
    auto P = [](int jp) { return Pad<LM>::col(jp); };
    // residual phase: thread (column j, chunk c) walks LC consecutive levels
    constexpr int NC = NTH / M, LC = NT / NC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* Y = reinterpret_cast<float2*>(smem_raw + Lo::oY);
    float* W = reinterpret_cast<float*>(smem_raw + Lo::oW);
    float2* bufs = reinterpret_cast<float2*>(smem_raw + Lo::oB);
    float2* tws = reinterpret_cast<float2*>(smem_raw + Lo::oTS);
    float2* twt = reinterpret_cast<float2*>(smem_raw + Lo::oTT);
    float2* gp = reinterpret_cast<float2*>(smem_raw + Lo::oGP);
    float2* gi = reinterpret_cast<float2*>(smem_raw + Lo::oGI);
    float2* ak = reinterpret_cast<float2*>(smem_raw + Lo::oAK);
    float2* F0 = reinterpret_cast<float2*>(smem_raw + Lo::oF0);
    float* lt = reinterpret_cast<float*>(smem_raw + Lo::oLT);
    float* sns = reinterpret_cast<float*>(smem_raw + Lo::oSN);
    float* sfull = reinterpret_cast<float*>(smem_raw + Lo::oSF);
    __shared__ float s_f[NTH / 32];
    __shared__ int s_e[NTH / 32];
    __shared__ int s_go;
    __shared__ float s_scale;
    const int tid = threadIdx.x;
    const long long b = blockIdx.x;

    for (int i = tid; i < M; i += NTH) tws[i] = a.tws[i];
    for (int i = tid; i <= M / 2; i += NTH) sns[i] = a.sns[i];
    for (int m = tid; m < 2 * M; m += NTH) {      // sin(pi m / M) from the half-period table
        const int r = m < M ? m : m - M;
        const float v = a.sns[r <= M / 2 ? r : M - r];
        sfull[m] = m < M ? v : -v;
    }
    for (int i = tid; i < H; i += NTH) {
        twt[i] = a.twt[i];
        gp[i] = a.gpow[b * H + i];
        gi[i] = a.gipw[b * H + i];
        ak[i] = a.ak[b * H + i];
    }
    for (int i = tid; i < n; i += NTH) lt[i] = a.lamtau[i];
    const float cnorm = a.cnorm[b], rho_h = a.rho_h[b], rho_hinv = a.rho_hinv[b];
    const dfloat om = {a.omega_df[b].x, a.omega_df[b].y};
    const dfloat ct = {a.ct.x, a.ct.y}, cx = {a.cx.x, a.cx.y};
    const double* fb = a.f + b * (a.delta ? (long long)n : (long long)NU);
    double* yb = a.y + b * (a.n0_only ? (long long)n : (long long)NU);

    // ---- the right-hand side: FP32 copy in W, its norm, its classification
    ScaledSsq nf;
    int bad = 0, nonzero = 0;
    if (a.delta) {
        const double f0s = -a.omega64[b] * a.inv_tau;            // f^0 = -omega g / tau
        for (int j = tid; j < n; j += NTH) {
            const double fd = f0s * fb[j];
            const dfloat fv = df_from_double_trunc(fd);
            F0[j] = make_float2(fv.hi, fv.lo);
            W[P(j)] = fv.hi;
            W[WS + P(j)] = 0.f;
            nf.add(fv.hi);
            bad |= !isfinite(fd);
            nonzero |= fd != 0.0;
        }
    } else {
        for (int e = tid; e < NU; e += NTH) {
            const int t = e / n, j = e - t * n;
            const double fd = fb[e];
            const dfloat fv = df_from_double_trunc(fd);
            W[t * WS + P(j)] = fv.hi;
            nf.add(fv.hi);
            bad |= !isfinite(fd);
            nonzero |= fd != 0.0;
        }
    }
    bad = __syncthreads_or(bad);
    nonzero = __syncthreads_or(nonzero);
    const double f2 = ssq_sum0(nf, s_f, s_e);                    // thread 0
    if (tid == 0) {
        const double rms = sqrt(f2 / (double)(a.delta ? n : NU));
        int st = ST_OK;
        if (bad) st = ST_NONFINITE_IN;
        else if ((rms > 0 && (rms < 1e-18 || rms > 1e28)) || (f2 == 0.0 && nonzero)) st = ST_RANGE;
        s_go = st != ST_OK ? 0 : f2 > 0.0 ? 1 : 2;
        // residual sums of squares are taken of r / 2^k, 2^k the power of two at
        // or below the root mean square of f (in range: rms in [1e-18, 1e28])
        s_scale = rms > 0 ? ldexpf(1.f, -(int)floorf(log2f((float)rms))) : 1.f;
        if (st != ST_OK || f2 == 0.0) {
            a.status[b] = st;
            a.iters[b] = 0;
            a.rel[b] = 0.0;
        }
    }
    __syncthreads();
    if (s_go != 1) {                              // zero data: y = 0; an unusable input writes nothing
        if (s_go == 2)
            for (int e = tid; e < (a.n0_only ? n : NU); e += NTH) yb[e] = 0.0;
        return;
    }

    double prev2 = INFINITY, r2 = f2;             // the stopping test runs in thread 0, on squares
    const float rsc = s_scale;
    int it = 0, status = ST_OK;
    const int rj = tid % M, rc = tid / M;
    for (bool first = true;; first = false) {
        // ---- one FP32 solve of A z = W; its inverse DST adds z to y
        const bool fdl = first && a.delta;                       // only level 0 is nonzero
        if (fdl) dst_row0_direct<LM>(W, sfull);
        else dst_rows<LM, 0>(W, NT, bufs, tws, sns, Y);
        __syncthreads();
        time_modes<LM, LH>(W, WS, n, bufs, twt, gp, gi, ak, lt, cnorm, rho_h, rho_hinv, fdl);
        __syncthreads();
        if (first) dst_rows<LM, 1>(W, NT, bufs, tws, sns, Y);
        else dst_rows<LM, 2>(W, NT, bufs, tws, sns, Y);
        __syncthreads();
        // ---- r = f - A y (eq. 3.3 / 3.6) in double-float, rounded to FP32 into W
        float nr = 0.f;                           // sum of (r / 2^k)^2
        if (rj < n) {
            const int j = rj, t0 = rc * LC, pj = P(j), pl = j > 0 ? P(j - 1) : 0, pr = j < n - 1 ? P(j + 1) : 0;
            int e = t0 * YS;                      // row offset of level t0 + q
            const double* fl = fb + (long long)t0 * n + j;
            dfloat pv;                            // y^{t-1}, or omega y^{N} at t = 0
            if (t0 == 0) {
                const float2 q = Y[(NT - 1) * YS + pj];
                pv = df_mul_un(om, dfloat{q.x, q.y});
            } else {
                pv = dfloat{Y[e - YS + pj].x, Y[e - YS + pj].y};
            }
            const dfloat zero = {0.f, 0.f};
#pragma unroll 4
            for (int q = 0; q < LC; ++q, e += YS) {
                const dfloat yc = {Y[e + pj].x, Y[e + pj].y};
                dfloat Ay = df_mul_un(ct, df_sub_un(yc, pv));
                const dfloat sl = j > 0 ? dfloat{Y[e + pl].x, Y[e + pl].y} : zero;
                const dfloat sr = j < n - 1 ? dfloat{Y[e + pr].x, Y[e + pr].y} : zero;
                const dfloat my = {2.f * yc.hi, 2.f * yc.lo};
                Ay = df_add_un(Ay, df_mul_un(cx, df_sub_un(my, df_add_un(sl, sr))));
                dfloat fv = zero;
                if (a.delta) {
                    if (t0 + q == 0) fv = dfloat{F0[j].x, F0[j].y};
                } else {
                    fv = df_from_double_trunc(fl[(long long)q * n]);
                }
                const dfloat r = df_sub_un(fv, Ay);
                const float rh = r.hi + r.lo;
                W[(t0 + q) * WS + pj] = rh;
                const float rs = rh * rsc;
                nr = fmaf(rs, rs, nr);
                pv = yc;
            }
        }
        const float r2s = fsum0(nr, s_f);
        if (tid == 0) {
            // ||r|| <= tol ||f||, ||r|| > ||r_prev|| / 2 and ||r|| > 1e-10 ||f||,
            // compared as squares (no division or square root in the loop)
            r2 = (double)r2s / ((double)rsc * (double)rsc);
            int go = 0;
            if (r2s != r2s) {                     // NaN residual
                status = ST_NONFINITE;
            } else if (isinf(r2s)) {              // (r / 2^k)^2 beyond the FP32 range: diverging
                status = ST_DIVERGED;
            } else if (r2 <= a.tol * a.tol * f2) {
            } else if (r2 > 0.25 * prev2) {       // no contraction
                if (r2 > 1e-20 * f2) status = ST_DIVERGED;
            } else if (it >= a.maxit) {
                status = ST_DIVERGED;
            } else {
                go = 1;
                prev2 = r2;
                ++it;
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
    }
    // ---- the FP64 solution (hi + lo, one rounding): thread (column j, chunk c)
    // writes its levels, a warp 32 consecutive values of one level
    if (rj < n) {
        const int pj = P(rj);
        const int t0 = a.n0_only ? 0 : rc * LC, t1 = a.n0_only ? (rc == 0 ? 1 : 0) : t0 + LC;
        for (int t = t0; t < t1; ++t) {
            const float2 v = Y[t * YS + pj];
            yb[(long long)t * n + rj] = qbvm_join_df_dadd(v.x, v.y);
        }
    }
    if (tid == 0) {
        a.status[b] = status;
        a.iters[b] = it;
        a.rel[b] = sqrt(r2 / f2);
    }
}

template <int LM, int LH>
cudaError_t launch_lm_lh(long long count, const Refine1dArgs& a, cudaStream_t s) {
    constexpr size_t bytes = Layout<LM, LH>::bytes;
    auto kern = k_refine1d<LM, LH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)count, NTH, bytes, s>>>(a);
    return cudaGetLastError();
}

// Shared memory of a shape the kernel is built for, else 0.
size_t shape_bytes(int lm, int lh) {
    if (lm == 6 && lh == 4) return Layout<6, 4>::bytes;
    if (lm == 6 && lh == 5) return Layout<6, 5>::bytes;
    if (lm == 6 && lh == 6) return Layout<6, 6>::bytes;
    if (lm == 7 && lh == 4) return Layout<7, 4>::bytes;
    if (lm == 7 && lh == 5) return Layout<7, 5>::bytes;
    if (lm == 8 && lh == 4) return Layout<8, 4>::bytes;
    return 0;
}

}  // namespace r1

int refine1d_supported(const Tables& tb) {
    if (tb.dim != 1 || !tb.sf || tb.gen) return 0;
    const int lm = tb.lpd[0], lh = tb.lnt - 1;
    if (tb.n[0] != (1 << lm) - 1) return 0;
    const size_t bytes = r1::shape_bytes(lm, lh);
    if (!bytes) return 0;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return bytes <= (size_t)optin;
}

cudaError_t launch_refine1d(const Tables& tb, long long count, const Refine1dArgs& a, cudaStream_t s) {
    if (count < 1 || count > 0x7fffffffLL || !refine1d_supported(tb)) return cudaErrorInvalidValue;
    const int lm = tb.lpd[0], lh = tb.lnt - 1;
    if (lm == 6 && lh == 4) return r1::launch_lm_lh<6, 4>(count, a, s);
    if (lm == 6 && lh == 5) return r1::launch_lm_lh<6, 5>(count, a, s);
    if (lm == 6 && lh == 6) return r1::launch_lm_lh<6, 6>(count, a, s);
    if (lm == 7 && lh == 4) return r1::launch_lm_lh<7, 4>(count, a, s);
    if (lm == 7 && lh == 5) return r1::launch_lm_lh<7, 5>(count, a, s);
    return r1::launch_lm_lh<8, 4>(count, a, s);
}

}  // namespace qbvm
