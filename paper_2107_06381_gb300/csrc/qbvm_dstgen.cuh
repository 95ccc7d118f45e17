// qbvm_dstgen.cuh -- DST-I of any length n = M - 1 (Step (b) in 2D/3D on a
// mesh of M intervals per axis, Section 2: h = L/M for any M).
//
// The transform is the one of qbvm_dst.cuh -- two real columns packed into one
// complex DFT of length M of w_j = s_j (x_j + x_{M-j}) + (x_j - x_{M-j})/2,
// y_{2k} = -Im W_k, y_{2k+1} - y_{2k-1} = Re W_k -- which holds for every M,
// even or odd.  What changes is the DFT of length M: a mixed-radix Stockham
// autosort FFT in shared memory, the factors of M taken as radix-4, -2, -3
// and -5 passes and, for any other prime factor p, a direct length-p DFT per
// butterfly (O(p) operations per element in that pass).
//
// Stage with radix p (L = product of the earlier radices, L' = L p,
// r' = M / L'): with X_s[k, j] = sum_{m<L} x[k + (M/L) m] w_L^{jm} held at
// k L + j, every (k', j), k' < r', j < L, reads X_s[k' + r' q, j] for q < p,
// multiplies input q by w_{L'}^{jq} and applies the length-p DFT:
//     X_{s+1}[k', j + L t] = sum_q w_p^{tq} w_{L'}^{jq} X_s[k' + r' q, j].
// After the last stage X[0, j] is the DFT in natural order.  Each stage reads
// one buffer and writes the other (ping-pong), so no register budget bounds
// the radix.  All twiddles index one table tw[m] = exp(-2 pi i m / M).
#pragma once
#include "qbvm_dst.cuh"

namespace qbvm {

constexpr int FFTGEN_MAX_STAGES = 16;

// The radices of a length-M transform, in the order they are applied.
struct FftGenPlan {
    int nrad = 0;
    int rad[FFTGEN_MAX_STAGES] = {};
};

// Radix factorisation of M >= 1: 4s first, then one 2, then 3s, 5s and the
// remaining prime factors in increasing order.  False if more than
// FFTGEN_MAX_STAGES factors would be needed (never for M <= 2^16).
inline bool fftgen_factor(int M, FftGenPlan* fp) {
    fp->nrad = 0;
    auto push = [&](int p) {
        if (fp->nrad >= FFTGEN_MAX_STAGES) return false;
        fp->rad[fp->nrad++] = p;
        return true;
    };
    while (M % 4 == 0) {
        if (!push(4)) return false;
        M /= 4;
    }
    if (M % 2 == 0) {
        if (!push(2)) return false;
        M /= 2;
    }
    for (int p = 3; M > 1; p += 2) {
        while (M % p == 0) {
            if (!push(p)) return false;
            M /= p;
        }
        if ((long long)p * p > M && M > 1) {
            if (!push(M)) return false;
            M = 1;
        }
    }
    return true;
}

// v * exp(S * 2 pi i m / M) from the table of exp(-2 pi i m / M)
template <int S, typename C>
__device__ __forceinline__ C tmul(const C* tw, int m, C v) {
    return cmul(v, twiddle<S>(tw, m));
}

// One radix-p stage of W = 2^lw columns (element (t, c) at t * W + c).
template <int S, typename R>
__device__ __forceinline__ void fftgen_stage(const cplx<R>* __restrict__ src, cplx<R>* __restrict__ dst,
                                             const cplx<R>* tw, int M, int lw, int p, int L) {
    using C = cplx<R>;
    const int W = 1 << lw, Lp = L * p, rq = M / Lp, Mp = M / p;
    const int ntask = Mp << lw;
    for (int b = threadIdx.x; b < ntask; b += blockDim.x) {
        const int c = b & (W - 1), rest = b >> lw;
        const int kq = rest / L, j = rest - kq * L;
        const C* in = src + ((size_t)(kq * L + j) << lw) + c;        // input q at in[q * rq * L * W]
        C* out = dst + ((size_t)(kq * Lp + j) << lw) + c;            // output t at out[t * L * W]
        const size_t istr = (size_t)rq * L << lw, ostr = (size_t)L << lw;
        const int wstep = j * rq;                                      // w_{L'}^{jq} = tw[q * j * rq]
        if (p == 2) {
            C a = in[0], v = in[istr];
            if (j) v = tmul<S>(tw, wstep, v);
            out[0] = cadd(a, v);
            out[ostr] = csub(a, v);
        } else if (p == 4) {
            C v0 = in[0], v1 = in[istr], v2 = in[2 * istr], v3 = in[3 * istr];
            if (j) {
                v1 = tmul<S>(tw, wstep, v1);
                v2 = tmul<S>(tw, 2 * wstep, v2);
                v3 = tmul<S>(tw, 3 * wstep, v3);
            }
            dft4<S>(v0, v1, v2, v3);
            out[0] = v0;
            out[ostr] = v1;
            out[2 * ostr] = v2;
            out[3 * ostr] = v3;
        } else if (p == 3) {
            // w_3 = -1/2 + S i sqrt(3)/2
            const R h3 = R(0.86602540378443864676);
            C a = in[0], v1 = in[istr], v2 = in[2 * istr];
            if (j) {
                v1 = tmul<S>(tw, wstep, v1);
                v2 = tmul<S>(tw, 2 * wstep, v2);
            }
            const C sm = cadd(v1, v2), df = csub(v1, v2);
            const C t1 = mkc(rfma(R(-0.5), sm.x, a.x), rfma(R(-0.5), sm.y, a.y));
            const C u = cmul_si<S>(mkc(h3 * df.x, h3 * df.y));        // S i sqrt(3)/2 (v1 - v2)
            out[0] = cadd(a, sm);
            out[ostr] = cadd(t1, u);
            out[2 * ostr] = csub(t1, u);
        } else if (p == 5) {
            // cos / sin of 2 pi/5 and 4 pi/5
            const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);
            const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);
            C x0 = in[0], x1 = in[istr], x2 = in[2 * istr], x3 = in[3 * istr], x4 = in[4 * istr];
            if (j) {
                x1 = tmul<S>(tw, wstep, x1);
                x2 = tmul<S>(tw, 2 * wstep, x2);
                x3 = tmul<S>(tw, 3 * wstep, x3);
                x4 = tmul<S>(tw, 4 * wstep, x4);
            }
            const C b1 = cadd(x1, x4), b2 = cadd(x2, x3), d1 = csub(x1, x4), d2 = csub(x2, x3);
            const C t1 = mkc(rfma(c1, b1.x, rfma(c2, b2.x, x0.x)), rfma(c1, b1.y, rfma(c2, b2.y, x0.y)));
            const C t2 = mkc(rfma(c2, b1.x, rfma(c1, b2.x, x0.x)), rfma(c2, b1.y, rfma(c1, b2.y, x0.y)));
            // S i (s1 d1 + s2 d2) and S i (s2 d1 - s1 d2)
            const C u1 = cmul_si<S>(mkc(rfma(s1, d1.x, s2 * d2.x), rfma(s1, d1.y, s2 * d2.y)));
            const C u2 = cmul_si<S>(mkc(rfma(s2, d1.x, -s1 * d2.x), rfma(s2, d1.y, -s1 * d2.y)));
            out[0] = cadd(x0, cadd(b1, b2));
            out[ostr] = cadd(t1, u1);
            out[4 * ostr] = csub(t1, u1);
            out[2 * ostr] = cadd(t2, u2);
            out[3 * ostr] = csub(t2, u2);
        } else {
            // direct length-p DFT: out_t = sum_q in_q w_M^{q u_t}, u_t = j r' + t M/p
            for (int t = 0; t < p; ++t) {
                const int u = (wstep + t * Mp) % M;
                C acc = in[0];
                int e = u;
                for (int q = 1; q < p; ++q) {
                    const C w = twiddle<S>(tw, e);
                    const C v = in[q * istr];
                    acc = mkc(rfma(v.x, w.x, rfma(-v.y, w.y, acc.x)), rfma(v.x, w.y, rfma(v.y, w.x, acc.y)));
                    e += u;
                    if (e >= M) e -= M;
                }
                out[t * ostr] = acc;
            }
        }
    }
    __syncthreads();
}

// FFT of W columns of length M held in `a`; `b` is scratch of the same size.
// Returns the buffer that holds the result.  Ends with __syncthreads().
template <int S, typename R>
__device__ __forceinline__ cplx<R>* fftgen_tile(cplx<R>* a, cplx<R>* b, const cplx<R>* tw, int M, int lw,
                                                const FftGenPlan& fp) {
    int L = 1;
    for (int s = 0; s < fp.nrad; ++s) {
        const int p = fp.rad[s];
        fftgen_stage<S, R>(a, b, tw, M, lw, p, L);
        L *= p;
        cplx<R>* t = a;
        a = b;
        b = t;
    }
    return a;
}

// Tile width log2(W) of a general-length DST tile: 2W real columns with
// M * W <= DST_TILE complex values.
__host__ __device__ inline int dstgen_lw(int M) {
    int lw = 0;
    while ((long long)M << (lw + 1) <= DST_TILE) ++lw;
    return lw;
}

template <typename R>
inline size_t dstgen_smem(int M, int lw) {
    const int W = 1 << lw, K = (M + 1) / 2;
    const int ncol = 2 * W;
    const size_t seg = (size_t)(TILE_THREADS >= ncol ? TILE_THREADS : ncol);
    return sizeof(cplx<R>) * (2 * (size_t)M * W + M) + sizeof(R) * ((size_t)K + 2 + seg);
}

// One general-length DST tile: 2W real columns of length n = M - 1 (as in
// dst_tile: inner == 1 selects rows of an [outer][n] array, else 2W
// consecutive inner indices of block o of an [outer][n][inner] array).
// Buffers: A, B of M x W complex (ping-pong FFT; B also stages the rows of
// the x pass and A or B holds the outputs), tables tw (M), sines (K + 1).
template <typename R, typename TIN, int OMODE, bool X4>
__device__ __forceinline__ void dstgen_tile(const TIN* in, void* out, int M, int lw, long long outer,
                                            long long inner, long long tile, const cplx<R>* __restrict__ tw,
                                            const R* __restrict__ sn, const FftGenPlan& fp,
                                            unsigned char* smem_raw) {
    using C = cplx<R>;
    const int n = M - 1, W = 1 << lw, K = (M + 1) / 2;   // spectrum entries W_0 .. W_{K-1} are used
    const int tid = threadIdx.x, nth = blockDim.x;
    const int ncol = 2 * W;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + (size_t)M * W;
    C* stw = B + (size_t)M * W;
    R* ssn = reinterpret_cast<R*>(stw + M);              // sin(j pi / M), j = 0..M/2
    R* seg = ssn + (K + 2);
    R* Ar = reinterpret_cast<R*>(A);

    pdl_trigger();
    for (int i = tid; i < M; i += nth) stw[i] = tw[i];
    for (int i = tid; i <= M / 2; i += nth) ssn[i] = X4 ? R(2) * sn[i] : sn[i];
    for (int p = tid; p < W; p += nth) A[p] = mkc(R(0), R(0));     // x_0 = 0
    pdl_wait();

    long long base_row = 0, o = 0, i0 = 0;
    int rows_here = ncol;
    if (inner == 1) {
        base_row = tile * ncol;
        rows_here = (int)min((long long)ncol, outer - base_row);
        const int count = rows_here * n;
        const TIN* src = in + base_row * n;
        R* raw = reinterpret_cast<R*>(B);
        for (int i = tid; i < count; i += nth) raw[i] = to_r<R, TIN>(src[i]);
        __syncthreads();
        for (int e = tid; e < ncol * n; e += nth) {
            const int j = e >> (lw + 1), r = e & (ncol - 1);
            Ar[((size_t)(j + 1) << (lw + 1)) + r] = r < rows_here ? raw[r * n + j] : R(0);
        }
    } else {
        const long long tiles_per_outer = (inner + ncol - 1) / ncol;
        o = tile / tiles_per_outer;
        i0 = (tile - o * tiles_per_outer) * ncol;
        const TIN* src = in + o * (long long)n * inner;
        for (int e = tid; e < ncol * n; e += nth) {
            const int j = e >> (lw + 1), r = e & (ncol - 1);
            const long long ii = i0 + r;
            Ar[((size_t)(j + 1) << (lw + 1)) + r] = ii < inner ? to_r<R, TIN>(src[(long long)j * inner + ii]) : R(0);
        }
    }
    __syncthreads();
    // w_j and w_{M-j} from the pair (x_j, x_{M-j}), j = 1 .. M/2 (x_M = 0)
    const int P = M / 2;
    for (int e = tid; e < (P << lw); e += nth) {
        const int j = (e >> lw) + 1, p = e & (W - 1);
        // for even M, j = M/2 pairs with itself: w_j = 2 s_j x_j (D vanishes)
        const C a = A[((size_t)j << lw) + p], b = A[((size_t)(M - j) << lw) + p];
        const R sj = ssn[j];
        const C S = mkc(a.x + b.x, a.y + b.y);
        const C D = X4 ? mkc(a.x - b.x, a.y - b.y) : mkc(R(0.5) * (a.x - b.x), R(0.5) * (a.y - b.y));
        A[((size_t)j << lw) + p] = mkc(rfma(sj, S.x, D.x), rfma(sj, S.y, D.y));
        if (j != M - j) A[((size_t)(M - j) << lw) + p] = mkc(rfma(sj, S.x, -D.x), rfma(sj, S.y, -D.y));
    }
    __syncthreads();
    C* Z = fftgen_tile<-1, R>(A, B, stw, M, lw, fp);
    C* other = Z == A ? B : A;
    R* obuf = reinterpret_cast<R*>(other);                 // [j'][2W] real, y_{j'+1} at row j'

    // separate the packed columns; even outputs and odd increments into obuf
    for (int e = tid; e < (K << lw); e += nth) {
        const int k = e >> lw, p = e & (W - 1);
        const C zk = Z[((size_t)k << lw) + p], zm = Z[((size_t)((M - k) % M) << lw) + p];
        const R hf = X4 ? R(1) : R(0.5);
        R ra = hf * (zk.x + zm.x), rb = hf * (zk.y + zm.y);
        if (k == 0) {
            ra *= R(0.5);
            rb *= R(0.5);
        } else if (2 * k <= n) {                           // y_{2k}
            C* ev = reinterpret_cast<C*>(obuf + ((size_t)(2 * k - 1) << (lw + 1)));
            ev[p] = mkc(hf * (zm.y - zk.y), hf * (zk.x - zm.x));
        }
        if (2 * k + 1 <= n) {                              // increment of y_{2k+1}
            C* od = reinterpret_cast<C*>(obuf + ((size_t)(2 * k) << (lw + 1)));
            od[p] = mkc(ra, rb);
        }
    }
    __syncthreads();
    // y_{2k+1} = sum of the increments up to k: segmented prefix sum per real column
    const int KO = n / 2 + (n & 1);                        // odd outputs y_1, y_3, ..., count ceil(n/2)
    const int segs = nth >= ncol ? nth / ncol : 1;
    const int Ls = (KO + segs - 1) / segs;
    for (int task = tid; task < ncol * segs; task += nth) {
        const int c = task % ncol, sg = task / ncol;
        const int k0 = sg * Ls, k1 = min(KO, k0 + Ls);
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
            const int c = task % ncol, sg = task / ncol;
            if (sg == 0) continue;
            R off = R(0);
            for (int s2 = 0; s2 < sg; ++s2) off += seg[s2 * ncol + c];
            const int k0 = sg * Ls, k1 = min(KO, k0 + Ls);
            for (int k = k0; k < k1; ++k) obuf[((size_t)(2 * k) << (lw + 1)) + c] += off;
        }
        __syncthreads();
    }
    if (inner == 1) {
        // transpose obuf [j][column] -> raw [column][j] in the free buffer, then store linearly
        R* raw = reinterpret_cast<R*>(Z);
        for (int e = tid; e < ncol * n; e += nth) {
            const int j = e >> (lw + 1), r = e & (ncol - 1);
            raw[r * n + j] = obuf[e];
        }
        __syncthreads();
        const int count = rows_here * n;
        const long long start = base_row * n;
        for (int i = tid; i < count; i += nth) dst_store<R, TIN, OMODE, 1>(out, start + i, raw[i]);
    } else {
        const long long base = o * (long long)n * inner;
        for (int e = tid; e < ncol * n; e += nth) {
            const int j = e >> (lw + 1), r = e & (ncol - 1);
            const long long ii = i0 + r;
            if (ii < inner) dst_store<R, TIN, OMODE, 1>(out, base + (long long)j * inner + ii, obuf[e]);
        }
    }
}

}  // namespace qbvm
