// qbvm_kernels.cu -- sm_103a kernels of the PinT-QBVM / PinT-MQBVM direct
// solve (Section 3.3, eq. 3.8).
//
// Space-first order (2D/3D): the factors of
//     A = (V (x) I)(D/tau (x) I - I (x) Delta_h)(V^{-1} (x) I)
// act on different Kronecker factors, and Delta_h = S diag(-Lambda) S^{-1}
// with the DST-I matrix S per axis, so the three steps of eq. 3.8 can be
// applied as: DST of the right-hand side along every space axis, then per
// spatial mode the scalar omega-circulant time problem (omega-scaling, FFT,
// divide by d_k/tau + Lambda_l, inverse FFT, unscaling), then the inverse DST.
// Intermediates stay real: the per-mode time system is real.
//
// 1D keeps the paper's order: omega-scaling + FFT along time into a complex
// workspace, one complex tridiagonal (Thomas) solve per frequency, inverse
// FFT + unscaling.
#include "qbvm_fft.cuh"
#include "qbvm_internal.h"

#include <type_traits>

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
template <typename R, int MAXB4>
__global__ void __launch_bounds__(TILE_THREADS)
k_dst(const R* in, R* out, int n, int lm, int lw, long long outer, long long inner,
      const cplx<R>* __restrict__ tw, const R* __restrict__ sn) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = 1 << lm, W = 1 << lw, H = M >> 1;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int ncol = 2 * W;                          // real columns in this tile
    C* buf = reinterpret_cast<C*>(smem_raw);         // M x W complex
    R* obuf = reinterpret_cast<R*>(buf + (M << lw)); // M x 2W real (outputs y_1..y_n at rows 0..n-1)
    C* stw = reinterpret_cast<C*>(obuf + ((size_t)M << (lw + 1)));
    R* ssn = reinterpret_cast<R*>(stw + M);          // sin(j pi / M), j = 0..H
    R* seg = ssn + (H + 2);                          // prefix-sum segment totals
    R* bufr = reinterpret_cast<R*>(buf);

    for (int i = tid; i < M; i += nth) stw[i] = tw[i];
    for (int i = tid; i <= H; i += nth) ssn[i] = sn[i];
    for (int p = tid; p < W; p += nth) buf[p] = mkc(R(0), R(0));

    long long base_row = 0, o = 0, i0 = 0;
    if (inner == 1) {
        base_row = (long long)blockIdx.x * ncol;
        for (int e = tid; e < ncol * n; e += nth) {
            int r = e / n, j = e - r * n;
            long long row = base_row + r;
            R v = row < outer ? in[row * n + j] : R(0);
            bufr[(((j + 1) << lw) + (r >> 1)) * 2 + (r & 1)] = v;
        }
    } else {
        long long tiles_per_outer = (inner + ncol - 1) / ncol;
        o = blockIdx.x / tiles_per_outer;
        i0 = (blockIdx.x - o * tiles_per_outer) * ncol;
        const R* src = in + o * (long long)n * inner;
        for (int e = tid; e < ncol * n; e += nth) {
            int j = e / ncol, r = e - j * ncol;
            long long ii = i0 + r;
            R v = ii < inner ? src[(long long)j * inner + ii] : R(0);
            bufr[(((j + 1) << lw) + (r >> 1)) * 2 + (r & 1)] = v;
        }
    }
    __syncthreads();
    // w_j and w_{M-j} from the pair (x_j, x_{M-j}), j = 1..H
    for (int e = tid; e < (H << lw); e += nth) {
        int j = (e >> lw) + 1, p = e & (W - 1);
        C a = buf[(j << lw) + p], b = buf[((M - j) << lw) + p];
        R sj = ssn[j];
        C A = mkc(sj * (a.x + b.x), sj * (a.y + b.y));
        C B = mkc(R(0.5) * (a.x - b.x), R(0.5) * (a.y - b.y));
        buf[(j << lw) + p] = cadd(A, B);
        if (j != H) buf[((M - j) << lw) + p] = csub(A, B);
    }
    __syncthreads();
    fft_tile<-1, MAXB4>(buf, stw, lm, lw);

    // separate the packed columns; even outputs and odd increments into obuf
    for (int e = tid; e < (H << lw); e += nth) {
        int k = e >> lw, p = e & (W - 1);
        C zk = buf[(k << lw) + p], zm = buf[(((M - k) & (M - 1)) << lw) + p];
        R ra = R(0.5) * (zk.x + zm.x), rb = R(0.5) * (zk.y + zm.y);
        if (k == 0) {
            ra *= R(0.5);
            rb *= R(0.5);
        } else {
            R* ev = obuf + ((size_t)(2 * k - 1) << (lw + 1));
            ev[2 * p] = R(0.5) * (zm.y - zk.y);
            ev[2 * p + 1] = R(0.5) * (zk.x - zm.x);
        }
        R* od = obuf + ((size_t)(2 * k) << (lw + 1));
        od[2 * p] = ra;
        od[2 * p + 1] = rb;
    }
    __syncthreads();
    // y_{2k+1} = sum_{kappa <= k} (odd increments): segmented prefix sum per real column
    const int segs = nth >= ncol ? nth / ncol : 1;
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
        for (int e = tid; e < ncol * n; e += nth) {
            int r = e / n, j = e - r * n;
            long long row = base_row + r;
            if (row < outer) out[row * n + j] = obuf[((size_t)j << (lw + 1)) + r];
        }
    } else {
        R* dst = out + o * (long long)n * inner;
        for (int e = tid; e < ncol * n; e += nth) {
            int j = e / ncol, r = e - j * ncol;
            long long ii = i0 + r;
            if (ii < inner) dst[(long long)j * inner + ii] = obuf[((size_t)j << (lw + 1)) + r];
        }
    }
}

constexpr int DST_TILE = 2048;     // complex elements per DST tile

static int dst_lw(int lm) {
    int lw = 0;
    while (((1 << lm) << (lw + 1)) <= DST_TILE) ++lw;
    return lw;
}

template <typename R>
size_t dst_smem(int lm) {
    const int M = 1 << lm, lw = dst_lw(lm), W = 1 << lw, H = M >> 1;
    const int ncol = 2 * W;
    size_t seg = (size_t)(TILE_THREADS >= ncol ? TILE_THREADS : ncol);
    return sizeof(cplx<R>) * ((size_t)M * W + M) + sizeof(R) * ((size_t)M * 2 * W + H + 2 + seg);
}

template <typename R>
cudaError_t launch_dst(const R* in, R* out, int n, int lm, long long outer, long long inner,
                       const void* tw, const void* sn, cudaStream_t s) {
    const int lw = dst_lw(lm), W = 1 << lw;
    long long blocks;
    if (inner == 1) blocks = (outer + 2 * W - 1) / (2 * W);
    else blocks = outer * ((inner + 2 * W - 1) / (2 * W));
    size_t smem = dst_smem<R>(lm);
    auto kern = k_dst<R, DST_TILE / 4 / TILE_THREADS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, TILE_THREADS, smem, s>>>(in, out, n, lm, lw, outer, inner,
                                                      reinterpret_cast<const cplx<R>*>(tw),
                                                      reinterpret_cast<const R*>(sn));
    return cudaGetLastError();
}

template cudaError_t launch_dst<double>(const double*, double*, int, int, long long, long long, const void*,
                                        const void*, cudaStream_t);
template cudaError_t launch_dst<float>(const float*, float*, int, int, long long, long long, const void*,
                                       const void*, cudaStream_t);

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
template <typename R, int MAXB4>
__global__ void __launch_bounds__(TILE_THREADS)
k_time_solve(const R* in, R* out, long long Nx, int lh, int lw, const cplx<R>* __restrict__ tw,
             const double2* __restrict__ gpow, const double2* __restrict__ gipw,
             const double2* __restrict__ ak, const double* __restrict__ lamtau, double cnorm,
             double rho_h, double rho_hinv, int delta_rhs, int n0_only) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = 1 << lh, W = 1 << lw;
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* stw = buf + (H << lw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const long long l0 = (long long)blockIdx.x * W;

    for (int i = tid; i < H; i += nth) stw[i] = tw[i];
    for (int e = tid; e < (H << lw); e += nth) {
        int t = e >> lw, c = e & (W - 1);
        long long l = l0 + c;
        double f0 = 0.0, f1 = 0.0;
        if (l < Nx) {
            if (delta_rhs) {
                if (t == 0) f0 = (double)in[l];
            } else {
                f0 = (double)in[(long long)t * Nx + l];
                f1 = rho_h * (double)in[(long long)(t + H) * Nx + l];
            }
        }
        double2 g = gpow[t];
        buf[e] = mkc(R(g.x * f0 - g.y * f1), R(g.y * f0 + g.x * f1));
    }
    __syncthreads();
    fft_tile<+1, MAXB4>(buf, stw, lh, lw);

    for (int e = tid; e < (H << lw); e += nth) {
        int k = e >> lw, c = e & (W - 1);
        long long l = l0 + c;
        double lt = l < Nx ? lamtau[l] : 0.0;
        double2 a = ak[k];
        double zr = a.x + lt, zi = a.y;
        double inv = cnorm / fma(zr, zr, zi * zi);
        C u = buf[e];
        buf[e] = mkc(R((u.x * zr + u.y * zi) * inv), R((u.y * zr - u.x * zi) * inv));
    }
    __syncthreads();
    fft_tile<-1, MAXB4>(buf, stw, lh, lw);

    const int tmax = n0_only ? 1 : H;
    for (int e = tid; e < (tmax << lw); e += nth) {
        int t = e >> lw, c = e & (W - 1);
        long long l = l0 + c;
        if (l < Nx) {
            double2 gi = gipw[t];
            C w = buf[e];
            double vx = gi.x * (double)w.x - gi.y * (double)w.y;
            out[(long long)t * Nx + l] = R(vx);
            if (!n0_only) {
                double vy = gi.x * (double)w.y + gi.y * (double)w.x;
                out[(long long)(t + H) * Nx + l] = R(rho_hinv * vy);
            }
        }
    }
}

static int tile_lw(int lp) {
    int lw = 0;
    while (((1 << lp) << (lw + 1)) <= TILE_ELEMS) ++lw;
    return lw;
}

template <typename R>
cudaError_t launch_time_solve(const R* in, R* out, const Tables& tb, double cnorm, int delta_rhs,
                              int n0_only, cudaStream_t s) {
    const int lh = tb.lnt - 1, H = 1 << lh;
    const int lw = tile_lw(lh), W = 1 << lw;
    long long blocks = (tb.Nx + W - 1) / W;
    size_t smem = sizeof(cplx<R>) * ((size_t)H * W + H);
    auto kern = k_time_solve<R, TILE_ELEMS / 4 / TILE_THREADS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const cplx<R>* tw = std::is_same<R, double>::value ? reinterpret_cast<const cplx<R>*>(tb.tw_t)
                                                       : reinterpret_cast<const cplx<R>*>(tb.tw_t32);
    kern<<<(unsigned)blocks, TILE_THREADS, smem, s>>>(in, out, tb.Nx, lh, lw, tw, tb.gpow, tb.gipw, tb.ak,
                                                      tb.lamtau, cnorm, tb.rho_h, tb.rho_hinv, delta_rhs,
                                                      n0_only);
    return cudaGetLastError();
}

template cudaError_t launch_time_solve<double>(const double*, double*, const Tables&, double, int, int, cudaStream_t);
template cudaError_t launch_time_solve<float>(const float*, float*, const Tables&, double, int, int, cudaStream_t);

// ------------------------------------------------------------------ 1D path
//
// The paper's order.  Step (a) is the half-length transform of the time
// solve above applied to every spatial point x, giving the even frequencies
// u^_{2m}(x) in the complex workspace wk[m][x]; Step (b) solves the complex
// tridiagonal systems of those frequencies (the odd ones are their conjugates
// and are never formed); Step (c) is the half-length inverse.

__global__ void __launch_bounds__(TILE_THREADS)
k_time_fwd_1d(const double* in, double2* wk, long long Nx, int lh, int lw, const double2* __restrict__ tw,
              const double2* __restrict__ gpow, double rho_h, int delta_rhs, double in_scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = 1 << lh, W = 1 << lw;
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    double2* stw = buf + (H << lw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const long long x0 = (long long)blockIdx.x * W;
    for (int i = tid; i < H; i += nth) stw[i] = tw[i];
    for (int e = tid; e < (H << lw); e += nth) {
        int t = e >> lw, c = e & (W - 1);
        long long x = x0 + c;
        double f0 = 0.0, f1 = 0.0;
        if (x < Nx) {
            if (delta_rhs) {
                if (t == 0) f0 = in_scale * in[x];
            } else {
                f0 = in[(long long)t * Nx + x];
                f1 = rho_h * in[(long long)(t + H) * Nx + x];
            }
        }
        double2 g = gpow[t];
        buf[e] = make_double2(g.x * f0 - g.y * f1, g.y * f0 + g.x * f1);
    }
    __syncthreads();
    fft_tile<+1, TILE_ELEMS / 4 / TILE_THREADS>(buf, stw, lh, lw);
    for (int e = tid; e < (H << lw); e += nth) {
        int k = e >> lw, c = e & (W - 1);
        long long x = x0 + c;
        if (x < Nx) wk[(long long)k * Nx + x] = buf[e];
    }
}

// Step (b) in 1D: for every even frequency 2m solve b_m w_i - w_{i-1} - w_{i+1} = rhs_i
// (the Dirichlet 3-point system times h^2; h^2 is folded into gpow) by the
// Thomas algorithm.  cp holds the modified super-diagonal.
__global__ void k_thomas_1d(double2* wk, double2* cp, int nsys, long long Nx, const double2* __restrict__ bk) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsys) return;
    double2* d = wk + (long long)k * Nx;
    double2* c = cp + (long long)k * Nx;
    const double2 b = bk[k];
    // forward sweep: den_i = b + c_{i-1}, c_i = -1/den_i, d_i = (d_i + d_{i-1})/den_i
    double2 cprev = make_double2(0.0, 0.0), dprev = make_double2(0.0, 0.0);
    for (long long i = 0; i < Nx; ++i) {
        double dr = b.x + cprev.x, di = b.y + cprev.y;
        double s = 1.0 / fma(dr, dr, di * di);
        double2 inv = make_double2(dr * s, -di * s);               // 1/den
        double2 rhs = d[i];
        rhs.x += dprev.x;
        rhs.y += dprev.y;
        double2 dn = cmul(rhs, inv);
        double2 cn = make_double2(-inv.x, -inv.y);
        d[i] = dn;
        c[i] = cn;
        cprev = cn;
        dprev = dn;
    }
    // back substitution: x_i = d_i - c_i x_{i+1}
    double2 xn = dprev;
    for (long long i = Nx - 2; i >= 0; --i) {
        double2 ci = c[i], di = d[i];
        double2 t = cmul(ci, xn);
        xn = make_double2(di.x - t.x, di.y - t.y);
        d[i] = xn;
    }
}

__global__ void __launch_bounds__(TILE_THREADS)
k_time_inv_1d(const double2* wk, double* out, long long Nx, int lh, int lw, const double2* __restrict__ tw,
              const double2* __restrict__ gipw, double rho_hinv, int n0_only) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int H = 1 << lh, W = 1 << lw;
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    double2* stw = buf + (H << lw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const long long x0 = (long long)blockIdx.x * W;
    for (int i = tid; i < H; i += nth) stw[i] = tw[i];
    for (int e = tid; e < (H << lw); e += nth) {
        int k = e >> lw, c = e & (W - 1);
        long long x = x0 + c;
        buf[e] = x < Nx ? wk[(long long)k * Nx + x] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    fft_tile<-1, TILE_ELEMS / 4 / TILE_THREADS>(buf, stw, lh, lw);
    const int tmax = n0_only ? 1 : H;
    for (int e = tid; e < (tmax << lw); e += nth) {
        int t = e >> lw, c = e & (W - 1);
        long long x = x0 + c;
        if (x < Nx) {
            double2 gi = gipw[t], w = buf[e];
            out[(long long)t * Nx + x] = gi.x * w.x - gi.y * w.y;
            if (!n0_only) out[(long long)(t + H) * Nx + x] = rho_hinv * (gi.x * w.y + gi.y * w.x);
        }
    }
}

cudaError_t launch_time_fwd_1d(const double* in, double2* wk, const Tables& tb, int delta_rhs, double in_scale,
                               cudaStream_t s) {
    const int lh = tb.lnt - 1, H = 1 << lh, lw = tile_lw(lh), W = 1 << lw;
    long long blocks = (tb.Nx + W - 1) / W;
    size_t smem = sizeof(double2) * ((size_t)H * W + H);
    cudaError_t e = cudaFuncSetAttribute(k_time_fwd_1d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_time_fwd_1d<<<(unsigned)blocks, TILE_THREADS, smem, s>>>(in, wk, tb.Nx, lh, lw, tb.tw_t, tb.gpow, tb.rho_h,
                                                                delta_rhs, in_scale);
    return cudaGetLastError();
}

cudaError_t launch_thomas_1d(double2* wk, double2* cp, const Tables& tb, cudaStream_t s) {
    const int nsys = tb.nt / 2;
    int threads = 64;
    int blocks = (nsys + threads - 1) / threads;
    k_thomas_1d<<<blocks, threads, 0, s>>>(wk, cp, nsys, tb.Nx, tb.bk);
    return cudaGetLastError();
}

cudaError_t launch_time_inv_1d(const double2* wk, double* out, const Tables& tb, int n0_only, cudaStream_t s) {
    const int lh = tb.lnt - 1, H = 1 << lh, lw = tile_lw(lh), W = 1 << lw;
    long long blocks = (tb.Nx + W - 1) / W;
    size_t smem = sizeof(double2) * ((size_t)H * W + H);
    cudaError_t e = cudaFuncSetAttribute(k_time_inv_1d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_time_inv_1d<<<(unsigned)blocks, TILE_THREADS, smem, s>>>(wk, out, tb.Nx, lh, lw, tb.tw_t, tb.gipw,
                                                                tb.rho_hinv, n0_only);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ residual
//
// (A y)^n = (y^n - y^{n-1})/tau - Delta_h y^n for n >= 1 and
// (A y)^0 = (y^0 - omega y^N)/tau - Delta_h y^0 (eq. 3.3 / 3.6, Kronecker form
// of Section 3.3); f^0 = -omega g / tau for the delta right-hand side.
constexpr int RES_THREADS = 256;

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

__global__ void __launch_bounds__(RES_THREADS)
k_residual(const double* __restrict__ y, const double* __restrict__ f, int delta_rhs, int nt,
           int nx, int ny, int nz, double inv_tau, double omega, double hx2, double hy2, double hz2,
           double* partials, double* r_out) {
    __shared__ double sh[32];
    const long long Nx = (long long)nx * ny * nz;
    const long long total = Nx * nt;
    double rr = 0.0, ff = 0.0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long t = idx / Nx, sidx = idx - t * Nx;
        int ix = (int)(sidx % nx);
        long long q = sidx / nx;
        int iy = (int)(q % ny), iz = (int)(q / ny);
        double yv = y[idx];
        double lap = -2.0 * yv * hx2;
        if (ix > 0) lap += y[idx - 1] * hx2;
        if (ix < nx - 1) lap += y[idx + 1] * hx2;
        if (ny > 1) {
            lap -= 2.0 * yv * hy2;
            if (iy > 0) lap += y[idx - nx] * hy2;
            if (iy < ny - 1) lap += y[idx + nx] * hy2;
        }
        if (nz > 1) {
            long long pl = (long long)nx * ny;
            lap -= 2.0 * yv * hz2;
            if (iz > 0) lap += y[idx - pl] * hz2;
            if (iz < nz - 1) lap += y[idx + pl] * hz2;
        }
        double prev = t > 0 ? y[idx - Nx] : omega * y[(long long)(nt - 1) * Nx + sidx];
        double Ay = (yv - prev) * inv_tau - lap;
        double fv;
        if (delta_rhs) fv = t == 0 ? -omega * inv_tau * f[sidx] : 0.0;
        else fv = f[idx];
        double r = fv - Ay;
        if (r_out) r_out[idx] = r;
        rr = fma(r, r, rr);
        ff = fma(fv, fv, ff);
    }
    rr = block_sum(rr, sh);
    ff = block_sum(ff, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = rr;
        partials[2 * blockIdx.x + 1] = ff;
    }
}

__global__ void k_reduce_pairs(const double* partials, int n, double* sums) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    a = block_sum(a, sh);
    b = block_sum(b, sh);
    if (threadIdx.x == 0) {
        sums[0] = a;
        sums[1] = b;
    }
}

int residual_blocks(const Tables& tb) {
    long long total = tb.Nx * tb.nt;
    long long b = (total + RES_THREADS * 4 - 1) / (RES_THREADS * 4);
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_residual(const double* y, const double* f, int delta_rhs, const Tables& tb,
                            const double h2inv[3], double* partials, int nblocks, double* sums,
                            double* r_out, cudaStream_t s) {
    k_residual<<<nblocks, RES_THREADS, 0, s>>>(y, f, delta_rhs, tb.nt, tb.n[0], tb.n[1], tb.n[2],
                                               1.0 / tb.tau, tb.omega, h2inv[0], h2inv[1], h2inv[2],
                                               partials, r_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_pairs<<<1, 1024, 0, s>>>(partials, nblocks, sums);
    return cudaGetLastError();
}

}  // namespace qbvm
