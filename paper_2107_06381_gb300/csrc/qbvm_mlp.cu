// qbvm_mlp.cu -- learned regularisation parameter: spectrum features of g_delta
// and a small MLP (forward, backward, Adam) trained on solves of the method.
//
// The paper chooses alpha a priori (Section 5: alpha = delta for PinT-QBVM,
// tau*delta for PinT-MQBVM).  Here a network predicts t = log10(alpha /
// alpha_rule) from
//   * 64 bins of the radial DST spectrum of g_delta: for the sine modes
//     (k_x, k_y) of the 2D grid, bin b holds log10 of the mean of c_l^2, c_l the
//     coefficient of mode l in g = sum_l c_l sin(k_x pi x) sin(k_y pi y) and
//     b = floor(64 |k| / (sqrt(2) (n + 1)));
//   * log10 delta, T and log2 N_t,
// standardised with per-feature mean and deviation before the first layer.
// Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3.h2 + b3 with
// bfloat16 weights in the products and FP32 accumulation (FP32 master weights
// for Adam); loss = (1/2B) sum (y - t)^2.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "qbvm.h"
#include "qbvm_internal.h"

namespace {

constexpr int MLP_THREADS = 256;

// ------------------------------------------------------------------ features
//
// The spectrum is taken of g_b 2^k_b, 2^k_b the power of two nearest 1/delta_b,
// so that data of any magnitude FP64 holds stays inside FP32's range through
// the FP32 DSTs and the squares; the bins are then corrected by the exact
// log10 2^(-2 k_b), so the features are those of g_b itself.

// The instance's scaling exponent k_b (0 for delta not positive and finite).
__device__ __forceinline__ int feat_scale_exp(double d) {
    if (!(d > 0.0) || !isfinite(d)) return 0;
    const int k = -(int)rint(log2(d));
    return k < -1000 ? -1000 : (k > 1000 ? 1000 : k);
}

// w[b][i] = FP32 rounding of g[b][i] 2^k_b (the scaling is exact in FP64).
__global__ void k_scaled_to_f32(const double* __restrict__ g, long long Nx, int B, const double* __restrict__ delta,
                                float* __restrict__ w) {
    const long long total = (long long)B * Nx;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / Nx);
        w[i] = __double2float_rn(ldexp(g[i], feat_scale_exp(delta[b])));
    }
}

__global__ void k_spectrum_bins(const float* __restrict__ ghat, long long Nx, const unsigned char* __restrict__ bin,
                                const float* __restrict__ inv_count, float coef_scale2, const double* __restrict__ delta,
                                float T, float lg_nt, int in_dim, float* __restrict__ feats) {
    __shared__ float acc[64];
    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) acc[i] = 0.f;
    __syncthreads();
    const float* g = ghat + (long long)b * Nx;
    for (long long l = threadIdx.x; l < Nx; l += blockDim.x) {
        float c = g[l];
        atomicAdd(&acc[bin[l]], c * c * coef_scale2);
    }
    __syncthreads();
    float* f = feats + (long long)b * in_dim;
    // log10(mean square + 1e-30) of g_b's own coefficients from the scaled mean
    // square m: a = log10 m - 2 k_b log10 2 (which may lie beyond FP64's range
    // as a power of ten), then log10(10^a + 10^-30) = max + log10(1 + 10^-|a + 30|)
    const int k = feat_scale_exp(delta[b]);
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        const double m = (double)(acc[i] * inv_count[i]);
        double v = -30.0;
        if (m > 0.0) {
            const double a = log10(m) - 2.0 * k * 0.30102999566398119521;
            v = a >= -30.0 ? a + log10(1.0 + exp10(-30.0 - a)) : -30.0 + log10(1.0 + exp10(a + 30.0));
        }
        f[i] = (float)v;
    }
    if (threadIdx.x == 0) {
        f[64] = (float)log10(delta[b]);
        f[65] = T;
        f[66] = lg_nt;
    }
}

// ------------------------------------------------------------------ MLP
__device__ __forceinline__ float bf(const __nv_bfloat16* w, long long i) { return __bfloat162float(w[i]); }

// y = H w3 + b3 (one warp per row).
__global__ void k_dense_out(const float* __restrict__ H, const __nv_bfloat16* __restrict__ w3, const float* __restrict__ b3,
                            int B, int N, float* __restrict__ y) {
    int warp = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= B) return;
    const float* h = H + (long long)warp * N;
    float s = 0.f;
    for (int n = lane; n < N; n += 32) s = fmaf(h[n], bf(w3, n), s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[warp] = s + b3[0];
}

// dy = (y - t)/B and the loss sum (1/2B) sum (y - t)^2.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, int B, float* __restrict__ dy,
                      double* __restrict__ loss) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.f;
    if (b < B) {
        r = y[b] - t[b];
        dy[b] = r / (float)B;
    }
    float s = 0.5f * r * r / (float)B;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, (double)s);
}

// dZ2 = dy w3^T masked by Z2 > 0.
__global__ void k_back_out(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ w3, const float* __restrict__ Z2,
                           int B, int N, float* __restrict__ dZ2) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)B * N) return;
    int b = (int)(idx / N), n = (int)(idx - (long long)b * N);
    dZ2[idx] = Z2[idx] > 0.f ? dy[b] * bf(w3, n) : 0.f;
}

// Gradient of the output layer (one output): dw[k] = sum_b D[b] A[b][k],
// db = sum_b D[b], the batch cut into WG_CHUNKS chunks.  Block c sums its
// chunk's rows -- the 8 warps take rows b, b + 8, ..., the lanes consecutive k,
// so every row of A is read coalesced -- into part[c][0..K]; k_wgrad1_sum adds
// the chunks in a fixed order (the result does not depend on scheduling).
constexpr int WG_CHUNKS = 64;
__global__ void k_wgrad1_part(const float* __restrict__ D, const float* __restrict__ A, int B, int K,
                              float* __restrict__ part) {
    constexpr int NW = MLP_THREADS / 32;
    __shared__ float sh[NW][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b0 = (int)((long long)B * blockIdx.x / gridDim.x);
    const int b1 = (int)((long long)B * (blockIdx.x + 1) / gridDim.x);
    for (int k0 = 0; k0 <= K; k0 += 32) {
        const int k = k0 + lane;
        float acc = 0.f;
        for (int b = b0 + w; b < b1; b += NW) {
            const float a = k < K ? A[(long long)b * K + k] : (k == K ? 1.f : 0.f);
            acc = fmaf(D[b], a, acc);
        }
        sh[w][lane] = acc;
        __syncthreads();
        if (w == 0 && k <= K) {
            float t = 0.f;
            for (int i = 0; i < NW; ++i) t += sh[i][lane];
            part[(long long)blockIdx.x * (K + 1) + k] = t;
        }
        __syncthreads();
    }
}
__global__ void k_wgrad1_sum(const float* __restrict__ part, int G, int K, float* __restrict__ dw,
                             float* __restrict__ db) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
        float t = 0.f;
        for (int c = 0; c < G; ++c) t += part[(long long)c * (K + 1) + k];
        if (k < K) dw[k] = t;
        else *db = t;
    }
}

// ---------------------------------------------- tensor-core products (BF16)
//
// C[m][n] = sum_k A(m, k) B(k, n) on the tensor cores: mma.sync m16n8k16 with
// BF16 operands and FP32 accumulation.  A is FP32 in memory (activations or
// gradients; optionally standardised on load, (a - mu[k]) * is[k], and so may
// be the FP32 B operand, (b - mub[n]) * isb[n]) and enters
// as its BF16 split a = a_hi + a_lo (a_hi = bf16(a), a_lo = bf16(a - a_hi): 16
// significant bits); B is either a BF16 weight matrix (one MMA per split part:
// A_hi W + A_lo W) or FP32 (split too: A_hi B_hi + A_hi B_lo + A_lo B_hi, the
// dropped A_lo B_lo below 2^-16 relative).  So the products keep the accuracy
// of the FP32-activation / BF16-weight arithmetic the network is defined with.
// Operand (m, k) of A sits at a[m * sam + k * sak], (k, n) of B at
// b[k * sbk + n * sbn]; rows and columns past M, N, K read as zero.
// One warp owns a 16 x 32 tile of C (four 16 x 8 MMA tiles); a CTA of four
// warps a 16 x 128 strip.  Fragments are gathered straight from global memory
// (the operands are a few hundred kilobytes and stay in L1/L2).
// Epilogue: EPI_BIAS_RELU  Z = C + bias[n], H = relu(Z);
//           EPI_MASK       C = (mask(m, n) > 0) ? C : 0 (mask row stride N);
//           EPI_STORE      C.
enum { EPI_BIAS_RELU = 0, EPI_MASK = 1, EPI_STORE = 2 };
constexpr int MMA_WARPS = 4;

__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo_col, __nv_bfloat16 hi_col) {
    return (unsigned)__bfloat16_as_ushort(lo_col) | ((unsigned)__bfloat16_as_ushort(hi_col) << 16);
}
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <bool BW, int EPI>
__global__ void __launch_bounds__(32 * MMA_WARPS)
k_mma_gemm(int M, int N, int K, const float* __restrict__ a, long long sam, long long sak,
           const float* __restrict__ mu, const float* __restrict__ is, const void* __restrict__ b, long long sbk,
           long long sbn, const float* __restrict__ mub, const float* __restrict__ isb,
           const float* __restrict__ bias, const float* __restrict__ mask, float* __restrict__ C,
           float* __restrict__ C2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;                 // fragment row group, thread in group
    const int m0 = blockIdx.x * 16, n0 = blockIdx.y * 128 + warp * 32;
    if (n0 >= N) return;
    auto ldA = [&](int m, int k) -> float {
        if (m >= M || k >= K) return 0.f;
        const float v = a[(long long)m * sam + (long long)k * sak];
        return mu ? (v - mu[k]) * is[k] : v;
    };
    auto ldB = [&](int k, int n) -> float {
        if (k >= K || n >= N) return 0.f;
        const long long i = (long long)k * sbk + (long long)n * sbn;
        if (BW) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(b)[i]);
        const float v = reinterpret_cast<const float*>(b)[i];
        return mub ? (v - mub[n]) * isb[n] : v;
    };
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        // A fragment: rows g, g + 8; columns 2 tg, 2 tg + 1 (+ 8)
        unsigned ah[4], al[4];
        {
            const int r[4] = {g, g + 8, g, g + 8}, c[4] = {2 * tg, 2 * tg, 2 * tg + 8, 2 * tg + 8};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __nv_bfloat16 h0, l0, h1, l1;
                split_bf16(ldA(m0 + r[q], k0 + c[q]), h0, l0);
                split_bf16(ldA(m0 + r[q], k0 + c[q] + 1), h1, l1);
                ah[q] = pack_bf16(h0, h1);
                al[q] = pack_bf16(l0, l1);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + 8 * j + g;                    // B fragment: column g; rows 2 tg, 2 tg + 1 (+ 8)
            __nv_bfloat16 h[4], l[4];
            const int kk[4] = {k0 + 2 * tg, k0 + 2 * tg + 1, k0 + 2 * tg + 8, k0 + 2 * tg + 9};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (BW) {
                    h[q] = __float2bfloat16_rn(ldB(kk[q], n));   // exact: the weights are BF16
                    l[q] = __float2bfloat16_rn(0.f);
                } else {
                    split_bf16(ldB(kk[q], n), h[q], l[q]);
                }
            }
            const unsigned bh0 = pack_bf16(h[0], h[1]), bh1 = pack_bf16(h[2], h[3]);
            mma_bf16(acc[j], ah, bh0, bh1);
            mma_bf16(acc[j], al, bh0, bh1);
            if (!BW) mma_bf16(acc[j], ah, pack_bf16(l[0], l[1]), pack_bf16(l[2], l[3]));
        }
    }
    // D fragment: rows g, g + 8; columns 2 tg, 2 tg + 1 of each n-tile
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int m = m0 + g + (e >= 2 ? 8 : 0), n = n0 + 8 * j + 2 * tg + (e & 1);
            if (m >= M || n >= N) continue;
            const long long o = (long long)m * N + n;
            float v = acc[j][e];
            if (EPI == EPI_BIAS_RELU) {
                v += bias[n];
                C[o] = v;
                C2[o] = fmaxf(v, 0.f);
            } else if (EPI == EPI_MASK) {
                C[o] = mask[o] > 0.f ? v : 0.f;
            } else {
                C[o] = v;
            }
        }
    }
}

template <bool BW, int EPI>
cudaError_t launch_mma(int M, int N, int K, const float* a, long long sam, long long sak, const float* mu,
                       const float* is, const void* b, long long sbk, long long sbn, const float* mub,
                       const float* isb, const float* bias, const float* mask, float* C, float* C2, cudaStream_t s) {
    const dim3 grid((unsigned)((M + 15) / 16), (unsigned)((N + 127) / 128));
    k_mma_gemm<BW, EPI><<<grid, 32 * MMA_WARPS, 0, s>>>(M, N, K, a, sam, sak, mu, is, b, sbk, sbn, mub, isb, bias,
                                                        mask, C, C2);
    return cudaGetLastError();
}

// db[n] = sum_b D[b][n] (the bias gradients).
__global__ void k_colsum(const float* __restrict__ D, int B, int N, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += D[(long long)b * N + n];
    db[n] = s;
}

// Adam (Kingma & Ba): FP32 master weights, bfloat16 copy for the products.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ pb, long long n, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

unsigned nblk(long long n) { return (unsigned)((n + MLP_THREADS - 1) / MLP_THREADS); }

}  // namespace

struct qbvm_mlp {
    int in_dim = 0, width = 0, bmax = 0;
    long long nparam = 0;
    long long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, ow3 = 0, ob3 = 0;
    float* p = nullptr;       // FP32 master
    float* g = nullptr;       // gradients
    float* m = nullptr;
    float* v = nullptr;
    __nv_bfloat16* pb = nullptr;
    float* mu = nullptr;
    float* inv_sd = nullptr;
    bool has_norm = false;
    float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *y = nullptr, *dy = nullptr, *dZ1 = nullptr,
          *dZ2 = nullptr;
    double* loss = nullptr;
    float* wpart = nullptr;   // output-layer gradient partial sums [WG_CHUNKS][width + 1]
    long long step = 0;
    std::vector<void*> allocs;
};

struct qbvm_features {
    int n = 0, M = 0, lm = 0, bmax = 0;
    double T = 0;
    int nt = 0;
    long long Nx = 0;
    float* work = nullptr;
    unsigned char* bin = nullptr;
    float* inv_count = nullptr;
    double* delta = nullptr;
    float2* tw = nullptr;
    float* sn = nullptr;
    std::vector<void*> allocs;
};

namespace {

template <typename T, typename H>
int m_alloc(H* h, T** ptr, size_t count) {
    *ptr = nullptr;
    if (!count) return QBVM_OK;
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_OOM;
    }
    h->allocs.push_back(q);
    *ptr = static_cast<T*>(q);
    return QBVM_OK;
}

// splitmix64 (Steele, Lea & Flood 2014): deterministic initial weights
unsigned long long splitmix(unsigned long long& s) {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The two hidden layers on the tensor cores: Z1 = A' W1^T + b1 (A' the
// standardised input), H1 = relu(Z1); Z2 = H1 W2^T + b2, H2 = relu(Z2).
cudaError_t mlp_hidden_layers(qbvm_mlp_t* h, const float* x, int B, cudaStream_t s) {
    const int K = h->in_dim, N = h->width;
    const float* mu = h->has_norm ? h->mu : nullptr;
    const float* is = h->has_norm ? h->inv_sd : nullptr;
    cudaError_t e = launch_mma<true, EPI_BIAS_RELU>(B, N, K, x, K, 1, mu, is, h->pb + h->oW1, 1, K, nullptr, nullptr,
                                                    h->p + h->ob1, nullptr, h->Z1, h->H1, s);
    if (e != cudaSuccess) return e;
    return launch_mma<true, EPI_BIAS_RELU>(B, N, N, h->H1, N, 1, nullptr, nullptr, h->pb + h->oW2, 1, N, nullptr,
                                           nullptr, h->p + h->ob2, nullptr, h->Z2, h->H2, s);
}

int mlp_grads(qbvm_mlp_t* h, const float* x, const float* t, int B, cudaStream_t s) {
    const int K = h->in_dim, N = h->width;
    const float* mu = h->has_norm ? h->mu : nullptr;
    const float* is = h->has_norm ? h->inv_sd : nullptr;
    if (cudaMemsetAsync(h->loss, 0, sizeof(double), s) != cudaSuccess) return QBVM_ERR_CUDA;
    if (mlp_hidden_layers(h, x, B, s) != cudaSuccess) return QBVM_ERR_CUDA;
    k_dense_out<<<nblk((long long)B * 32), MLP_THREADS, 0, s>>>(h->H2, h->pb + h->ow3, h->p + h->ob3, B, N, h->y);
    k_mse<<<nblk(B), MLP_THREADS, 0, s>>>(h->y, t, B, h->dy, h->loss);
    // w3, b3: dW = dy^T H2 (one output row)
    k_wgrad1_part<<<WG_CHUNKS, MLP_THREADS, 0, s>>>(h->dy, h->H2, B, N, h->wpart);
    k_wgrad1_sum<<<nblk((long long)(N + 1)), MLP_THREADS, 0, s>>>(h->wpart, WG_CHUNKS, N, h->g + h->ow3,
                                                                h->g + h->ob3);
    k_back_out<<<nblk((long long)B * N), MLP_THREADS, 0, s>>>(h->dy, h->pb + h->ow3, h->Z2, B, N, h->dZ2);
    // dW2 = dZ2^T H1 (N x N, reduction over the batch), db2 = column sums of dZ2
    if (launch_mma<false, EPI_STORE>(N, N, B, h->dZ2, 1, N, nullptr, nullptr, h->H1, N, 1, nullptr, nullptr,
                                     nullptr, nullptr, h->g + h->oW2, nullptr, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    k_colsum<<<nblk(N), MLP_THREADS, 0, s>>>(h->dZ2, B, N, h->g + h->ob2);
    // dZ1 = (dZ2 W2) masked by Z1 > 0
    if (launch_mma<true, EPI_MASK>(B, N, N, h->dZ2, N, 1, nullptr, nullptr, h->pb + h->oW2, N, 1, nullptr, nullptr,
                                   nullptr, h->Z1, h->dZ1, nullptr, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    // dW1 = dZ1^T A' (N x K, A' the standardised input, standardised on load), db1
    if (launch_mma<false, EPI_STORE>(N, K, B, h->dZ1, 1, N, nullptr, nullptr, x, K, 1, mu, is, nullptr, nullptr,
                                     h->g + h->oW1, nullptr, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    k_colsum<<<nblk(N), MLP_THREADS, 0, s>>>(h->dZ1, B, N, h->g + h->ob1);
    return cudaGetLastError() == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

}  // namespace

extern "C" {

int qbvm_mlp_create(int in_dim, int width, int max_batch, unsigned long long seed, qbvm_mlp_t** out) {
    if (!out || in_dim < 1 || in_dim > 4096 || width < 1 || width > 4096 || max_batch < 1) return QBVM_ERR_BAD_ARG;
    *out = nullptr;
    qbvm_mlp_t* h = new (std::nothrow) qbvm_mlp();
    if (!h) return QBVM_ERR_OOM;
    h->in_dim = in_dim;
    h->width = width;
    h->bmax = max_batch;
    const long long K = in_dim, N = width;
    h->oW1 = 0;
    h->ob1 = N * K;
    h->oW2 = h->ob1 + N;
    h->ob2 = h->oW2 + N * N;
    h->ow3 = h->ob2 + N;
    h->ob3 = h->ow3 + N;
    h->nparam = h->ob3 + 1;
    // He-uniform weights, zero biases (deterministic from `seed`)
    std::vector<float> init((size_t)h->nparam, 0.f);
    unsigned long long st = seed;
    auto uni = [&](double a) { return (float)((2.0 * ((splitmix(st) >> 11) * (1.0 / 9007199254740992.0)) - 1.0) * a); };
    for (long long i = 0; i < N * K; ++i) init[h->oW1 + i] = uni(std::sqrt(6.0 / K));
    for (long long i = 0; i < N * N; ++i) init[h->oW2 + i] = uni(std::sqrt(6.0 / N));
    for (long long i = 0; i < N; ++i) init[h->ow3 + i] = uni(std::sqrt(3.0 / N));
    int rc = m_alloc(h, &h->p, h->nparam);
    if (!rc) rc = m_alloc(h, &h->g, h->nparam);
    if (!rc) rc = m_alloc(h, &h->m, h->nparam);
    if (!rc) rc = m_alloc(h, &h->v, h->nparam);
    if (!rc) rc = m_alloc(h, &h->pb, h->nparam);
    if (!rc) rc = m_alloc(h, &h->mu, K);
    if (!rc) rc = m_alloc(h, &h->inv_sd, K);
    if (!rc) rc = m_alloc(h, &h->Z1, (size_t)max_batch * N);
    if (!rc) rc = m_alloc(h, &h->H1, (size_t)max_batch * N);
    if (!rc) rc = m_alloc(h, &h->Z2, (size_t)max_batch * N);
    if (!rc) rc = m_alloc(h, &h->H2, (size_t)max_batch * N);
    if (!rc) rc = m_alloc(h, &h->dZ1, (size_t)max_batch * N);
    if (!rc) rc = m_alloc(h, &h->dZ2, (size_t)max_batch * N);
    if (!rc) rc = m_alloc(h, &h->y, (size_t)max_batch);
    if (!rc) rc = m_alloc(h, &h->dy, (size_t)max_batch);
    if (!rc) rc = m_alloc(h, &h->wpart, (size_t)WG_CHUNKS * (N + 1));
    if (!rc) rc = m_alloc(h, &h->loss, 1);
    if (!rc && cudaMemcpy(h->p, init.data(), sizeof(float) * init.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = QBVM_ERR_CUDA;
    if (!rc && (cudaMemset(h->m, 0, sizeof(float) * h->nparam) != cudaSuccess ||
                cudaMemset(h->v, 0, sizeof(float) * h->nparam) != cudaSuccess))
        rc = QBVM_ERR_CUDA;
    if (!rc) {
        k_to_bf16<<<nblk(h->nparam), MLP_THREADS>>>(h->p, h->pb, h->nparam);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = QBVM_ERR_CUDA;
    }
    if (rc) {
        for (void* q : h->allocs) cudaFree(q);
        delete h;
        return rc;
    }
    *out = h;
    return QBVM_OK;
}

long long qbvm_mlp_num_params(const qbvm_mlp_t* h) { return h ? h->nparam : -1; }

int qbvm_mlp_set_norm(qbvm_mlp_t* h, const float* mean, const float* sd) {
    if (!h || !mean || !sd) return QBVM_ERR_BAD_ARG;
    std::vector<float> is(h->in_dim);
    for (int k = 0; k < h->in_dim; ++k) is[k] = sd[k] > 0 ? 1.f / sd[k] : 1.f;
    if (cudaMemcpy(h->mu, mean, sizeof(float) * h->in_dim, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->inv_sd, is.data(), sizeof(float) * h->in_dim, cudaMemcpyHostToDevice) != cudaSuccess)
        return QBVM_ERR_CUDA;
    h->has_norm = true;
    return QBVM_OK;
}

int qbvm_mlp_get_params(const qbvm_mlp_t* h, float* params, float* adam_m, float* adam_v, long long* step) {
    if (!h) return QBVM_ERR_BAD_ARG;
    const size_t b = sizeof(float) * h->nparam;
    if (params && cudaMemcpy(params, h->p, b, cudaMemcpyDeviceToHost) != cudaSuccess) return QBVM_ERR_CUDA;
    if (adam_m && cudaMemcpy(adam_m, h->m, b, cudaMemcpyDeviceToHost) != cudaSuccess) return QBVM_ERR_CUDA;
    if (adam_v && cudaMemcpy(adam_v, h->v, b, cudaMemcpyDeviceToHost) != cudaSuccess) return QBVM_ERR_CUDA;
    if (step) *step = h->step;
    return QBVM_OK;
}

int qbvm_mlp_set_params(qbvm_mlp_t* h, const float* params, const float* adam_m, const float* adam_v, long long step) {
    if (!h || !params) return QBVM_ERR_BAD_ARG;
    const size_t b = sizeof(float) * h->nparam;
    if (cudaMemcpy(h->p, params, b, cudaMemcpyHostToDevice) != cudaSuccess) return QBVM_ERR_CUDA;
    if (adam_m && cudaMemcpy(h->m, adam_m, b, cudaMemcpyHostToDevice) != cudaSuccess) return QBVM_ERR_CUDA;
    if (adam_v && cudaMemcpy(h->v, adam_v, b, cudaMemcpyHostToDevice) != cudaSuccess) return QBVM_ERR_CUDA;
    h->step = step;
    k_to_bf16<<<nblk(h->nparam), MLP_THREADS>>>(h->p, h->pb, h->nparam);
    return cudaDeviceSynchronize() == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

int qbvm_mlp_forward(qbvm_mlp_t* h, const float* x, int B, float* y, void* stream) {
    if (!h || !x || !y || B < 1 || B > h->bmax) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int N = h->width;
    if (mlp_hidden_layers(h, x, B, s) != cudaSuccess) return QBVM_ERR_CUDA;
    k_dense_out<<<nblk((long long)B * 32), MLP_THREADS, 0, s>>>(h->H2, h->pb + h->ow3, h->p + h->ob3, B, N, y);
    return cudaGetLastError() == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

int qbvm_mlp_gradients(qbvm_mlp_t* h, const float* x, const float* t, int B, float* grads, double* loss_out,
                       void* stream) {
    if (!h || !x || !t || B < 1 || B > h->bmax) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = mlp_grads(h, x, t, B, s);
    if (rc) return rc;
    if (grads && cudaMemcpyAsync(grads, h->g, sizeof(float) * h->nparam, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (loss_out && cudaMemcpyAsync(loss_out, h->loss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

int qbvm_mlp_train_step(qbvm_mlp_t* h, const float* x, const float* t, int B, float lr, void* stream) {
    if (!h || !x || !t || B < 1 || B > h->bmax || !(lr > 0)) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = mlp_grads(h, x, t, B, s);
    if (rc) return rc;
    h->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)h->step), c2 = 1.f - std::pow(b2, (float)h->step);
    k_adam<<<nblk(h->nparam), MLP_THREADS, 0, s>>>(h->p, h->g, h->m, h->v, h->pb, h->nparam, lr, b1, b2, c1, c2, 1e-8f);
    return cudaGetLastError() == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

int qbvm_mlp_last_loss(qbvm_mlp_t* h, double* loss, void* stream) {
    if (!h || !loss) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return QBVM_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

int qbvm_mlp_destroy(qbvm_mlp_t* h) {
    if (!h) return QBVM_OK;
    for (void* q : h->allocs) cudaFree(q);
    delete h;
    return QBVM_OK;
}

// ------------------------------------------------------------------ features

int qbvm_features_plan(int m, double T, int nt, int max_batch, qbvm_features_t** out) {
    if (!out || m < 4 || m > 1024 || (m & (m - 1)) || max_batch < 1 || !(T > 0) || nt < 2) return QBVM_ERR_BAD_ARG;
    *out = nullptr;
    qbvm_features_t* f = new (std::nothrow) qbvm_features();
    if (!f) return QBVM_ERR_OOM;
    f->M = m;
    f->n = m - 1;
    f->lm = 0;
    while ((1 << f->lm) < m) ++f->lm;
    f->T = T;
    f->nt = nt;
    f->bmax = max_batch;
    f->Nx = (long long)f->n * f->n;
    std::vector<unsigned char> bin((size_t)f->Nx);
    std::vector<float> cnt(64, 0.f), inv(64, 0.f);
    const double rmax = std::sqrt(2.0) * (f->n + 1);
    for (int ky = 1; ky <= f->n; ++ky)
        for (int kx = 1; kx <= f->n; ++kx) {
            int b = (int)std::floor(64.0 * std::sqrt((double)kx * kx + (double)ky * ky) / rmax);
            b = b > 63 ? 63 : b;
            bin[(size_t)(ky - 1) * f->n + (kx - 1)] = (unsigned char)b;
            cnt[b] += 1.f;
        }
    for (int b = 0; b < 64; ++b) inv[b] = cnt[b] > 0 ? 1.f / cnt[b] : 0.f;
    std::vector<float2> tw(m);
    std::vector<float> sn(m / 2 + 2, 0.f);
    for (int i = 0; i < m; ++i) {
        double a = M_PI * (2.0 * i / m);
        tw[i] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    for (int j = 0; j <= m / 2; ++j) sn[j] = (float)std::sin(M_PI * j / m);
    int rc = m_alloc(f, &f->work, (size_t)max_batch * f->Nx);
    if (!rc) rc = m_alloc(f, &f->bin, (size_t)f->Nx);
    if (!rc) rc = m_alloc(f, &f->inv_count, 64);
    if (!rc) rc = m_alloc(f, &f->delta, (size_t)max_batch);
    if (!rc) rc = m_alloc(f, &f->tw, (size_t)m);
    if (!rc) rc = m_alloc(f, &f->sn, sn.size());
    if (!rc && (cudaMemcpy(f->bin, bin.data(), bin.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(f->inv_count, inv.data(), 64 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(f->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(f->sn, sn.data(), sn.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess))
        rc = QBVM_ERR_CUDA;
    if (rc) {
        for (void* q : f->allocs) cudaFree(q);
        delete f;
        return rc;
    }
    *out = f;
    return QBVM_OK;
}

int qbvm_features_run(qbvm_features_t* f, const double* g, const double* delta_host, int B, float* feats,
                      void* stream) {
    if (!f || !g || !delta_host || !feats || B < 1 || B > f->bmax) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = f->n;
    if (cudaMemcpyAsync(f->delta, delta_host, sizeof(double) * B, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    // g_b 2^k_b in FP32, then the unnormalised DST-I along x then y of every instance
    {
        const long long total = (long long)B * f->Nx;
        const unsigned blocks = (unsigned)std::min<long long>((total + MLP_THREADS - 1) / MLP_THREADS, 152LL * 16);
        k_scaled_to_f32<<<blocks, MLP_THREADS, 0, s>>>(g, f->Nx, B, f->delta, f->work);
        if (cudaGetLastError() != cudaSuccess) return QBVM_ERR_CUDA;
    }
    if (qbvm::launch_dst<float, float, 0>(f->work, f->work, f->n, f->lm, (long long)B * n, 1, f->tw, f->sn, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (qbvm::launch_dst<float, float, 0>(f->work, f->work, f->n, f->lm, (long long)B, n, f->tw, f->sn, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    const float scale = (float)((2.0 / f->M) * (2.0 / f->M));       // DST coefficient -> sine-series coefficient
    k_spectrum_bins<<<B, MLP_THREADS, 0, s>>>(f->work, f->Nx, f->bin, f->inv_count, scale * scale, f->delta,
                                              (float)f->T, (float)std::log2((double)f->nt), 67, feats);
    return cudaGetLastError() == cudaSuccess ? QBVM_OK : QBVM_ERR_CUDA;
}

int qbvm_features_destroy(qbvm_features_t* f) {
    if (!f) return QBVM_OK;
    for (void* q : f->allocs) cudaFree(q);
    delete f;
    return QBVM_OK;
}

}  // extern "C"
