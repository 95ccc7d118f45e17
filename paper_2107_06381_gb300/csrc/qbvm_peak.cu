// qbvm_peak.cu -- qbvm_measure_peak: the fused multiply-add throughput of the
// current GPU, measured, as the ALU roofline of the solver's kernels.
//
// The FP64 transforms of the solve are bound by the FP64 pipe, not by HBM, on
// a part whose FP64 rate is a small fraction of its FP32 rate; the roofline
// they are rated against is therefore this GPU's own sustained FP64 FMA rate,
// taken the way a copy kernel measures the HBM peak: a kernel that does
// nothing but independent FMA chains on every SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "qbvm.h"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_BLOCKS_PER_SM = 4;       // 32 warps per SM
constexpr int PEAK_CHAINS = 8;              // independent FMA chains per thread

__device__ double g_peak_sink;

// a <- a * b + c on PEAK_CHAINS independent accumulators, `iters` times.
// |b| < 1 keeps every chain bounded (it converges to c / (1 - b)), so no
// overflow or subnormal slows the pipe.  The sum is stored only when it
// equals `never`, which the host picks so that it cannot happen; the compiler
// cannot know that and keeps every FMA.
template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(long long iters, T b, T c, T never) {
    T a[PEAK_CHAINS];
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (long long it = 0; it < iters; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int i = 0; i < PEAK_CHAINS; ++i) a[i] = fma(a[i], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < PEAK_CHAINS; ++i) s += a[i];
    if (s == never) g_peak_sink = (double)s;
}

template <typename T>
int measure(long long iters, double* out, cudaStream_t s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    const unsigned grid = (unsigned)(sms * PEAK_BLOCKS_PER_SM);
    const double fmas = (double)grid * PEAK_THREADS * PEAK_CHAINS * (double)iters;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return QBVM_ERR_CUDA;
    }
    int rc = QBVM_OK;
    double best = 0.0;
    const T b = (T)0.999, c = (T)1e-3, never = (T)-12345.678;
    for (int rep = 0; rep < 6 && rc == QBVM_OK; ++rep) {       // one warm-up, then the best of five
        cudaEventRecord(e0, s);
        k_fma_peak<T><<<grid, PEAK_THREADS, 0, s>>>(iters, b, c, never);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = QBVM_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
            rc = QBVM_ERR_CUDA;
            break;
        }
        const double rate = fmas / (ms * 1e-3);
        if (rep > 0 && rate > best) best = rate;
    }
    if (rc) cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == QBVM_OK) *out = best;
    return rc;
}

}  // namespace

extern "C" int qbvm_measure_peak(int kind, double* fma_per_s_out, void* stream) {
    if (!fma_per_s_out) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // iteration counts sized for a few milliseconds per launch on a GB300
    // (about 0.6 T FP64 and 40 T FP32 FMA/s)
    if (kind == QBVM_PEAK_FP64_FMA) return measure<double>(2048, fma_per_s_out, s);
    if (kind == QBVM_PEAK_FP32_FMA) return measure<float>(131072, fma_per_s_out, s);
    return QBVM_ERR_BAD_ARG;
}
