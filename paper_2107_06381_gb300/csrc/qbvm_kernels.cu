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
#include "qbvm_dst.cuh"
#include "qbvm_dstgen.cuh"
#include "qbvm_fft.cuh"
#include "qbvm_df.cuh"
#include "qbvm_regdst.cuh"
#include "qbvm_timesolve.cuh"
#include "qbvm_internal.h"

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>
#include <type_traits>

namespace qbvm {

// Raise a kernel's dynamic shared-memory limit and prefer the largest
// shared-memory carve-out.  The attribute calls are driver calls, so they are
// made once per (device, kernel) and whenever a launch needs more than the
// limit set so far; launches of small problems are otherwise host-bound.
struct SmemSet {
    int dev;
    const void* fn;
    size_t bytes;
};
static std::mutex g_smem_mu;
static std::vector<SmemSet> g_smem_set;

template <typename K>
static cudaError_t set_smem(K kern, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
    const void* fn = reinterpret_cast<const void*>(kern);
    {
        std::lock_guard<std::mutex> lk(g_smem_mu);
        for (const SmemSet& r : g_smem_set)
            if (r.dev == dev && r.fn == fn && r.bytes >= smem) return cudaSuccess;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_smem_mu);
    for (SmemSet& r : g_smem_set)
        if (r.dev == dev && r.fn == fn) {
            r.bytes = std::max(r.bytes, smem);
            return cudaSuccess;
        }
    g_smem_set.push_back({dev, fn, smem});
    return cudaSuccess;
}

static int device_sms();

// Launch with programmatic stream serialisation (see pdl_wait) when the grid
// is small -- at most two CTAs per SM, as in the latency-bound chains of the
// y^0-only solve or of small grids, where the successor's launch and table
// loads then overlap the predecessor's tail (y^0-only on 255^2: 53 -> 42 us).
// Larger grids launch the ordinary way: with the attribute the 3D refined
// solve (127^3 x 128) measured 20.7 ms against 18.8 ms without.  Only kernels
// that call pdl_wait before touching a predecessor's data come through here
// (for the others the attribute would not be safe; for these, pdl_wait is a
// no-op in an ordinary launch).
template <typename... P, typename... A>
static cudaError_t launch_pdl(void (*kern)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              A... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    const int sms = device_sms();
    cfg.numAttrs = (sms > 0 && grid <= 2u * (unsigned)sms) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

#define QBVM_PDL(...)                                   \
    do {                                                \
        cudaError_t le__ = launch_pdl(__VA_ARGS__);     \
        if (le__ != cudaSuccess) return le__;           \
    } while (0)

// SMs of the current device, queried once per device.
static int device_sms() {
    static std::mutex mu;
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (sms[dev] == 0 && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms[dev] = 0;
    }
    return sms[dev];
}

template <typename R, typename TIN, int OMODE, int MAXB4, bool X4>
__global__ void __launch_bounds__(TILE_THREADS)
k_dst(const TIN* in, void* out, int n, int lm, int lw, long long outer, long long inner,
      const cplx<R>* __restrict__ tw, const R* __restrict__ sn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dst_tile<R, TIN, OMODE, MAXB4, false, X4, true>(in, out, n, lm, lw, outer, inner, (long long)blockIdx.x, tw,
                                                    sn, smem_raw);
}

// The same tile with the transform length fixed at compile time (the tile
// width follows from it), so that the whole pipeline inlines with constant
// sizes; used for the common lengths M = 64 ... 512.
template <typename R, typename TIN, int OMODE, int LM, bool X4>
__global__ void __launch_bounds__(TILE_THREADS)
k_dst_ct(const TIN* in, void* out, long long outer, long long inner, const cplx<R>* __restrict__ tw,
         const R* __restrict__ sn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LW = 11 - LM;                     // 2^LM * 2^LW = DST_TILE complex values
    static_assert((1 << (LM + LW)) == DST_TILE, "DST tile size");
    dst_tile<R, TIN, OMODE, DST_TILE / 4 / TILE_THREADS, false, X4, true>(in, out, (1 << LM) - 1, LM, LW, outer, inner,
                                                                    (long long)blockIdx.x, tw, sn, smem_raw);
}

template <typename R, typename TIN, int OMODE, int LM, bool X4>
static cudaError_t launch_dst_ct(const TIN* in, void* out, long long outer, long long inner, const void* tw,
                                 const void* sn, long long blocks, size_t smem, cudaStream_t s) {
    auto kern = k_dst_ct<R, TIN, OMODE, LM, X4>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    QBVM_PDL(kern, (unsigned)blocks, TILE_THREADS, smem, s, in, out, outer, inner, reinterpret_cast<const cplx<R>*>(tw),
                                                      reinterpret_cast<const R*>(sn));
    return cudaGetLastError();
}

// FP32 DST with the transform in registers (rd::tile), M = 64, 128, 256.
// Minimum CTAs per SM: shared memory admits 5 (M = 256) / 10 (M = 128) CTAs;
// the y/z passes fit that in 48 registers without spills, the x passes keep
// 64 (measured: the x pass slows down when squeezed to 48).
template <typename TIN, int OMODE, int LM, bool XAX>
__global__ void __launch_bounds__(rd::threads<LM>(), LM == 8 ? (XAX ? 4 : 5) : LM == 7 ? (XAX ? 8 : 10) : (XAX ? 9 : 12))
k_dst_reg(const TIN* in, void* out, long long outer, long long inner, const float2* __restrict__ tw,
          const float* __restrict__ sn) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    rd::tile<TIN, OMODE, LM, XAX>(in, out, outer, inner, (long long)blockIdx.x, tw, sn, smem_raw);
}

template <typename TIN, int OMODE, int LM, bool XAX>
static cudaError_t launch_dst_reg(const TIN* in, void* out, long long outer, long long inner, const void* tw,
                                  const void* sn, cudaStream_t s) {
    auto kern = k_dst_reg<TIN, OMODE, LM, XAX>;
    constexpr size_t smem = rd::smem_bytes<LM, XAX>();
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const long long blocks = XAX ? (outer + rd::NCOL - 1) / rd::NCOL : outer * ((inner + rd::NCOL - 1) / rd::NCOL);
    QBVM_PDL(kern, (unsigned)blocks, rd::threads<LM>(), smem, s, in, out, outer, inner,
                                                           reinterpret_cast<const float2*>(tw),
                                                           reinterpret_cast<const float*>(sn));
    return cudaGetLastError();
}

template <typename TIN, int OMODE>
static cudaError_t launch_dst_reg_any(const TIN* in, void* out, int lm, long long outer, long long inner,
                                      const void* tw, const void* sn, cudaStream_t s) {
    const bool x = inner == 1;
    switch (lm) {
        case 6: return x ? launch_dst_reg<TIN, OMODE, 6, true>(in, out, outer, inner, tw, sn, s)
                         : launch_dst_reg<TIN, OMODE, 6, false>(in, out, outer, inner, tw, sn, s);
        case 7: return x ? launch_dst_reg<TIN, OMODE, 7, true>(in, out, outer, inner, tw, sn, s)
                         : launch_dst_reg<TIN, OMODE, 7, false>(in, out, outer, inner, tw, sn, s);
        default: return x ? launch_dst_reg<TIN, OMODE, 8, true>(in, out, outer, inner, tw, sn, s)
                          : launch_dst_reg<TIN, OMODE, 8, false>(in, out, outer, inner, tw, sn, s);
    }
}

// DST-I of any length n = M - 1 (mixed-radix transform, qbvm_dstgen.cuh).
template <typename R, typename TIN, int OMODE, bool X4>
__global__ void __launch_bounds__(TILE_THREADS)
k_dst_gen(const TIN* in, void* out, int M, int lw, long long outer, long long inner,
          const cplx<R>* __restrict__ tw, const R* __restrict__ sn, FftGenPlan fp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dstgen_tile<R, TIN, OMODE, X4>(in, out, M, lw, outer, inner, (long long)blockIdx.x, tw, sn, fp, smem_raw);
}

template <typename R, typename TIN, int OMODE, bool X4>
static cudaError_t launch_dst_gen(const TIN* in, void* out, int M, long long outer, long long inner,
                                  const void* tw, const void* sn, cudaStream_t s) {
    FftGenPlan fp;
    if (M < 2 || !fftgen_factor(M, &fp)) return cudaErrorInvalidValue;
    int lw = dstgen_lw(M);
    auto nblocks = [&](int l) {
        const long long W2 = 2LL << l;
        return inner == 1 ? (outer + W2 - 1) / W2 : outer * ((inner + W2 - 1) / W2);
    };
    // as for the power-of-two tiles: few tiles spread over at least two per SM
    const int sms = device_sms();
    while (sms > 0 && lw > 0 && nblocks(lw) < 2LL * sms) --lw;
    const size_t smem = dstgen_smem<R>(M, lw);
    auto kern = k_dst_gen<R, TIN, OMODE, X4>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    QBVM_PDL(kern, (unsigned)nblocks(lw), TILE_THREADS, smem, s, in, out, M, lw, outer, inner,
                                                   reinterpret_cast<const cplx<R>*>(tw),
                                                   reinterpret_cast<const R*>(sn), fp);
    return cudaGetLastError();
}

template <typename R>
size_t dst_smem_bytes(int lm) { return dst_smem<R>(lm); }
template size_t dst_smem_bytes<double>(int);
template size_t dst_smem_bytes<float>(int);
int dst_tile_lw(int lm) { return dst_lw(lm); }

template <typename R, typename TIN, int OMODE, bool X4>
cudaError_t launch_dst(const TIN* in, void* out, int n, int lm, long long outer, long long inner,
                       const void* tw, const void* sn, cudaStream_t s) {
    // lengths the power-of-two tiles do not take: the mixed-radix tile
    if (n + 1 != (1 << lm) || lm < 2 || lm > 10) return launch_dst_gen<R, TIN, OMODE, X4>(in, out, n + 1, outer, inner, tw, sn, s);
    const int lw0 = dst_lw(lm);
    auto nblocks = [&](int l) {
        const long long W2 = 2LL << l;               // real columns per tile
        return inner == 1 ? (outer + W2 - 1) / W2 : outer * ((inner + W2 - 1) / W2);
    };
    int lw = lw0;
    if (std::is_same<R, double>::value) {
        // Few tiles (one or a few levels, e.g. the y^0-only solve): an FP64 tile
        // is ~15 us of FP64-pipe work on its SM, so narrower tiles spread the
        // pass over at least two per SM.  Column pairs and prefix-sum segments
        // are those of the full-width tiles, so the results are bitwise the same.
        const int sms = device_sms();
        while (sms > 0 && lw > 0 && nblocks(lw) < 2LL * sms) --lw;
    }
    const long long blocks = nblocks(lw);
    size_t smem = dst_smem<R>(lm, lw);
    if (std::is_same<R, float>::value && !X4 && n == (1 << lm) - 1 && lm >= 6 && lm <= 8)
        return launch_dst_reg_any<TIN, OMODE>(in, out, lm, outer, inner, tw, sn, s);
    if (n == (1 << lm) - 1 && lw == lw0) {
        switch (lm) {
            case 6: return launch_dst_ct<R, TIN, OMODE, 6, X4>(in, out, outer, inner, tw, sn, blocks, smem, s);
            case 7: return launch_dst_ct<R, TIN, OMODE, 7, X4>(in, out, outer, inner, tw, sn, blocks, smem, s);
            case 8: return launch_dst_ct<R, TIN, OMODE, 8, X4>(in, out, outer, inner, tw, sn, blocks, smem, s);
            case 9: return launch_dst_ct<R, TIN, OMODE, 9, X4>(in, out, outer, inner, tw, sn, blocks, smem, s);
            default: break;
        }
    }
    auto kern = k_dst<R, TIN, OMODE, DST_TILE / 4 / TILE_THREADS, X4>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    QBVM_PDL(kern, (unsigned)blocks, TILE_THREADS, smem, s, in, out, n, lm, lw, outer, inner,
                                                      reinterpret_cast<const cplx<R>*>(tw),
                                                      reinterpret_cast<const R*>(sn));
    return cudaGetLastError();
}

#define QBVM_DST_INST(R, TIN, OM, X4)                                                                   \
    template cudaError_t launch_dst<R, TIN, OM, X4>(const TIN*, void*, int, int, long long, long long, \
                                                    const void*, const void*, cudaStream_t);
QBVM_DST_INST(double, double, 0, true)
QBVM_DST_INST(float, float, 0, false)
QBVM_DST_INST(float, double, 0, false)
QBVM_DST_INST(float, float, 1, false)
QBVM_DST_INST(float, float, 2, false)
#undef QBVM_DST_INST

template <typename R, int MAXB4>
__global__ void __launch_bounds__(TILE_THREADS)
k_time_solve(const R* in, R* out, long long Nx, int lh, int lw, const cplx<R>* __restrict__ tw,
             const cplx<R>* __restrict__ gpow, const cplx<R>* __restrict__ gipw,
             const cplx<R>* __restrict__ ak, const R* __restrict__ lamtau, R cnorm,
             const cplx<R>* __restrict__ gpowr, const cplx<R>* __restrict__ gipr, const cplx<R>* __restrict__ qinv,
             int delta_rhs, int n0_only) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    time_solve_tile<R, MAXB4>(in, out, Nx, lh, lw, tw, gpow, gipw, ak, lamtau, cnorm, gpowr, gipr, qinv, delta_rhs,
                              n0_only, (long long)blockIdx.x, smem_raw);
}

// Compile-time half length LH and tile width LW (H * W = 4 * MAXB4 * TILE_THREADS).
template <typename R, int MAXB4, int LH>
__global__ void __launch_bounds__(TILE_THREADS)
k_time_solve_ct(const R* in, R* out, long long Nx, const cplx<R>* __restrict__ tw,
                const cplx<R>* __restrict__ gpow, const cplx<R>* __restrict__ gipw,
                const cplx<R>* __restrict__ ak, const R* __restrict__ lamtau, R cnorm,
                const cplx<R>* __restrict__ gpowr, const cplx<R>* __restrict__ gipr,
                const cplx<R>* __restrict__ qinv, int delta_rhs, int n0_only) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LT = (MAXB4 == 4 ? 12 : MAXB4 == 2 ? 11 : 10);     // log2 of the tile size
    time_solve_tile<R, MAXB4>(in, out, Nx, LH, LT - LH, tw, gpow, gipw, ak, lamtau, cnorm, gpowr, gipr, qinv,
                              delta_rhs, n0_only, (long long)blockIdx.x, smem_raw);
}

// The FP64 time solve of `count` instances of one shape stored back to back
// (instance b reads in + b in_stride and writes out + b out_stride), each with
// its own omega: gpow, gipw, gpowr, gipr are [count][H] and qinv [count][H][Nx].
// Block = b * tiles + mode tile.  The tile is W = 2^lw modes wide (at most
// the single-instance width, fewer when Nx is small); LH < 0: lh is taken at
// run time.
template <int MAXB4, int LH>
__global__ void __launch_bounds__(TILE_THREADS, 3)
k_time_solve_batched(const double* in, double* out, long long Nx, int lh, int lw, long long tiles,
                     long long in_stride, long long out_stride, const double2* __restrict__ tw,
                     const double2* __restrict__ gpow, const double2* __restrict__ gipw,
                     const double2* __restrict__ gpowr, const double2* __restrict__ gipr,
                     const double2* __restrict__ qinv, int delta_rhs, int n0_only) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int h = LH >= 0 ? LH : lh, w = lw;
    const long long b = (long long)blockIdx.x / tiles, tile = (long long)blockIdx.x - b * tiles;
    const long long H = 1LL << h;
    time_solve_tile<double, MAXB4>(in + b * in_stride, out + b * out_stride, Nx, h, w, tw, gpow + b * H,
                                   gipw + b * H, nullptr, nullptr, 0.0, gpowr + b * H, gipr + b * H,
                                   qinv + b * H * Nx, delta_rhs, n0_only, tile, smem_raw);
}

// FP32 time solve with the transforms in registers, H = nt/2 = 32 ... 256.
// The same three steps as time_solve_tile, per spatial mode l, with the
// length-H DFT split as N1 x N2 (n = N2 n1 + n2, k = k1 + N1 k2): thread n2 of
// the T = N2 threads of mode l does the length-N1 DFT over n1 of its time
// indices, the padded shared-memory transpose hands each thread the k1 rows it
// owns, and the length-N2 DFTs give it the frequencies k1 + N1 k2.  After the
// divide the inverse runs in mirror order (length-N2 DFTs over k2, twiddle,
// transpose back, length-N1 DFTs over k1), which leaves each thread holding
// exactly the time indices it loaded.  A CTA takes TS_MODES consecutive modes:
// the [nt][TS_MODES] tile is staged through shared memory with coalesced row
// accesses (row stride RS chosen so that the threads' strided time reads are
// bank-conflict free), and each mode's column is read and rewritten only by
// its own threads.  With the delta right-hand side the forward transform of
// f^0 e_0 is the constant f^0 and is not computed.
template <int LH> struct TsCfg;
// TS_MODES spatial modes per CTA: 32 (128-byte row segments in the load and
// store phases) up to H = 64, where it measured 9 % faster on 127^3 x 128 than
// 16; 16 for H = 128, 256, where 32 measured 3 % slower on 255^2 x 256.
template <> struct TsCfg<8> { static constexpr int N1 = 16, N2 = 16, BS = 17, FB = 272, RS = 18, TS_MODES = 16; };
template <> struct TsCfg<7> { static constexpr int N1 = 16, N2 = 8, BS = 9, FB = 152, RS = 20, TS_MODES = 16; };
template <> struct TsCfg<6> { static constexpr int N1 = 8, N2 = 8, BS = 9, FB = 72, RS = 36, TS_MODES = 32; };
template <> struct TsCfg<5> { static constexpr int N1 = 8, N2 = 4, BS = 5, FB = 52, RS = 40, TS_MODES = 32; };

// The staging tile [nt][RS] and the per-mode transpose buffers share one
// region: the tile is free between the first reads and the final writes.
template <int LH>
constexpr size_t ts_region_bytes() {
    return (size_t)(2 << LH) * TsCfg<LH>::RS * sizeof(float) > (size_t)TsCfg<LH>::TS_MODES * TsCfg<LH>::FB * sizeof(float2)
               ? (size_t)(2 << LH) * TsCfg<LH>::RS * sizeof(float)
               : (size_t)TsCfg<LH>::TS_MODES * TsCfg<LH>::FB * sizeof(float2);
}
template <int LH>
constexpr size_t ts_reg_smem() { return (size_t)4 * (1 << LH) * sizeof(float2) + ts_region_bytes<LH>(); }

// Minimum CTAs per SM: 64 registers for H = 256 / 128 (from 80: 24 -> 32
// resident warps, 4 % faster at H = 128), 48 below.
template <int LH>
__device__ __forceinline__ void time_solve_reg_tile(const float* in, float* out, long long Nx,
                                                    const float2* __restrict__ tw, const float2* __restrict__ gpow,
                                                    const float2* __restrict__ gipw, const float2* __restrict__ ak,
                                                    const float* __restrict__ lamtau, float cnorm, float rho_h,
                                                    float rho_hinv, int delta_rhs, int n0_only, long long tile) {
    using G = TsCfg<LH>;
    constexpr int H = 1 << LH, NT = 2 * H, N1 = G::N1, N2 = G::N2, T = N2, NTH = TsCfg<LH>::TS_MODES * T, Q = N1 / T;
    constexpr int RS = G::RS, RSTEP = NTH / TsCfg<LH>::TS_MODES;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* stw = reinterpret_cast<float2*>(smem_raw);
    float2* sgp = stw + H;
    float2* sgi = sgp + H;
    float2* sak = sgi + H;
    float2* fbuf = sak + H;                                            // transpose buffers ...
    float* st = reinterpret_cast<float*>(fbuf);                        // ... aliasing the tile [NT][RS]
    const int tid = threadIdx.x;
    pdl_trigger();
    for (int i = tid; i < H; i += NTH) {
        stw[i] = tw[i];
        sgp[i] = gpow[i];
        sgi[i] = gipw[i];
        sak[i] = ak[i];
    }
    pdl_wait();                                                        // the input is a predecessor's output
    const long long l0 = tile * TsCfg<LH>::TS_MODES;
    {   // load phase: rows of TS_MODES consecutive modes, a batch of loads in flight per thread
        const int cc = tid % TsCfg<LH>::TS_MODES, r0 = tid / TsCfg<LH>::TS_MODES;
        const bool ok = l0 + cc < Nx;
        const float* src = in + l0 + cc;
        const int rows = delta_rhs ? 1 : NT;
        constexpr int BATCH = 16;
        for (int rb = r0; rb < rows; rb += RSTEP * BATCH) {
            float v[BATCH];
#pragma unroll
            for (int q = 0; q < BATCH; ++q) {
                const int r = rb + q * RSTEP;
                v[q] = (ok && r < rows) ? src[(long long)r * Nx] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < BATCH; ++q) {
                const int r = rb + q * RSTEP;
                if (r < rows) st[r * RS + cc] = v[q];
            }
        }
    }
    __syncthreads();
    const int c = tid / T, n2 = tid % T;
    const long long l = l0 + c;
    const bool ok = l < Nx;
    float2* buf = fbuf + c * G::FB;
    float2 X[Q][N2];
    float2 v[N1];
    if (delta_rhs) {
        const float f0 = st[c];
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) X[q][k2] = make_float2(f0, 0.f);
    } else {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {                  // gamma^t (f_t + i rho^H f_{t+H})
            const int n = N2 * n1 + n2;
            const float2 g = sgp[n];
            const float fa = st[n * RS + c], f1 = rho_h * st[(n + H) * RS + c];
            v[n1] = make_float2(fmaf(g.x, fa, -g.y * f1), fmaf(g.y, fa, g.x * f1));
        }
    }
    __syncthreads();                                       // every column read: the tile becomes the buffers
    if (!delta_rhs) {
        rd::rdft<N1, +1>(v);
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1)
            if (n2) v[k1] = cmulc(v[k1], stw[n2 * k1]);    // exp(+2 pi i n2 k1 / H)
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
    }
    // Step (b): divide by d_{2k} + tau Lambda_l
    const float lt = ok ? lamtau[l] : 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k1 = n2 + T * q;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const float2 a = sak[k1 + N1 * k2];
            const float zr = a.x + lt, zi = a.y;
            // |d + tau Lambda|^2 lies far inside the fast division's range (2 ulp):
            // this FP32 solve is the refinement's correction step
            const float inv = __fdividef(cnorm, fmaf(zr, zr, zi * zi));
            const float2 u = X[q][k2];
            X[q][k2] = make_float2(fmaf(u.x, zr, u.y * zi) * inv, fmaf(u.y, zr, -u.x * zi) * inv);
        }
    }
    // Step (c): inverse DFT in mirror order
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k1 = n2 + T * q;
        rd::rdft<N2, -1>(X[q]);
#pragma unroll
        for (int j = 1; j < N2; ++j)
            if (k1) X[q][j] = cmul(X[q][j], stw[j * k1]);  // exp(-2 pi i j k1 / H)
    }
    __syncwarp();
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
    __syncthreads();                                       // every buffer read: the region is the tile again
    rd::rdft<N1, -1>(w);
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {                      // outputs into this mode's own column
        const int n = N2 * n1 + n2;
        const float2 gi = sgi[n], qv = w[n1];
        st[n * RS + c] = fmaf(gi.x, qv.x, -gi.y * qv.y);
        st[(n + H) * RS + c] = rho_hinv * fmaf(gi.x, qv.y, gi.y * qv.x);
    }
    __syncthreads();
    {   // store phase
        const int cc = tid % TsCfg<LH>::TS_MODES, r0 = tid / TsCfg<LH>::TS_MODES;
        if (l0 + cc < Nx) {
            float* dst = out + l0 + cc;
            const int rows = n0_only ? 1 : NT;
            for (int r = r0; r < rows; r += RSTEP) dst[(long long)r * Nx] = st[r * RS + cc];
        }
    }
}

template <int LH>
__global__ void __launch_bounds__(TsCfg<LH>::TS_MODES * TsCfg<LH>::N2, LH == 8 ? 4 : LH == 7 ? 8 : LH == 6 ? 5 : 10)
k_time_solve_reg(const float* in, float* out, long long Nx, const float2* __restrict__ tw,
                 const float2* __restrict__ gpow, const float2* __restrict__ gipw, const float2* __restrict__ ak,
                 const float* __restrict__ lamtau, float cnorm, float rho_h, float rho_hinv, int delta_rhs,
                 int n0_only) {
    time_solve_reg_tile<LH>(in, out, Nx, tw, gpow, gipw, ak, lamtau, cnorm, rho_h, rho_hinv, delta_rhs, n0_only,
                            (long long)blockIdx.x);
}

// The same solve for `count` instances of one shape stored back to back, each
// with its own omega: block = b * tiles + mode tile; instance b reads
// in + b in_stride, writes out + b out_stride and takes the rows b of the
// [count][H] tables gpow, gipw, ak and of cnorm, rho_h, rho_hinv.
template <int LH>
__global__ void __launch_bounds__(TsCfg<LH>::TS_MODES * TsCfg<LH>::N2, LH == 8 ? 4 : LH == 7 ? 8 : LH == 6 ? 5 : 10)
k_time_solve_reg_batched(const float* in, float* out, long long Nx, long long tiles, long long in_stride,
                         long long out_stride, const float2* __restrict__ tw, const float2* __restrict__ gpow,
                         const float2* __restrict__ gipw, const float2* __restrict__ ak,
                         const float* __restrict__ lamtau, const float* __restrict__ cnorm,
                         const float* __restrict__ rho_h, const float* __restrict__ rho_hinv, int delta_rhs,
                         int n0_only) {
    const long long b = (long long)blockIdx.x / tiles, tile = (long long)blockIdx.x - b * tiles;
    constexpr int H = 1 << LH;
    time_solve_reg_tile<LH>(in + b * in_stride, out + b * out_stride, Nx, tw, gpow + b * H, gipw + b * H,
                            ak + b * H, lamtau, cnorm[b], rho_h[b], rho_hinv[b], delta_rhs, n0_only, tile);
}

template <int LH>
static cudaError_t launch_time_solve_reg(const float* in, float* out, const Tables& tb, float cnorm, int delta_rhs,
                                         int n0_only, cudaStream_t s) {
    auto kern = k_time_solve_reg<LH>;
    constexpr size_t smem = ts_reg_smem<LH>();
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (tb.Nx + TsCfg<LH>::TS_MODES - 1) / TsCfg<LH>::TS_MODES;
    QBVM_PDL(kern, (unsigned)blocks, TsCfg<LH>::TS_MODES * TsCfg<LH>::N2, smem, s, 
        in, out, tb.Nx, reinterpret_cast<const float2*>(tb.tw_t32), reinterpret_cast<const float2*>(tb.gpow32),
        reinterpret_cast<const float2*>(tb.gipw32), reinterpret_cast<const float2*>(tb.ak32),
        reinterpret_cast<const float*>(tb.lamtau32), cnorm, (float)tb.rho_h, (float)tb.rho_hinv, delta_rhs, n0_only);
    return cudaGetLastError();
}

__global__ void k_make_qinv(const double2* __restrict__ ak, const double* __restrict__ lamtau, double cnorm, int H,
                            long long Nx, double2* __restrict__ q) {
    const long long n = (long long)H * Nx;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / Nx, l = i - k * Nx;
        const double zr = ak[k].x + lamtau[l], zi = ak[k].y;
        const double inv = cnorm / (zr * zr + zi * zi);
        q[i] = make_double2(zr * inv, -zi * inv);
    }
}

cudaError_t launch_make_qinv(const Tables& tb, double cnorm, double2* q, cudaStream_t s) {
    const long long n = (long long)(tb.nt / 2) * tb.Nx;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_make_qinv<<<(unsigned)blocks, 256, 0, s>>>(tb.ak, tb.lamtau, cnorm, tb.nt / 2, tb.Nx, q);
    return cudaGetLastError();
}

__global__ void k_y0fac_pow2(const double2* __restrict__ q, int H, long long Nx, double* __restrict__ out) {
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < Nx; l += (long long)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int m = 0; m < H; ++m) a += q[(long long)m * Nx + l].x;
        out[l] = 2.0 * a;                                // the odd frequencies are the conjugates
    }
}

__global__ void k_y0fac_gen(const double2* __restrict__ dk, const double* __restrict__ lamtau, double cnorm, int P,
                            long long Nx, double* __restrict__ out) {
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < Nx; l += (long long)gridDim.x * blockDim.x) {
        double a = 0.0;
        const double lt = lamtau[l];
        for (int k = 0; k < P; ++k) {
            const double zr = dk[k].x + lt, zi = dk[k].y;
            a += cnorm * zr / (zr * zr + zi * zi);
        }
        out[l] = a;
    }
}

__global__ void k_mul_modes(const double* __restrict__ x, const double* __restrict__ fac, double* __restrict__ y,
                            long long n) {
    pdl_trigger();
    pdl_wait();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fac[i] * x[i];
}

cudaError_t launch_make_y0fac(const Tables& tb, double cnorm, double* out, cudaStream_t s) {
    long long blocks = (tb.Nx + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (tb.gen) k_y0fac_gen<<<(unsigned)blocks, 256, 0, s>>>(tb.dk_full, tb.lamtau, cnorm, tb.nt, tb.Nx, out);
    else k_y0fac_pow2<<<(unsigned)blocks, 256, 0, s>>>(tb.qinv, tb.nt / 2, tb.Nx, out);
    return cudaGetLastError();
}

cudaError_t launch_mul_modes(const double* x, const double* fac, double* y, long long n, cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    QBVM_PDL(k_mul_modes, (unsigned)blocks, 256, 0, s, x, fac, y, n);
    return cudaGetLastError();
}

static int tile_lw(int lp, int tile = TILE_ELEMS) {
    int lw = 0;
    while (((1 << lp) << (lw + 1)) <= tile) ++lw;
    return lw;
}

// FP64 tiles hold 4096 complex values (the FP64 pipe is the limit); FP32
// tiles 2048, which halves the registers and doubles the CTAs per SM that
// hide global-memory latency.
template <typename R>
constexpr int time_tile_maxb4() { return std::is_same<R, double>::value ? 4 : 2; }

template <typename R>
cudaError_t launch_time_solve(const R* in, R* out, const Tables& tb, double cnorm, int delta_rhs,
                              int n0_only, cudaStream_t s) {
    constexpr int MB = time_tile_maxb4<R>();
    constexpr int TILE = 4 * MB * TILE_THREADS;
    const int lh = tb.lnt - 1, H = 1 << lh;
    const int lw0 = tile_lw(lh, TILE);
    int lw = lw0;
    {
        // few modes (small grids): narrower tiles spread the FP64 work over more
        // SMs; every mode's transforms are the same arithmetic at any width
        const int sms = device_sms();
        while (sms > 0 && lw > 0 && (tb.Nx + (1LL << lw) - 1) >> lw < 2LL * sms) --lw;
    }
    const int W = 1 << lw;
    long long blocks = (tb.Nx + W - 1) / W;
    size_t smem = sizeof(cplx<R>) * ((size_t)H * W + H);
    const bool f64 = std::is_same<R, double>::value;
    auto pick = [f64](const void* a, const void* b) { return reinterpret_cast<const cplx<R>*>(f64 ? a : b); };
    const R* lt = reinterpret_cast<const R*>(f64 ? (const void*)tb.lamtau : (const void*)tb.lamtau32);
    const cplx<R>* qv = f64 ? reinterpret_cast<const cplx<R>*>(tb.qinv) : nullptr;
    if (std::is_same<R, float>::value) {
        const float* fin = reinterpret_cast<const float*>(in);
        float* fout = reinterpret_cast<float*>(out);
        switch (lh) {
            case 5: return launch_time_solve_reg<5>(fin, fout, tb, (float)cnorm, delta_rhs, n0_only, s);
            case 6: return launch_time_solve_reg<6>(fin, fout, tb, (float)cnorm, delta_rhs, n0_only, s);
            case 7: return launch_time_solve_reg<7>(fin, fout, tb, (float)cnorm, delta_rhs, n0_only, s);
            case 8: return launch_time_solve_reg<8>(fin, fout, tb, (float)cnorm, delta_rhs, n0_only, s);
            default: break;
        }
    }
#define QBVM_TS_CT(LHV)                                                                                        \
    case LHV: {                                                                                                \
        auto kern = k_time_solve_ct<R, MB, LHV>;                                                               \
        cudaError_t e = set_smem(kern, smem);                                                                  \
        if (e != cudaSuccess) return e;                                                                        \
        QBVM_PDL(kern, (unsigned)blocks, TILE_THREADS, smem, s, in, out, tb.Nx, pick(tb.tw_t, tb.tw_t32),            \
                                                          pick(tb.gpow, tb.gpow32), pick(tb.gipw, tb.gipw32),  \
                                                          pick(tb.ak, tb.ak32), lt, R(cnorm),                  \
                                                          pick(tb.gpowr, tb.gpowr32), pick(tb.gipr, tb.gipr32), \
                                                          qv, delta_rhs, n0_only);                             \
        return cudaGetLastError();                                                                             \
    }
    if (lw == lw0) {
        switch (lh) {
            QBVM_TS_CT(5)
            QBVM_TS_CT(6)
            QBVM_TS_CT(7)
            QBVM_TS_CT(8)
            default: break;
        }
    }
#undef QBVM_TS_CT
    auto kern = k_time_solve<R, MB>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    QBVM_PDL(kern, (unsigned)blocks, TILE_THREADS, smem, s, in, out, tb.Nx, lh, lw, pick(tb.tw_t, tb.tw_t32),
                                                      pick(tb.gpow, tb.gpow32), pick(tb.gipw, tb.gipw32),
                                                      pick(tb.ak, tb.ak32), lt, R(cnorm), pick(tb.gpowr, tb.gpowr32),
                                                      pick(tb.gipr, tb.gipr32), qv, delta_rhs, n0_only);
    return cudaGetLastError();
}

template cudaError_t launch_time_solve<double>(const double*, double*, const Tables&, double, int, int, cudaStream_t);
template cudaError_t launch_time_solve<float>(const float*, float*, const Tables&, double, int, int, cudaStream_t);

cudaError_t launch_time_solve_batched(const double* in, double* out, const Tables& tb, long long count,
                                      long long in_stride, long long out_stride, const double2* gpow,
                                      const double2* gipw, const double2* gpowr, const double2* gipr,
                                      const double2* qinv, int delta_rhs, int n0_only, cudaStream_t s) {
    constexpr int MB = time_tile_maxb4<double>();
    constexpr int TILE = 4 * MB * TILE_THREADS;
    const int lh = tb.lnt - 1, H = 1 << lh;
    int lw = tile_lw(lh, TILE);
    while (lw > 0 && (1LL << (lw - 1)) >= tb.Nx) --lw;         // no wider than the modes
    const int sms = device_sms();                               // and at least two tiles per SM
    while (sms > 0 && lw > 0 && count * ((tb.Nx + (1LL << lw) - 1) >> lw) < 2LL * sms) --lw;
    const int W = 1 << lw;
    const long long tiles = (tb.Nx + W - 1) / W;
    const long long blocks = tiles * count;
    if (count < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = sizeof(double2) * ((size_t)H * W + H);
#define QBVM_TSB(LHV)                                                                                            \
    {                                                                                                            \
        auto kern = k_time_solve_batched<MB, LHV>;                                                               \
        cudaError_t e = set_smem(kern, smem);                                                                    \
        if (e != cudaSuccess) return e;                                                                          \
        QBVM_PDL(kern, (unsigned)blocks, TILE_THREADS, smem, s, in, out, tb.Nx, lh, lw, tiles, in_stride, out_stride,  \
                                                          tb.tw_t, gpow, gipw, gpowr, gipr, qinv, delta_rhs,     \
                                                          n0_only);                                              \
        return cudaGetLastError();                                                                               \
    }
    switch (lh) {
        case 5: QBVM_TSB(5)
        case 6: QBVM_TSB(6)
        case 7: QBVM_TSB(7)
        case 8: QBVM_TSB(8)
        default: QBVM_TSB(-1)
    }
#undef QBVM_TSB
}

template <int LH>
static cudaError_t launch_time_solve_reg_batched_lh(const float* in, float* out, const Tables& tb, long long count,
                                                    long long in_stride, long long out_stride, const float2* gpow,
                                                    const float2* gipw, const float2* ak, const float* cnorm,
                                                    const float* rho_h, const float* rho_hinv, int delta_rhs,
                                                    int n0_only, cudaStream_t s) {
    auto kern = k_time_solve_reg_batched<LH>;
    constexpr size_t smem = ts_reg_smem<LH>();
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (tb.Nx + TsCfg<LH>::TS_MODES - 1) / TsCfg<LH>::TS_MODES;
    if (count < 1 || tiles * count > 0x7fffffffLL) return cudaErrorInvalidValue;
    QBVM_PDL(kern, (unsigned)(tiles * count), TsCfg<LH>::TS_MODES * TsCfg<LH>::N2, smem, s, in, out, tb.Nx, tiles, in_stride,
             out_stride, reinterpret_cast<const float2*>(tb.tw_t32), gpow, gipw, ak,
             reinterpret_cast<const float*>(tb.lamtau32), cnorm, rho_h, rho_hinv, delta_rhs, n0_only);
    return cudaGetLastError();
}

// The generic FP32 tile for the other time lengths (nt = 2 ... 32, 1024):
// instance b takes rows b of the [count][H] tables and cnorm[b].
template <int MAXB4>
__global__ void __launch_bounds__(TILE_THREADS)
k_time_solve_batched32(const float* in, float* out, long long Nx, int lh, int lw, long long tiles,
                       long long in_stride, long long out_stride, const float2* __restrict__ tw,
                       const float2* __restrict__ gpow, const float2* __restrict__ gipw,
                       const float2* __restrict__ gpowr, const float2* __restrict__ gipr,
                       const float2* __restrict__ ak, const float* __restrict__ lamtau,
                       const float* __restrict__ cnorm, int delta_rhs, int n0_only) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long b = (long long)blockIdx.x / tiles, tile = (long long)blockIdx.x - b * tiles;
    const long long H = 1LL << lh;
    time_solve_tile<float, MAXB4>(in + b * in_stride, out + b * out_stride, Nx, lh, lw, tw, gpow + b * H,
                                  gipw + b * H, ak + b * H, lamtau, cnorm[b], gpowr + b * H, gipr + b * H, nullptr,
                                  delta_rhs, n0_only, tile, smem_raw);
}

cudaError_t launch_time_solve_batched32(const float* in, float* out, const Tables& tb, long long count,
                                        long long in_stride, long long out_stride, const BatchTables32& bt,
                                        int delta_rhs, int n0_only, cudaStream_t s) {
    switch (tb.lnt - 1) {
        case 5: return launch_time_solve_reg_batched_lh<5>(in, out, tb, count, in_stride, out_stride, bt.gpow, bt.gipw, bt.ak, bt.cnorm, bt.rho_h, bt.rho_hinv, delta_rhs, n0_only, s);
        case 6: return launch_time_solve_reg_batched_lh<6>(in, out, tb, count, in_stride, out_stride, bt.gpow, bt.gipw, bt.ak, bt.cnorm, bt.rho_h, bt.rho_hinv, delta_rhs, n0_only, s);
        case 7: return launch_time_solve_reg_batched_lh<7>(in, out, tb, count, in_stride, out_stride, bt.gpow, bt.gipw, bt.ak, bt.cnorm, bt.rho_h, bt.rho_hinv, delta_rhs, n0_only, s);
        case 8: return launch_time_solve_reg_batched_lh<8>(in, out, tb, count, in_stride, out_stride, bt.gpow, bt.gipw, bt.ak, bt.cnorm, bt.rho_h, bt.rho_hinv, delta_rhs, n0_only, s);
        default: break;
    }
    constexpr int MB = time_tile_maxb4<float>();
    constexpr int TILE = 4 * MB * TILE_THREADS;
    const int lh = tb.lnt - 1, H = 1 << lh;
    int lw = tile_lw(lh, TILE);
    while (lw > 0 && (1LL << (lw - 1)) >= tb.Nx) --lw;         // no wider than the modes
    const int W = 1 << lw;
    const long long tiles = (tb.Nx + W - 1) / W;
    if (count < 1 || tiles * count > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float2) * ((size_t)H * W + H);
    auto kern = k_time_solve_batched32<MB>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    QBVM_PDL(kern, (unsigned)(tiles * count), TILE_THREADS, smem, s, in, out, tb.Nx, lh, lw, tiles, in_stride,
             out_stride, reinterpret_cast<const float2*>(tb.tw_t32), bt.gpow, bt.gipw, bt.gpowr, bt.gipr, bt.ak,
             reinterpret_cast<const float*>(tb.lamtau32), bt.cnorm, delta_rhs, n0_only);
    return cudaGetLastError();
}

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
    if (delta_rhs) {
        // f = f^0 e_0: the transform is gamma^0 f^0 at every frequency
        const double2 g = gpow[0];
        for (int e = tid; e < (H << lw); e += nth) {
            const long long x = x0 + (e & (W - 1));
            const double f0 = x < Nx ? in_scale * in[x] : 0.0;
            buf[e] = make_double2(g.x * f0, g.y * f0);
        }
        __syncthreads();
    } else {
        for (int i = tid; i < H; i += nth) stw[i] = tw[i];
        for (int e = tid; e < (H << lw); e += nth) {
            int t = e >> lw, c = e & (W - 1);
            long long x = x0 + c;
            double f0 = 0.0, f1 = 0.0;
            if (x < Nx) {
                f0 = in[(long long)t * Nx + x];
                f1 = rho_h * in[(long long)(t + H) * Nx + x];
            }
            double2 g = gpow[t];
            buf[e] = make_double2(g.x * f0 - g.y * f1, g.y * f0 + g.x * f1);
        }
        __syncthreads();
        fft_tile<+1, TILE_ELEMS / 4 / TILE_THREADS>(buf, stw, lh, lw);
    }
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
    cudaError_t e = set_smem(k_time_fwd_1d, smem);
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
    cudaError_t e = set_smem(k_time_inv_1d, smem);
    if (e != cudaSuccess) return e;
    k_time_inv_1d<<<(unsigned)blocks, TILE_THREADS, smem, s>>>(wk, out, tb.Nx, lh, lw, tb.tw_t, tb.gipw,
                                                                tb.rho_hinv, n0_only);
    return cudaGetLastError();
}

// ------------------------------------------------------- general nt (Bluestein)
//
// For a number of time levels P that is not a power of two (the paper's meshes
// have N_t = N + 1) the length-P DFTs of Steps (a) and (c) use Bluestein's
// chirp-z identity (L. I. Bluestein, "A linear filtering approach to the
// computation of the discrete Fourier transform", 1970): with
// c_m = exp(S i pi m^2 / P),
//     sum_{t<P} x_t exp(S 2 pi i k t / P) = c_k sum_t (x_t c_t) conj(c_{k-t}),
// a linear convolution, evaluated as a cyclic one of power-of-two length
// L >= 2P - 1 with the FFT engine: FFT(x c), times the plan's table
// B = FFT(conj c, wrapped) / L, inverse FFT, times c_k.  Every frequency is
// formed (no half-spectrum shortcut).  Modes:
//   BS_FWD_DIV  Step (a) + Step (b) of the space-first solve: real [P][N] in
//               (one level for the delta right-hand side), pre-factor
//               gamma^t, out [P][N] complex cnorm u^_k / (d_k + tau Lambda_l);
//   BS_FWD      Step (a) of the 1D solve: as above without the divide
//               (cnorm scales the delta right-hand side);
//   BS_INV      Step (c): complex [P][N] in, out y_t = Re(post_t q_t) real.
// The forward transform of the delta right-hand side f^0 e_0 is the constant
// f^0 and is written without transforming.
enum { BS_FWD_DIV = 0, BS_FWD = 1, BS_INV = 2 };

template <typename R, int S, int MODE>
__global__ void __launch_bounds__(TILE_THREADS)
k_bluestein(const void* in, void* out, long long N, int P, int lL, int lw, const cplx<R>* __restrict__ tw,
            const cplx<R>* __restrict__ chirp, const cplx<R>* __restrict__ B, const cplx<R>* __restrict__ fac,
            const cplx<R>* __restrict__ dk, const R* __restrict__ lamtau, R cnorm, int delta_rhs,
            int n0_only) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = 1 << lL, W = 1 << lw;
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* stw = buf + ((size_t)L << lw);
    const int tid = threadIdx.x, nth = blockDim.x;
    const long long l0 = (long long)blockIdx.x * W;
    auto csgn = [](C c) { return S > 0 ? c : mkc(c.x, -c.y); };   // c_m of sign S
    auto epilogue = [&](int k, long long l, C v) {
        if (MODE == BS_FWD_DIV) {
            const C a = dk[k];
            const R zr = a.x + lamtau[l], zi = a.y;
            const R inv = cnorm / (zr * zr + zi * zi);
            reinterpret_cast<C*>(out)[(long long)k * N + l] = mkc((v.x * zr + v.y * zi) * inv, (v.y * zr - v.x * zi) * inv);
        } else if (MODE == BS_FWD) {
            reinterpret_cast<C*>(out)[(long long)k * N + l] = v;
        } else {
            const C g = fac[k];
            reinterpret_cast<R*>(out)[(long long)k * N + l] = g.x * v.x - g.y * v.y;
        }
    };
    if (MODE != BS_INV && delta_rhs) {
        const R sc = MODE == BS_FWD ? cnorm : R(1);
        for (int e = tid; e < (P << lw); e += nth) {
            const int k = e >> lw, c = e & (W - 1);
            const long long l = l0 + c;
            if (l < N) {
                const R f0 = sc * reinterpret_cast<const R*>(in)[l];
                epilogue(k, l, mkc(fac[0].x * f0, fac[0].y * f0));
            }
        }
        return;
    }
    for (int i = tid; i < L; i += nth) stw[i] = tw[i];
    for (int e = tid; e < (L << lw); e += nth) {
        const int t = e >> lw, c = e & (W - 1);
        const long long l = l0 + c;
        C v = mkc(R(0), R(0));
        if (t < P && l < N) {
            if (MODE == BS_INV) {
                v = reinterpret_cast<const C*>(in)[(long long)t * N + l];
            } else {
                const R f = reinterpret_cast<const R*>(in)[(long long)t * N + l];
                v = mkc(fac[t].x * f, fac[t].y * f);
            }
            v = cmul(v, csgn(chirp[t]));
        }
        buf[e] = v;
    }
    __syncthreads();
    fft_tile<-1, TILE_ELEMS / 4 / TILE_THREADS>(buf, stw, lL, lw);
    for (int e = tid; e < (L << lw); e += nth) buf[e] = cmul(buf[e], B[e >> lw]);
    __syncthreads();
    fft_tile<+1, TILE_ELEMS / 4 / TILE_THREADS>(buf, stw, lL, lw);
    const int kmax = (MODE == BS_INV && n0_only) ? 1 : P;
    for (int e = tid; e < (kmax << lw); e += nth) {
        const int k = e >> lw, c = e & (W - 1);
        const long long l = l0 + c;
        if (l < N) epilogue(k, l, cmul(buf[e], csgn(chirp[k])));
    }
}

template <typename R>
static cudaError_t launch_bluestein_r(int mode, const void* in, void* out, long long N, const Tables& tb, R cnorm,
                                     int delta_rhs, int n0_only, const cplx<R>* twL, const cplx<R>* chirp,
                                     const cplx<R>* bsf, const cplx<R>* bsi, const cplx<R>* gpw,
                                     const cplx<R>* gip, const cplx<R>* dk, const R* lamtau, cudaStream_t s) {
    const int lL = tb.lL, L = 1 << lL;
    int lw = 0;
    while ((L << (lw + 1)) <= TILE_ELEMS) ++lw;
    const long long blocks = (N + (1 << lw) - 1) >> lw;
    const size_t smem = sizeof(cplx<R>) * (((size_t)L << lw) + L);
    cudaError_t e = cudaSuccess;
    const int P = tb.nt;
    if (mode == BS_FWD_DIV) {
        auto kern = k_bluestein<R, +1, BS_FWD_DIV>;
        if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
        kern<<<(unsigned)blocks, TILE_THREADS, smem, s>>>(in, out, N, P, lL, lw, twL, chirp, bsf, gpw, dk, lamtau,
                                                          cnorm, delta_rhs, 0);
    } else if (mode == BS_FWD) {
        auto kern = k_bluestein<R, +1, BS_FWD>;
        if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
        kern<<<(unsigned)blocks, TILE_THREADS, smem, s>>>(in, out, N, P, lL, lw, twL, chirp, bsf, gpw, nullptr,
                                                          nullptr, cnorm, delta_rhs, 0);
    } else {
        auto kern = k_bluestein<R, -1, BS_INV>;
        if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
        kern<<<(unsigned)blocks, TILE_THREADS, smem, s>>>(in, out, N, P, lL, lw, twL, chirp, bsi, gip, nullptr,
                                                          nullptr, R(0), 0, n0_only);
    }
    return cudaGetLastError();
}

cudaError_t launch_bluestein(int mode, const void* in, void* out, long long N, const Tables& tb, double cnorm,
                             int delta_rhs, int n0_only, cudaStream_t s) {
    return launch_bluestein_r<double>(mode, in, out, N, tb, cnorm, delta_rhs, n0_only, tb.tw_L, tb.chirp, tb.bs_fwd,
                                      tb.bs_inv, tb.gpw_full, tb.gip_full, tb.dk_full, tb.lamtau, s);
}

cudaError_t launch_bluestein32(int mode, const void* in, void* out, long long N, const Tables& tb, float cnorm,
                               int delta_rhs, int n0_only, cudaStream_t s) {
    if (!tb.tw_L32) return cudaErrorInvalidValue;              // built by FP32-refinement plans only
    return launch_bluestein_r<float>(mode, in, out, N, tb, cnorm, delta_rhs, n0_only, tb.tw_L32, tb.chirp32,
                                     tb.bs_fwd32, tb.bs_inv32, tb.gpw_full32, tb.gip_full32, tb.dk_full32,
                                     tb.lamtau32, s);
}

cudaError_t launch_thomas_1d_n(double2* wk, double2* cp, int nsys, const Tables& tb, cudaStream_t s) {
    int threads = 64;
    int blocks = (nsys + threads - 1) / threads;
    k_thomas_1d<<<blocks, threads, 0, s>>>(wk, cp, nsys, tb.Nx, tb.bk);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ residual
//
// (A y)^n = (y^n - y^{n-1})/tau - Delta_h y^n for n >= 1 and
// (A y)^0 = (y^0 - omega y^N)/tau - Delta_h y^0 (eq. 3.3 / 3.6, Kronecker form
// of Section 3.3); f^0 = -omega g / tau for the delta right-hand side.
constexpr int RES_THREADS = 256;

// Rows of n_x contiguous values: row index -> (t, z, y) in 32-bit arithmetic;
// the threads of a block stride over x.
__global__ void __launch_bounds__(RES_THREADS)
k_residual(const double* __restrict__ y, const double* __restrict__ f, int delta_rhs, int nt,
           int nx, int ny, int nz, double inv_tau, double omega, double hx2, double hy2, double hz2,
           double* partials, double* r_out) {
    __shared__ double sh[32];
    const long long Nx = (long long)nx * ny * nz;
    const long long pl = (long long)nx * ny;
    const int rows = nt * ny * nz;
    double rr = 0.0, ff = 0.0;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int t = row / (ny * nz), rz = row - t * (ny * nz);
        const int iz = rz / ny, iy = rz - iz * ny;
        const long long base = (long long)row * nx;
        const long long sbase = base - (long long)t * Nx;
        for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
            const long long idx = base + ix;
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
                lap -= 2.0 * yv * hz2;
                if (iz > 0) lap += y[idx - pl] * hz2;
                if (iz < nz - 1) lap += y[idx + pl] * hz2;
            }
            double prev = t > 0 ? y[idx - Nx] : omega * y[(long long)(nt - 1) * Nx + sbase + ix];
            double Ay = (yv - prev) * inv_tau - lap;
            double fv;
            if (delta_rhs) fv = t == 0 ? -omega * inv_tau * f[sbase + ix] : 0.0;
            else fv = f[idx];
            double r = fv - Ay;
            if (r_out) r_out[idx] = r;
            rr = fma(r, r, rr);
            ff = fma(fv, fv, ff);
        }
    }
    rr = block_sum(rr, sh);
    ff = block_sum(ff, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = rr;
        partials[2 * blockIdx.x + 1] = ff;
    }
}

// The refinement residual of 1D plans in FP64 arithmetic: y is the
// double-float iterate, each value joined exactly into FP64 (the bit-built
// widenings and one FP64 add, qbvm_join_df_dadd), the stencil as in
// k_residual, r rounded once to FP32 (r.hi of the correction), norms in FP64.
// Its error, O(2^-53) of the terms against O(2^-48) for the double-float
// stencil, sets the floor the refinement stalls at (about kappa(A) times it);
// 1D plans hold at most 2047 x 2048 unknowns, so the FP64 pipe's cost stays
// small (tens of microseconds).
__global__ void __launch_bounds__(RES_THREADS)
k_residual_1d_dd(const float2* __restrict__ y, const double* __restrict__ f, int delta_rhs, int fnorm, int nt,
                 int nx, double inv_tau, double omega, double hx2, float* __restrict__ r_out, double* partials) {
    pdl_trigger();
    pdl_wait();
    __shared__ double sh[32];
    const long long N = (long long)nt * nx;
    auto ld = [&](long long i) {
        const float2 v = y[i];
        return qbvm_join_df_dadd(v.x, v.y);
    };
    double rr = 0.0, ff = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int t = (int)(i / nx), ix = (int)(i - (long long)t * nx);
        const double yv = ld(i);
        double lap = -2.0 * yv;
        if (ix > 0) lap += ld(i - 1);
        if (ix < nx - 1) lap += ld(i + 1);
        const double prev = t > 0 ? ld(i - nx) : omega * ld((long long)(nt - 1) * nx + ix);
        const double Ay = (yv - prev) * inv_tau - lap * hx2;
        double fv;
        if (delta_rhs) fv = t == 0 ? -omega * inv_tau * f[ix] : 0.0;
        else fv = f[i];
        const double r = fv - Ay;
        r_out[i] = __double2float_rn(r);
        rr = fma(r, r, rr);
        if (fnorm) ff = fma(fv, fv, ff);
    }
    rr = block_sum(rr, sh);
    ff = block_sum(ff, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = rr;
        partials[2 * blockIdx.x + 1] = ff;
    }
}

__global__ void k_reduce_pairs(const double* partials, int n, double* sums) {
    pdl_trigger();
    pdl_wait();
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

// Double-float residual for the refinement: y is a double-float array (hi, lo),
// f is FP64 (split exactly on load, integer pipes); the stencil runs in
// double-float on the FP32 pipes.  Writes r.hi (FP32: the right-hand side of
// the next FP32 correction solve) and per-block partial sums of ||r||^2,
// ||f||^2 (r.hi^2, f.hi^2; enough digits for a stopping test).
//   (A y)^n = ct (y^n - p^n) + sum_d c_d (2 y^n - y_{i-e_d} - y_{i+e_d}),
//   ct = 1/tau, c_d = 1/h_d^2, p^n = y^{n-1} (n >= 1) or omega y^{N} (n = 0).
// Differences are formed before the (inexact) scalings; with equal spacing on
// every axis (EQ) the axes share one product: c (2d y - sum of neighbours).
// Sums use df_add_sloppy: its error, O(u^2) times the magnitudes of the terms,
// is of the size the double-float inputs already carry.
struct DfCoef {
    dfloat ct, omega, cx, cy, cz;
};

template <bool EQ>
__global__ void __launch_bounds__(RES_THREADS)
k_residual_df(const float2* __restrict__ y, const double* __restrict__ f, int delta_rhs, int nt, int nx, int ny,
              int nz, DfCoef k, double f0_scale, float* __restrict__ r_out, double* partials) {
    pdl_trigger();
    pdl_wait();
    __shared__ double sh[32];
    const long long Nx = (long long)nx * ny * nz;
    const long long pl = (long long)nx * ny;
    const int rows = nt * ny * nz;
    const int dims = 1 + (ny > 1) + (nz > 1);
    float rr = 0.f, ff = 0.f;
    auto ld = [&](long long i) { float2 v = y[i]; return dfloat{v.x, v.y}; };
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int t = row / (ny * nz), rz = row - t * (ny * nz);
        const int iz = rz / ny, iy = rz - iz * ny;
        const long long base = (long long)row * nx;
        const long long sbase = base - (long long)t * Nx;
        for (int ix = threadIdx.x; ix < nx; ix += blockDim.x) {
            const long long idx = base + ix;
            const dfloat yv = ld(idx);
            dfloat d1;
            if (t > 0) d1 = df_add_sloppy(yv, df_neg(ld(idx - Nx)));
            else d1 = df_add_sloppy(yv, df_neg(df_mul(k.omega, ld((long long)(nt - 1) * Nx + sbase + ix))));
            dfloat Ay = df_mul(k.ct, d1);
            dfloat sx = {0.f, 0.f};
            if (ix > 0) sx = ld(idx - 1);
            if (ix < nx - 1) sx = df_add_sloppy(sx, ld(idx + 1));
            dfloat sy = {0.f, 0.f}, sz = {0.f, 0.f};
            if (ny > 1) {
                if (iy > 0) sy = ld(idx - nx);
                if (iy < ny - 1) sy = df_add_sloppy(sy, ld(idx + nx));
            }
            if (nz > 1) {
                if (iz > 0) sz = ld(idx - pl);
                if (iz < nz - 1) sz = df_add_sloppy(sz, ld(idx + pl));
            }
            if (EQ) {
                dfloat S = sx;
                if (ny > 1) S = df_add_sloppy(S, sy);
                if (nz > 1) S = df_add_sloppy(S, sz);
                // 2 d y: scalings by 2 and 4 are exact; 6 y = 4 y + 2 y in double-float
                dfloat my = dims == 3 ? df_add_sloppy(dfloat{4.f * yv.hi, 4.f * yv.lo}, dfloat{2.f * yv.hi, 2.f * yv.lo})
                                      : dfloat{2.f * dims * yv.hi, 2.f * dims * yv.lo};
                dfloat lap = df_add_sloppy(my, df_neg(S));
                Ay = df_add_sloppy(Ay, df_mul(k.cx, lap));
            } else {
                Ay = df_add_sloppy(Ay, df_mul(k.cx, df_add_sloppy(dfloat{2.f * yv.hi, 2.f * yv.lo}, df_neg(sx))));
                if (ny > 1) Ay = df_add_sloppy(Ay, df_mul(k.cy, df_add_sloppy(dfloat{2.f * yv.hi, 2.f * yv.lo}, df_neg(sy))));
                if (nz > 1) Ay = df_add_sloppy(Ay, df_mul(k.cz, df_add_sloppy(dfloat{2.f * yv.hi, 2.f * yv.lo}, df_neg(sz))));
            }
            dfloat fv = {0.f, 0.f};
            if (delta_rhs) {
                if (t == 0) fv = df_from_double(f0_scale * f[sbase + ix]);
            } else {
                fv = df_from_double(f[idx]);
            }
            dfloat r = df_add_sloppy(fv, df_neg(Ay));
            r_out[idx] = r.hi;
            rr = fmaf(r.hi, r.hi, rr);
            ff = fmaf(fv.hi, fv.hi, ff);
        }
    }
    double a = block_sum((double)rr, sh);
    double b = block_sum((double)ff, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

// The same residual, four consecutive unknowns of the flattened [nt][nz][ny][nx]
// array per thread: the iterate, f and r move as 16-byte vectors, the x
// neighbours across a group boundary come from the adjacent lanes, and the
// (t, z, y, x) position is advanced incrementally (no divisions in the loop).
// Requires 16-byte aligned y, f and r_out.
// Intermediate pairs are left unnormalised (the high parts combined by exact
// two-sums, the low parts and rounding errors summed in FP32: error O(u^2)
// times the terms' magnitudes, the size the double-float inputs carry), f is
// split by truncation (df_from_double_trunc), 6 y is an exact product pair,
// and ||f||^2 is summed only when `fnorm` is set (the first residual of a
// solve).  Bounded to 64 registers (4 CTAs per SM): the 3D stencil took 97
// and ran at a quarter of the warp slots.  FAST (the residuals after the
// first, whose ||f|| is known): ||r||^2 as a plain FP32 sum of (r rscale)^2,
// rscale the power of two near 1 / rms(f), instead of the scaled sum that
// follows the magnitudes (about 13 instructions per term); the block's sum is
// returned times inv_s2 = 1 / rscale^2 (exact).
template <bool EQ, int DIMS, bool FAST = false, typename IT = long long>
__device__ __forceinline__ void residual_df4_body(const float2* __restrict__ y, const double* __restrict__ f,
                                                  int delta_rhs, int nt, int nx, int ny, int nz, const DfCoef& k,
                                                  double f0_scale, int fnorm, float* __restrict__ r_out,
                                                  IT blk, IT nblk, double* part2,
                                                  float rscale = 0.f, double inv_s2 = 0.0) {
    __shared__ double sh[32];
    const IT Nx = (IT)nx * ny * nz, N = (IT)nt * Nx, pl = (IT)nx * ny;
    const IT ngroups = (N + 3) >> 2;
    const int lane = threadIdx.x & 31;
    const IT wid = (blk * blockDim.x + threadIdx.x) >> 5;
    const IT nw = (nblk * blockDim.x) >> 5;
    // (t, z, y, x) of a flat index: 32-bit divisions when the index fits (a
    // 64-bit division is a long software sequence, and short-lived threads --
    // small instances of a batch -- pay it for few elements)
    auto split = [&](IT i, int& t, int& z, int& yy, int& x) {
        if (i < 0x7fffffffLL && Nx < 0x7fffffffLL) {
            const unsigned ui = (unsigned)i, uN = (unsigned)Nx, up = (unsigned)pl, ux = (unsigned)nx;
            const unsigned ut = ui / uN;
            unsigned r = ui - ut * uN;
            const unsigned uz = r / up;
            r -= uz * up;
            const unsigned uy = r / ux;
            t = (int)ut;
            z = (int)uz;
            yy = (int)uy;
            x = (int)(r - uy * ux);
            return;
        }
        t = (int)(i / Nx);
        IT r = i - (IT)t * Nx;
        z = (int)(r / pl);
        r -= (IT)z * pl;
        yy = (int)(r / nx);
        x = (int)(r - (IT)yy * nx);
    };
    int t, iz, iy, ix, St, Sz, Sy, Sx;
    split((wid * 32 + lane) * 4, t, iz, iy, ix);
    split(nw * 128, St, Sz, Sy, Sx);
    auto ld = [&](IT i) { float2 v = y[i]; return dfloat{v.x, v.y}; };
    const float4* y4 = reinterpret_cast<const float4*>(y);
    const double2* f2 = reinterpret_cast<const double2*>(f);
    ScaledSsq nr, nf;
    float nr2 = 0.f;
    for (IT gb = wid * 32; gb < ngroups; gb += nw * 32) {
        const IT g = gb + lane, i0 = 4 * g;
        const bool act = g < ngroups, full = act && i0 + 3 < N;
        dfloat yv[4];
        if (full) {
            const float4 a = y4[2 * g], b = y4[2 * g + 1];
            yv[0] = {a.x, a.y};
            yv[1] = {a.z, a.w};
            yv[2] = {b.x, b.y};
            yv[3] = {b.z, b.w};
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) yv[e] = (act && i0 + e < N) ? ld(i0 + e) : dfloat{0.f, 0.f};
        }
        double fd[4] = {0.0, 0.0, 0.0, 0.0};
        if (!delta_rhs) {
            if (full) {
                const double2 a = f2[2 * g], b = f2[2 * g + 1];
                fd[0] = a.x;
                fd[1] = a.y;
                fd[2] = b.x;
                fd[3] = b.y;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (act && i0 + e < N) fd[e] = f[i0 + e];
            }
        }
        // x neighbours of the group's first and last element
        dfloat xl = {__shfl_up_sync(0xffffffffu, yv[3].hi, 1), __shfl_up_sync(0xffffffffu, yv[3].lo, 1)};
        dfloat xr = {__shfl_down_sync(0xffffffffu, yv[0].hi, 1), __shfl_down_sync(0xffffffffu, yv[0].lo, 1)};
        if (lane == 0) xl = (act && i0 >= 1) ? ld(i0 - 1) : dfloat{0.f, 0.f};
        if (lane == 31) xr = (act && i0 + 4 < N) ? ld(i0 + 4) : dfloat{0.f, 0.f};
        float rv[4];
        int et = t, ez = iz, ey = iy, ex = ix;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (e > 0 && ++ex == nx) {
                ex = 0;
                if (++ey == ny) {
                    ey = 0;
                    if (++ez == nz) {
                        ez = 0;
                        ++et;
                    }
                }
            }
            const IT idx = i0 + e;
            rv[e] = 0.f;
            if (!(act && idx < N)) continue;
            const dfloat yc = yv[e];
            dfloat pv = et > 0 ? ld(idx - Nx) : ld(idx + (IT)(nt - 1) * Nx);
            if (et == 0) pv = df_mul_un(k.omega, pv);
            dfloat Ay = df_mul_un(k.ct, df_sub_un(yc, pv));
            const dfloat L = e > 0 ? yv[e - 1] : xl, R = e < 3 ? yv[e + 1] : xr;
            const dfloat zero = {0.f, 0.f};
            const dfloat sxl = ex > 0 ? L : zero, sxr = ex < nx - 1 ? R : zero;
            dfloat ys = zero, yn = zero, zd = zero, zu = zero;
            if (DIMS >= 2) {
                if (ey > 0) ys = ld(idx - nx);
                if (ey < ny - 1) yn = ld(idx + nx);
            }
            if (DIMS >= 3) {
                if (ez > 0) zd = ld(idx - pl);
                if (ez < nz - 1) zu = ld(idx + pl);
            }
            if (EQ) {
                dfloat S = df_add_un(sxl, sxr);
                if (DIMS >= 2) S = df_add_un(S, df_add_un(ys, yn));
                if (DIMS >= 3) S = df_add_un(S, df_add_un(zd, zu));
                const float c2d = 2.f * DIMS;
                dfloat my = {c2d * yc.hi, c2d * yc.lo};
                if (DIMS == 3) my.lo = fmaf(c2d, yc.hi, -my.hi) + my.lo;       // 6 y exactly
                Ay = df_add_un(Ay, df_mul_un(k.cx, df_sub_un(my, S)));
            } else {
                const dfloat y2 = {2.f * yc.hi, 2.f * yc.lo};
                Ay = df_add_un(Ay, df_mul_un(k.cx, df_sub_un(y2, df_add_un(sxl, sxr))));
                if (DIMS >= 2) Ay = df_add_un(Ay, df_mul_un(k.cy, df_sub_un(y2, df_add_un(ys, yn))));
                if (DIMS >= 3) Ay = df_add_un(Ay, df_mul_un(k.cz, df_sub_un(y2, df_add_un(zd, zu))));
            }
            // f - A y; with the delta right-hand side f is zero past level 0
            dfloat fv = zero, r;
            if (delta_rhs && et != 0) {
                r = dfloat{-Ay.hi, -Ay.lo};
            } else {
                if (delta_rhs) fv = df_from_double_trunc(f0_scale * f[((IT)ez * ny + ey) * nx + ex]);
                else fv = df_from_double_trunc(fd[e]);
                r = df_sub_un(fv, Ay);
            }
            const float rh = r.hi + r.lo;
            rv[e] = rh;
            if (FAST) {
                const float rs = rh * rscale;
                nr2 = fmaf(rs, rs, nr2);
            } else {
                nr.add(rh);
                if (fnorm) nf.add(fv.hi);
            }
        }
        if (full) {
            reinterpret_cast<float4*>(r_out)[g] = make_float4(rv[0], rv[1], rv[2], rv[3]);
        } else if (act) {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (i0 + e < N) r_out[i0 + e] = rv[e];
        }
        // advance (t, z, y, x) by the grid stride (each component wraps at most once)
        ix += Sx;
        int c = ix >= nx;
        if (c) ix -= nx;
        iy += Sy + c;
        c = iy >= ny;
        if (c) iy -= ny;
        iz += Sz + c;
        c = iz >= nz;
        if (c) iz -= nz;
        t += St + c;
    }
    if (FAST) {
        // warp sums in FP32, the warps' sums in FP64 by one thread
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nr2 += __shfl_xor_sync(0xffffffffu, nr2, o);
        __shared__ float shf[RES_THREADS / 32];
        if (lane == 0) shf[threadIdx.x >> 5] = nr2;
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += (double)shf[i];
            part2[0] = a * inv_s2;
            part2[1] = 0.0;
        }
        return;
    }
    double a = block_sum(nr.value(), sh);
    double b = block_sum(nf.value(), sh);
    if (threadIdx.x == 0) {
        part2[0] = a;
        part2[1] = b;
    }
}

// IT: the index type, int when the array has fewer than 2^31 values (the
// 64-bit index arithmetic had cost 22 % more instructions and 8 % more time
// on 127^3 x 128).
template <bool EQ, int DIMS, bool FAST, typename IT>
__global__ void __launch_bounds__(RES_THREADS, 4)
k_residual_df4(const float2* __restrict__ y, const double* __restrict__ f, int delta_rhs, int nt, int nx, int ny,
               int nz, DfCoef k, double f0_scale, int fnorm, float* __restrict__ r_out, double* partials,
               float rscale, double inv_s2) {
    pdl_trigger();
    pdl_wait();
    residual_df4_body<EQ, DIMS, FAST, IT>(y, f, delta_rhs, nt, nx, ny, nz, k, f0_scale, fnorm, r_out,
                                          (IT)blockIdx.x, (IT)gridDim.x, partials + 2 * (long long)blockIdx.x,
                                          rscale, inv_s2);
}

// `count` instances back to back, bpi blocks per instance: block (b, j) runs
// the instance's residual with its own omega (and f^0 = -omega_b g_b / tau).
template <bool EQ, int DIMS, typename IT>
__global__ void __launch_bounds__(RES_THREADS, 4)
k_residual_df4_batched(const float2* __restrict__ y, const double* __restrict__ f, int delta_rhs, int nt, int nx,
                       int ny, int nz, DfCoef k, const float2* __restrict__ omega_df,
                       const double* __restrict__ omega64, double inv_tau, int fnorm, int bpi,
                       float* __restrict__ r_out, double* partials) {
    pdl_trigger();
    pdl_wait();
    const long long b = blockIdx.x / bpi, j = blockIdx.x - b * bpi;
    const long long per = (long long)nt * nx * ny * nz, Nx = (long long)nx * ny * nz;
    DfCoef kb = k;
    const float2 om = omega_df[b];
    kb.omega = dfloat{om.x, om.y};
    residual_df4_body<EQ, DIMS, false, IT>(y + b * per, f + b * (delta_rhs ? Nx : per), delta_rhs, nt, nx, ny, nz, kb,
                                           -omega64[b] * inv_tau, fnorm, r_out + b * per, (IT)j, (IT)bpi,
                                           partials + 2 * (long long)blockIdx.x);
}

// sums[2 b], sums[2 b + 1] = the instance's partial pairs summed (one warp each).
__global__ void k_reduce_instances(const double* partials, int bpi, long long count, double* sums) {
    pdl_trigger();
    pdl_wait();
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    double a = 0.0, c = 0.0;
    for (int i = lane; i < bpi; i += 32) {
        a += partials[2 * (w * bpi + i)];
        c += partials[2 * (w * bpi + i) + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        sums[2 * w] = a;
        sums[2 * w + 1] = c;
    }
}

// In place: a double-float array (8 bytes per value) becomes the FP64 array.
__global__ void k_df_to_double(void* buf, long long n) {
    pdl_trigger();
    pdl_wait();
    const float2* src = reinterpret_cast<const float2*>(buf);
    double* dst = reinterpret_cast<double*>(buf);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float2 v = src[i];
        dst[i] = qbvm_join_df(v.x, v.y);
    }
}

// The same conversion, four values per thread (the join with one FP64 add per
// value, qbvm_join_df_dadd: the integer join made this kernel instruction-bound
// at 3.8 TB/s): two 16-byte loads of the pairs,
// then two 16-byte stores of the doubles over the same 32 bytes (every thread
// reads its bytes before writing them, and no other thread touches them).
// Requires a 16-byte aligned buffer; values past the last group of four are
// taken one per thread by the first threads of the grid.
__global__ void __launch_bounds__(256) k_df_to_double4(void* buf, long long n) {
    pdl_trigger();
    pdl_wait();
    const long long ng = n >> 2;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const float4* src = reinterpret_cast<const float4*>(buf);
    double2* dst = reinterpret_cast<double2*>(buf);
    for (long long g = tid; g < ng; g += stride) {
        const float4 a = src[2 * g], b = src[2 * g + 1];
        dst[2 * g] = make_double2(qbvm_join_df_dadd(a.x, a.y), qbvm_join_df_dadd(a.z, a.w));
        dst[2 * g + 1] = make_double2(qbvm_join_df_dadd(b.x, b.y), qbvm_join_df_dadd(b.z, b.w));
    }
    const long long i = 4 * ng + tid;
    if (i < n) {
        const float2 v = reinterpret_cast<const float2*>(buf)[i];
        reinterpret_cast<double*>(buf)[i] = qbvm_join_df(v.x, v.y);
    }
}

static dfloat df_const(double c) {
    float h = (float)c;
    return {h, (float)(c - (double)h)};
}

cudaError_t launch_residual_df(const void* y_df, const double* f, int delta_rhs, const Tables& tb,
                               const double h2inv[3], float* r_out, double* partials, int nblocks, double* sums,
                               int fnorm, cudaStream_t s, float rscale) {
    DfCoef k;
    const double it = 1.0 / tb.tau;
    k.ct = df_const(it);
    k.omega = df_const(tb.omega);
    k.cx = df_const(h2inv[0]);
    k.cy = df_const(h2inv[1]);
    k.cz = df_const(h2inv[2]);
    const bool eq = (tb.dim < 2 || h2inv[1] == h2inv[0]) && (tb.dim < 3 || h2inv[2] == h2inv[0]);
    const bool aligned = ((reinterpret_cast<uintptr_t>(y_df) | reinterpret_cast<uintptr_t>(f) |
                           reinterpret_cast<uintptr_t>(r_out)) & 15) == 0;
    if (tb.dim == 1) {
        const long long n = (long long)tb.nt * tb.Nx;
        long long nb = (n + RES_THREADS - 1) / RES_THREADS;
        if (nb > nblocks) nb = nblocks;
        QBVM_PDL(k_residual_1d_dd, (unsigned)nb, RES_THREADS, 0, s, reinterpret_cast<const float2*>(y_df), f,
                 delta_rhs, fnorm, tb.nt, tb.n[0], it, tb.omega, h2inv[0], r_out, partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        QBVM_PDL(k_reduce_pairs, 1, 1024, 0, s, partials, (int)nb, sums);
        return cudaGetLastError();
    }
    if (aligned) {
        const long long groups = ((long long)tb.nt * tb.Nx + 3) / 4;
        long long nb = (groups + RES_THREADS - 1) / RES_THREADS;
        if (nb > nblocks) nb = nblocks;
        const float2* yy = reinterpret_cast<const float2*>(y_df);
        const double fs = -tb.omega * it;
        const int nx = tb.n[0], ny = tb.n[1], nz = tb.n[2];
        const bool fast = rscale > 0.f && !fnorm;
        const double is2 = fast ? 1.0 / ((double)rscale * (double)rscale) : 0.0;
        const bool i32 = (long long)tb.nt * tb.Nx < 0x7ffff000LL;
#define QBVM_RD4F(E, D, F)                                                                                      \
        do {                                                                                                    \
            if (i32)                                                                                            \
                QBVM_PDL(k_residual_df4<E, D, F, int>, (unsigned)nb, RES_THREADS, 0, s, yy, f, delta_rhs, tb.nt, nx,\
                         ny, nz, k, fs, fnorm, r_out, partials, rscale, is2);                                  \
            else                                                                                                \
                QBVM_PDL(k_residual_df4<E, D, F, long long>, (unsigned)nb, RES_THREADS, 0, s, yy, f, delta_rhs,     \
                         tb.nt, nx, ny, nz, k, fs, fnorm, r_out, partials, rscale, is2);                       \
        } while (0)
#define QBVM_RD4(E, D)                                                                                          \
        do {                                                                                                    \
            if (fast) QBVM_RD4F(E, D, true);                                                                    \
            else QBVM_RD4F(E, D, false);                                                                        \
        } while (0)
        if (tb.dim == 2) {
            if (eq) QBVM_RD4(true, 2);
            else QBVM_RD4(false, 2);
        } else {
            if (eq) QBVM_RD4(true, 3);
            else QBVM_RD4(false, 3);
        }
#undef QBVM_RD4
#undef QBVM_RD4F
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        QBVM_PDL(k_reduce_pairs, 1, 1024, 0, s, partials, (int)nb, sums);
        return cudaGetLastError();
    }
    if (eq)
        QBVM_PDL(k_residual_df<true>, nblocks, RES_THREADS, 0, s, reinterpret_cast<const float2*>(y_df), f, delta_rhs, tb.nt,
                                                            tb.n[0], tb.n[1], tb.n[2], k, -tb.omega * it, r_out,
                                                            partials);
    else
        QBVM_PDL(k_residual_df<false>, nblocks, RES_THREADS, 0, s, reinterpret_cast<const float2*>(y_df), f, delta_rhs,
                                                             tb.nt, tb.n[0], tb.n[1], tb.n[2], k, -tb.omega * it,
                                                             r_out, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    QBVM_PDL(k_reduce_pairs, 1, 1024, 0, s, partials, nblocks, sums);
    return cudaGetLastError();
}

int residual_blocks_per_instance(const Tables& tb) {
    const long long groups = ((long long)tb.nt * tb.Nx + 3) / 4;
    long long b = (groups + 4 * RES_THREADS - 1) / (4 * RES_THREADS);        // four groups per thread
    if (b > 1024) b = 1024;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_residual_df_batched(const void* y_df, const double* f, int delta_rhs, const Tables& tb,
                                       const double h2inv[3], long long count, const float2* omega_df,
                                       const double* omega64, float* r_out, double* partials, double* sums,
                                       int fnorm, int bpi, cudaStream_t s) {
    if (((long long)tb.nt * tb.Nx) % 4 != 0 || count * bpi > 0x7fffffffLL) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(y_df) | reinterpret_cast<uintptr_t>(r_out) |
         (delta_rhs ? 0 : reinterpret_cast<uintptr_t>(f))) & 15)
        return cudaErrorInvalidValue;
    DfCoef k;
    const double it = 1.0 / tb.tau;
    k.ct = df_const(it);
    k.omega = df_const(tb.omega);
    k.cx = df_const(h2inv[0]);
    k.cy = df_const(h2inv[1]);
    k.cz = df_const(h2inv[2]);
    const bool eq = (tb.dim < 2 || h2inv[1] == h2inv[0]) && (tb.dim < 3 || h2inv[2] == h2inv[0]);
    const float2* yy = reinterpret_cast<const float2*>(y_df);
    const int nx = tb.n[0], ny = tb.n[1], nz = tb.n[2];
    const unsigned nb = (unsigned)(count * bpi);
    const bool i32 = (long long)tb.nt * tb.Nx < 0x7ffff000LL;       // one instance's values
#define QBVM_RDB(E, D)                                                                                        \
    do {                                                                                                      \
        if (i32)                                                                                              \
            QBVM_PDL(k_residual_df4_batched<E, D, int>, nb, RES_THREADS, 0, s, yy, f, delta_rhs, tb.nt, nx, ny, nz, \
                     k, omega_df, omega64, it, fnorm, bpi, r_out, partials);                                   \
        else                                                                                                  \
            QBVM_PDL(k_residual_df4_batched<E, D, long long>, nb, RES_THREADS, 0, s, yy, f, delta_rhs, tb.nt, nx,    \
                     ny, nz, k, omega_df, omega64, it, fnorm, bpi, r_out, partials);                           \
    } while (0)
    if (tb.dim == 1) QBVM_RDB(true, 1);
    else if (tb.dim == 2) { if (eq) QBVM_RDB(true, 2); else QBVM_RDB(false, 2); }
    else { if (eq) QBVM_RDB(true, 3); else QBVM_RDB(false, 3); }
#undef QBVM_RDB
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long thr = count * 32;
    QBVM_PDL(k_reduce_instances, (unsigned)((thr + 255) / 256), 256, 0, s, partials, bpi, count, sums);
    return cudaGetLastError();
}

cudaError_t launch_df_to_double(void* buf, long long n, cudaStream_t s) {
    if ((reinterpret_cast<uintptr_t>(buf) & 15) == 0) {
        long long blocks = ((n >> 2) + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        if (blocks < 1) blocks = 1;
        QBVM_PDL(k_df_to_double4, (unsigned)blocks, 256, 0, s, buf, n);
        return cudaGetLastError();
    }
    long long blocks = (n + 1023) / 1024;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (blocks < 1) blocks = 1;
    QBVM_PDL(k_df_to_double, (unsigned)blocks, 256, 0, s, buf, n);
    return cudaGetLastError();
}

// flags[0] = 1 if any of x[0..n) is NaN or infinite (exponent field all
// ones), flags[1] = 1 if any is nonzero; tested on the words of each value
// (integer pipes).
__global__ void k_classify(const double* __restrict__ x, long long n, int* flags) {
    int bad = 0, nonzero = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned int h = qbvm_dhi(x[i]), l = qbvm_dlo(x[i]);
        bad |= ((h >> 20) & 0x7FFu) == 0x7FFu;
        nonzero |= ((h << 1) | l) != 0u;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, 1);
    if (__syncthreads_or(nonzero) && threadIdx.x == 0) atomicOr(flags + 1, 1);
}

cudaError_t launch_classify(const double* x, long long n, int* flags, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_classify<<<(unsigned)blocks, 256, 0, s>>>(x, n, flags);
    return cudaGetLastError();
}

int residual_blocks(const Tables& tb) {
    long long rows = (long long)tb.nt * tb.n[1] * tb.n[2];
    long long b = rows;
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
    QBVM_PDL(k_reduce_pairs, 1, 1024, 0, s, partials, nblocks, sums);
    return cudaGetLastError();
}

}  // namespace qbvm
