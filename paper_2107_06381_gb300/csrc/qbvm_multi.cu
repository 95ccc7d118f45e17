// qbvm_multi.cu -- full PinT-QBVM / PinT-MQBVM solves (every time level) of
// many instances of uneven shape, each with its own alpha and right-hand
// side, in ONE persistent kernel launch replayed from a captured CUDA graph.
//
// Every instance is an ordinary FP64 space-first plan (qbvm_plan builds its
// tables: sine roots and sines per axis, gamma^t, the Step (b) reciprocals
// cnorm / (d_{2m} + tau Lambda_l), and for the delta right-hand side one level
// of workspace).  The kernel runs the three steps of eq. 3.8 for all of them
// as one work queue of tiles, in topological order:
//   DX, DY, DZ   forward DST-I along x, y, z (of g for the delta right-hand
//                side, of every level of F otherwise), in place after DX;
//   TS           the time solve per tile of spatial modes (Steps (a)-(c));
//   IX, IY, IZ   the inverse DST-I of every level, in place in y.
// A stage of an instance starts when every tile of the instance's previous
// stage is done (per-instance counters); the tiles of different instances and
// stages interleave freely.  Items are claimed with an atomic ticket in queue
// order and every CTA of the grid is resident, so the smallest unfinished
// item is always being worked on; the waits are bounded anyway and give up
// with an error flag (QBVM_ERR_TIMEOUT from qbvm_multi_check).  Data written
// earlier in the launch by other CTAs is read through L2 (ld.global.cg).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "qbvm.h"
#include "qbvm_dst.cuh"
#include "qbvm_internal.h"
#include "qbvm_timesolve.cuh"

namespace {

enum MStage { MS_DX = 0, MS_DY, MS_DZ, MS_TS, MS_IX, MS_IY, MS_IZ, MS_N };

constexpr int M_THREADS = qbvm::TILE_THREADS;
constexpr int M_TIME_TILE = 4096;                 // complex values of one FP64 time-solve tile
constexpr long long M_SPIN_LIMIT = 1ll << 22;     // bounded waits (about half a second with the back-off)

struct MInst {
    int dim, delta, nt, lh, tlw;
    int n[3], lm[3], lw[3];
    long long Nx;
    int tiles[MS_N];
    int prev[MS_N];                  // the stage each stage waits for (-1: none)
    const double* in;                // g (one level) or F [nt][Nx]
    double* y;                       // [nt][Nx]
    double* ghat;                    // delta right-hand side: the DST of g
    const double2* tw_s[3];
    const double* sn_s[3];
    const double2 *tw_t, *gpow, *gipw, *gpowr, *gipr, *qinv;
};

struct MRun {
    const MInst* inst;
    const int4* items;
    int nitems;
    int* counters;                   // count x MS_N
    int* next;
    int* errflag;
};

__device__ __forceinline__ int ld_vol(const int* p) { return *(const volatile int*)p; }

// Thread 0 waits until *counter >= target (bounded); every thread learns the outcome.
__device__ bool m_wait(const int* counter, int target, int* errflag) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        long long it = 0;
        int good = 1;
        while (ld_vol(counter) < target) {
            if (ld_vol(errflag) != 0 || ++it > M_SPIN_LIMIT) {
                good = 0;
                atomicCAS(errflag, 0, 1);
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    const int r = ok;
    __syncthreads();
    return r != 0;
}

// One DST tile along axis ax of `lev` levels of `buf` (in -> out); LM > 0
// fixes the transform length (and so the tile width) at compile time, as the
// per-pass kernels do, so that the tile's loops unroll without spilling.
template <int LM>
__device__ __noinline__ void m_dst_l(const MInst& I, int ax, const double* in, double* out, long long lev, int tile,
                                     unsigned char* smem) {
    const long long nx = I.n[0], ny = I.n[1], nz = I.n[2];
    long long outer, inner;
    if (ax == 0) {
        outer = lev * ny * nz;
        inner = 1;
    } else if (ax == 1) {
        outer = lev * nz;
        inner = nx;
    } else {
        outer = lev;
        inner = nx * ny;
    }
    const int lm = LM > 0 ? LM : I.lm[ax];
    const int lw = LM > 0 ? 11 - LM : I.lw[ax];          // M * W = DST_TILE
    qbvm::dst_tile<double, double, 0, qbvm::DST_TILE / 4 / M_THREADS, true, true, false>(
        in, out, (1 << lm) - 1, lm, lw, outer, inner, tile, I.tw_s[ax], I.sn_s[ax], smem);
}
__device__ __forceinline__ void m_dst(const MInst& I, int ax, const double* in, double* out, long long lev, int tile,
                                      unsigned char* smem) {
    switch (I.lm[ax]) {
        case 6: m_dst_l<6>(I, ax, in, out, lev, tile, smem); break;
        case 7: m_dst_l<7>(I, ax, in, out, lev, tile, smem); break;
        case 8: m_dst_l<8>(I, ax, in, out, lev, tile, smem); break;
        case 9: m_dst_l<9>(I, ax, in, out, lev, tile, smem); break;
        default: m_dst_l<0>(I, ax, in, out, lev, tile, smem); break;
    }
}

// The time-solve tile, its half length LH > 0 fixed at compile time (common
// lengths), else taken at run time.
template <int LH>
__device__ __noinline__ void m_time_l(const MInst& I, int tile, unsigned char* smem) {
    const double* src = I.delta ? I.ghat : I.y;
    const int lh = LH > 0 ? LH : I.lh;
    const int lw = LH > 0 ? 12 - LH : I.tlw;             // H * W = M_TIME_TILE
    qbvm::time_solve_tile<double, M_TIME_TILE / 4 / M_THREADS, true, false>(
        src, I.y, I.Nx, lh, lw, I.tw_t, I.gpow, I.gipw, nullptr, nullptr, 0.0, I.gpowr, I.gipr, I.qinv, I.delta, 0,
        tile, smem);
}
__device__ __forceinline__ void m_time(const MInst& I, int tile, unsigned char* smem) {
    switch (I.lh) {
        case 5: m_time_l<5>(I, tile, smem); break;
        case 6: m_time_l<6>(I, tile, smem); break;
        case 7: m_time_l<7>(I, tile, smem); break;
        case 8: m_time_l<8>(I, tile, smem); break;
        default: m_time_l<0>(I, tile, smem); break;
    }
}

__global__ void __launch_bounds__(M_THREADS, 2) k_multi(MRun run) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    __shared__ MInst I;
    for (;;) {
        if (threadIdx.x == 0) s_item = ld_vol(run.errflag) ? run.nitems : atomicAdd(run.next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= run.nitems) return;
        const int4 w = run.items[it];
        if (threadIdx.x == 0) I = run.inst[w.y];
        __syncthreads();
        int* cnt = run.counters + (long long)w.y * MS_N;
        const int pv = I.prev[w.x];
        if (pv >= 0 && !m_wait(cnt + pv, I.tiles[pv], run.errflag)) return;
        const long long levf = I.delta ? 1 : I.nt;       // levels of the forward DSTs
        double* fwd = I.delta ? I.ghat : I.y;
        switch (w.x) {
            case MS_DX: m_dst(I, 0, I.in, fwd, levf, w.z, smem); break;
            case MS_DY: m_dst(I, 1, fwd, fwd, levf, w.z, smem); break;
            case MS_DZ: m_dst(I, 2, fwd, fwd, levf, w.z, smem); break;
            case MS_TS: m_time(I, w.z, smem); break;
            case MS_IX: m_dst(I, 0, I.y, I.y, I.nt, w.z, smem); break;
            case MS_IY: m_dst(I, 1, I.y, I.y, I.nt, w.z, smem); break;
            case MS_IZ: m_dst(I, 2, I.y, I.y, I.nt, w.z, smem); break;
            default: break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(cnt + w.x, 1);
        }
    }
}

bool is_p2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int log2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

struct qbvm_multi {
    int count = 0;
    std::vector<qbvm_plan_t*> plans;
    std::vector<MInst> host;
    std::vector<void*> allocs;
    MInst* d_inst = nullptr;
    int4* d_items = nullptr;
    int nitems = 0;
    int* d_counters = nullptr;       // count x MS_N, then `next`, then the error flag
    int grid = 0;
    size_t smem = 0;
    long long unknowns = 0;
    cudaGraphExec_t graph = nullptr;
};

namespace {

void m_destroy(qbvm_multi_t* mp) {
    if (!mp) return;
    if (mp->graph) cudaGraphExecDestroy(mp->graph);
    for (void* v : mp->allocs) cudaFree(v);
    for (qbvm_plan_t* p : mp->plans) qbvm_destroy(p);
    delete mp;
}

template <typename T>
int m_upload(qbvm_multi_t* mp, T** ptr, const std::vector<T>& h) {
    void* v = nullptr;
    if (cudaMalloc(&v, std::max<size_t>(1, h.size()) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_OOM;
    }
    mp->allocs.push_back(v);
    *ptr = static_cast<T*>(v);
    if (!h.empty() && cudaMemcpy(v, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    return QBVM_OK;
}

bool device_ptr(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

extern "C" {

int qbvm_multi_plan(const qbvm_multi_instance* inst, int count, qbvm_multi_t** out) {
    if (!inst || !out || count < 1) return QBVM_ERR_BAD_ARG;
    *out = nullptr;
    // host-side checks first: the shapes the persistent tiles take
    for (int i = 0; i < count; ++i) {
        const qbvm_desc& d = inst[i].desc;
        int rc = qbvm::validate_desc(&d);
        if (rc) return rc;
        if (!inst[i].g_or_F || !inst[i].y) return QBVM_ERR_BAD_ARG;
        if (d.precision != QBVM_FP64 || d.order == QBVM_ORDER_TIME_FIRST) return QBVM_ERR_UNSUPPORTED;
        if (!is_p2(d.nt) || d.nt > 1024) return QBVM_ERR_UNSUPPORTED;
        for (int a = 0; a < d.dim; ++a)
            if (!is_p2(d.m[a]) || d.m[a] < 4 || d.m[a] > 2048) return QBVM_ERR_UNSUPPORTED;
    }
    qbvm_multi_t* mp = new (std::nothrow) qbvm_multi();
    if (!mp) return QBVM_ERR_OOM;
    mp->count = count;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        m_destroy(mp);
        return QBVM_ERR_CUDA;
    }
    std::vector<int4> items;
    size_t smem = 0;
    for (int i = 0; i < count; ++i) {
        qbvm_desc d = inst[i].desc;
        d.order = QBVM_ORDER_SPACE_FIRST;
        if (!device_ptr(inst[i].g_or_F, dev) || !device_ptr(inst[i].y, dev)) {
            m_destroy(mp);
            return QBVM_ERR_BAD_ARG;
        }
        qbvm_plan_t* p = nullptr;
        int rc = qbvm_plan(&d, &p);
        if (rc) {
            m_destroy(mp);
            return rc;
        }
        mp->plans.push_back(p);
        qbvm::PlanView v;
        qbvm::plan_view(p, &v);
        const qbvm::Tables& tb = *v.tb;
        MInst I{};
        I.dim = d.dim;
        I.delta = d.rhs_kind == QBVM_RHS_DELTA;
        I.nt = d.nt;
        I.lh = log2i(d.nt) - 1;
        if (I.lh < 0) I.lh = 0;
        I.tlw = std::max(0, log2i(M_TIME_TILE) - I.lh);
        I.Nx = tb.Nx;
        for (int a = 0; a < 3; ++a) {
            I.n[a] = tb.n[a];
            I.lm[a] = a < d.dim ? log2i(d.m[a]) : 0;
            I.lw[a] = a < d.dim ? qbvm::dst_lw(I.lm[a]) : 0;
            I.tw_s[a] = tb.tw_s[a];
            I.sn_s[a] = tb.sn_s[a];
        }
        I.in = inst[i].g_or_F;
        I.y = inst[i].y;
        I.ghat = v.ghat;
        I.tw_t = tb.tw_t;
        I.gpow = tb.gpow;
        I.gipw = tb.gipw;
        I.gpowr = tb.gpowr;
        I.gipr = tb.gipr;
        I.qinv = tb.qinv;
        if (!I.qinv || (I.delta && !I.ghat)) {
            m_destroy(mp);
            return QBVM_ERR_UNSUPPORTED;
        }
        // tiles per stage
        const long long nx = I.n[0], ny = I.n[1], nz = I.n[2];
        auto dst_tiles = [&](int ax, long long lev) -> long long {
            const long long W2 = 2LL << I.lw[ax];
            if (ax == 0) return (lev * ny * nz + W2 - 1) / W2;
            if (ax == 1) return lev * nz * ((nx + W2 - 1) / W2);
            return lev * ((nx * ny + W2 - 1) / W2);
        };
        const long long levf = I.delta ? 1 : I.nt;
        long long t[MS_N] = {dst_tiles(0, levf), d.dim >= 2 ? dst_tiles(1, levf) : 0,
                             d.dim == 3 ? dst_tiles(2, levf) : 0, (I.Nx + (1LL << I.tlw) - 1) >> I.tlw,
                             dst_tiles(0, I.nt), d.dim >= 2 ? dst_tiles(1, I.nt) : 0,
                             d.dim == 3 ? dst_tiles(2, I.nt) : 0};
        int last = -1;
        for (int st = 0; st < MS_N; ++st) {
            if (t[st] > 0x3fffffffLL) {
                m_destroy(mp);
                return QBVM_ERR_UNSUPPORTED;
            }
            I.tiles[st] = (int)t[st];
            I.prev[st] = t[st] > 0 ? last : -1;
            if (t[st] > 0) last = st;
        }
        for (int a = 0; a < d.dim; ++a) smem = std::max(smem, qbvm::dst_smem_bytes<double>(I.lm[a]));
        smem = std::max(smem, sizeof(double2) * (((size_t)1 << (I.lh + I.tlw)) + ((size_t)1 << I.lh)));
        mp->host.push_back(I);
        mp->unknowns += tb.Nx * d.nt;
    }
    // the queue: stage by stage, instance by instance (every dependency has a smaller ticket)
    for (int st = 0; st < MS_N; ++st)
        for (int i = 0; i < count; ++i)
            for (int k = 0; k < mp->host[i].tiles[st]; ++k) items.push_back(make_int4(st, i, k, 0));
    if (items.size() > 0x7fffffffULL) {
        m_destroy(mp);
        return QBVM_ERR_UNSUPPORTED;
    }
    mp->nitems = (int)items.size();
    mp->smem = smem;
    int rc = m_upload(mp, &mp->d_inst, mp->host);
    if (!rc) rc = m_upload(mp, &mp->d_items, items);
    if (!rc) rc = m_upload(mp, &mp->d_counters, std::vector<int>((size_t)count * MS_N + 2, 0));
    if (!rc) {
        int per_sm = 0, sms = 0;
        if (cudaFuncSetAttribute(k_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi, M_THREADS, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            rc = QBVM_ERR_CUDA;
        }
        mp->grid = std::min(per_sm * sms, std::max(1, mp->nitems));     // every CTA resident
    }
    if (rc) {
        m_destroy(mp);
        return rc;
    }
    *out = mp;
    return QBVM_OK;
}

int qbvm_multi_run(qbvm_multi_t* mp, void* stream) {
    if (!mp) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!mp->graph) {
        // capture once: counter reset + the persistent launch; replayed by every run
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return QBVM_ERR_CUDA;
        }
        MRun run{mp->d_inst, mp->d_items, mp->nitems, mp->d_counters,
                 mp->d_counters + (size_t)mp->count * MS_N, mp->d_counters + (size_t)mp->count * MS_N + 1};
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            cudaMemsetAsync(mp->d_counters, 0, sizeof(int) * ((size_t)mp->count * MS_N + 2), cs);
            k_multi<<<mp->grid, M_THREADS, mp->smem, cs>>>(run);
            ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && g;
        }
        if (ok) ok = cudaGraphInstantiate(&mp->graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (!ok) {
            cudaGetLastError();
            mp->graph = nullptr;
            return QBVM_ERR_CUDA;
        }
    }
    if (cudaGraphLaunch(mp->graph, s) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    return QBVM_OK;
}

int qbvm_multi_check(qbvm_multi_t* mp, void* stream) {
    if (!mp) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int flag = 0;
    if (cudaMemcpyAsync(&flag, mp->d_counters + (size_t)mp->count * MS_N + 1, sizeof(int), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    return flag ? QBVM_ERR_TIMEOUT : QBVM_OK;
}

int qbvm_multi_info(const qbvm_multi_t* mp, long long* unknowns, int* work_items, int* grid) {
    if (!mp) return QBVM_ERR_BAD_ARG;
    if (unknowns) *unknowns = mp->unknowns;
    if (work_items) *work_items = mp->nitems;
    if (grid) *grid = mp->grid;
    return QBVM_OK;
}

int qbvm_multi_destroy(qbvm_multi_t* mp) {
    m_destroy(mp);
    return QBVM_OK;
}

}  // extern "C"
