// qbvm_plan.cu -- plan construction, orchestration and the C ABI of qbvm.h.
//
// A plan derives tau, alpha and omega (Sections 3.1/3.2, the a-priori rule of
// Section 5), builds the FP64 tables of the diagonalisation of Section 3.3
// on the host, uploads them, and owns the device workspace.  qbvm_solve
// enqueues the three steps of eq. 3.8 on the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qbvm.h"
#include "qbvm_internal.h"

using qbvm::Tables;

struct qbvm_plan {
    qbvm_desc d{};
    Tables tb{};
    int dev = 0;
    double alpha = 0, omega = 0, tau = 0;
    double h[3] = {1, 1, 1};
    double h2inv[3] = {0, 0, 0};
    int lp[3] = {0, 0, 0};
    // workspace
    double2* wk = nullptr;        // 1D: complex [nt][Nx]
    double2* wcp = nullptr;       // 1D: Thomas modified super-diagonal
    double* ghat = nullptr;       // 2D/3D delta rhs: DST of g (Nx)
    double* wreal = nullptr;      // 2D/3D general rhs with n0_only: [nt][Nx]
    double* partials = nullptr;   // residual partial sums
    float rscale = 0.f;           // 2^-k, 2^k <= rms(f) of the solve in progress (refinement residual norms)
    double* sums = nullptr;       // residual sums (2)
    int nres = 0;
    double* stage_in = nullptr;   // host-pointer staging
    double* stage_out = nullptr;
    // FP32 refinement workspace
    float* f32 = nullptr;         // [nt][Nx] FP32 work array (and the residual's r.hi)
    double* fcopy = nullptr;      // FP32_REFINE: copy of an F that aliases y
    int* flag = nullptr;          // FP32_REFINE: non-finite input test
    // host-pointer solves: a copy stream and events that pipeline the staging
    cudaStream_t copy_stream = nullptr;
    cudaStream_t aux_stream = nullptr;   // second compute stream for alternate chunks
    std::vector<cudaEvent_t> copy_events;
    float* g32 = nullptr;         // Nx FP32 (delta rhs)
    long long ws_bytes = 0;
    int last_iters = 0;
    double last_relres = 0.0;
    int kernels_per_solve = 0;
    std::vector<void*> allocs;
    // tracing: (kernel name, start, stop) per launch while profiling is on
    bool profiling = false;
    struct Mark { const char* name; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(long long v) { int l = 0; while ((1LL << l) < v) ++l; return l; }

// DST-I lengths n = m - 1 the kernels take: m a power of two in [4, 1024] by
// the radix-4/2 tiles, any other m in [2, 2048] by the mixed-radix tile.
bool dst_length_ok(int m) { return m >= 2 && m <= 2048; }
// Space-first always in 2D/3D; in 1D on request, or by default when m allows the DST.
bool space_first(const qbvm_desc* d) {
    if (d->dim > 1) return true;
    if (d->order == QBVM_ORDER_TIME_FIRST) return false;
    if (d->order == QBVM_ORDER_SPACE_FIRST) return true;
    return dst_length_ok(d->m[0]);
}

int validate(const qbvm_desc* d) {
    if (!d) return QBVM_ERR_BAD_ARG;
    if (d->dim < 1 || d->dim > 3) return QBVM_ERR_BAD_ARG;
    for (int i = 0; i < d->dim; ++i)
        if (d->m[i] < 2) return QBVM_ERR_BAD_ARG;
    if (d->nt < 2) return QBVM_ERR_BAD_ARG;
    if (!(d->T > 0) || !std::isfinite(d->T)) return QBVM_ERR_BAD_ARG;
    if (!(d->L > 0) || !std::isfinite(d->L)) return QBVM_ERR_BAD_ARG;
    if (d->form != QBVM_FORM_PQ && d->form != QBVM_FORM_PM) return QBVM_ERR_BAD_ARG;
    if (d->precision != QBVM_FP64 && d->precision != QBVM_FP32_REFINE) return QBVM_ERR_BAD_ARG;
    if (d->rhs_kind != QBVM_RHS_DELTA && d->rhs_kind != QBVM_RHS_GENERAL) return QBVM_ERR_BAD_ARG;
    if (!std::isfinite(d->alpha) || std::isnan(d->delta)) return QBVM_ERR_BAD_ARG;
    if (!(d->alpha > 0) && !(d->delta > 0 && std::isfinite(d->delta))) return QBVM_ERR_BAD_ARG;
    // sizes the kernels implement
    if (is_pow2(d->nt)) {
        if (d->nt > 1024) return QBVM_ERR_UNSUPPORTED;
    } else {
        // other lengths: Bluestein time DFTs of power-of-two length L >= 2 nt - 1 <= 4096
        if (d->nt > 2048) return QBVM_ERR_UNSUPPORTED;
    }
    if (d->order < QBVM_ORDER_AUTO || d->order > QBVM_ORDER_SPACE_FIRST) return QBVM_ERR_BAD_ARG;
    if (d->order == QBVM_ORDER_TIME_FIRST && d->dim != 1) return QBVM_ERR_BAD_ARG;
    const bool sf = space_first(d);
    if (d->precision == QBVM_FP32_REFINE && !sf) return QBVM_ERR_UNSUPPORTED;   // refinement runs space-first
    if (sf) {
        for (int i = 0; i < d->dim; ++i)
            if (!dst_length_ok(d->m[i])) return QBVM_ERR_UNSUPPORTED;
    } else if (d->m[0] - 1 > (1 << 20)) {
        return QBVM_ERR_UNSUPPORTED;
    }
    return QBVM_OK;
}

template <typename T>
int dalloc(qbvm_plan_t* p, T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) return QBVM_OK;
    void* v = nullptr;
    if (cudaMalloc(&v, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_OOM;
    }
    p->allocs.push_back(v);
    p->ws_bytes += (long long)(count * sizeof(T));
    *ptr = static_cast<T*>(v);
    return QBVM_OK;
}

template <typename T>
int upload(qbvm_plan_t* p, T** ptr, const std::vector<T>& host) {
    int rc = dalloc(p, ptr, host.size());
    if (rc) return rc;
    if (cudaMemcpy(*ptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return QBVM_ERR_CUDA;
    return QBVM_OK;
}

// exp(-2 pi i m / P) for m < P (FP64, angle reduced to pi * (2m/P) with 2m/P exact)
void roots(int P, std::vector<double2>& w64, std::vector<float2>& w32) {
    w64.resize(P);
    w32.resize(P);
    for (int m = 0; m < P; ++m) {
        double a = M_PI * (2.0 * m / P);
        double c = std::cos(a), s = -std::sin(a);
        w64[m] = make_double2(c, s);
        w32[m] = make_float2((float)c, (float)s);
    }
}

// Tables of the Bluestein time DFTs for nt not a power of two (Section 3.3,
// Steps (a) and (c) with every frequency): chirp c_m = exp(i pi m^2/nt), the
// transforms B = DFT_L(b)/L of the wrapped kernels b_m = conj(c_|m|) (for the
// +theta transform) and c_|m| (for -theta), gamma^t and gamma^{-t} for t < nt,
// d_k = 1 - gamma theta^k.  Angles are reduced exactly in integers
// (m^2 mod 2 nt, j m mod L) before the FP64 sine and cosine.
int bluestein_tables(qbvm_plan_t* p, double mag, double scale1d) {
    Tables& tb = p->tb;
    const int P = tb.nt;
    int lL = 0;
    while ((1 << lL) < 2 * P - 1) ++lL;
    const int L = 1 << lL;
    tb.gen = 1;
    tb.lL = lL;
    std::vector<double2> twL, chirp(P), bf(L), bi(L), gp(P), gi(P), dk(P);
    std::vector<float2> tw32;
    roots(L, twL, tw32);
    for (int m = 0; m < P; ++m) {
        const long long r = ((long long)m * m) % (2LL * P);
        const double a = M_PI * ((double)r / P);
        chirp[m] = make_double2(std::cos(a), std::sin(a));
    }
    std::vector<double2> kf(L, make_double2(0, 0)), ki(L, make_double2(0, 0));
    for (int m = 0; m < P; ++m) {
        const double2 c = chirp[m], cc = make_double2(c.x, -c.y);
        kf[m] = cc;
        ki[m] = c;
        if (m > 0) {
            kf[L - m] = cc;
            ki[L - m] = c;
        }
    }
    for (int j = 0; j < L; ++j) {                         // direct DFT_L with exp(-2 pi i j m / L)
        double fr = 0, fi = 0, ir = 0, ii = 0;
        for (int m = 0; m < L; ++m) {
            const double2 w = twL[((long long)j * m) % L];
            fr += kf[m].x * w.x - kf[m].y * w.y;
            fi += kf[m].x * w.y + kf[m].y * w.x;
            ir += ki[m].x * w.x - ki[m].y * w.y;
            ii += ki[m].x * w.y + ki[m].y * w.x;
        }
        bf[j] = make_double2(fr / L, fi / L);
        bi[j] = make_double2(ir / L, ii / L);
    }
    const double g1 = std::pow(mag, 1.0 / P);
    for (int t = 0; t < P; ++t) {
        const double a = M_PI * ((double)t / P);
        const double r = std::pow(mag, (double)t / P), ri = std::pow(mag, -(double)t / P);
        gp[t] = make_double2(scale1d * r * std::cos(a), scale1d * r * std::sin(a));
        gi[t] = make_double2(ri * std::cos(a), -ri * std::sin(a));
        const double b = M_PI * ((2.0 * t + 1.0) / P);   // arg(gamma theta^k), k = t
        dk[t] = make_double2(1.0 - g1 * std::cos(b), -g1 * std::sin(b));
    }
    int rc = upload(p, &tb.tw_L, twL);
    if (!rc) rc = upload(p, &tb.chirp, chirp);
    if (!rc) rc = upload(p, &tb.bs_fwd, bf);
    if (!rc) rc = upload(p, &tb.bs_inv, bi);
    if (!rc) rc = upload(p, &tb.gpw_full, gp);
    if (!rc) rc = upload(p, &tb.gip_full, gi);
    if (!rc) rc = upload(p, &tb.dk_full, dk);
    if (!rc && p->d.precision == QBVM_FP32_REFINE) {
        auto to32 = [](const std::vector<double2>& v) {
            std::vector<float2> o(v.size());
            for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
            return o;
        };
        rc = upload(p, &tb.tw_L32, tw32);
        if (!rc) rc = upload(p, &tb.chirp32, to32(chirp));
        if (!rc) rc = upload(p, &tb.bs_fwd32, to32(bf));
        if (!rc) rc = upload(p, &tb.bs_inv32, to32(bi));
        if (!rc) rc = upload(p, &tb.gpw_full32, to32(gp));
        if (!rc) rc = upload(p, &tb.gip_full32, to32(gi));
        if (!rc) rc = upload(p, &tb.dk_full32, to32(dk));
    }
    return rc;
}

void destroy_plan(qbvm_plan_t* p) {
    if (!p) return;
    for (cudaEvent_t e : p->copy_events) cudaEventDestroy(e);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->aux_stream) cudaStreamDestroy(p->aux_stream);
    for (void* v : p->allocs) cudaFree(v);
    for (auto& m : p->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    delete p;
}

cudaEvent_t take_event(qbvm_plan_t* p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Brackets one kernel launch with events when the plan is profiling.
// One stage of a solve: an NVTX range around its launches (header-only NVTX;
// a no-op without a tool attached) and, while profiling is on, CUDA events
// on the stream around its kernel.
struct Span {
    qbvm_plan_t* p;
    const char* name;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Span(qbvm_plan_t* p_, const char* n, cudaStream_t s_) : p(p_), name(n), s(s_) {
        nvtxRangePushA(n);
        if (p->profiling && (a = take_event(p)) != nullptr) cudaEventRecord(a, s);
    }
    ~Span() {
        nvtxRangePop();
        if (!a) return;
        cudaEvent_t b = take_event(p);
        if (!b) {
            p->event_pool.push_back(a);
            return;
        }
        cudaEventRecord(b, s);
        p->marks.push_back({name, a, b});
    }
};

enum { KIND_DEV = 0, KIND_HOST = 1, KIND_FOREIGN = 2 };
// Device memory of the plan's device `dev` (or managed memory), host memory,
// or device memory of another GPU (KIND_FOREIGN: the plan's kernels would read
// it as a peer, an illegal address without peer mapping; refused as BAD_ARG).
int ptr_kind(const void* ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return KIND_HOST;
    }
    if (a.type == cudaMemoryTypeManaged) return KIND_DEV;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? KIND_DEV : KIND_FOREIGN;
    return KIND_HOST;
}

#define CK(...)                                     \
    do {                                            \
        cudaError_t e__ = (__VA_ARGS__);            \
        if (e__ != cudaSuccess) return QBVM_ERR_CUDA; \
    } while (0)

// --- FP64 pipeline on device pointers -------------------------------------

// Normalisation of the FP64 space-first solve: the inverse-DST factors 2/(n+1)
// per axis, 1/nt of the inverse time DFT, and 4^(-2 dim) for the FP64 DSTs,
// which produce 4x the transform (an exact power of two).
double fp64_cn(const Tables& tb) {
    double cn = 1.0;
    for (int i = 0; i < tb.dim; ++i) cn *= 2.0 / (tb.n[i] + 1);
    cn /= tb.nt;
    return std::ldexp(cn, -4 * tb.dim);
}
// The time-solve constant of the plan's right-hand side kind.
double fp64_cnorm(const qbvm_plan_t* p) {
    const double cn = fp64_cn(p->tb);
    return p->d.rhs_kind == QBVM_RHS_DELTA ? -p->tb.omega * cn : p->tb.tau * cn;
}

// FP64 space-first solve in three phases, so that the host-pointer path can
// overlap its copies with the per-level DSTs.
// DST-I along every axis of the levels [l0, l1) of [nt][Nx] arrays, in -> out.
int fp64_dst_levels(qbvm_plan_t* p, const double* in, double* out, long long l0, long long l1, cudaStream_t s,
                    int* launches) {
    const Tables& tb = p->tb;
    const long long nx = tb.n[0], ny = tb.n[1], nz = tb.n[2], lev = l1 - l0, off = l0 * tb.Nx;
    { Span sp_(p, "dst_x", s); CK(qbvm::launch_dst<double, double, 0, true>(in + off, out + off, tb.n[0], p->lp[0], lev * ny * nz, 1, tb.tw_s[0], tb.sn_s[0], s)); }
    if (tb.dim >= 2) { Span sp_(p, "dst_y", s); CK(qbvm::launch_dst<double, double, 0, true>(out + off, out + off, tb.n[1], p->lp[1], lev * nz, nx, tb.tw_s[1], tb.sn_s[1], s)); }
    if (tb.dim == 3) { Span sp_(p, "dst_z", s); CK(qbvm::launch_dst<double, double, 0, true>(out + off, out + off, tb.n[2], p->lp[2], lev, nx * ny, tb.tw_s[2], tb.sn_s[2], s)); }
    *launches += tb.dim;
    return QBVM_OK;
}

// Steps (a)-(c) in time for every spatial mode: the sine-basis spectrum `spec`
// (one level for the delta right-hand side, [nt][Nx] otherwise) -> y.
int fp64_time_part(qbvm_plan_t* p, const double* spec, double* y, int delta, int n0_only, cudaStream_t s,
                   int* launches) {
    const Tables& tb = p->tb;
    const double cn = fp64_cn(tb);
    // f^0 = -omega g / tau: fold -omega/tau into the time-solve constant
    const double cnorm = delta ? -tb.omega * cn : tb.tau * cn;
    if (delta && n0_only && tb.y0fac) {
        // y^0 only: Step (c) at t = 0 of a constant spectrum is one factor per mode
        { Span sp_(p, "y0_modes", s); CK(qbvm::launch_mul_modes(spec, tb.y0fac, y, tb.Nx, s)); }
        *launches += 1;
    } else if (tb.gen) {
        { Span sp_(p, "time_fwd", s); CK(qbvm::launch_bluestein(0, spec, p->wk, tb.Nx, tb, cnorm, delta, 0, s)); }
        { Span sp_(p, "time_inv", s); CK(qbvm::launch_bluestein(2, p->wk, y, tb.Nx, tb, 0.0, 0, n0_only, s)); }
        *launches += 2;
    } else {
        { Span sp_(p, "time_solve", s); CK(qbvm::launch_time_solve<double>(spec, y, tb, cnorm, delta, n0_only, s)); }
        *launches += 1;
    }
    return QBVM_OK;
}

int solve_fp64_dev(qbvm_plan_t* p, const double* in, double* y, int n0_only, cudaStream_t s) {
    const Tables& tb = p->tb;
    const int delta = p->d.rhs_kind == QBVM_RHS_DELTA;
    int launches = 0;
    if (!tb.sf && tb.gen) {
        // general nt: Bluestein time DFTs over every frequency, Thomas for each
        { Span sp_(p, "time_fwd_1d", s); CK(qbvm::launch_bluestein(1, in, p->wk, tb.Nx, tb, delta ? -tb.omega / tb.tau : 1.0, delta, 0, s)); }
        { Span sp_(p, "thomas_1d", s); CK(qbvm::launch_thomas_1d_n(p->wk, p->wcp, tb.nt, tb, s)); }
        { Span sp_(p, "time_inv_1d", s); CK(qbvm::launch_bluestein(2, p->wk, y, tb.Nx, tb, 0.0, 0, n0_only, s)); }
        launches = 3;
    } else if (!tb.sf) {
        // Step (a), Step (b) (Thomas per frequency), Step (c)
        { Span sp_(p, "time_fwd_1d", s); CK(qbvm::launch_time_fwd_1d(in, p->wk, tb, delta, delta ? -tb.omega / tb.tau : 1.0, s)); }
        { Span sp_(p, "thomas_1d", s); CK(qbvm::launch_thomas_1d(p->wk, p->wcp, tb, s)); }
        { Span sp_(p, "time_inv_1d", s); CK(qbvm::launch_time_inv_1d(p->wk, y, tb, n0_only, s)); }
        launches = 3;
    } else {
        if (delta) {
            // DST of g along every axis -> ghat, then the time part reads level 0
            int rc = fp64_dst_levels(p, in, p->ghat, 0, 1, s, &launches);
            if (!rc) rc = fp64_time_part(p, p->ghat, y, 1, n0_only, s, &launches);
            if (rc) return rc;
        } else {
            double* work = n0_only ? p->wreal : y;
            int rc = fp64_dst_levels(p, in, work, 0, tb.nt, s, &launches);
            if (!rc) rc = fp64_time_part(p, work, y, 0, n0_only, s, &launches);
            if (rc) return rc;
        }
        // inverse DST (the (2/M) factors are in the time-solve constant)
        int rc = fp64_dst_levels(p, y, y, 0, n0_only ? 1 : tb.nt, s, &launches);
        if (rc) return rc;
    }
    p->kernels_per_solve = launches;
    return QBVM_OK;
}

// --- FP32 transforms + iterative refinement (2D/3D) ---------------------------
//
// y_0 = A32^{-1} f;  repeat: r = f - A y, stop when ||r||/||f|| <= tol, else
// y += A32^{-1} r.  A32^{-1} is the space-first pipeline in FP32 (roots,
// gamma^t, d_k and tau*Lambda computed in FP64 on the host and rounded once).
// The iterate y and the residual are carried in double-float (hi + lo, ~48
// significand bits, computed on the FP32 pipes: GB300 runs FP64 at 1/64 of
// the FP32 rate); y is stored as float2 pairs in the caller's 8-byte-per-value
// output array and converted to FP64 in place at the end.

int fp32_solve(qbvm_plan_t* p, const void* rhs, int rhs_fp64, int delta, void* ydf, int accumulate,
               cudaStream_t s) {
    const Tables& tb = p->tb;
    const long long nx = tb.n[0], ny = tb.n[1], nz = tb.n[2], nt = tb.nt;
    double cn = 1.0;
    for (int i = 0; i < tb.dim; ++i) cn *= 2.0 / (tb.n[i] + 1);
    cn /= tb.nt;
    float* w = p->f32;
    if (delta) {
        { Span sp_(p, "dst_x", s); CK(qbvm::launch_dst<float, double, 0>((const double*)rhs, p->g32, tb.n[0], p->lp[0], ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s)); }
        if (tb.dim >= 2) { Span sp_(p, "dst_y", s); CK(qbvm::launch_dst<float, float, 0>(p->g32, p->g32, tb.n[1], p->lp[1], nz, nx, tb.tw_s32[1], tb.sn_s32[1], s)); }
        if (tb.dim == 3) { Span sp_(p, "dst_z", s); CK(qbvm::launch_dst<float, float, 0>(p->g32, p->g32, tb.n[2], p->lp[2], 1, nx * ny, tb.tw_s32[2], tb.sn_s32[2], s)); }
        if (tb.gen) {
            // nt not a power of two: Bluestein time DFTs (every frequency) in FP32
            { Span sp_(p, "time_fwd", s); CK(qbvm::launch_bluestein32(0, p->g32, p->wk, tb.Nx, tb, (float)(-tb.omega * cn), 1, 0, s)); }
            { Span sp_(p, "time_inv", s); CK(qbvm::launch_bluestein32(2, p->wk, w, tb.Nx, tb, 0.f, 0, 0, s)); }
        } else {
            Span sp_(p, "time_solve", s);
            CK(qbvm::launch_time_solve<float>(p->g32, w, tb, -tb.omega * cn, 1, 0, s));
        }
    } else {
        if (rhs_fp64) { Span sp_(p, "dst_x", s); CK(qbvm::launch_dst<float, double, 0>((const double*)rhs, w, tb.n[0], p->lp[0], nt * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s)); }
        else { Span sp_(p, "dst_x", s); CK(qbvm::launch_dst<float, float, 0>((const float*)rhs, w, tb.n[0], p->lp[0], nt * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s)); }
        if (tb.dim >= 2) { Span sp_(p, "dst_y", s); CK(qbvm::launch_dst<float, float, 0>(w, w, tb.n[1], p->lp[1], nt * nz, nx, tb.tw_s32[1], tb.sn_s32[1], s)); }
        if (tb.dim == 3) { Span sp_(p, "dst_z", s); CK(qbvm::launch_dst<float, float, 0>(w, w, tb.n[2], p->lp[2], nt, nx * ny, tb.tw_s32[2], tb.sn_s32[2], s)); }
        if (tb.gen) {
            { Span sp_(p, "time_fwd", s); CK(qbvm::launch_bluestein32(0, w, p->wk, tb.Nx, tb, (float)(tb.tau * cn), 0, 0, s)); }
            { Span sp_(p, "time_inv", s); CK(qbvm::launch_bluestein32(2, p->wk, w, tb.Nx, tb, 0.f, 0, 0, s)); }
        } else {
            Span sp_(p, "time_solve", s);
            CK(qbvm::launch_time_solve<float>(w, w, tb, tb.tau * cn, 0, 0, s));
        }
    }
    if (tb.dim == 3) { Span sp_(p, "dst_z", s); CK(qbvm::launch_dst<float, float, 0>(w, w, tb.n[2], p->lp[2], nt, nx * ny, tb.tw_s32[2], tb.sn_s32[2], s)); }
    if (tb.dim >= 2) { Span sp_(p, "dst_y", s); CK(qbvm::launch_dst<float, float, 0>(w, w, tb.n[1], p->lp[1], nt * nz, nx, tb.tw_s32[1], tb.sn_s32[1], s)); }
    if (accumulate) {
        Span sp_(p, "dst_x", s);
        CK(qbvm::launch_dst<float, float, 1>(w, ydf, tb.n[0], p->lp[0], nt * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s));
    } else {
        Span sp_(p, "dst_x", s);
        CK(qbvm::launch_dst<float, float, 2>(w, ydf, tb.n[0], p->lp[0], nt * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s));
    }
    return QBVM_OK;
}

// ||f - A y|| / ||f|| with r.hi written to p->f32.  *fnorm2 < 0 on entry: sum
// ||f||^2 too and return it there (the first residual of a solve); otherwise
// it holds ||f||^2 from that first call.
int residual_norm_df(qbvm_plan_t* p, const void* ydf, const double* in, int delta, double* rel, double* fnorm2,
                     cudaStream_t s) {
    const int want_f = *fnorm2 < 0;
    // after the first residual ||r||^2 is a plain FP32 sum of (r / 2^k)^2, 2^k the
    // power of two at or below rms(f) (2D / 3D; 1D sums in FP64)
    const float rscale = want_f ? 0.f : p->rscale;
    { Span sp_(p, "residual_df", s); CK(qbvm::launch_residual_df(ydf, in, delta, p->tb, p->h2inv, p->f32, p->partials, p->nres, p->sums, want_f, s, rscale)); }
    double h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, p->sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (want_f) {
        *fnorm2 = h[1];
        const double cnt = (double)p->tb.Nx * (delta ? 1 : p->tb.nt);
        const double rms = std::sqrt(h[1] / cnt);
        p->rscale = (std::isfinite(rms) && rms > 1e-30 && rms < 1e30) ? (float)std::ldexp(1.0, -(int)std::floor(std::log2(rms))) : 0.f;
    } else {
        h[1] = *fnorm2;
    }
    if (!want_f && rscale > 0.f && h[0] == INFINITY && std::isfinite(h[1])) {
        *rel = INFINITY;                              // (r / 2^k)^2 beyond the FP32 range: the iteration diverges
        return QBVM_OK;
    }
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return QBVM_ERR_NONFINITE;
    *rel = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return QBVM_OK;
}

// FP32 holds the right-hand side and the residuals of the refinement only for
// data of moderate magnitude; outside [FP32_RMS_LO, FP32_RMS_HI] (root mean
// square of f over its nonzero-capable entries) the plan's FP64 pipeline solves.
constexpr double FP32_RMS_LO = 1e-18, FP32_RMS_HI = 1e28;

int solve_fp32r_dev(qbvm_plan_t* p, const double* in, double* y, int n0_only, cudaStream_t s) {
    const Tables& tb = p->tb;
    const int delta = p->d.rhs_kind == QBVM_RHS_DELTA;
    double* yfull = n0_only ? p->wreal : y;        // holds the double-float iterate, 8 bytes per value
    const double tol = p->d.refine_tol > 0 ? p->d.refine_tol : 1e-13;
    const int maxit = p->d.refine_max_iters > 0 ? p->d.refine_max_iters : 10;
    int rc = fp32_solve(p, in, 1, delta, yfull, 0, s);
    if (rc) return rc;
    const int launches_solve = 2 * tb.dim + (tb.gen ? 2 : 1);
    int launches = launches_solve;
    double rel = 0.0, prev = INFINITY;
    int it = 0;
    int status = QBVM_OK;
    bool first = true;
    double fn2 = -1.0;                               // ||f||^2, summed by the first residual
    for (;;) {
        rc = residual_norm_df(p, yfull, in, delta, &rel, &fn2, s);     // r.hi lands in p->f32
        launches += 2;
        if (rc && !(first && rc == QBVM_ERR_NONFINITE)) return rc;
        if (first) {
            first = false;
            const double cnt = (double)tb.Nx * (delta ? 1 : tb.nt);
            const double rms = std::sqrt(fn2 / cnt);
            bool fp64 = rms > 0 && (rms < FP32_RMS_LO || rms > FP32_RMS_HI);
            if (rc == QBVM_ERR_NONFINITE || fn2 == 0.0) {
                // NaN or Inf in the input itself, or finite data FP32 cannot hold
                // (beyond its range, or so small that every value flushes to zero):
                // the former is an error, the latter goes to the FP64 pipeline
                if (!p->flag) {
                    rc = dalloc(p, &p->flag, 2);
                    if (rc) return rc;
                }
                int fl[2] = {0, 0};
                CK(qbvm::launch_classify(in, (long long)cnt, p->flag, s));
                CK(cudaMemcpyAsync(fl, p->flag, sizeof(fl), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                ++launches;
                if (fl[0]) return QBVM_ERR_NONFINITE;
                fp64 = fp64 || rc == QBVM_ERR_NONFINITE || fl[1];
                rc = QBVM_OK;
            }
            if (fp64) {
                rc = solve_fp64_dev(p, in, y, n0_only, s);     // wreal exists for n0_only (solve_dev)
                if (rc) return rc;
                double r64 = 0.0;
                if (!n0_only) {
                    rc = qbvm_residual(p, y, in, &r64, s);
                    if (rc) return rc;
                }
                p->last_iters = 0;
                p->last_relres = n0_only ? NAN : r64;
                p->kernels_per_solve = launches + p->kernels_per_solve;
                return QBVM_OK;
            }
        }
        if (rel <= tol) break;
        if (rel > 0.5 * prev) {
            // no contraction: the double-float floor if the residual is already tiny,
            // else the FP32 transforms are too inaccurate for this omega
            if (rel > 1e-10) status = QBVM_ERR_DIVERGED;
            break;
        }
        if (it >= maxit) {        // still contracting but the cap is reached above tol
            status = QBVM_ERR_DIVERGED;
            break;
        }
        prev = rel;
        rc = fp32_solve(p, p->f32, 0, 0, yfull, 1, s);
        if (rc) return rc;
        launches += launches_solve;
        ++it;
    }
    { Span sp_(p, "df_to_double", s); CK(qbvm::launch_df_to_double(yfull, tb.Nx * tb.nt, s)); }
    ++launches;
    if (n0_only) CK(cudaMemcpyAsync(y, yfull, sizeof(double) * tb.Nx, cudaMemcpyDeviceToDevice, s));
    p->last_iters = it;
    p->last_relres = rel;
    p->kernels_per_solve = launches;
    return status;
}

}  // namespace

int qbvm::validate_desc(const qbvm_desc* d) { return validate(d); }
double qbvm::time_cn(const Tables& tb) { return fp64_cn(tb); }

int qbvm::plan_view(const struct ::qbvm_plan* p, PlanView* out) {
    if (!p || !out) return QBVM_ERR_BAD_ARG;
    out->tb = &p->tb;
    out->form = p->d.form;
    out->precision = p->d.precision;
    out->rhs_kind = p->d.rhs_kind;
    out->dim = p->d.dim;
    out->dev = p->dev;
    out->ghat = p->ghat;
    out->alpha = p->alpha;
    out->tau = p->tau;
    for (int i = 0; i < 3; ++i) out->h2inv[i] = p->h2inv[i];
    return QBVM_OK;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

int qbvm_version(void) { return 100; }

const char* qbvm_strerror(int code) {
    switch (code) {
        case QBVM_OK: return "success";
        case QBVM_ERR_BAD_ARG: return "invalid argument or descriptor";
        case QBVM_ERR_OOM: return "out of memory";
        case QBVM_ERR_NONFINITE: return "non-finite value in input or result";
        case QBVM_ERR_DIVERGED: return "iteration stopped above its tolerance (FP32 refinement or GMRES)";
        case QBVM_ERR_TIMEOUT: return "a bounded device wait gave up";
        case QBVM_ERR_CUDA: return "CUDA runtime error";
        case QBVM_ERR_UNSUPPORTED: return "size not implemented by the kernels";
        default: return "unknown status code";
    }
}

int qbvm_plan(const qbvm_desc* desc, qbvm_plan_t** out) {
    if (!out) return QBVM_ERR_BAD_ARG;
    *out = nullptr;
    int rc = validate(desc);
    if (rc) return rc;
    qbvm_plan_t* p = new (std::nothrow) struct qbvm_plan();
    if (!p) return QBVM_ERR_OOM;
    p->d = *desc;
    const qbvm_desc& d = p->d;
    Tables& tb = p->tb;
    tb.dim = d.dim;
    tb.sf = space_first(&d) ? 1 : 0;
    tb.nt = d.nt;
    tb.lnt = ilog2(d.nt);
    tb.Nx = 1;
    for (int i = 0; i < 3; ++i) {
        tb.n[i] = i < d.dim ? d.m[i] - 1 : 1;
        p->h[i] = i < d.dim ? d.L / d.m[i] : 1.0;
        p->h2inv[i] = i < d.dim ? 1.0 / (p->h[i] * p->h[i]) : 0.0;
        tb.Nx *= tb.n[i];
    }
    p->tau = d.T / (d.nt - 1);
    p->alpha = d.alpha > 0 ? d.alpha : (d.form == QBVM_FORM_PQ ? d.delta : p->tau * d.delta);
    p->omega = d.form == QBVM_FORM_PQ ? -1.0 / p->alpha : -p->tau / p->alpha;
    tb.tau = p->tau;
    tb.omega = p->omega;
    if (!(std::isfinite(p->alpha) && p->alpha > 0 && std::isfinite(p->omega))) {
        delete p;
        return QBVM_ERR_BAD_ARG;
    }
    if (cudaGetDevice(&p->dev) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return QBVM_ERR_CUDA;
    }

    // ---- FP64 tables of Section 3.3 ----
    const int nt = d.nt, H = nt / 2;
    const double mag = std::fabs(p->omega);
    // principal root of omega < 0: gamma = |omega|^{1/nt} exp(i pi/nt)
    std::vector<double2> tw64, gpow(H), gipw(H), gpowr(H), gipr(H), ak(H), bk;
    std::vector<float2> tw32;
    roots(H, tw64, tw32);
    const double scale1d = !tb.sf ? p->h[0] * p->h[0] / nt : 1.0;   // time-first 1D: h^2 and 1/nt in gamma^t
    for (int t = 0; t < H; ++t) {
        double r = std::pow(mag, (double)t / nt);
        double a = M_PI * ((double)t / nt);
        gpow[t] = make_double2(scale1d * r * std::cos(a), scale1d * r * std::sin(a));
        double ri = 2.0 * std::pow(mag, -(double)t / nt);
        gipw[t] = make_double2(ri * std::cos(a), -ri * std::sin(a));
        // with rho^H = |omega|^{1/2} folded in: i rho^H gamma^t and rho^{-H} 2 gamma^{-t}
        double rr = std::pow(mag, (double)(t + H) / nt), rir = 2.0 * std::pow(mag, -(double)(t + H) / nt);
        gpowr[t] = make_double2(-scale1d * rr * std::sin(a), scale1d * rr * std::cos(a));
        gipr[t] = make_double2(rir * std::cos(a), -rir * std::sin(a));
    }
    tb.rho_h = std::sqrt(mag);
    tb.rho_hinv = 1.0 / tb.rho_h;
    const double g1 = std::pow(mag, 1.0 / nt);
    for (int m = 0; m < H; ++m) {
        double a = M_PI * ((4.0 * m + 1.0) / nt);        // arg(gamma theta^{2m})
        ak[m] = make_double2(1.0 - g1 * std::cos(a), -g1 * std::sin(a));
    }
    auto to32 = [](const std::vector<double2>& v) {
        std::vector<float2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
        return o;
    };
    rc = upload(p, &tb.tw_t, tw64);
    if (!rc) rc = upload(p, &tb.tw_t32, tw32);
    if (!rc) rc = upload(p, &tb.gpow, gpow);
    if (!rc) rc = upload(p, &tb.gipw, gipw);
    if (!rc) rc = upload(p, &tb.ak, ak);
    if (!rc) rc = upload(p, &tb.gpow32, to32(gpow));
    if (!rc) rc = upload(p, &tb.gipw32, to32(gipw));
    if (!rc) rc = upload(p, &tb.gpowr, gpowr);
    if (!rc) rc = upload(p, &tb.gipr, gipr);
    if (!rc) rc = upload(p, &tb.gpowr32, to32(gpowr));
    if (!rc) rc = upload(p, &tb.gipr32, to32(gipr));
    if (!rc) rc = upload(p, &tb.ak32, to32(ak));
    if (!rc && !is_pow2(nt)) rc = bluestein_tables(p, mag, scale1d);
    if (!rc && !tb.sf) {
        const double h2 = p->h[0] * p->h[0];
        if (tb.gen) {                                     // every frequency k < nt
            bk.resize(nt);
            const double g1n = std::pow(mag, 1.0 / nt);
            for (int k = 0; k < nt; ++k) {
                const double a = M_PI * ((2.0 * k + 1.0) / nt);
                bk[k] = make_double2(h2 * (1.0 - g1n * std::cos(a)) / p->tau + 2.0, -h2 * g1n * std::sin(a) / p->tau);
            }
        } else {
            bk.resize(H);
            for (int m = 0; m < H; ++m)
                bk[m] = make_double2(h2 * ak[m].x / p->tau + 2.0, h2 * ak[m].y / p->tau);
        }
        rc = upload(p, &tb.bk, bk);
    }
    if (!rc && tb.sf) {
        // Dirichlet eigenvalues (4/h^2) sin^2(k pi/(2M)) per axis, summed per mode
        std::vector<std::vector<double>> lam(3);
        for (int i = 0; i < 3; ++i) {
            lam[i].assign(tb.n[i], 0.0);
            if (i < d.dim)
                for (int k = 1; k <= tb.n[i]; ++k) {
                    double s = std::sin(M_PI * k / (2.0 * d.m[i]));
                    lam[i][k - 1] = 4.0 * p->h2inv[i] * s * s;
                }
        }
        std::vector<double> lt((size_t)tb.Nx);
        size_t idx = 0;
        for (int z = 0; z < tb.n[2]; ++z)
            for (int yy = 0; yy < tb.n[1]; ++yy)
                for (int x = 0; x < tb.n[0]; ++x)
                    lt[idx++] = p->tau * (lam[0][x] + lam[1][yy] + lam[2][z]);
        rc = upload(p, &tb.lamtau, lt);
        std::vector<float> lt32(lt.begin(), lt.end());
        if (!rc) rc = upload(p, &tb.lamtau32, lt32);
        for (int i = 0; i < d.dim && !rc; ++i) {
            const int M = d.m[i];
            p->lp[i] = ilog2(M);
            tb.lpd[i] = p->lp[i];
            std::vector<double2> s64;
            std::vector<float2> s32;
            roots(M, s64, s32);
            rc = upload(p, &tb.tw_s[i], s64);
            if (!rc) rc = upload(p, &tb.tw_s32[i], s32);
            std::vector<double> sn(M / 2 + 2, 0.0);
            std::vector<float> sn32(M / 2 + 2, 0.f);
            for (int j = 0; j <= M / 2; ++j) {
                sn[j] = std::sin(M_PI * j / M);
                sn32[j] = (float)sn[j];
            }
            if (!rc) rc = upload(p, &tb.sn_s[i], sn);
            if (!rc) rc = upload(p, &tb.sn_s32[i], sn32);
        }
    }
    // ---- workspace ----
    const size_t total = (size_t)tb.Nx * nt;
    if (!rc && !tb.sf) {
        rc = dalloc(p, &p->wk, total);
        if (!rc) rc = dalloc(p, &p->wcp, total);
    }
    if (!rc && tb.sf) rc = dalloc(p, &p->ghat, (size_t)tb.Nx);
    if (!rc && tb.sf && tb.gen) rc = dalloc(p, &p->wk, total);      // Bluestein spectrum [nt][Nx]
    if (!rc && tb.sf && d.precision == QBVM_FP64 && !tb.gen) {
        // Step (b) reciprocals, once per plan
        rc = dalloc(p, &tb.qinv, (size_t)(nt / 2) * (size_t)tb.Nx);
        if (!rc && (qbvm::launch_make_qinv(tb, fp64_cnorm(p), tb.qinv, 0) != cudaSuccess ||
                    cudaStreamSynchronize(0) != cudaSuccess))
            rc = QBVM_ERR_CUDA;
    }
    if (!rc && tb.sf && d.precision == QBVM_FP64 && d.rhs_kind == QBVM_RHS_DELTA) {
        // y^0-only fast mode of the delta right-hand side
        rc = dalloc(p, &tb.y0fac, (size_t)tb.Nx);
        if (!rc && (qbvm::launch_make_y0fac(tb, fp64_cnorm(p), tb.y0fac, 0) != cudaSuccess ||
                    cudaStreamSynchronize(0) != cudaSuccess))
            rc = QBVM_ERR_CUDA;
    }
    if (!rc) {
        p->nres = qbvm::residual_blocks(tb);
        rc = dalloc(p, &p->partials, (size_t)2 * p->nres);
        if (!rc) rc = dalloc(p, &p->sums, 2);
    }
    if (rc) {
        destroy_plan(p);
        return rc;
    }
    *out = p;
    return QBVM_OK;
}

int qbvm_plan_info(const qbvm_plan_t* p, qbvm_info* out) {
    if (!p || !out) return QBVM_ERR_BAD_ARG;
    out->alpha = p->alpha;
    out->omega = p->omega;
    out->tau = p->tau;
    out->unknowns = p->tb.Nx * p->tb.nt;
    out->workspace_bytes = p->ws_bytes;
    out->last_refine_iters = p->last_iters;
    out->last_rel_residual = p->last_relres;
    out->kernels_per_solve = p->kernels_per_solve;
    return QBVM_OK;
}

int qbvm_profile_enable(qbvm_plan_t* p, int on) {
    if (!p) return QBVM_ERR_BAD_ARG;
    for (auto& m : p->marks) {
        p->event_pool.push_back(m.a);
        p->event_pool.push_back(m.b);
    }
    p->marks.clear();
    p->profiling = on != 0;
    return QBVM_OK;
}

int qbvm_profile_read(qbvm_plan_t* p, qbvm_kernel_stat* out, int capacity, int* count) {
    if (!p || !count || (capacity > 0 && !out)) return QBVM_ERR_BAD_ARG;
    int n = 0;
    int rc = QBVM_OK;
    for (auto& m : p->marks) {
        float ms = 0.f;
        if (cudaEventSynchronize(m.b) != cudaSuccess || cudaEventElapsedTime(&ms, m.a, m.b) != cudaSuccess) {
            cudaGetLastError();
            rc = QBVM_ERR_CUDA;
        }
        int i = 0;
        while (i < n && std::strncmp(out[i].name, m.name, sizeof(out[i].name)) != 0) ++i;
        if (i == n) {
            if (n >= capacity) continue;
            std::memset(&out[n], 0, sizeof(out[n]));
            std::strncpy(out[n].name, m.name, sizeof(out[n].name) - 1);
            ++n;
        }
        out[i].launches += 1;
        out[i].total_ms += ms;
        p->event_pool.push_back(m.a);
        p->event_pool.push_back(m.b);
    }
    p->marks.clear();
    *count = n;
    return rc;
}

int qbvm_destroy(qbvm_plan_t* p) {
    destroy_plan(p);
    return QBVM_OK;
}

static int ensure_stage(qbvm_plan_t* p) {
    const size_t total = (size_t)p->tb.Nx * p->tb.nt;
    int rc = QBVM_OK;
    if (!p->stage_in) rc = dalloc(p, &p->stage_in, total);
    if (!rc && !p->stage_out) rc = dalloc(p, &p->stage_out, total);
    return rc;
}

static int ensure_wreal(qbvm_plan_t* p) {
    if (p->wreal) return QBVM_OK;
    return dalloc(p, &p->wreal, (size_t)p->tb.Nx * p->tb.nt);
}

static int ensure_fp32(qbvm_plan_t* p) {
    const size_t total = (size_t)p->tb.Nx * p->tb.nt;
    int rc = QBVM_OK;
    if (!p->f32) rc = dalloc(p, &p->f32, total);
    if (!rc && !p->g32) rc = dalloc(p, &p->g32, (size_t)p->tb.Nx);
    return rc;
}

static int solve_dev(qbvm_plan_t* p, const double* in, double* y, int n0_only, cudaStream_t s) {
    const bool refine = p->d.precision == QBVM_FP32_REFINE;
    if (p->tb.sf && n0_only && (p->d.rhs_kind == QBVM_RHS_GENERAL || refine)) {
        int rc = ensure_wreal(p);
        if (rc) return rc;
    }
    if (!refine) return solve_fp64_dev(p, in, y, n0_only, s);
    if (!p->tb.sf) return QBVM_ERR_UNSUPPORTED;
    int rc = ensure_fp32(p);
    if (rc) return rc;
    if (p->d.rhs_kind == QBVM_RHS_GENERAL) {
        // the refinement re-reads F after y has been written: an F that overlaps
        // y is copied first (the FP64 path is alias-safe as it stands)
        const size_t total = (size_t)p->tb.Nx * p->tb.nt;
        const char *a = reinterpret_cast<const char*>(in), *b = reinterpret_cast<const char*>(y);
        const size_t na = total * sizeof(double), nb = (n0_only ? (size_t)p->tb.Nx : total) * sizeof(double);
        if (a < b + nb && b < a + na) {
            if (!p->fcopy) rc = dalloc(p, &p->fcopy, total);
            if (rc) return rc;
            CK(cudaMemcpyAsync(p->fcopy, in, na, cudaMemcpyDeviceToDevice, s));
            in = p->fcopy;
        }
    }
    return solve_fp32r_dev(p, in, y, n0_only, s);
}

// Host-pointer FP64 space-first solve with the copies overlapped: chunks of
// time levels go host -> device on the copy stream while the DSTs of the
// chunks already there run; after the time part each chunk's inverse DSTs are
// followed by its device -> host copy, again on the copy stream.  Chunks
// alternate between the caller's stream and a second compute stream, so the
// partly filled last wave of one chunk's DST shares the SMs with the first
// CTAs of the next (a chunk alone fills about one wave and a fraction).
// Events order the three streams; the caller's stream ends after the last
// copy; only the first chunk's input copy and the last chunk's output copy
// are exposed.  (Overlap needs pinned host memory; pageable memory still
// gives the right answer.)
constexpr int HOST_CHUNKS = 8;

static int solve_fp64_host(qbvm_plan_t* p, const double* hin, double* hout, int n0_only, cudaStream_t s) {
    const Tables& tb = p->tb;
    const long long Nx = tb.Nx, nt = tb.nt;
    const int delta = p->d.rhs_kind == QBVM_RHS_DELTA;
    // events: [0, H) chunk inputs copied, [H, 2H) chunk outputs ready, then
    // start, copies done, forward chunks joined, time part done
    const int E_START = 2 * HOST_CHUNKS, E_DONE = E_START + 1, E_JOIN = E_START + 2, E_FORK = E_START + 3;
    if (!p->copy_stream) {
        CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking));
        p->copy_events.resize(E_FORK + 1);
        for (auto& e : p->copy_events) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    cudaStream_t cs = p->copy_stream, as = p->aux_stream;
    cudaEvent_t* ev = p->copy_events.data();
    auto cst = [&](int c) { return (c & 1) ? as : s; };
    // chunks start at even levels: the x-DST packs rows in pairs from its first
    // row, so the pairs (and the rounding) are those of the whole-array pass.
    // (Measured on 255^2 x 256: 8 equal chunks beat 16 equal ones, chunks
    // growing 7/5 per step with the output ones shrinking, and a one-level-pair
    // first input and last output chunk with the rest split evenly.)
    const int nch = (int)std::max(1LL, std::min((long long)HOST_CHUNKS, nt / 2));
    auto lev0 = [&](int c) { return c == nch ? nt : ((nt * c / nch) & ~1LL); };
    double *din = p->stage_in, *dy = p->stage_out;
    int launches = 0, rc = QBVM_OK;
    CK(cudaEventRecord(ev[E_START], s));                     // everything starts after the caller's work
    CK(cudaStreamWaitEvent(cs, ev[E_START], 0));
    CK(cudaStreamWaitEvent(as, ev[E_START], 0));
    if (delta) {
        CK(cudaMemcpyAsync(din, hin, sizeof(double) * Nx, cudaMemcpyHostToDevice, s));
        rc = fp64_dst_levels(p, din, p->ghat, 0, 1, s, &launches);
        if (!rc) rc = fp64_time_part(p, p->ghat, dy, 1, n0_only, s, &launches);
    } else {
        double* work = n0_only ? p->wreal : dy;
        for (int c = 0; c < nch && !rc; ++c) {
            const long long a = lev0(c), b = lev0(c + 1);
            CK(cudaMemcpyAsync(din + a * Nx, hin + a * Nx, sizeof(double) * (b - a) * Nx, cudaMemcpyHostToDevice, cs));
            CK(cudaEventRecord(ev[c], cs));
            CK(cudaStreamWaitEvent(cst(c), ev[c], 0));
            rc = fp64_dst_levels(p, din, work, a, b, cst(c), &launches);
        }
        if (rc) return rc;
        CK(cudaEventRecord(ev[E_JOIN], as));
        CK(cudaStreamWaitEvent(s, ev[E_JOIN], 0));
        rc = fp64_time_part(p, work, dy, 0, n0_only, s, &launches);
    }
    if (rc) return rc;
    CK(cudaEventRecord(ev[E_FORK], s));
    CK(cudaStreamWaitEvent(as, ev[E_FORK], 0));
    const int nco = n0_only ? 1 : nch;
    for (int c = 0; c < nco && !rc; ++c) {
        const long long a = n0_only ? 0 : lev0(c), b = n0_only ? 1 : lev0(c + 1);
        rc = fp64_dst_levels(p, dy, dy, a, b, cst(c), &launches);
        if (rc) break;
        CK(cudaEventRecord(ev[HOST_CHUNKS + c], cst(c)));
        CK(cudaStreamWaitEvent(cs, ev[HOST_CHUNKS + c], 0));
        CK(cudaMemcpyAsync(hout + a * Nx, dy + a * Nx, sizeof(double) * (b - a) * Nx, cudaMemcpyDeviceToHost, cs));
    }
    if (rc) return rc;
    // the last copy waited for every chunk of either compute stream
    CK(cudaEventRecord(ev[E_DONE], cs));
    CK(cudaStreamWaitEvent(s, ev[E_DONE], 0));
    CK(cudaStreamSynchronize(s));
    p->kernels_per_solve = launches;
    return QBVM_OK;
}

int qbvm_solve(qbvm_plan_t* p, const double* g_or_F, double* y, int n0_only, void* stream) {
    struct Range {
        Range() { nvtxRangePushA("qbvm_solve"); }
        ~Range() { nvtxRangePop(); }
    } range_;
    if (!p || !g_or_F || !y) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int kin = ptr_kind(g_or_F, p->dev), kout = ptr_kind(y, p->dev);
    if (kin != kout || kin == KIND_FOREIGN) return QBVM_ERR_BAD_ARG;
    if (kin == KIND_DEV) return solve_dev(p, g_or_F, y, n0_only, s);
    // host pointers: stage through plan buffers
    int rc = ensure_stage(p);
    if (rc) return rc;
    if (p->d.precision == QBVM_FP64 && p->tb.sf) {
        if (n0_only && p->d.rhs_kind == QBVM_RHS_GENERAL) rc = ensure_wreal(p);
        if (rc) return rc;
        return solve_fp64_host(p, g_or_F, y, n0_only, s);
    }
    const size_t nin = (size_t)p->tb.Nx * (p->d.rhs_kind == QBVM_RHS_DELTA ? 1 : p->tb.nt);
    const size_t nout = (size_t)p->tb.Nx * (n0_only ? 1 : p->tb.nt);
    CK(cudaMemcpyAsync(p->stage_in, g_or_F, nin * sizeof(double), cudaMemcpyHostToDevice, s));
    rc = solve_dev(p, p->stage_in, p->stage_out, n0_only, s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(y, p->stage_out, nout * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return QBVM_OK;
}

int qbvm_residual(qbvm_plan_t* p, const double* y, const double* g_or_F, double* rel_norm_out, void* stream) {
    if (!p || !y || !g_or_F || !rel_norm_out) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ky = ptr_kind(y, p->dev), kf = ptr_kind(g_or_F, p->dev);
    if (ky != kf || ky == KIND_FOREIGN) return QBVM_ERR_BAD_ARG;
    const int delta = p->d.rhs_kind == QBVM_RHS_DELTA;
    const double* dy = y;
    const double* df = g_or_F;
    if (ky == KIND_HOST) {
        int rc = ensure_stage(p);
        if (rc) return rc;
        const size_t total = (size_t)p->tb.Nx * p->tb.nt;
        const size_t nin = delta ? (size_t)p->tb.Nx : total;
        CK(cudaMemcpyAsync(p->stage_out, y, total * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(p->stage_in, g_or_F, nin * sizeof(double), cudaMemcpyHostToDevice, s));
        dy = p->stage_out;
        df = p->stage_in;
    }
    { Span sp_(p, "residual", s); CK(qbvm::launch_residual(dy, df, delta, p->tb, p->h2inv, p->partials, p->nres, p->sums, nullptr, s)); }
    double h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, p->sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return QBVM_ERR_NONFINITE;
    *rel_norm_out = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return QBVM_OK;
}

}  // extern "C"
