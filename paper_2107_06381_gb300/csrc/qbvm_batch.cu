// qbvm_batch.cu -- many PinT-QBVM / PinT-MQBVM instances of one shape, each
// with its own regularisation parameter alpha (so its own omega of eq. 3.3 /
// 3.6), solved together: the DST-I passes run once over all instances' time
// levels (the DST does not depend on omega), the time solve of eq. 3.8 once
// over every (instance, mode tile) with per-instance omega tables.  A batch
// of B instances costs the launches of ONE solve, whatever B is.
//
// The shape tables (time and space roots, sines, tau Lambda) are those of a
// base plan built from the descriptor; the omega-dependent ones are built
// here in FP64 on the host exactly as the base plan builds its own:
//   gpow[t] = gamma^t, gipw[t] = 2 gamma^{-t}, gpowr[t] = i rho^H gamma^t,
//   gipr[t] = 2 rho^{-H} gamma^{-t}  (t < H = nt/2, gamma = |omega|^{1/nt} e^{i pi/nt}),
//   d_{2m} = 1 - gamma theta^{2m},
// and on the device the Step (b) reciprocals cnorm / (d_{2m} + tau Lambda_l).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "qbvm.h"
#include "qbvm_internal.h"

namespace {

__global__ void k_make_qinv_batched(const double2* __restrict__ ak, const double* __restrict__ lamtau,
                                    const double* __restrict__ cnorm, int H, long long Nx, long long count,
                                    double2* __restrict__ q) {
    const long long per = (long long)H * Nx, n = per * count;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / per, r = i - b * per, k = r / Nx, l = r - k * Nx;
        const double2 a = ak[b * H + k];
        const double zr = a.x + lamtau[l], zi = a.y;
        const double inv = cnorm[b] / (zr * zr + zi * zi);
        q[i] = make_double2(zr * inv, -zi * inv);
    }
}

// y^0 of the delta right-hand side: Step (c) at t = 0 of the constant
// spectrum is the sum over the formed (even) frequencies, twice its real part.
__global__ void k_y0fac_batched(const double2* __restrict__ q, int H, long long Nx, long long count,
                                double* __restrict__ out) {
    const long long n = Nx * count;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / Nx, l = i - b * Nx;
        const double2* qb = q + b * H * Nx;
        double a = 0.0;
        for (int m = 0; m < H; ++m) a += qb[(long long)m * Nx + l].x;
        out[i] = 2.0 * a;
    }
}

unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

struct qbvm_batch {
    qbvm_plan_t* base = nullptr;
    qbvm_desc d{};
    long long count = 0;
    std::vector<double> alpha;
    double2 *gpow = nullptr, *gipw = nullptr, *gpowr = nullptr, *gipr = nullptr, *ak = nullptr, *qinv = nullptr;
    double* cnorm = nullptr;
    double* y0fac = nullptr;      // delta right-hand side: [count][Nx]
    double* ghat = nullptr;       // delta right-hand side: the DST of every g, [count][Nx]
    double* work = nullptr;       // general right-hand side with n0_only: [count][nt][Nx]
    double* stage_in = nullptr;   // host-pointer solves: device copies of the input and output
    double* stage_out = nullptr;
    // FP32 transforms + double-float refinement (precision QBVM_FP32_REFINE)
    std::vector<double2> h_gpow, h_gipw, h_gpowr, h_gipr, h_ak;   // FP64 omega tables, kept for the FP64 pipeline
    std::vector<double> h_cnorm;
    bool fp64_ready = false;      // FP64 tables on the device (FP64 batches, or an FP32 batch's fallback)
    qbvm::BatchTables32 t32_delta, t32_gen;   // the FP32 tables with the delta / general cnorm
    float2* omega_df = nullptr;   // omega_b as a double-float pair, [count]
    double* omega64 = nullptr;    // omega_b, [count]
    float* f32 = nullptr;         // FP32 work array [count][nt][Nx] (also r.hi of the residual)
    float* g32 = nullptr;         // delta right-hand side: the FP32 DST of every g, [count][Nx]
    double* partials = nullptr;   // residual partial sums [count][bpi][2]
    double* sums = nullptr;       // per-instance ||r||^2, ||f||^2 [count][2]
    int* flags = nullptr;         // input classification (NaN/Inf, nonzero)
    bool r1 = false;              // 1D shapes the fused refinement kernel takes (qbvm_refine1d.cu)
    int* r1_stat = nullptr;       // its per-instance status and steps, [count][2]
    double* r1_rel = nullptr;     // its per-instance final relative residual, [count]
    int bpi = 1;
    int last_iters = 0;
    double last_rel = 0.0;        // largest relative residual over the instances at the end
    std::vector<void*> allocs;
};

namespace {

template <typename T>
int balloc(qbvm_batch* b, T** ptr, size_t n) {
    *ptr = nullptr;
    void* v = nullptr;
    if (cudaMalloc(&v, (n ? n : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_OOM;
    }
    b->allocs.push_back(v);
    *ptr = static_cast<T*>(v);
    return QBVM_OK;
}

template <typename T>
int bupload(qbvm_batch* b, T** ptr, const std::vector<T>& h) {
    int rc = balloc(b, ptr, h.size());
    if (rc) return rc;
    if (cudaMemcpy(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    return QBVM_OK;
}

void destroy_batch(qbvm_batch* b) {
    if (!b) return;
    for (void* v : b->allocs) cudaFree(v);
    if (b->base) qbvm_destroy(b->base);
    delete b;
}

// DST-I along every axis of `lev` consecutive levels (the FP64 4x transform).
int dst_levels(const qbvm::Tables& tb, const double* in, double* out, long long lev, cudaStream_t s) {
    const long long nx = tb.n[0], ny = tb.n[1], nz = tb.n[2];
    if (qbvm::launch_dst<double, double, 0, true>(in, out, tb.n[0], tb.lpd[0], lev * ny * nz, 1, tb.tw_s[0],
                                                  tb.sn_s[0], s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (tb.dim >= 2 && qbvm::launch_dst<double, double, 0, true>(out, out, tb.n[1], tb.lpd[1], lev * nz, nx,
                                                                 tb.tw_s[1], tb.sn_s[1], s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    if (tb.dim == 3 && qbvm::launch_dst<double, double, 0, true>(out, out, tb.n[2], tb.lpd[2], lev, nx * ny,
                                                                 tb.tw_s[2], tb.sn_s[2], s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    return QBVM_OK;
}

// The FP64 device tables of the batch (its per-instance omega factors, the
// Step (b) reciprocals and, for the delta right-hand side, the y^0 factors)
// from the FP64 host tables.
int fp64_tables(qbvm_batch* bt) {
    if (bt->fp64_ready) return QBVM_OK;
    qbvm::PlanView v;
    qbvm::plan_view(bt->base, &v);
    const qbvm::Tables& tb = *v.tb;
    const long long count = bt->count, H = tb.nt / 2, Nx = tb.Nx;
    int rc = bupload(bt, &bt->gpow, bt->h_gpow);
    if (!rc) rc = bupload(bt, &bt->gipw, bt->h_gipw);
    if (!rc) rc = bupload(bt, &bt->gpowr, bt->h_gpowr);
    if (!rc) rc = bupload(bt, &bt->gipr, bt->h_gipr);
    if (!rc) rc = bupload(bt, &bt->ak, bt->h_ak);
    if (!rc) rc = bupload(bt, &bt->cnorm, bt->h_cnorm);
    if (!rc) rc = balloc(bt, &bt->qinv, (size_t)(count * H * Nx));
    if (!rc) {
        // the FP64 plan's lamtau: the base plan of an FP32 batch has it too
        k_make_qinv_batched<<<grid_for(count * H * Nx), 256>>>(bt->ak, tb.lamtau, bt->cnorm, (int)H, Nx, count,
                                                              bt->qinv);
        if (cudaGetLastError() != cudaSuccess) rc = QBVM_ERR_CUDA;
    }
    if (!rc && bt->d.rhs_kind == QBVM_RHS_DELTA) {
        if (!bt->ghat) rc = balloc(bt, &bt->ghat, (size_t)(count * Nx));
        if (!rc) rc = balloc(bt, &bt->y0fac, (size_t)(count * Nx));
        if (!rc) {
            k_y0fac_batched<<<grid_for(count * Nx), 256>>>(bt->qinv, (int)H, Nx, count, bt->y0fac);
            if (cudaGetLastError() != cudaSuccess) rc = QBVM_ERR_CUDA;
        }
    }
    if (!rc) bt->fp64_ready = true;
    return rc;
}

// The FP32 tables (the FP64 ones rounded once), omega per instance, and the
// workspace of the refinement.
int fp32_tables(qbvm_batch* bt) {
    qbvm::PlanView v;
    qbvm::plan_view(bt->base, &v);
    const qbvm::Tables& tb = *v.tb;
    const long long count = bt->count, Nx = tb.Nx, nt = tb.nt;
    auto to32 = [](const std::vector<double2>& a) {
        std::vector<float2> o(a.size());
        for (size_t i = 0; i < a.size(); ++i) o[i] = make_float2((float)a[i].x, (float)a[i].y);
        return o;
    };
    double cn = 1.0;                               // FP32 DSTs: prod 2/(n_d + 1) (not the FP64 4x), 1/nt
    for (int i = 0; i < tb.dim; ++i) cn *= 2.0 / (tb.n[i] + 1);
    cn /= nt;
    std::vector<float> cd((size_t)count), cg((size_t)count, (float)(v.tau * cn)), rh((size_t)count), ri((size_t)count);
    std::vector<float2> odf((size_t)count);
    std::vector<double> o64((size_t)count);
    for (long long b = 0; b < count; ++b) {
        const double a = bt->alpha[(size_t)b];
        const double om = bt->d.form == QBVM_FORM_PQ ? -1.0 / a : -v.tau / a;
        o64[(size_t)b] = om;
        const float oh = (float)om;
        odf[(size_t)b] = make_float2(oh, (float)(om - (double)oh));
        cd[(size_t)b] = (float)(-om * cn);
        rh[(size_t)b] = (float)std::sqrt(std::fabs(om));
        ri[(size_t)b] = (float)(1.0 / std::sqrt(std::fabs(om)));
    }
    float2 *gp, *gi, *gr, *gir, *ak;
    float *pcd, *pcg, *prh, *pri;
    int rc = bupload(bt, &gp, to32(bt->h_gpow));
    if (!rc) rc = bupload(bt, &gi, to32(bt->h_gipw));
    if (!rc) rc = bupload(bt, &gr, to32(bt->h_gpowr));
    if (!rc) rc = bupload(bt, &gir, to32(bt->h_gipr));
    if (!rc) rc = bupload(bt, &ak, to32(bt->h_ak));
    if (!rc) rc = bupload(bt, &pcd, cd);
    if (!rc) rc = bupload(bt, &pcg, cg);
    if (!rc) rc = bupload(bt, &prh, rh);
    if (!rc) rc = bupload(bt, &pri, ri);
    if (!rc) rc = bupload(bt, &bt->omega_df, odf);
    if (!rc) rc = bupload(bt, &bt->omega64, o64);
    if (rc) return rc;
    bt->t32_delta = {gp, gi, gr, gir, ak, pcd, prh, pri};
    bt->t32_gen = {gp, gi, gr, gir, ak, pcg, prh, pri};
    bt->r1 = qbvm::refine1d_supported(tb) != 0;
    if (bt->r1) {                                  // the fused kernel needs no work arrays
        rc = balloc(bt, &bt->r1_stat, (size_t)(2 * count));
        if (!rc) rc = balloc(bt, &bt->r1_rel, (size_t)count);
        return rc;
    }
    // blocks per instance: about four groups of four unknowns per thread
    // (measured on 10 000 instances of 63 x 64: one, two and four groups per
    // thread took 2.51, 2.12 and 1.93 ms per refined batch)
    bt->bpi = qbvm::residual_blocks_per_instance(tb);
    if (count * (long long)bt->bpi > 0x7fffffffLL) bt->bpi = (int)std::max(1LL, 0x7fffffffLL / count);
    rc = balloc(bt, &bt->f32, (size_t)(count * nt * Nx));
    if (!rc && bt->d.rhs_kind == QBVM_RHS_DELTA) rc = balloc(bt, &bt->g32, (size_t)(count * Nx));
    if (!rc) rc = balloc(bt, &bt->partials, (size_t)(2 * count * bt->bpi));
    if (!rc) rc = balloc(bt, &bt->sums, (size_t)(2 * count));
    if (!rc) rc = balloc(bt, &bt->flags, 2);
    return rc;
}

// 1: memory of device `dev` (or managed), 0: host memory, -1: another GPU's
// memory (the batch's kernels would read it as a peer: refused).
int dev_kind(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? 1 : -1;
    return 0;
}

int solve_batched_dev(qbvm_batch_t* bt, const double* g_or_F, double* y, int n0_only, cudaStream_t s);
int solve_batched_fp64(qbvm_batch_t* bt, const double* g_or_F, double* y, int n0_only, cudaStream_t s);

}  // namespace

extern "C" {

int qbvm_batch_plan(const qbvm_desc* desc, int count, const double* alphas, qbvm_batch_t** out) {
    if (!desc || !out || count < 1) return QBVM_ERR_BAD_ARG;
    *out = nullptr;
    qbvm_desc d0 = *desc;                         // validated with the first instance's alpha
    if (alphas) d0.alpha = alphas[0];
    if (!(std::isfinite(d0.alpha) && (d0.alpha > 0 || d0.delta > 0))) return QBVM_ERR_BAD_ARG;
    int rc = qbvm::validate_desc(&d0);
    if (rc) return rc;
    if ((desc->nt & (desc->nt - 1)) != 0) return QBVM_ERR_UNSUPPORTED;       // half-length time transforms only
    if (desc->precision == QBVM_FP32_REFINE) {
        // the batched residual moves groups of four unknowns per thread
        long long nx = 1;
        for (int i = 0; i < desc->dim; ++i) nx *= desc->m[i] - 1;
        if ((nx * desc->nt) % 4 != 0) return QBVM_ERR_UNSUPPORTED;
    }
    // the batch runs space-first; AUTO is space-first whenever m allows the DST
    // (m <= 2048), which the descriptor check already required of every m when
    // the order is space-first
    if (desc->dim == 1 && (desc->order == QBVM_ORDER_TIME_FIRST || desc->m[0] > 2048)) return QBVM_ERR_UNSUPPORTED;
    const double tau = desc->T / (desc->nt - 1);
    std::vector<double> al((size_t)count);
    for (int b = 0; b < count; ++b) {
        double a = alphas ? alphas[b]
                          : (desc->alpha > 0 ? desc->alpha : (desc->form == QBVM_FORM_PQ ? desc->delta : tau * desc->delta));
        if (!(std::isfinite(a) && a > 0)) return QBVM_ERR_BAD_ARG;
        al[(size_t)b] = a;
    }
    qbvm_batch* bt = new (std::nothrow) qbvm_batch();
    if (!bt) return QBVM_ERR_OOM;
    bt->d = d0;
    bt->d.alpha = al[0];
    bt->count = count;
    bt->alpha = al;
    rc = qbvm_plan(&bt->d, &bt->base);
    if (rc) {
        destroy_batch(bt);
        return rc;
    }
    qbvm::PlanView v;
    qbvm::plan_view(bt->base, &v);
    const qbvm::Tables& tb = *v.tb;
    if (!tb.sf || tb.gen) {                       // time-first 1D (m beyond the DST lengths) or Bluestein nt
        destroy_batch(bt);
        return QBVM_ERR_UNSUPPORTED;
    }
    const int nt = desc->nt, H = nt / 2;
    const double cn = qbvm::time_cn(tb);
    std::vector<double2> gpow((size_t)count * H), gipw(gpow.size()), gpowr(gpow.size()), gipr(gpow.size()),
        ak(gpow.size());
    std::vector<double> cnv((size_t)count);
    for (int b = 0; b < count; ++b) {
        const double omega = desc->form == QBVM_FORM_PQ ? -1.0 / al[(size_t)b] : -tau / al[(size_t)b];
        const double mag = std::fabs(omega);
        if (!std::isfinite(omega) || !(mag > 0)) {
            destroy_batch(bt);
            return QBVM_ERR_BAD_ARG;
        }
        cnv[(size_t)b] = desc->rhs_kind == QBVM_RHS_DELTA ? -omega * cn : tau * cn;
        double2* g = gpow.data() + (size_t)b * H;
        double2* gi = gipw.data() + (size_t)b * H;
        double2* gr = gpowr.data() + (size_t)b * H;
        double2* gir = gipr.data() + (size_t)b * H;
        for (int t = 0; t < H; ++t) {
            const double a = M_PI * ((double)t / nt);
            const double r = std::pow(mag, (double)t / nt), ri = 2.0 * std::pow(mag, -(double)t / nt);
            const double rr = std::pow(mag, (double)(t + H) / nt), rir = 2.0 * std::pow(mag, -(double)(t + H) / nt);
            g[t] = make_double2(r * std::cos(a), r * std::sin(a));
            gi[t] = make_double2(ri * std::cos(a), -ri * std::sin(a));
            gr[t] = make_double2(-rr * std::sin(a), rr * std::cos(a));
            gir[t] = make_double2(rir * std::cos(a), -rir * std::sin(a));
        }
        const double g1 = std::pow(mag, 1.0 / nt);
        double2* d = ak.data() + (size_t)b * H;
        for (int m = 0; m < H; ++m) {
            const double a = M_PI * ((4.0 * m + 1.0) / nt);
            d[m] = make_double2(1.0 - g1 * std::cos(a), -g1 * std::sin(a));
        }
    }
    bt->h_gpow = std::move(gpow);
    bt->h_gipw = std::move(gipw);
    bt->h_gpowr = std::move(gpowr);
    bt->h_gipr = std::move(gipr);
    bt->h_ak = std::move(ak);
    bt->h_cnorm = std::move(cnv);
    rc = desc->precision == QBVM_FP64 ? fp64_tables(bt) : fp32_tables(bt);
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        rc = QBVM_ERR_CUDA;
    }
    if (rc) {
        destroy_batch(bt);
        return rc;
    }
    *out = bt;
    return QBVM_OK;
}

int qbvm_solve_batched(qbvm_batch_t* bt, const double* g_or_F, double* y, int n0_only, void* stream) {
    if (!bt || !g_or_F || !y) return QBVM_ERR_BAD_ARG;
    qbvm::PlanView v;
    qbvm::plan_view(bt->base, &v);
    const int din = dev_kind(g_or_F, v.dev), dout = dev_kind(y, v.dev);
    // both on the batch's device or both on the host
    if (din != dout || din < 0) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (din) return solve_batched_dev(bt, g_or_F, y, n0_only, s);
    // host arrays: through batch-owned device copies, synchronous
    const long long B = bt->count, Nx = v.tb->Nx, nt = v.tb->nt;
    const size_t nin = (size_t)(B * Nx * (bt->d.rhs_kind == QBVM_RHS_DELTA ? 1 : nt));
    const size_t nout = (size_t)(B * Nx * (n0_only ? 1 : nt));
    if (!bt->stage_in) {
        int rc = balloc(bt, &bt->stage_in, (size_t)(B * Nx * nt));
        if (!rc) rc = balloc(bt, &bt->stage_out, (size_t)(B * Nx * nt));
        if (rc) return rc;
    }
    if (cudaMemcpyAsync(bt->stage_in, g_or_F, nin * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    int rc = solve_batched_dev(bt, bt->stage_in, bt->stage_out, n0_only, s);
    if (rc) return rc;
    if (cudaMemcpyAsync(y, bt->stage_out, nout * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    return QBVM_OK;
}

}  // extern "C"

namespace {

// ---- FP32 transforms + double-float refinement over the whole batch --------
//
// As the single plan's refinement (y_0 = A32^{-1} f, then r = f - A y,
// y += A32^{-1} r), every stage once over all instances: the FP32 DST passes
// over count * nt levels, the FP32 time solve with each instance's omega
// tables, one batched double-float residual with per-instance norms.  The
// batch stops when the largest relative residual is at most the tolerance;
// a stall above 1e-10 or the cap above the tolerance is QBVM_ERR_DIVERGED.

#define BCK(...)                                      \
    do {                                              \
        if ((__VA_ARGS__) != cudaSuccess) {           \
            cudaGetLastError();                       \
            return QBVM_ERR_CUDA;                     \
        }                                             \
    } while (0)

// One FP32 solve of every instance: rhs (FP64 when rhs_fp64, else the FP32
// work array; one level per instance when delta) -> ydf (store, or add when
// accumulate, into the double-float iterate).
int fp32_solve_batched(qbvm_batch* bt, const qbvm::Tables& tb, const void* rhs, int rhs_fp64, int delta, void* ydf,
                       int accumulate, cudaStream_t s) {
    const long long B = bt->count, nx = tb.n[0], ny = tb.n[1], nz = tb.n[2], nt = tb.nt, Nx = tb.Nx;
    const long long lev = B * nt;
    float* w = bt->f32;
    if (delta) {
        BCK(qbvm::launch_dst<float, double, 0>((const double*)rhs, bt->g32, tb.n[0], tb.lpd[0], B * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s));
        if (tb.dim >= 2) BCK(qbvm::launch_dst<float, float, 0>(bt->g32, bt->g32, tb.n[1], tb.lpd[1], B * nz, nx, tb.tw_s32[1], tb.sn_s32[1], s));
        if (tb.dim == 3) BCK(qbvm::launch_dst<float, float, 0>(bt->g32, bt->g32, tb.n[2], tb.lpd[2], B, nx * ny, tb.tw_s32[2], tb.sn_s32[2], s));
        BCK(qbvm::launch_time_solve_batched32(bt->g32, w, tb, B, Nx, nt * Nx, bt->t32_delta, 1, 0, s));
    } else {
        if (rhs_fp64) BCK(qbvm::launch_dst<float, double, 0>((const double*)rhs, w, tb.n[0], tb.lpd[0], lev * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s));
        else BCK(qbvm::launch_dst<float, float, 0>((const float*)rhs, w, tb.n[0], tb.lpd[0], lev * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s));
        if (tb.dim >= 2) BCK(qbvm::launch_dst<float, float, 0>(w, w, tb.n[1], tb.lpd[1], lev * nz, nx, tb.tw_s32[1], tb.sn_s32[1], s));
        if (tb.dim == 3) BCK(qbvm::launch_dst<float, float, 0>(w, w, tb.n[2], tb.lpd[2], lev, nx * ny, tb.tw_s32[2], tb.sn_s32[2], s));
        BCK(qbvm::launch_time_solve_batched32(w, w, tb, B, nt * Nx, nt * Nx, bt->t32_gen, 0, 0, s));
    }
    if (tb.dim == 3) BCK(qbvm::launch_dst<float, float, 0>(w, w, tb.n[2], tb.lpd[2], lev, nx * ny, tb.tw_s32[2], tb.sn_s32[2], s));
    if (tb.dim >= 2) BCK(qbvm::launch_dst<float, float, 0>(w, w, tb.n[1], tb.lpd[1], lev * nz, nx, tb.tw_s32[1], tb.sn_s32[1], s));
    if (accumulate) BCK(qbvm::launch_dst<float, float, 1>(w, ydf, tb.n[0], tb.lpd[0], lev * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s));
    else BCK(qbvm::launch_dst<float, float, 2>(w, ydf, tb.n[0], tb.lpd[0], lev * ny * nz, 1, tb.tw_s32[0], tb.sn_s32[0], s));
    return QBVM_OK;
}

// The fused 1D refinement: one launch, then the per-instance statuses.
int solve_batched_r1(qbvm_batch* bt, const double* in, double* y, int n0_only, cudaStream_t s) {
    qbvm::PlanView v;
    qbvm::plan_view(bt->base, &v);
    const qbvm::Tables& tb = *v.tb;
    const long long B = bt->count;
    auto df = [](double x) {
        const float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    };
    qbvm::Refine1dArgs a;
    a.f = in;
    a.y = y;
    a.delta = bt->d.rhs_kind == QBVM_RHS_DELTA;
    a.n0_only = n0_only;
    a.tws = tb.tw_s32[0];
    a.sns = tb.sn_s32[0];
    a.twt = tb.tw_t32;
    a.lamtau = tb.lamtau32;
    a.gpow = bt->t32_gen.gpow;
    a.gipw = bt->t32_gen.gipw;
    a.ak = bt->t32_gen.ak;
    a.cnorm = bt->t32_gen.cnorm;
    a.rho_h = bt->t32_gen.rho_h;
    a.rho_hinv = bt->t32_gen.rho_hinv;
    a.omega_df = bt->omega_df;
    a.omega64 = bt->omega64;
    a.ct = df(1.0 / tb.tau);
    a.cx = df(v.h2inv[0]);
    a.inv_tau = 1.0 / tb.tau;
    a.tol = bt->d.refine_tol > 0 ? bt->d.refine_tol : 1e-13;
    a.maxit = bt->d.refine_max_iters > 0 ? bt->d.refine_max_iters : 10;
    a.iters = bt->r1_stat + B;
    a.rel = bt->r1_rel;
    a.status = bt->r1_stat;
    BCK(qbvm::launch_refine1d(tb, B, a, s));
    std::vector<int> st((size_t)(2 * B));
    std::vector<double> rl((size_t)B);
    BCK(cudaMemcpyAsync(st.data(), bt->r1_stat, sizeof(int) * 2 * B, cudaMemcpyDeviceToHost, s));
    BCK(cudaMemcpyAsync(rl.data(), bt->r1_rel, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    bool nonfinite_in = false, unusable = false, nonfinite = false, diverged = false;
    int iters = 0;
    double rel = 0.0;
    for (long long b = 0; b < B; ++b) {
        const int sb = st[(size_t)b];
        if (sb == qbvm::R1_NONFINITE_IN) nonfinite_in = true;
        if (sb == qbvm::R1_NONFINITE_IN || sb == qbvm::R1_RANGE) unusable = true;
        if (sb == qbvm::R1_DIVERGED) diverged = true;
        if (sb == qbvm::R1_NONFINITE) nonfinite = true;
        iters = std::max(iters, st[(size_t)(B + b)]);
        rel = std::max(rel, rl[(size_t)b]);
    }
    if (unusable) {
        // NaN / Inf, or data outside the FP32 range, in some instance: the FP64
        // pipeline solves the batch, as in the staged refinement
        int rc = fp64_tables(bt);
        if (rc) return rc;
        rc = solve_batched_fp64(bt, in, y, n0_only, s);
        bt->last_iters = 0;
        bt->last_rel = NAN;
        return rc ? rc : (nonfinite_in ? QBVM_ERR_NONFINITE : QBVM_OK);
    }
    bt->last_iters = iters;
    bt->last_rel = rel;
    if (nonfinite) return QBVM_ERR_NONFINITE;
    return diverged ? QBVM_ERR_DIVERGED : QBVM_OK;
}

int solve_batched_fp32r(qbvm_batch* bt, const double* in, double* y, int n0_only, cudaStream_t s) {
    if (bt->r1) return solve_batched_r1(bt, in, y, n0_only, s);
    qbvm::PlanView v;
    qbvm::plan_view(bt->base, &v);
    const qbvm::Tables& tb = *v.tb;
    const long long B = bt->count, Nx = tb.Nx, nt = tb.nt;
    const int delta = bt->d.rhs_kind == QBVM_RHS_DELTA;
    const double tol = bt->d.refine_tol > 0 ? bt->d.refine_tol : 1e-13;
    const int maxit = bt->d.refine_max_iters > 0 ? bt->d.refine_max_iters : 10;
    double* yfull = y;
    if (n0_only) {                                   // the iterate needs every level
        if (!bt->work) {
            int rc = balloc(bt, &bt->work, (size_t)(B * nt * Nx));
            if (rc) return rc;
        }
        yfull = bt->work;
    }
    int rc = fp32_solve_batched(bt, tb, in, 1, delta, yfull, 0, s);
    if (rc) return rc;
    std::vector<double> h((size_t)(2 * B)), fn2((size_t)B, 0.0);
    double prev = INFINITY, rel = 0.0;
    int it = 0, status = QBVM_OK;
    for (bool first = true;; first = false) {
        BCK(qbvm::launch_residual_df_batched(yfull, in, delta, tb, v.h2inv, B, bt->omega_df, bt->omega64, bt->f32,
                                             bt->partials, bt->sums, first ? 1 : 0, bt->bpi, s));
        BCK(cudaMemcpyAsync(h.data(), bt->sums, sizeof(double) * 2 * B, cudaMemcpyDeviceToHost, s));
        BCK(cudaStreamSynchronize(s));
        rel = 0.0;
        bool finite = true, fp32_range = true;
        for (long long b = 0; b < B; ++b) {
            if (first) {
                fn2[(size_t)b] = h[(size_t)(2 * b + 1)];
                const double cnt = (double)Nx * (delta ? 1 : nt);
                const double rms = std::sqrt(fn2[(size_t)b] / cnt);
                // data FP32 cannot hold (beyond its range, or flushed to zero)
                if (rms > 0 && (rms < 1e-18 || rms > 1e28)) fp32_range = false;
            }
            const double r2 = h[(size_t)(2 * b)], f2 = fn2[(size_t)b];
            if (!std::isfinite(r2) || !std::isfinite(f2)) finite = false;
            rel = std::max(rel, f2 > 0 ? std::sqrt(r2 / f2) : std::sqrt(r2));
        }
        if (first && finite && fp32_range) {
            // ||f_b|| = 0: all-zero data (y_b = 0 is right) or data so small that
            // FP32 flushed it to zero -- the input decides
            const long long per_in = delta ? Nx : nt * Nx;
            for (long long b = 0; b < B && fp32_range; ++b) {
                if (fn2[(size_t)b] != 0.0) continue;
                int fl[2] = {0, 0};
                BCK(qbvm::launch_classify(in + b * per_in, per_in, bt->flags, s));
                BCK(cudaMemcpyAsync(fl, bt->flags, sizeof(fl), cudaMemcpyDeviceToHost, s));
                BCK(cudaStreamSynchronize(s));
                if (fl[0]) finite = false;
                if (fl[1]) fp32_range = false;
            }
        }
        if (first && (!finite || !fp32_range)) {
            // NaN / Inf anywhere, or data outside the FP32 range: the FP64
            // pipeline solves the batch (it carries NaN / Inf through IEEE
            // arithmetic, as the single FP64 solve does)
            rc = fp64_tables(bt);
            if (rc) return rc;
            rc = solve_batched_fp64(bt, in, y, n0_only, s);
            bt->last_iters = 0;
            bt->last_rel = NAN;
            return rc ? rc : (finite ? QBVM_OK : QBVM_ERR_NONFINITE);
        }
        if (!finite) return QBVM_ERR_NONFINITE;
        if (rel <= tol) break;
        if (rel > 0.5 * prev) {                      // no contraction
            if (rel > 1e-10) status = QBVM_ERR_DIVERGED;
            break;
        }
        if (it >= maxit) {
            status = QBVM_ERR_DIVERGED;
            break;
        }
        prev = rel;
        rc = fp32_solve_batched(bt, tb, bt->f32, 0, 0, yfull, 1, s);
        if (rc) return rc;
        ++it;
    }
    BCK(qbvm::launch_df_to_double(yfull, B * nt * Nx, s));
    if (n0_only)
        BCK(cudaMemcpy2DAsync(y, sizeof(double) * Nx, yfull, sizeof(double) * nt * Nx, sizeof(double) * Nx, B,
                              cudaMemcpyDeviceToDevice, s));
    bt->last_iters = it;
    bt->last_rel = rel;
    return status;
}

int solve_batched_dev(qbvm_batch_t* bt, const double* g_or_F, double* y, int n0_only, cudaStream_t s) {
    if (bt->d.precision == QBVM_FP32_REFINE) return solve_batched_fp32r(bt, g_or_F, y, n0_only, s);
    return solve_batched_fp64(bt, g_or_F, y, n0_only, s);
}

int solve_batched_fp64(qbvm_batch_t* bt, const double* g_or_F, double* y, int n0_only, cudaStream_t s) {
    qbvm::PlanView v;
    qbvm::plan_view(bt->base, &v);
    const qbvm::Tables& tb = *v.tb;
    const long long B = bt->count, Nx = tb.Nx, nt = tb.nt, lev = B * nt;
    const int delta = bt->d.rhs_kind == QBVM_RHS_DELTA;
    int rc;
    if (delta) {
        rc = dst_levels(tb, g_or_F, bt->ghat, B, s);                       // one level per instance
        if (rc) return rc;
        if (n0_only) {
            qbvm::launch_mul_modes(bt->ghat, bt->y0fac, y, B * Nx, s);
            if (cudaGetLastError() != cudaSuccess) return QBVM_ERR_CUDA;
            return dst_levels(tb, y, y, B, s);
        }
        if (qbvm::launch_time_solve_batched(bt->ghat, y, tb, B, Nx, nt * Nx, bt->gpow, bt->gipw, bt->gpowr, bt->gipr,
                                            bt->qinv, 1, 0, s) != cudaSuccess)
            return QBVM_ERR_CUDA;
        return dst_levels(tb, y, y, lev, s);
    }
    double* work = y;
    if (n0_only) {
        if (!bt->work) {
            rc = balloc(bt, &bt->work, (size_t)lev * Nx);
            if (rc) return rc;
        }
        work = bt->work;
    }
    rc = dst_levels(tb, g_or_F, work, lev, s);
    if (rc) return rc;
    if (qbvm::launch_time_solve_batched(work, y, tb, B, nt * Nx, n0_only ? Nx : nt * Nx, bt->gpow, bt->gipw,
                                        bt->gpowr, bt->gipr, bt->qinv, 0, n0_only, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    return dst_levels(tb, y, y, n0_only ? B : lev, s);
}

}  // namespace

extern "C" {

int qbvm_batch_info(const qbvm_batch_t* bt, double* alphas, long long* unknowns_per_instance) {
    if (!bt) return QBVM_ERR_BAD_ARG;
    qbvm::PlanView v;
    qbvm::plan_view(bt->base, &v);
    if (alphas)
        for (long long b = 0; b < bt->count; ++b) alphas[b] = bt->alpha[(size_t)b];
    if (unknowns_per_instance) *unknowns_per_instance = v.tb->Nx * v.tb->nt;
    return QBVM_OK;
}

int qbvm_batch_refine_info(const qbvm_batch_t* bt, int* iters, double* max_rel_residual) {
    if (!bt) return QBVM_ERR_BAD_ARG;
    if (iters) *iters = bt->last_iters;
    if (max_rel_residual) *max_rel_residual = bt->last_rel;
    return QBVM_OK;
}

int qbvm_batch_refine_fused(const qbvm_batch_t* bt, int* fused) {
    if (!bt || !fused) return QBVM_ERR_BAD_ARG;
    *fused = bt->r1 ? 1 : 0;
    return QBVM_OK;
}

int qbvm_batch_destroy(qbvm_batch_t* bt) {
    if (!bt) return QBVM_OK;                      // NULL is accepted, as by every destroy
    destroy_batch(bt);
    return QBVM_OK;
}

}  // extern "C"
