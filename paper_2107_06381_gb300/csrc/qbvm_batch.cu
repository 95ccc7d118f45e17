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
    if (desc->precision != QBVM_FP64) return QBVM_ERR_UNSUPPORTED;
    if ((desc->nt & (desc->nt - 1)) != 0) return QBVM_ERR_UNSUPPORTED;       // half-length time transforms only
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
    rc = bupload(bt, &bt->gpow, gpow);
    if (!rc) rc = bupload(bt, &bt->gipw, gipw);
    if (!rc) rc = bupload(bt, &bt->gpowr, gpowr);
    if (!rc) rc = bupload(bt, &bt->gipr, gipr);
    if (!rc) rc = bupload(bt, &bt->ak, ak);
    if (!rc) rc = bupload(bt, &bt->cnorm, cnv);
    const long long Nx = tb.Nx;
    if (!rc) rc = balloc(bt, &bt->qinv, (size_t)count * H * Nx);
    if (!rc) {
        k_make_qinv_batched<<<grid_for((long long)count * H * Nx), 256>>>(bt->ak, tb.lamtau, bt->cnorm, H, Nx, count,
                                                                          bt->qinv);
        if (cudaGetLastError() != cudaSuccess) rc = QBVM_ERR_CUDA;
    }
    if (!rc && desc->rhs_kind == QBVM_RHS_DELTA) {
        rc = balloc(bt, &bt->ghat, (size_t)count * Nx);
        if (!rc) rc = balloc(bt, &bt->y0fac, (size_t)count * Nx);
        if (!rc) {
            k_y0fac_batched<<<grid_for((long long)count * Nx), 256>>>(bt->qinv, H, Nx, count, bt->y0fac);
            if (cudaGetLastError() != cudaSuccess) rc = QBVM_ERR_CUDA;
        }
    }
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

int solve_batched_dev(qbvm_batch_t* bt, const double* g_or_F, double* y, int n0_only, cudaStream_t s) {
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

int qbvm_batch_destroy(qbvm_batch_t* bt) {
    if (!bt) return QBVM_OK;                      // NULL is accepted, as by every destroy
    destroy_batch(bt);
    return QBVM_OK;
}

}  // extern "C"
