// qbvm_gmres.cu -- the original QBVM (A_h, eq. 2.3) and MQBVM (B_h, eq. 2.6)
// all-at-once systems of Section 2, solved by flexible right-preconditioned
// GMRES(m) (Saad, "A flexible inner-outer preconditioned GMRES algorithm",
// 1993) with the PinT direct solve of Section 3 as the preconditioner.
//
// Both systems share the backward Euler rows of the PinT systems,
//     (y^n - y^{n-1})/tau - Delta_h y^n = 0,   n = 1..N,
// and differ in the first block row:
//     A_h:  alpha y^0 + y^N = g,      B_h:  (alpha/tau)(y^0 - y^1) + y^N = g,
// while the PinT systems of eqs. 3.3/3.6, first row scaled by tau*alpha (PQ)
// or alpha (PM), read alpha (I - tau Delta_h) y^0 + y^N = g and
// alpha (I/tau - Delta_h) y^0 + y^N = g.  So M^{-1} v = PinT^{-1}(D^{-1} v)
// with D scaling block 0 by tau*alpha or alpha, and A M^{-1} = I + (a first
// block row term).
//
// Device work: the operator (a stencil kernel), batched dot products and
// updates for classical Gram-Schmidt applied twice, the preconditioner
// (qbvm_solve).  Host work: the (m+1) x m Hessenberg least-squares problem by
// Givens rotations.  Everything is FP64.
#include <cmath>
#include <new>
#include <vector>

#include "qbvm.h"
#include "qbvm_internal.h"

namespace {

constexpr int GT = 256;        // threads per block of the vector kernels
constexpr int KC = 8;          // dot products per k_mdot launch

long long grid_for(long long n) {
    long long b = (n + GT - 1) / GT;
    if (b > 152 * 8) b = 152 * 8;
    return b < 1 ? 1 : b;
}

// out = A y (method 0: A_h) or B_h y (method 1), y and out [nt][nz][ny][nx].
__global__ void k_apply_original(const double* __restrict__ y, double* __restrict__ out, int method, int nt, int nx,
                                 int ny, int nz, double inv_tau, double alpha, double cx, double cy, double cz) {
    const long long Nx = (long long)nx * ny * nz, N = (long long)nt * Nx, pl = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / Nx, s = i - t * Nx;
        double v;
        if (t == 0) {
            const double yN = y[(long long)(nt - 1) * Nx + s];
            if (method == QBVM_ORIGINAL_QBVM) v = alpha * y[s] + yN;
            else v = alpha * inv_tau * (y[s] - y[Nx + s]) + yN;
        } else {
            const long long iz = s / pl, rz = s - iz * pl, iy = rz / nx, ix = rz - iy * nx;
            const double yc = y[i];
            double lap = cx * (2.0 * yc - (ix > 0 ? y[i - 1] : 0.0) - (ix < nx - 1 ? y[i + 1] : 0.0));
            if (ny > 1) lap += cy * (2.0 * yc - (iy > 0 ? y[i - nx] : 0.0) - (iy < ny - 1 ? y[i + nx] : 0.0));
            if (nz > 1) lap += cz * (2.0 * yc - (iz > 0 ? y[i - pl] : 0.0) - (iz < nz - 1 ? y[i + pl] : 0.0));
            v = (yc - y[i - Nx]) * inv_tau + lap;
        }
        out[i] = v;
    }
}

// part[q * gridDim.x + block] = partial sums of <V_{j0+q}, w>, q < kc.
__global__ void __launch_bounds__(GT)
k_mdot(const double* __restrict__ V, long long ld, int j0, int kc, const double* __restrict__ w, long long N,
       double* __restrict__ part) {
    __shared__ double sh[KC][GT / 32];
    double acc[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) acc[q] = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int q = 0; q < KC; ++q)
            if (q < kc) acc[q] = fma(V[(long long)(j0 + q) * ld + i], wi, acc[q]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < KC; ++q) {
        double a = acc[q];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[q][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < KC && threadIdx.x < kc) {
        double a = 0.0;
        for (int k = 0; k < GT / 32; ++k) a += sh[threadIdx.x][k];
        part[(long long)threadIdx.x * gridDim.x + blockIdx.x] = a;
    }
}

// out[j0 + q] = sum over blocks of part[q][.], one block per q.
__global__ void k_mdot_reduce(const double* __restrict__ part, int nb, int j0, double* __restrict__ out) {
    __shared__ double sh[GT / 32];
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[(long long)blockIdx.x * nb + i];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
        out[j0 + blockIdx.x] = t;
    }
}

// w += sgn * sum_{j<k} c[j] V_j   (c on the device)
__global__ void k_mupdate(double* __restrict__ w, const double* __restrict__ V, long long ld, int k,
                          const double* __restrict__ c, double sgn, long long N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int j = 0; j < k; ++j) a = fma(c[j], V[(long long)j * ld + i], a);
        w[i] = fma(sgn, a, w[i]);
    }
}

// dst = a * (src - sub) (sub may be null); the first n0 entries get the extra factor a0
__global__ void k_scale(double* __restrict__ dst, const double* __restrict__ src, const double* __restrict__ sub,
                        double a, long long n0, double a0, long long N) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double v = sub ? src[i] - sub[i] : src[i];
        dst[i] = (i < n0 ? a * a0 : a) * v;
    }
}

}  // namespace

struct qbvm_gmres {
    qbvm_plan_t* plan = nullptr;
    qbvm::PlanView pv{};
    int method = 0, m = 0;
    long long Nx = 0, N = 0;
    int nb = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *tmp = nullptr, *f = nullptr;
    double *part = nullptr, *dots = nullptr;   // dots: [0, m+1) pass 1, [m+1, 2m+2) pass 2, [2m+2] norm
};

namespace {

#define GK(...)                                       \
    do {                                              \
        if ((__VA_ARGS__) != cudaSuccess) {           \
            cudaGetLastError();                       \
            return QBVM_ERR_CUDA;                     \
        }                                             \
    } while (0)

void free_gmres(qbvm_gmres_t* g) {
    if (!g) return;
    for (double* p : {g->V, g->Z, g->w, g->tmp, g->f, g->part, g->dots}) cudaFree(p);
    delete g;
}

int apply_op(qbvm_gmres_t* g, const double* y, double* out, cudaStream_t s) {
    const qbvm::Tables& tb = *g->pv.tb;
    k_apply_original<<<(unsigned)grid_for(g->N), GT, 0, s>>>(y, out, g->method, tb.nt, tb.n[0], tb.n[1], tb.n[2],
                                                               1.0 / g->pv.tau, g->pv.alpha, g->pv.h2inv[0],
                                                               g->pv.h2inv[1], g->pv.h2inv[2]);
    GK(cudaGetLastError());
    return QBVM_OK;
}

// dots[off + j] = <V_j, w>, j < k  (V may be w itself with k = 1)
int mdot(qbvm_gmres_t* g, const double* V, int k, const double* w, int off, cudaStream_t s) {
    for (int j0 = 0; j0 < k; j0 += KC) {
        const int kc = k - j0 < KC ? k - j0 : KC;
        k_mdot<<<g->nb, GT, 0, s>>>(V, g->N, j0, kc, w, g->N, g->part);
        GK(cudaGetLastError());
        k_mdot_reduce<<<kc, GT, 0, s>>>(g->part, g->nb, off + j0, g->dots);
        GK(cudaGetLastError());
    }
    return QBVM_OK;
}

int norm2(qbvm_gmres_t* g, const double* w, double* out, cudaStream_t s) {
    int rc = mdot(g, w, 1, w, 2 * g->m + 2, s);
    if (rc) return rc;
    double h = 0.0;
    GK(cudaMemcpyAsync(&h, g->dots + 2 * g->m + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    GK(cudaStreamSynchronize(s));
    if (!std::isfinite(h)) return QBVM_ERR_NONFINITE;
    *out = std::sqrt(h);
    return QBVM_OK;
}

}  // namespace

extern "C" {

int qbvm_gmres_create(qbvm_plan_t* plan, int method, int restart, qbvm_gmres_t** out) {
    if (!plan || !out || restart < 1 || restart > 64) return QBVM_ERR_BAD_ARG;
    if (method != QBVM_ORIGINAL_QBVM && method != QBVM_ORIGINAL_MQBVM) return QBVM_ERR_BAD_ARG;
    *out = nullptr;
    qbvm::PlanView pv;
    int rc = qbvm::plan_view(plan, &pv);
    if (rc) return rc;
    if (pv.precision != QBVM_FP64 || pv.rhs_kind != QBVM_RHS_GENERAL) return QBVM_ERR_UNSUPPORTED;
    if ((method == QBVM_ORIGINAL_QBVM) != (pv.form == QBVM_FORM_PQ)) return QBVM_ERR_BAD_ARG;
    qbvm_gmres_t* g = new (std::nothrow) qbvm_gmres();
    if (!g) return QBVM_ERR_OOM;
    g->plan = plan;
    g->pv = pv;
    g->method = method;
    g->m = restart;
    g->Nx = pv.tb->Nx;
    g->N = pv.tb->Nx * pv.tb->nt;
    g->nb = (int)grid_for(g->N);
    const size_t n = (size_t)g->N;
    bool ok = cudaMalloc(&g->V, sizeof(double) * n * (restart + 1)) == cudaSuccess &&
              cudaMalloc(&g->Z, sizeof(double) * n * restart) == cudaSuccess &&
              cudaMalloc(&g->w, sizeof(double) * n) == cudaSuccess &&
              cudaMalloc(&g->tmp, sizeof(double) * n) == cudaSuccess &&
              cudaMalloc(&g->f, sizeof(double) * n) == cudaSuccess &&
              cudaMalloc(&g->part, sizeof(double) * (size_t)g->nb * KC) == cudaSuccess &&
              cudaMalloc(&g->dots, sizeof(double) * (2 * restart + 3)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_gmres(g);
        return QBVM_ERR_OOM;
    }
    *out = g;
    return QBVM_OK;
}

int qbvm_gmres_solve(qbvm_gmres_t* g, const double* gin, double* y, double tol, int max_iters, int* iters,
                     double* rel_residual, void* stream) {
    if (!g || !gin || !y || !(tol > 0) || max_iters < 1) return QBVM_ERR_BAD_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long N = g->N, Nx = g->Nx;
    const int m = g->m;
    const double pre = g->method == QBVM_ORIGINAL_QBVM ? 1.0 / (g->pv.tau * g->pv.alpha) : 1.0 / g->pv.alpha;
    int rc;
    // f = (g, 0, ..., 0); y = 0
    GK(cudaMemsetAsync(g->f, 0, sizeof(double) * N, s));
    GK(cudaMemcpyAsync(g->f, gin, sizeof(double) * Nx, cudaMemcpyDeviceToDevice, s));
    GK(cudaMemsetAsync(y, 0, sizeof(double) * N, s));
    double beta0 = 0.0;
    if ((rc = norm2(g, g->f, &beta0, s))) return rc;
    if (iters) *iters = 0;
    if (beta0 == 0.0) {
        if (rel_residual) *rel_residual = 0.0;
        return QBVM_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hcol(2 * m + 3);
    auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    int total = 0;
    double rel = 1.0, prev_rel = INFINITY;
    for (;;) {
        // true residual r = f - A y into V_0
        if ((rc = apply_op(g, y, g->w, s))) return rc;
        k_scale<<<(unsigned)grid_for(N), GT, 0, s>>>(g->V, g->f, g->w, 1.0, 0, 1.0, N);
        GK(cudaGetLastError());
        double beta = 0.0;
        if ((rc = norm2(g, g->V, &beta, s))) return rc;
        rel = beta / beta0;
        if (rel <= tol || total >= max_iters) break;
        // a whole restart cycle that gains less than 10 %: the FP64 floor of the
        // true residual of the original system lies above tol
        if (rel > 0.9 * prev_rel) break;
        prev_rel = rel;
        k_scale<<<(unsigned)grid_for(N), GT, 0, s>>>(g->V, g->V, nullptr, 1.0 / beta, 0, 1.0, N);
        GK(cudaGetLastError());
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int j = 0;
        for (; j < m && total < max_iters; ++j) {
            double* Vj = g->V + (size_t)j * N;
            double* Zj = g->Z + (size_t)j * N;
            // preconditioner: Z_j = PinT^{-1} (D^{-1} V_j)
            k_scale<<<(unsigned)grid_for(N), GT, 0, s>>>(g->tmp, Vj, nullptr, 1.0, Nx, pre, N);
            GK(cudaGetLastError());
            if ((rc = qbvm_solve(g->plan, g->tmp, Zj, 0, s))) return rc;
            if ((rc = apply_op(g, Zj, g->w, s))) return rc;
            // classical Gram-Schmidt, twice
            for (int pass = 0; pass < 2; ++pass) {
                const int off = pass * (m + 1);
                if ((rc = mdot(g, g->V, j + 1, g->w, off, s))) return rc;
                k_mupdate<<<(unsigned)grid_for(N), GT, 0, s>>>(g->w, g->V, N, j + 1, g->dots + off, -1.0, N);
                GK(cudaGetLastError());
            }
            if ((rc = mdot(g, g->w, 1, g->w, 2 * m + 2, s))) return rc;
            GK(cudaMemcpyAsync(hcol.data(), g->dots, sizeof(double) * (2 * m + 3), cudaMemcpyDeviceToHost, s));
            GK(cudaStreamSynchronize(s));
            const double hn = std::sqrt(hcol[2 * m + 2]);
            if (!std::isfinite(hn)) return QBVM_ERR_NONFINITE;
            for (int i = 0; i <= j; ++i) Hij(i, j) = hcol[i] + hcol[m + 1 + i];
            Hij(j + 1, j) = hn;
            ++total;
            if (hn > 0) {
                k_scale<<<(unsigned)grid_for(N), GT, 0, s>>>(g->V + (size_t)(j + 1) * N, g->w, nullptr, 1.0 / hn, 0,
                                                              1.0, N);
                GK(cudaGetLastError());
            }
            // Givens rotations on the new column
            for (int i = 0; i < j; ++i) {
                const double a = Hij(i, j), b = Hij(i + 1, j);
                Hij(i, j) = cs[i] * a + sn[i] * b;
                Hij(i + 1, j) = -sn[i] * a + cs[i] * b;
            }
            const double a = Hij(j, j), b = Hij(j + 1, j), r = std::hypot(a, b);
            cs[j] = r > 0 ? a / r : 1.0;
            sn[j] = r > 0 ? b / r : 0.0;
            Hij(j, j) = r;
            Hij(j + 1, j) = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            if (std::fabs(gv[j + 1]) <= tol * beta0 || hn == 0.0) {
                ++j;
                break;
            }
        }
        // y += Z c with H(0:j, 0:j) c = gv(0:j)
        std::vector<double> c(j, 0.0);
        for (int i = j - 1; i >= 0; --i) {
            double t = gv[i];
            for (int k = i + 1; k < j; ++k) t -= Hij(i, k) * c[k];
            c[i] = Hij(i, i) != 0.0 ? t / Hij(i, i) : 0.0;
        }
        if (j > 0) {
            GK(cudaMemcpyAsync(g->dots, c.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
            k_mupdate<<<(unsigned)grid_for(N), GT, 0, s>>>(y, g->Z, N, j, g->dots, 1.0, N);
            GK(cudaGetLastError());
        }
    }
    if (iters) *iters = total;
    if (rel_residual) *rel_residual = rel;
    return rel <= tol ? QBVM_OK : QBVM_ERR_DIVERGED;
}

int qbvm_gmres_destroy(qbvm_gmres_t* g) {
    free_gmres(g);
    return QBVM_OK;
}

}  // extern "C"
