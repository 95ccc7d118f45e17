// qbvm_noalloc.cu -- qbvm_residual_noalloc: the relative all-at-once residual
// computed without a plan and without allocating any device memory.
//
// Its only scratch (the residual kernel's per-block partial sums and their
// two totals) lives in the file-scope array below, which every GPU that loads
// this library holds until the process exits.  Host code cannot use the
// array's name as a device address, so every call looks the address up with
// cudaGetSymbolAddress, with the call's device current.  The lookup allocates
// nothing and is not cached: a cached address would go stale if the caller
// reset the device (cudaDeviceReset) and the module were loaded again in a
// new context.
#include <cmath>

#include "qbvm.h"
#include "qbvm_internal.h"

namespace {

constexpr int NOALLOC_BLOCKS = 4096;                      // residual blocks the scratch holds
constexpr int NOALLOC_DOUBLES = 2 * NOALLOC_BLOCKS + 2;   // (r^2, f^2) per block + the two totals

static __device__ __align__(256) double qbvm_noalloc_scratch[NOALLOC_DOUBLES];

// Device address of the scratch array in the current device's context.
int scratch_address(double** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, qbvm_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    *out = static_cast<double*>(p);
    return QBVM_OK;
}

// True when `ptr` is device (or managed) memory of device `dev`, the device
// that owns the scratch and runs the kernel: memory of another GPU would be a
// peer access, which without peer mapping is an illegal address.
bool on_device(const void* ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" int qbvm_residual_noalloc(const qbvm_desc* desc, const double* y, const double* g_or_F,
                                     double* rel_norm_out, void* stream) {
    if (!desc || !y || !g_or_F || !rel_norm_out) return QBVM_ERR_BAD_ARG;
    int rc = qbvm::validate_desc(desc);
    if (rc) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    // host data would need staging memory; another GPU's memory is not ours to read
    if (!on_device(y, dev) || !on_device(g_or_F, dev)) return QBVM_ERR_BAD_ARG;

    // tau, alpha and omega exactly as qbvm_plan derives them (Sections 3.1/3.2, 5)
    const qbvm_desc& d = *desc;
    qbvm::Tables tb;
    tb.dim = d.dim;
    tb.nt = d.nt;
    tb.Nx = 1;
    double h2inv[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        tb.n[i] = i < d.dim ? d.m[i] - 1 : 1;
        if (i < d.dim) {
            double h = d.L / d.m[i];
            h2inv[i] = 1.0 / (h * h);
        }
        tb.Nx *= tb.n[i];
    }
    tb.tau = d.T / (d.nt - 1);
    const double alpha = d.alpha > 0 ? d.alpha : (d.form == QBVM_FORM_PQ ? d.delta : tb.tau * d.delta);
    tb.omega = d.form == QBVM_FORM_PQ ? -1.0 / alpha : -tb.tau / alpha;
    if (!(std::isfinite(alpha) && alpha > 0 && std::isfinite(tb.omega))) return QBVM_ERR_BAD_ARG;

    const int nblocks = qbvm::residual_blocks(tb);
    if (nblocks > NOALLOC_BLOCKS) return QBVM_ERR_UNSUPPORTED;       // more partial sums than the scratch holds
    double* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc) return rc;

    // Every block writes its own partial pair and the reduction overwrites the
    // totals, so nothing in the scratch has to be cleared between calls.
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* totals = scratch + 2 * NOALLOC_BLOCKS;
    if (qbvm::launch_residual(y, g_or_F, d.rhs_kind == QBVM_RHS_DELTA, tb, h2inv, scratch, nblocks, totals,
                              nullptr, s) != cudaSuccess)
        return QBVM_ERR_CUDA;
    double h[2] = {0, 0};
    if (cudaMemcpyAsync(h, totals, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return QBVM_ERR_CUDA;
    }
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return QBVM_ERR_NONFINITE;
    *rel_norm_out = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return QBVM_OK;
}
