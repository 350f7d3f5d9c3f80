// An FP32 + FP64-refinement solve that allocates no device memory.
//
// sptrsv_solve with SPTRSV_F32_IR precision needs two scratch arrays per
// call (the FP32 correction and the FP64 residual, n * nrhs elements each)
// and allocates them with cudaMalloc the first time a plan sees a given size.
// Some callers cannot allocate at solve time: code recording a CUDA graph,
// applications whose device memory is handed out by their own pool or fixed
// at start-up, real-time loops that must not synchronise the device.  This
// entry point runs the same kernels with that scratch taken from a
// file-scope __device__ array of fixed size instead.
#include <mutex>

#include "plan.cuh"

namespace sptrsv {
namespace {

// Largest n * nrhs the no-allocation solve accepts.
constexpr int64_t kNoAllocMaxElems = 1ll << 20;
constexpr size_t kR64Bytes = (size_t)kNoAllocMaxElems * sizeof(double);
constexpr size_t kD32Bytes = (size_t)kNoAllocMaxElems * sizeof(float);

// FP64 residuals first, then FP32 corrections: 12 MiB held by every device
// that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_ir_scratch[kR64Bytes + kD32Bytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_ir_scratch on the current device.  In host code the
// symbol is only a host-side handle; the address comes from the runtime,
// once per device, with that device current.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ir_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

sptrsv_status_t to_status(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA;
}

}  // namespace
}  // namespace sptrsv

using namespace sptrsv;

extern "C" SPTRSV_API sptrsv_status_t sptrsv_solve_ir_noalloc(sptrsv_plan_t p, const double *d_b,
                                                              double *d_x, int32_t nrhs,
                                                              sptrsv_stream_t stream) {
    if (!p) return SPTRSV_ERR_INVALID_ARG;
    if (p->latched != SPTRSV_OK) return SPTRSV_ERR_BAD_STATE;
    if (nrhs < 1) return SPTRSV_ERR_INVALID_ARG;
    if (p->prm.precision != SPTRSV_F32_IR || (p->n > 0 && !p->s32.built))
        return SPTRSV_ERR_BAD_STATE;
    const int32_t n = p->n;
    if (n == 0) return SPTRSV_OK;
    if (!d_b || !d_x) return SPTRSV_ERR_INVALID_ARG;
    const int64_t count = (int64_t)n * nrhs;
    if (count > kNoAllocMaxElems) return SPTRSV_ERR_UNSUPPORTED;
    const size_t bytes = (size_t)count * sizeof(double);
    const char *b0 = (const char *)d_b, *x0 = (const char *)d_x;
    if (b0 < x0 + bytes && x0 < b0 + bytes) return SPTRSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;

    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return to_status(e);
    double *r64 = (double *)base;
    float *d32 = (float *)((char *)base + kR64Bytes);

    const uint64_t tmo = (uint64_t)(p->prm.wait_timeout_ms > 0 ? p->prm.wait_timeout_ms : 5000) *
                         1000000ull;
    const SolveConfig &c = p->cfg;
    SolveData<float> sd = p->s32.view();
    sd.backoff_ns = c.backoff_ns;
    auto solve32 = [&](const double *rhs, bool skip) -> cudaError_t {
        for (int32_t c0 = 0; c0 < nrhs; c0 += 32) {
            const int nr = nrhs - c0 < 32 ? nrhs - c0 : 32;
            const int mx = max_coresident_ctas<float>(c.L, nr, c.syncfree, c.block_threads,
                                                      p->num_sms, p->s32.run_slots);
            if (mx <= 0) return cudaErrorInvalidConfiguration;
            LaunchCfg lc{c.block_threads, c.grid > 0 && c.grid < mx ? c.grid : mx};
            cudaError_t le = launch_solve<float>(sd, rhs + c0, d32 + c0, n, nrhs, nr, c.syncfree,
                                                 lc, p->status.p, tmo, skip, s);
            if (le != cudaSuccess) return le;
        }
        return cudaSuccess;
    };
    if ((e = launch_ir_begin(p->status.p, d_b, count, s)) != cudaSuccess) return to_status(e);
    if ((e = solve32(d_b, false)) != cudaSuccess) return to_status(e);
    if ((e = launch_ir_update(d_x, d32, count, true, p->status.p, s)) != cudaSuccess)
        return to_status(e);
    for (int it = 0; it < p->prm.ir_max_iter; ++it) {
        if ((e = launch_residual(n, p->row_ptr.p, p->col.p, p->val.p, p->rev, d_b, d_x, r64, nrhs, nrhs,
                                 p->status.p, s)) != cudaSuccess)
            return to_status(e);
        if ((e = launch_ir_decide(p->status.p, p->prm.ir_tol, p->lnorm.p, s)) != cudaSuccess)
            return to_status(e);
        if ((e = solve32(r64, true)) != cudaSuccess) return to_status(e);
        if ((e = launch_ir_update(d_x, d32, count, false, p->status.p, s)) != cudaSuccess)
            return to_status(e);
    }
    return SPTRSV_OK;
}
