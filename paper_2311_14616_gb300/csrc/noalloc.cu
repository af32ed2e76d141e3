// Residual entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they need a residual: code running
// inside a framework whose caching allocator already owns the device memory
// (a driver allocation there can fail or fragment the pool), latency-critical
// loops where cudaMalloc's implicit device synchronisation and unpredictable
// cost are not acceptable, and deployments whose policy allows allocation only
// at start-up.  ir_residual_noalloc serves them: its only workspace (the
// split-K partial sums of the residual) lives in a fixed array in device
// global memory that is part of this library's image.  Every GPU that loads
// the library holds that array (IR_RESIDUAL_NOALLOC_SCRATCH doubles, 8 MiB)
// until the process exits.
//
// Setup: the first successful call on a device (with that device current)
// looks up the array's device address with cudaGetSymbolAddress, once per
// device; make that first call before any stream capture begins.  A lookup
// that fails is not remembered: the next call tries again.  The address is
// kept for the life of the process, so resetting the device or its primary
// context after the first call is not supported.  The host-side name of the
// array is only a stand-in and is never handed to a kernel.
//
// Sharing: all calls use the same array.  Every partial sum a call reads was
// written by that call's first kernel, and the norm output is cleared by the
// call itself, so leftover contents of an earlier call do no harm -- but two
// calls whose work overlaps on the GPU (different streams, no ordering
// between them) race on the array and give wrong results.
#include <mutex>

#include "ir_internal.cuh"

namespace {

constexpr int64_t kScratchDoubles = IR_RESIDUAL_NOALLOC_SCRATCH;
static __device__ __align__(256) double g_resid_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double *g_scratch_dev[kMaxDevices];            // device address of the array, per device (null: not set up)
std::mutex g_setup_mutex;

// The array's device address on device `dev` (current), looked up on the first
// successful call; a failed lookup is retried by the next call.
cudaError_t scratch_address(int dev, double **out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[dev]) {
        double *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void **)&p, g_resid_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ir_status ir_residual_noalloc(int64_t n, ir_dtype TW, const void *A, int64_t lda,
                                         const void *b, const double *x, double *r,
                                         double *rnorm, void *stream) {
    if (n < 0 || (TW != IR_F64 && TW != IR_F32) || lda < (n > 1 ? n : 1)) return IR_EINVAL;
    if (n > 0 && (!A || !b || !x || !r || !rnorm)) return IR_EINVAL;
    if (n > IR_RESIDUAL_NOALLOC_MAX_N) return IR_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (n == 0) {
        if (rnorm && (e = cudaMemsetAsync(rnorm, 0, sizeof(double), s)) != cudaSuccess)
            return ir::record_cuda_error(e, "cudaMemsetAsync(rnorm)");
        return IR_OK;
    }
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return ir::record_cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return IR_EUNSUPPORTED;
    double *scratch = nullptr;
    if ((e = scratch_address(dev, &scratch)) != cudaSuccess)
        return ir::record_cuda_error(e, "cudaGetSymbolAddress(residual scratch)");
    int sms = 1;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return ir::record_cuda_error(e, "cudaDeviceGetAttribute");
    // fewer column splits when the partial sums would not fit the array
    while (sms > 1 && ir::residual_partials_needed(n, sms) > kScratchDoubles) sms /= 2;
    if (ir::residual_partials_needed(n, sms) > kScratchDoubles) return IR_EUNSUPPORTED;
    e = ir::launch_residual(n, TW, A, lda, b, x, r, scratch, kScratchDoubles,
                            reinterpret_cast<unsigned long long *>(rnorm), sms, s);
    return e == cudaSuccess ? IR_OK : ir::record_cuda_error(e, "launch_residual (noalloc)");
}
