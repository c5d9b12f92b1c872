// gp_mll_grad_pathwise_noalloc: the pathwise gradient estimator with its scratch
// memory in a fixed, file-scope device array instead of a caller-provided buffer.
//
// Who needs it: callers that cannot allocate device memory at the point of the
// call -- code running while a stream is being captured into a CUDA graph
// (allocation calls are not permitted in the captured region), host callbacks
// enqueued on a stream (which may not call the CUDA API), and embedded or
// real-time hosts that fix their device memory budget up front.  The regular
// gp_mll_grad_pathwise needs a workspace that somebody has to allocate; this
// variant needs none beyond its inputs and outputs.
//
// The scratch holds the per-block partial sums of the fused reduction; every
// launch writes each partial it later reads, so nothing has to be cleared
// between calls.  All calls on one device share the one array: calls whose
// work overlaps on the GPU (different streams, no ordering between them) race
// on it and must not be issued.
#include "solvers.cuh"

#include <mutex>

namespace gp {

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[GP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The first call on
// a device looks it up (cudaGetSymbolAddress with that device current); the host
// symbol itself is only a stand-in and must never be passed to a kernel.
int scratch_for_current_device(void **out) {
    int dev = 0;
    GP_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d out of range", dev);
        return GP_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
            return GP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GP_OK;
}

}  // namespace

}  // namespace gp

using namespace gp;

extern "C" int gp_mll_grad_pathwise_noalloc(int kind, const double *theta, int d, const float *X, int64_t n,
                                            const float *Vsol, int s, double *grad, int prec, cudaStream_t stream) {
    clear_error();
    try {
        KP<float> kp;
        GP_TRY(make_kp<float>(kind, theta, d, &kp));
        if (n < 1 || s < 1) {
            set_error("need n >= 1 and s >= 1");
            return GP_ERR_INVALID_ARG;
        }
        if (!X || !Vsol || !grad) {
            set_error("null pointer argument");
            return GP_ERR_INVALID_ARG;
        }
        if (prec != GP_PREC_FP32 && prec != GP_PREC_TC16) {
            set_error("prec must be GP_PREC_FP32 (1) or GP_PREC_TC16 (2), got %d", prec);
            return GP_ERR_INVALID_ARG;
        }
        const size_t need = grad_workspace<float>(n, d, s + 1, prec);
        if (need > (size_t)GP_NOALLOC_SCRATCH_BYTES) {
            set_error("n=%lld, d=%d needs %zu bytes of scratch; the static scratch of "
                      "gp_mll_grad_pathwise_noalloc holds %zu bytes (use gp_mll_grad_pathwise)",
                      (long long)n, d, need, (size_t)GP_NOALLOC_SCRATCH_BYTES);
            return GP_ERR_INVALID_ARG;
        }
        void *scratch = nullptr;
        GP_TRY(scratch_for_current_device(&scratch));
        GradArgs<float> a;
        a.kp = kp;
        a.X = X;
        a.n = n;
        a.U0 = Vsol;
        a.U = Vsol + n;
        a.ldu = n;
        a.W0 = Vsol;
        a.W = Vsol + n;
        a.ldw = n;
        a.R = s + 1;
        a.lam0 = 0.5;
        a.lam_rest = -0.5 / (double)s;
        a.grad = grad;
        return apply_grad<float>(a, prec, scratch, (size_t)GP_NOALLOC_SCRATCH_BYTES, stream);
    } catch (...) {
        set_error("internal error");
        return GP_ERR_CUDA;
    }
}
