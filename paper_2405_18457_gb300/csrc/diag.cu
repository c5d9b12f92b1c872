// Unit-rate probe: instruction throughput of the pipes that bound the hot-path kernels, per SM
// and per SM clock, measured on the device the library runs on (the MUFU rates are not
// published per chip, and the roofline of the kernel-matrix kernels is set by them).
//
// One CTA of 1024 threads per SM; every thread runs `iters` rounds of 8 independent chains of
// the probed instruction (enough independent work to keep the pipe full), bracketed by
// clock64() reads after a CTA barrier, so the rate is (instructions executed by the CTA) /
// (SM cycles between the barriers) and does not depend on the clock frequency.
#include "gp_internal.cuh"

#include <algorithm>
#include <vector>

namespace gp {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 8;

enum ProbeOp { P_EX2 = 0, P_RSQRT, P_SIN, P_COS, P_FFMA, P_DFMA, P_COUNT };

template <int OP>
__device__ __forceinline__ float probe_step(float a) {
    float r;
    if (OP == P_EX2) {
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-a));
    } else if (OP == P_RSQRT) {
        asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    } else if (OP == P_SIN) {
        asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    } else if (OP == P_COS) {
        asm volatile("cos.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    } else {
        asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(0.999f), "f"(0.001f));
    }
    return r;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads, 1) unit_rate_kernel(int iters, float *sink, long long *cycles) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 0.5f + 0.01f * (float)((threadIdx.x + k) & 15);
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = probe_step<OP>(a[k]);
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0f) sink[threadIdx.x] = s;  // never true: keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kProbeThreads, 1) unit_rate_f64_kernel(int iters, double *sink, long long *cycles) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 0.5 + 0.01 * (double)((threadIdx.x + k) & 15);
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(0.999), "d"(0.001));
    }
    __syncthreads();
    const long long t1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) sink[threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace
}  // namespace gp

using namespace gp;

// rates[0..5]: ex2, rsqrt, sin, cos (MUFU), FP32 FMA, FP64 FMA -- thread-instructions per SM per
// SM clock (median over the SMs).  ws: device scratch of gp_diag_unit_rates_workspace() bytes.
extern "C" size_t gp_diag_unit_rates_workspace(void) {
    return (size_t)(kProbeThreads * sizeof(double) + 4096 * sizeof(long long));
}

extern "C" int gp_diag_unit_rates(int iters, double *rates, void *ws, size_t ws_bytes, cudaStream_t st) {
    clear_error();
    if (!rates || !ws || iters < 1) {
        set_error("rates and ws must be non-null and iters >= 1");
        return GP_ERR_INVALID_ARG;
    }
    if (ws_bytes < gp_diag_unit_rates_workspace()) {
        set_error("unit-rate probe workspace holds %zu bytes, %zu required", ws_bytes, gp_diag_unit_rates_workspace());
        return GP_ERR_INVALID_ARG;
    }
    const int sms = std::min(device_sm_count(), 4096);
    double *sink = static_cast<double *>(ws);
    long long *cyc = reinterpret_cast<long long *>(static_cast<char *>(ws) + kProbeThreads * sizeof(double));
    std::vector<long long> h((size_t)sms);
    for (int op = 0; op < P_COUNT; ++op) {
        switch (op) {
            case P_EX2: unit_rate_kernel<P_EX2><<<sms, kProbeThreads, 0, st>>>(iters, (float *)sink, cyc); break;
            case P_RSQRT: unit_rate_kernel<P_RSQRT><<<sms, kProbeThreads, 0, st>>>(iters, (float *)sink, cyc); break;
            case P_SIN: unit_rate_kernel<P_SIN><<<sms, kProbeThreads, 0, st>>>(iters, (float *)sink, cyc); break;
            case P_COS: unit_rate_kernel<P_COS><<<sms, kProbeThreads, 0, st>>>(iters, (float *)sink, cyc); break;
            case P_FFMA: unit_rate_kernel<P_FFMA><<<sms, kProbeThreads, 0, st>>>(iters, (float *)sink, cyc); break;
            default: unit_rate_f64_kernel<<<sms, kProbeThreads, 0, st>>>(iters / 8 + 1, sink, cyc); break;
        }
        GP_TRY(check_launch("unit_rate_kernel"));
        GP_TRY_CUDA(cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost, st));
        GP_TRY_CUDA(cudaStreamSynchronize(st));
        std::sort(h.begin(), h.end());
        const double med = (double)h[h.size() / 2];
        const double it = (op == P_DFMA) ? (double)(iters / 8 + 1) : (double)iters;
        rates[op] = med > 0.0 ? it * kChains * kProbeThreads / med : 0.0;
    }
    return GP_OK;
}
