// C-ABI entry points: argument validation, error reporting and dispatch.
#include "gp_internal.cuh"
#include "solvers.cuh"

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

namespace gp {

static thread_local char g_err[1024];

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

static std::atomic<long long> g_launches{0};

int check_launch(const char *what, int count) {
    g_launches.fetch_add(count, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
        return GP_ERR_CUDA;
    }
    return GP_OK;
}

// Event pool for the optional product-kernel timing.
namespace {
struct Span {
    cudaEvent_t start, end;
    int tag;
};
struct Prof {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<Span> spans;
    cudaEvent_t open = nullptr;
    int open_tag = 0;
};
Prof &prof() {
    static Prof p;
    return p;
}
cudaEvent_t take_event(Prof &p) {
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

void prof_begin(cudaStream_t st, int tag) {
    Prof &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    if (!p.on) return;
    p.open = take_event(p);
    p.open_tag = tag;
    cudaEventRecord(p.open, st);
}

void prof_end(cudaStream_t st) {
    Prof &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    if (!p.on || p.open == nullptr) return;
    cudaEvent_t e = take_event(p);
    cudaEventRecord(e, st);
    p.spans.push_back(Span{p.open, e, p.open_tag});
    p.open = nullptr;
}

namespace {
std::mutex g_dev_mu;                                   // guards the two per-device caches below
std::set<std::pair<int, const void *>> g_smem_raised;  // (device, kernel) pairs already set up
std::map<int, int> g_sm_count;                          // device -> SM count
}  // namespace

int ensure_max_dyn_smem(const void *kernel) {
    int dev = 0;
    GP_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (g_smem_raised.count({dev, kernel})) return GP_OK;
    GP_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
    g_smem_raised.insert({dev, kernel});
    return GP_OK;
}

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 152;
    }
    std::lock_guard<std::mutex> g(g_dev_mu);
    auto it = g_sm_count.find(dev);
    if (it != g_sm_count.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    g_sm_count[dev] = sms;
    return sms;
}

int check_ws(void *ws, size_t ws_bytes, size_t need) {
    if (need == 0) return GP_OK;
    if (ws == nullptr) {
        set_error("workspace is null but %zu bytes are required", need);
        return GP_ERR_WORKSPACE;
    }
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
        set_error("workspace must be 256-byte aligned");
        return GP_ERR_WORKSPACE;
    }
    if (ws_bytes < need) {
        set_error("workspace holds %zu bytes, %zu required", ws_bytes, need);
        return GP_ERR_WORKSPACE;
    }
    return GP_OK;
}

template <typename T>
int make_kp(int kind, const double *theta, int d, KP<T> *kp) {
    if (kind != GP_RBF && kind != GP_MATERN32) {
        set_error("kind must be GP_RBF (0) or GP_MATERN32 (1), got %d", kind);
        return GP_ERR_INVALID_ARG;
    }
    if (d < 1 || d > GP_MAX_D) {
        set_error("d must be in [1, %d], got %d", GP_MAX_D, d);
        return GP_ERR_INVALID_ARG;
    }
    if (theta == nullptr) {
        set_error("theta is null");
        return GP_ERR_INVALID_ARG;
    }
    for (int k = 0; k < d + 2; ++k) {
        if (!(std::isfinite(theta[k]) && theta[k] > 0.0)) {
            set_error("theta[%d] = %g must be finite and positive", k, theta[k]);
            return GP_ERR_INVALID_ARG;
        }
    }
    std::memset(kp, 0, sizeof(*kp));
    kp->kind = kind;
    kp->d = d;
    for (int k = 0; k < d; ++k) {
        kp->ell[k] = (T)theta[k];
        kp->inv_ell[k] = (T)(1.0 / theta[k]);
    }
    kp->sf = (T)theta[d];
    kp->sf2 = (T)(theta[d] * theta[d]);
    kp->sigma = (T)theta[d + 1];
    kp->sigma2 = (T)(theta[d + 1] * theta[d + 1]);
    return GP_OK;
}
template int make_kp<float>(int, const double *, int, KP<float> *);
template int make_kp<double>(int, const double *, int, KP<double> *);

}  // namespace gp

using namespace gp;

#define GP_API_BEGIN \
    clear_error();   \
    try {
#define GP_API_END                                          \
    }                                                       \
    catch (const std::exception &ex) {                      \
        set_error("internal error: %s", ex.what());         \
        return GP_ERR_CUDA;                                 \
    }                                                       \
    catch (...) {                                           \
        set_error("internal error");                        \
        return GP_ERR_CUDA;                                 \
    }

#define REQ(cond, ...)                     \
    do {                                   \
        if (!(cond)) {                     \
            set_error(__VA_ARGS__);        \
            return GP_ERR_INVALID_ARG;     \
        }                                  \
    } while (0)

namespace {

int check_prec(int prec) {
    if (prec != GP_PREC_FP32 && prec != GP_PREC_TC16) {
        set_error("prec must be GP_PREC_FP32 (1) or GP_PREC_TC16 (2), got %d", prec);
        return GP_ERR_INVALID_ARG;
    }
    if (prec == GP_PREC_TC16 && !tc_available()) {
        set_error("GP_PREC_TC16 needs an sm_103 device with tcgen05");
        return GP_ERR_UNSUPPORTED;
    }
    return GP_OK;
}

// The products also take the split tensor-core form.
int check_prec_mvm(int prec) {
    if (prec == GP_PREC_TC16X3) return check_prec(GP_PREC_TC16);
    return check_prec(prec);
}

template <typename T>
int mvm_common(int kind, const double *theta, int d, const T *X1, int64_t n1, const T *X2, int64_t n2,
               const T *V, int64_t ldv, int nrhs, T *Y, int64_t ldy, int add_noise, int prec, void *ws,
               size_t ws_bytes, cudaStream_t st) {
    REQ(n1 >= 0 && n2 >= 0 && nrhs >= 0, "sizes must be non-negative");
    if (n1 == 0 || nrhs == 0) return GP_OK;
    REQ(Y != nullptr && X1 != nullptr, "X1 and Y must not be null");
    REQ(ldy >= n1, "ldy (%lld) must be >= n1 (%lld)", (long long)ldy, (long long)n1);
    if (n2 > 0) {
        REQ(X2 != nullptr && V != nullptr, "X2 and V must not be null");
        REQ(ldv >= n2, "ldv (%lld) must be >= n2 (%lld)", (long long)ldv, (long long)n2);
    }
    REQ(add_noise == 0 || (X1 == X2 && n1 == n2), "add_noise requires X1 == X2 and n1 == n2");
    if (sizeof(T) == sizeof(float)) GP_TRY(check_prec_mvm(prec));
    KP<T> kp;
    GP_TRY(make_kp<T>(kind, theta, d, &kp));
    if (n2 == 0) {
        for (int c = 0; c < nrhs; ++c) GP_TRY_CUDA(cudaMemsetAsync(Y + (int64_t)c * ldy, 0, sizeof(T) * n1, st));
        return GP_OK;
    }
    return apply_mvm<T>(kp, X1, n1, X2, n2, V, ldv, nrhs, Y, ldy, add_noise, prec, ws, ws_bytes, st);
}

template <typename T>
int solver_args(int kind, const double *theta, int d, const T *X, int64_t n, const T *B, int nrhs,
                T *V, int64_t max_iters, double tol, int stop_rule, gp_solve_info_t *info, KP<T> *kp) {
    REQ(X != nullptr && B != nullptr && V != nullptr && info != nullptr, "null pointer argument");
    REQ(n >= 1, "n must be >= 1");
    REQ(nrhs >= 1, "nrhs must be >= 1");
    REQ(max_iters >= 0, "max_iters must be >= 0");
    REQ(tol >= 0.0 && std::isfinite(tol), "tol must be finite and >= 0");
    REQ(stop_rule == GP_STOP_BOTH || stop_rule == GP_STOP_EITHER, "stop_rule must be 0 or 1");
    std::memset(info, 0, sizeof(*info));
    return make_kp<T>(kind, theta, d, kp);
}

template <typename T>
int rkhs_common(int kind, const double *theta, int d, const T *X, int64_t n, const T *Uinit, const T *U, int R,
                double *dist, int prec, void *ws, size_t ws_bytes, cudaStream_t stream) {
    KP<T> kp;
    GP_TRY(make_kp<T>(kind, theta, d, &kp));
    REQ(n >= 1 && R >= 0, "need n >= 1 and R >= 0");
    if (R == 0) return GP_OK;
    REQ(X && U && dist, "null pointer argument");
    if (sizeof(T) == sizeof(float)) GP_TRY(check_prec(prec));
    return rkhs_sqdist<T>(kp, X, n, Uinit, U, R, dist, prec, ws, ws_bytes, stream);
}

}  // namespace

extern "C" {

const char *gp_last_error(void) { return gp::g_err; }

int gp_version(void) { return 10000; }

void gp_diag_reset(int time_products) {
    Prof &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (auto &s : p.spans) {
        p.pool.push_back(s.start);
        p.pool.push_back(s.end);
    }
    p.spans.clear();
    p.on = time_products != 0;
    g_launches.store(0);
}

long long gp_diag_launches(void) { return g_launches.load(); }

int gp_device_check(cudaStream_t stream) {
    GP_API_BEGIN
    return tc_timeout_status(stream);
    GP_API_END
}

int gp_diag_timeout_probe(long long wait_cycles, cudaStream_t stream) {
    GP_API_BEGIN
    REQ(wait_cycles >= 0 && wait_cycles <= 4000000000LL, "wait_cycles must be in [0, 4e9]");
    return tc_timeout_probe(wait_cycles, stream);
    GP_API_END
}

int gp_diag_kernel_time(int which, double *total_ms, long long *count) {
    GP_API_BEGIN
    REQ(total_ms && count, "null pointer argument");
    REQ(which == 0 || which == 1, "which must be 0 (products) or 1 (gradients)");
    Prof &p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    double tot = 0.0;
    long long cnt = 0;
    for (auto &s : p.spans) {
        if (s.tag != which) continue;
        GP_TRY_CUDA(cudaEventSynchronize(s.end));
        float ms = 0.0f;
        GP_TRY_CUDA(cudaEventElapsedTime(&ms, s.start, s.end));
        tot += ms;
        ++cnt;
    }
    *total_ms = tot;
    *count = cnt;
    return GP_OK;
    GP_API_END
}

int gp_diag_product_time(double *total_ms, long long *count) { return gp_diag_kernel_time(0, total_ms, count); }

// ------------------------------------------------------------------ MVM
size_t gp_kernel_mvm_workspace(int64_t n1, int64_t n2, int d, int nrhs, int prec) {
    return mvm_workspace<float>(n1, n2, d, nrhs, prec);
}
size_t gp_kernel_mvm_f64_workspace(int64_t n1, int64_t n2, int d, int nrhs) {
    return mvm_workspace<double>(n1, n2, d, nrhs, GP_PREC_FP32);
}

int gp_kernel_mvm(int kind, const double *theta, int d, const float *X1, int64_t n1, const float *X2,
                  int64_t n2, const float *V, int64_t ldv, int nrhs, float *Y, int64_t ldy, int add_noise,
                  int prec, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    return mvm_common<float>(kind, theta, d, X1, n1, X2, n2, V, ldv, nrhs, Y, ldy, add_noise, prec, ws,
                             ws_bytes, stream);
    GP_API_END
}

int gp_kernel_mvm_f64(int kind, const double *theta, int d, const double *X1, int64_t n1,
                      const double *X2, int64_t n2, const double *V, int64_t ldv, int nrhs, double *Y,
                      int64_t ldy, int add_noise, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    return mvm_common<double>(kind, theta, d, X1, n1, X2, n2, V, ldv, nrhs, Y, ldy, add_noise,
                              GP_PREC_FP32, ws, ws_bytes, stream);
    GP_API_END
}

// ------------------------------------------------------------------ CG
size_t gp_solve_cg_workspace(int64_t n, int d, int nrhs, int prec) {
    return cg_workspace<float>(n, d, nrhs, prec);
}
size_t gp_solve_cg_f64_workspace(int64_t n, int d, int nrhs) {
    return cg_workspace<double>(n, d, nrhs, GP_PREC_FP32);
}

int gp_solve_cg(int kind, const double *theta, int d, const float *X, int64_t n, const float *B, int nrhs,
                float *V_inout, int64_t max_iters, double tol, int stop_rule, int prec,
                gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(solver_args<float>(kind, theta, d, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, info, &kp));
    GP_TRY(check_prec(prec));
    return cg_solve<float>(kp, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, prec, info, ws, ws_bytes,
                           stream);
    GP_API_END
}

int gp_solve_cg_f64(int kind, const double *theta, int d, const double *X, int64_t n, const double *B,
                    int nrhs, double *V_inout, int64_t max_iters, double tol, int stop_rule,
                    gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<double> kp;
    GP_TRY(solver_args<double>(kind, theta, d, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, info, &kp));
    return cg_solve<double>(kp, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, GP_PREC_FP32, info, ws,
                            ws_bytes, stream);
    GP_API_END
}

// ------------------------------------------------------------------ preconditioned CG
size_t gp_solve_pcg_workspace(int64_t n, int d, int nrhs, int prec, int rank) {
    return cg_workspace<float>(n, d, nrhs, prec, std::max(0, std::min<int>(rank, (int)std::min<int64_t>(n, 128))));
}
size_t gp_solve_pcg_f64_workspace(int64_t n, int d, int nrhs, int rank) {
    return cg_workspace<double>(n, d, nrhs, GP_PREC_FP32,
                                std::max(0, std::min<int>(rank, (int)std::min<int64_t>(n, 128))));
}

int gp_solve_pcg(int kind, const double *theta, int d, const float *X, int64_t n, const float *B, int nrhs,
                 float *V_inout, int64_t max_iters, double tol, int stop_rule, int prec, int rank,
                 gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(solver_args<float>(kind, theta, d, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, info, &kp));
    GP_TRY(check_prec(prec));
    REQ(rank >= 0 && rank <= 128, "rank must be in [0, 128]");
    const int k = (int)std::min<int64_t>(rank, n);
    return cg_solve<float>(kp, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, prec, info, ws, ws_bytes,
                           stream, k);
    GP_API_END
}

int gp_solve_pcg_f64(int kind, const double *theta, int d, const double *X, int64_t n, const double *B,
                     int nrhs, double *V_inout, int64_t max_iters, double tol, int stop_rule, int rank,
                     gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<double> kp;
    GP_TRY(solver_args<double>(kind, theta, d, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, info, &kp));
    REQ(rank >= 0 && rank <= 128, "rank must be in [0, 128]");
    const int k = (int)std::min<int64_t>(rank, n);
    return cg_solve<double>(kp, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, GP_PREC_FP32, info, ws,
                            ws_bytes, stream, k);
    GP_API_END
}

// ------------------------------------------------------------------ AP
size_t gp_solve_ap_workspace(int64_t n, int d, int nrhs, int64_t block_size, int prec) {
    return ap_workspace<float>(n, d, nrhs, block_size, prec);
}
size_t gp_solve_ap_f64_workspace(int64_t n, int d, int nrhs, int64_t block_size) {
    return ap_workspace<double>(n, d, nrhs, block_size, GP_PREC_FP32);
}

int gp_solve_ap(int kind, const double *theta, int d, const float *X, int64_t n, const float *B, int nrhs,
                float *V_inout, int64_t block_size, int64_t max_iters, double tol, int stop_rule, int prec,
                gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(solver_args<float>(kind, theta, d, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, info, &kp));
    GP_TRY(check_prec(prec));
    REQ(block_size >= 1 && block_size <= 1024, "block_size must be in [1, 1024]");
    return ap_solve<float>(kp, X, n, B, nrhs, V_inout, block_size, max_iters, tol, stop_rule, prec, info, ws,
                           ws_bytes, stream);
    GP_API_END
}

int gp_solve_ap_f64(int kind, const double *theta, int d, const double *X, int64_t n, const double *B,
                    int nrhs, double *V_inout, int64_t block_size, int64_t max_iters, double tol,
                    int stop_rule, gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<double> kp;
    GP_TRY(solver_args<double>(kind, theta, d, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, info, &kp));
    REQ(block_size >= 1 && block_size <= 1024, "block_size must be in [1, 1024]");
    return ap_solve<double>(kp, X, n, B, nrhs, V_inout, block_size, max_iters, tol, stop_rule, GP_PREC_FP32,
                            info, ws, ws_bytes, stream);
    GP_API_END
}

// ------------------------------------------------------------------ SGD
size_t gp_solve_sgd_workspace(int64_t n, int d, int nrhs, int64_t batch, int prec) {
    return sgd_workspace<float>(n, d, nrhs, batch, prec);
}
size_t gp_solve_sgd_f64_workspace(int64_t n, int d, int nrhs, int64_t batch) {
    return sgd_workspace<double>(n, d, nrhs, batch, GP_PREC_FP32);
}

int gp_solve_sgd(int kind, const double *theta, int d, const float *X, int64_t n, const float *B, int nrhs,
                 float *V_inout, int64_t batch, const int32_t *batch_idx, double lr, double momentum,
                 int64_t max_iters, double tol, int stop_rule, int prec, gp_solve_info_t *info, void *ws,
                 size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(solver_args<float>(kind, theta, d, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, info, &kp));
    GP_TRY(check_prec(prec));
    REQ(batch >= 1 && batch <= n, "batch must be in [1, n]");
    REQ(batch_idx != nullptr || max_iters == 0, "batch_idx is null");
    REQ(std::isfinite(lr) && lr > 0 && std::isfinite(momentum) && momentum >= 0 && momentum < 1,
        "need lr > 0 and 0 <= momentum < 1");
    return sgd_solve<float>(kp, X, n, B, nrhs, V_inout, batch, batch_idx, lr, momentum, max_iters, tol,
                            stop_rule, prec, info, ws, ws_bytes, stream);
    GP_API_END
}

int gp_solve_sgd_f64(int kind, const double *theta, int d, const double *X, int64_t n, const double *B,
                     int nrhs, double *V_inout, int64_t batch, const int32_t *batch_idx, double lr,
                     double momentum, int64_t max_iters, double tol, int stop_rule, gp_solve_info_t *info,
                     void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<double> kp;
    GP_TRY(solver_args<double>(kind, theta, d, X, n, B, nrhs, V_inout, max_iters, tol, stop_rule, info, &kp));
    REQ(batch >= 1 && batch <= n, "batch must be in [1, n]");
    REQ(batch_idx != nullptr || max_iters == 0, "batch_idx is null");
    REQ(std::isfinite(lr) && lr > 0 && std::isfinite(momentum) && momentum >= 0 && momentum < 1,
        "need lr > 0 and 0 <= momentum < 1");
    return sgd_solve<double>(kp, X, n, B, nrhs, V_inout, batch, batch_idx, lr, momentum, max_iters, tol,
                             stop_rule, GP_PREC_FP32, info, ws, ws_bytes, stream);
    GP_API_END
}

// ------------------------------------------------------------------ RFF
int gp_rff_prior_sample(int kind, const double *theta, int d, const float *X, int64_t n, int m,
                        const float *omega_hat, const float *chi2, const float *W, int s, float *F,
                        int64_t ldf, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(make_kp<float>(kind, theta, d, &kp));
    REQ(n >= 0 && s >= 0, "sizes must be non-negative");
    REQ(m >= 2 && m % 2 == 0, "m must be even and >= 2");
    if (n == 0 || s == 0) return GP_OK;
    REQ(X && omega_hat && W && F, "null pointer argument");
    REQ(kind == GP_RBF || chi2 != nullptr, "chi2 is required for Matern-3/2");
    REQ(ldf >= n, "ldf must be >= n");
    return rff_prior<float>(kp, X, n, m, omega_hat, chi2, W, s, F, ldf, stream);
    GP_API_END
}

size_t gp_rff_prior_sample_workspace(int d, int m, int s, int prec) { return rff_workspace(d, m, s, prec); }

int gp_rff_prior_sample_ws(int kind, const double *theta, int d, const float *X, int64_t n, int m,
                           const float *omega_hat, const float *chi2, const float *W, int s, float *F, int64_t ldf,
                           int prec, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(make_kp<float>(kind, theta, d, &kp));
    REQ(n >= 0 && s >= 0, "sizes must be non-negative");
    REQ(m >= 2 && m % 2 == 0, "m must be even and >= 2");
    if (n == 0 || s == 0) return GP_OK;
    REQ(X && omega_hat && W && F, "null pointer argument");
    REQ(kind == GP_RBF || chi2 != nullptr, "chi2 is required for Matern-3/2");
    REQ(ldf >= n, "ldf must be >= n");
    GP_TRY(check_prec(prec));
    return rff_prior_ws(kp, X, n, m, omega_hat, chi2, W, s, F, ldf, prec, ws, ws_bytes, stream);
    GP_API_END
}

int gp_rff_prior_sample_f64(int kind, const double *theta, int d, const double *X, int64_t n, int m,
                            const double *omega_hat, const double *chi2, const double *W, int s, double *F,
                            int64_t ldf, cudaStream_t stream) {
    GP_API_BEGIN
    KP<double> kp;
    GP_TRY(make_kp<double>(kind, theta, d, &kp));
    REQ(n >= 0 && s >= 0, "sizes must be non-negative");
    REQ(m >= 2 && m % 2 == 0, "m must be even and >= 2");
    if (n == 0 || s == 0) return GP_OK;
    REQ(X && omega_hat && W && F, "null pointer argument");
    REQ(kind == GP_RBF || chi2 != nullptr, "chi2 is required for Matern-3/2");
    REQ(ldf >= n, "ldf must be >= n");
    return rff_prior<double>(kp, X, n, m, omega_hat, chi2, W, s, F, ldf, stream);
    GP_API_END
}

int gp_pathwise_rhs(const double *theta, int d, const float *y, const float *F, const float *w, int64_t n,
                    int s, float *B, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(make_kp<float>(GP_RBF, theta, d, &kp));
    REQ(n >= 0 && s >= 0, "sizes must be non-negative");
    if (n == 0) return GP_OK;
    REQ(y && B && (s == 0 || (F && w)), "null pointer argument");
    return pathwise_rhs(kp.sigma, y, F, w, n, s, B, stream);
    GP_API_END
}

// ------------------------------------------------------------------ gradients
size_t gp_mll_grad_workspace(int64_t n, int d, int s, int prec) {
    return grad_workspace<float>(n, d, s + 1, prec);
}
size_t gp_mll_grad_f64_workspace(int64_t n, int d, int s) {
    return grad_workspace<double>(n, d, s + 1, GP_PREC_FP32);
}

}  // extern "C"

template <typename T>
static int grad_common(int kind, const double *theta, int d, const T *X, int64_t n, const T *Vsol,
                       const T *Z, int s, double *grad, int prec, void *ws, size_t ws_bytes,
                       cudaStream_t st, int pathwise) {
    KP<T> kp;
    GP_TRY(make_kp<T>(kind, theta, d, &kp));
    REQ(n >= 1 && s >= 1, "need n >= 1 and s >= 1");
    REQ(X && Vsol && grad && (pathwise || Z), "null pointer argument");
    if (sizeof(T) == sizeof(float)) GP_TRY(check_prec(prec));
    GradArgs<T> a;
    a.kp = kp;
    a.X = X;
    a.n = n;
    a.U0 = Vsol;
    a.U = Vsol + n;
    a.ldu = n;
    a.W0 = Vsol;
    a.W = pathwise ? Vsol + n : Z;
    a.ldw = n;
    a.R = s + 1;
    a.lam0 = 0.5;
    a.lam_rest = -0.5 / (double)s;
    a.grad = grad;
    return apply_grad<T>(a, prec, ws, ws_bytes, st);
}

extern "C" {

int gp_mll_grad_standard(int kind, const double *theta, int d, const float *X, int64_t n, const float *Vsol,
                         const float *Z, int s, double *grad, int prec, void *ws, size_t ws_bytes,
                         cudaStream_t stream) {
    GP_API_BEGIN
    return grad_common<float>(kind, theta, d, X, n, Vsol, Z, s, grad, prec, ws, ws_bytes, stream, 0);
    GP_API_END
}
int gp_mll_grad_pathwise(int kind, const double *theta, int d, const float *X, int64_t n, const float *Vsol,
                         int s, double *grad, int prec, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    return grad_common<float>(kind, theta, d, X, n, Vsol, nullptr, s, grad, prec, ws, ws_bytes, stream, 1);
    GP_API_END
}
int gp_mll_grad_standard_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                             const double *Vsol, const double *Z, int s, double *grad, void *ws,
                             size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    return grad_common<double>(kind, theta, d, X, n, Vsol, Z, s, grad, GP_PREC_FP32, ws, ws_bytes, stream, 0);
    GP_API_END
}
int gp_mll_grad_pathwise_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                             const double *Vsol, int s, double *grad, void *ws, size_t ws_bytes,
                             cudaStream_t stream) {
    GP_API_BEGIN
    return grad_common<double>(kind, theta, d, X, n, Vsol, nullptr, s, grad, GP_PREC_FP32, ws, ws_bytes,
                               stream, 1);
    GP_API_END
}

// ------------------------------------------------------------------ predictions
size_t gp_predict_workspace(int64_t nstar, int64_t n, int d, int s, int prec) {
    return predict_workspace(nstar, n, d, s, prec);
}

int gp_predict(int kind, const double *theta, int d, const float *Xstar, int64_t nstar, const float *X, int64_t n,
               const float *Vsol, int s, const float *Fstar, const float *ystar, float *mean, float *var,
               double *metrics, int prec, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(make_kp<float>(kind, theta, d, &kp));
    REQ(nstar >= 0 && n >= 1 && s >= 1, "need nstar >= 0, n >= 1 and s >= 1");
    if (nstar == 0) return GP_OK;
    REQ(Xstar && X && Vsol && Fstar && mean && var, "null pointer argument");
    GP_TRY(check_prec(prec));
    return predict(kp, Xstar, nstar, X, n, Vsol, s, Fstar, ystar, mean, var, metrics, prec, ws, ws_bytes, stream);
    GP_API_END
}

// ------------------------------------------------------------------ solver diagnostics
size_t gp_rkhs_sqdist_workspace(int64_t n, int d, int R, int prec) { return rkhs_workspace<float>(n, d, R, prec); }
size_t gp_rkhs_sqdist_f64_workspace(int64_t n, int d, int R) {
    return rkhs_workspace<double>(n, d, R, GP_PREC_FP32);
}


int gp_rkhs_sqdist(int kind, const double *theta, int d, const float *X, int64_t n, const float *Uinit,
                   const float *U, int R, double *dist, int prec, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    return rkhs_common<float>(kind, theta, d, X, n, Uinit, U, R, dist, prec, ws, ws_bytes, stream);
    GP_API_END
}

int gp_rkhs_sqdist_f64(int kind, const double *theta, int d, const double *X, int64_t n, const double *Uinit,
                       const double *U, int R, double *dist, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    return rkhs_common<double>(kind, theta, d, X, n, Uinit, U, R, dist, GP_PREC_FP32, ws, ws_bytes, stream);
    GP_API_END
}

// ------------------------------------------------------------------ autotuning
size_t gp_autotune_mvm_workspace(int64_t n, int d, int nrhs) {
    Carver c(nullptr);
    c.take<char>(tc_points_bytes(n, d));
    c.take<char>(tc_autotune_workspace(n, std::min(nrhs, 128)));
    return c.bytes();
}

int gp_autotune_mvm(int kind, const double *theta, int d, const float *X, int64_t n, const float *V, int nrhs,
                    float *Y, int reps, int *best_split, double *best_ms, void *ws, size_t ws_bytes,
                    cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(make_kp<float>(kind, theta, d, &kp));
    REQ(n >= 1 && nrhs >= 1 && nrhs <= 128, "need n >= 1 and 1 <= nrhs <= 128");
    REQ(X && V && Y && best_split && best_ms, "null pointer argument");
    REQ(reps >= 1 && reps <= 100, "reps must be in [1, 100]");
    GP_TRY(check_prec(GP_PREC_TC16));
    Carver c(ws);
    void *pbuf = c.take<char>(tc_points_bytes(n, d));
    const size_t twb = tc_autotune_workspace(n, nrhs);
    void *tw = c.take<char>(twb);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    TcMvmArgs a{};
    a.kind = kind;
    GP_TRY(tc_prepare_points(kp, X, n, pbuf, &a.rows, stream));
    a.cols = a.rows;
    a.V = V;
    a.ldv = n;
    a.R = nrhs;
    a.Y = Y;
    a.ldy = n;
    a.sf2 = kp.sf2;
    a.alpha = 1.0f;
    a.beta = 0.0f;
    a.diag_coef = kp.sigma2;
    a.Vd = V;
    a.ldvd = n;
    a.ndiag = n;
    return tc_autotune(a, reps, tw, twb, stream, best_split, best_ms);
    GP_API_END
}

void gp_autotune_reset(void) { tc_autotune_reset(); }

size_t gp_autotune_grad_workspace(int64_t n, int d, int s) {
    Carver c(nullptr);
    c.take<double>((size_t)d + 2);
    c.take<char>(grad_workspace<float>(n, d, s + 1, GP_PREC_TC16));
    return c.bytes();
}

int gp_autotune_grad(int kind, const double *theta, int d, const float *X, int64_t n, const float *Vsol, int s,
                     const float *Z, int reps, int64_t *best_param, double *best_ms, void *ws, size_t ws_bytes,
                     cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(make_kp<float>(kind, theta, d, &kp));
    REQ(n >= 1 && s >= 1, "need n >= 1 and s >= 1");
    REQ(X && Vsol && best_param && best_ms, "null pointer argument");
    REQ(reps >= 1 && reps <= 100, "reps must be in [1, 100]");
    GP_TRY(check_prec(GP_PREC_TC16));
    Carver c(ws);
    double *g = c.take<double>((size_t)d + 2);
    const size_t gwb = grad_workspace<float>(n, d, s + 1, GP_PREC_TC16);
    void *gw = c.take<char>(gwb);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    GradArgs<float> a;
    a.kp = kp;
    a.X = X;
    a.n = n;
    a.U0 = Vsol;
    a.U = Vsol + n;
    a.ldu = n;
    a.W0 = Vsol;
    a.W = Z ? Z : Vsol + n;  // standard estimator: (v_j, z_j); pathwise: (zhat_j, zhat_j)
    a.ldw = n;
    a.R = s + 1;
    a.lam0 = 0.5;
    a.lam_rest = -0.5 / (double)s;
    a.grad = g;
    return tc_autotune_grad(a, reps, gw, gwb, stream, best_param, best_ms);
    GP_API_END
}

int gp_autotune_save(const char *path) {
    GP_API_BEGIN
    REQ(path != nullptr && *path, "path must be a non-empty string");
    return tc_autotune_save(path);
    GP_API_END
}

int gp_autotune_load(const char *path) {
    GP_API_BEGIN
    REQ(path != nullptr && *path, "path must be a non-empty string");
    return tc_autotune_load(path);
    GP_API_END
}

int64_t gp_autotune_count(void) { return tc_autotune_count(); }

// ------------------------------------------------------------------ bilinear-form derivatives
}  // extern "C"

template <typename T>
static size_t bilinear_ws(int64_t n, int d, int R, int prec) {
    Carver c(nullptr);
    c.take<double>((size_t)d + 2);
    c.take<char>(grad_workspace<T>(n, d, R, prec));
    c.take<char>(bilinear_dx_workspace<T>(n, d));
    return c.bytes();
}

template <typename T>
static int bilinear_common(int kind, const double *theta, int d, const T *X, int64_t n, const T *U, int64_t ldu,
                           const T *W, int64_t ldw, int R, double lam0, double lam_rest, double *value,
                           double *dtheta, T *dX, int prec, void *ws, size_t ws_bytes, cudaStream_t st) {
    KP<T> kp;
    GP_TRY(make_kp<T>(kind, theta, d, &kp));
    REQ(n >= 1 && R >= 1, "need n >= 1 and R >= 1");
    REQ(X && U && W, "null pointer argument");
    REQ(ldu >= n && ldw >= n, "ldu and ldw must be >= n");
    REQ(std::isfinite(lam0) && std::isfinite(lam_rest), "lam0 and lam_rest must be finite");
    if (sizeof(T) == sizeof(float)) GP_TRY(check_prec(prec));
    if (!value && !dtheta && !dX) return GP_OK;
    Carver c(ws);
    double *gbuf = c.take<double>((size_t)d + 2);
    const size_t gwb = grad_workspace<T>(n, d, R, prec);
    void *gws = c.take<char>(gwb);
    const size_t xwb = bilinear_dx_workspace<T>(n, d);
    void *xws = c.take<char>(xwb);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    GradArgs<T> a;
    a.kp = kp;
    a.X = X;
    a.n = n;
    a.U0 = U;
    a.U = U + ldu;
    a.ldu = ldu;
    a.W0 = W;
    a.W = W + ldw;
    a.ldw = ldw;
    a.R = R;
    a.lam0 = lam0;
    a.lam_rest = lam_rest;
    a.grad = dtheta ? dtheta : gbuf;
    if (value || dtheta) {
        GP_TRY(apply_grad<T>(a, prec, gws, gwb, st));
        if (value) GP_TRY(bilinear_value<T>(kp, a.grad, value, st));
    }
    if (dX) GP_TRY(bilinear_dx<T>(a, (U == W && ldu == ldw) ? 1 : 0, dX, xws, xwb, st));
    return GP_OK;
}

extern "C" {

size_t gp_bilinear_grad_workspace(int64_t n, int d, int R, int prec) {
    return bilinear_ws<float>(n, d, R, prec);
}
size_t gp_bilinear_grad_f64_workspace(int64_t n, int d, int R) {
    return bilinear_ws<double>(n, d, R, GP_PREC_FP32);
}

int gp_bilinear_grad(int kind, const double *theta, int d, const float *X, int64_t n, const float *U,
                     int64_t ldu, const float *W, int64_t ldw, int R, double lam0, double lam_rest, double *value,
                     double *dtheta, float *dX, int prec, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    return bilinear_common<float>(kind, theta, d, X, n, U, ldu, W, ldw, R, lam0, lam_rest, value, dtheta, dX,
                                  prec, ws, ws_bytes, stream);
    GP_API_END
}

int gp_bilinear_grad_f64(int kind, const double *theta, int d, const double *X, int64_t n, const double *U,
                         int64_t ldu, const double *W, int64_t ldw, int R, double lam0, double lam_rest,
                         double *value, double *dtheta, double *dX, void *ws, size_t ws_bytes,
                         cudaStream_t stream) {
    GP_API_BEGIN
    return bilinear_common<double>(kind, theta, d, X, n, U, ldu, W, ldw, R, lam0, lam_rest, value, dtheta, dX,
                                   GP_PREC_FP32, ws, ws_bytes, stream);
    GP_API_END
}

// ------------------------------------------------------------------ posterior samples
size_t gp_posterior_samples_workspace(int64_t nstar, int64_t n, int d, int s, int prec) {
    return posterior_workspace(nstar, n, d, s, prec);
}

int gp_posterior_samples(int kind, const double *theta, int d, const float *Xstar, int64_t nstar,
                         const float *X, int64_t n, const float *Vsol, int s, const float *Fstar, float *out,
                         int prec, void *ws, size_t ws_bytes, cudaStream_t stream) {
    GP_API_BEGIN
    KP<float> kp;
    GP_TRY(make_kp<float>(kind, theta, d, &kp));
    REQ(nstar >= 0 && n >= 1 && s >= 1, "need nstar >= 0, n >= 1, s >= 1");
    if (nstar == 0) return GP_OK;
    REQ(Xstar && X && Vsol && Fstar && out, "null pointer argument");
    GP_TRY(check_prec(prec));
    return posterior_samples(kp, Xstar, nstar, X, n, Vsol, s, Fstar, out, prec, ws, ws_bytes, stream);
    GP_API_END
}

// ------------------------------------------------------------------ outer loop
int gp_adam_softplus_step(int P, double *nu, double *m, double *v, int64_t t, const double *grad_theta,
                          double lr, double beta1, double beta2, double eps, double *theta_out) {
    GP_API_BEGIN
    REQ(P >= 1 && nu && m && v && grad_theta && theta_out, "null pointer argument");
    REQ(t >= 1, "t must be >= 1");
    REQ(lr > 0 && beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps > 0, "bad Adam settings");
    for (int p = 0; p < P; ++p) {
        if (!std::isfinite(grad_theta[p])) {
            set_error("grad_theta[%d] is not finite", p);
            return GP_ERR_INVALID_ARG;
        }
    }
    // theta = softplus(nu); d theta / d nu = sigmoid(nu); ascent on L.
    for (int p = 0; p < P; ++p) {
        double sig = 1.0 / (1.0 + std::exp(-nu[p]));
        double g = grad_theta[p] * sig;
        m[p] = beta1 * m[p] + (1.0 - beta1) * g;
        v[p] = beta2 * v[p] + (1.0 - beta2) * g * g;
        double mh = m[p] / (1.0 - std::pow(beta1, (double)t));
        double vh = v[p] / (1.0 - std::pow(beta2, (double)t));
        nu[p] += lr * mh / (std::sqrt(vh) + eps);
        theta_out[p] = nu[p] > 30.0 ? nu[p] : std::log1p(std::exp(nu[p]));
    }
    return GP_OK;
    GP_API_END
}

}  // extern "C"
