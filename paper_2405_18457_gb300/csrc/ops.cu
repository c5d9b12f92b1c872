// Operator dispatch (CUDA-core vs tcgen05), random Fourier features, pathwise
// right-hand sides and pathwise-conditioned posterior samples.
#include "solvers.cuh"

#include <algorithm>
#include <type_traits>

namespace gp {

// ===========================================================================
// H V / K V dispatch
// ===========================================================================
template <typename T>
size_t mvm_workspace(int64_t n1, int64_t n2, int d, int R, int prec) {
    if (std::is_same<T, float>::value && (prec == GP_PREC_TC16 || prec == GP_PREC_TC16X3)) {
        Carver c(nullptr);
        c.take<char>(tc_points_bytes(n1, d));
        c.take<char>(tc_points_bytes(n2, d));
        c.take<char>(tc_mvm_workspace(n1, n2, R));
        return c.bytes();
    }
    return mvm_simt_workspace<T>(n1, n2, R);
}

template <typename T>
int apply_mvm(const KP<T> &kp, const T *X1, int64_t n1, const T *X2, int64_t n2, const T *V, int64_t ldv,
              int R, T *Y, int64_t ldy, int add_noise, int prec, void *ws, size_t ws_bytes, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (prec == GP_PREC_TC16 || prec == GP_PREC_TC16X3) {
            Carver c(ws);
            void *pa = c.take<char>(tc_points_bytes(n1, kp.d));
            void *pb = c.take<char>(tc_points_bytes(n2, kp.d));
            size_t tcw = tc_mvm_workspace(n1, n2, R);
            void *tw = c.take<char>(tcw);
            GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
            TcMvmArgs a{};
            a.kind = kp.kind;
            if (X2 == X1 && n2 == n1) {
                GP_TRY(tc_prepare_points(kp, X1, n1, pa, &a.rows, st));
                a.cols = a.rows;
            } else {
                GP_TRY(tc_prepare_pair(kp, X1, n1, X2, n2, pa, pb, &a.rows, &a.cols, st));
            }
            a.V = V;
            a.ldv = ldv;
            a.R = R;
            a.Y = Y;
            a.ldy = ldy;
            a.sf2 = kp.sf2;
            a.alpha = 1.0f;
            a.beta = 0.0f;
            a.diag_coef = add_noise ? kp.sigma2 : 0.0f;
            a.Vd = V;
            a.ldvd = ldv;
            a.drow0 = 0;
            a.ndiag = add_noise ? n1 : 0;
            a.done = nullptr;
            a.split = prec == GP_PREC_TC16X3 ? 1 : 0;
            return tc_mvm(a, tw, tcw, st);
        }
    }
    MvmArgs<T> a{};
    a.kp = kp;
    a.X1 = X1;
    a.n1 = n1;
    a.X2 = X2;
    a.n2 = n2;
    a.n2_total = n2;
    a.col0_dev = nullptr;
    a.V = V;
    a.ldv = ldv;
    a.R = R;
    a.Y = Y;
    a.ldy = ldy;
    a.alpha = T(1);
    a.beta = T(0);
    a.diag_coef = add_noise ? kp.sigma2 : T(0);
    a.Vd = V;
    a.ldvd = ldv;
    a.drow0 = 0;
    a.ndiag = add_noise ? n1 : 0;
    a.diag_from_col0 = 0;
    a.done = nullptr;
    return mvm_simt<T>(a, ws, ws_bytes, st);
}

template size_t mvm_workspace<float>(int64_t, int64_t, int, int, int);
template size_t mvm_workspace<double>(int64_t, int64_t, int, int, int);
template int apply_mvm<float>(const KP<float> &, const float *, int64_t, const float *, int64_t, const float *,
                              int64_t, int, float *, int64_t, int, int, void *, size_t, cudaStream_t);
template int apply_mvm<double>(const KP<double> &, const double *, int64_t, const double *, int64_t,
                               const double *, int64_t, int, double *, int64_t, int, int, void *, size_t,
                               cudaStream_t);

// Gradient dispatch.  The fused tensor-core estimator lives in tc.cu; the
// CUDA-core reduction serves FP32 and FP64.
size_t tc_grad_workspace(int64_t n, int d, int R);
int tc_grad(const GradArgs<float> &a, void *ws, size_t ws_bytes, cudaStream_t st);

template <typename T>
size_t grad_workspace(int64_t n, int d, int R, int prec) {
    if (std::is_same<T, float>::value && prec == GP_PREC_TC16) return tc_grad_workspace(n, d, R);
    return grad_simt_workspace<T>(n, d, R);
}

template <typename T>
int apply_grad(const GradArgs<T> &a, int prec, void *ws, size_t ws_bytes, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (prec == GP_PREC_TC16) return tc_grad(a, ws, ws_bytes, st);
    }
    return grad_simt<T>(a, ws, ws_bytes, st);
}
template size_t grad_workspace<float>(int64_t, int, int, int);
template size_t grad_workspace<double>(int64_t, int, int, int);
template int apply_grad<float>(const GradArgs<float> &, int, void *, size_t, cudaStream_t);
template int apply_grad<double>(const GradArgs<double> &, int, void *, size_t, cudaStream_t);

// ===========================================================================
// Random Fourier features (App. B "Kernel Function and Random Features")
// ===========================================================================
namespace {

constexpr int RP = 64;   // points per block
constexpr int RFC = 32;  // frequencies per chunk
constexpr int RS = 64;   // samples per block

__device__ __forceinline__ void sc(float a, float *s, float *c) { sincosf(a, s, c); }
__device__ __forceinline__ void sc(double a, double *s, double *c) { sincos(a, s, c); }

// Four consecutive shared-memory values (16-byte aligned for float).
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

// F[j][i] = s_f sqrt(2/m) sum_l W[j][l] cos(w_l.x_i) + W[j][h+l] sin(w_l.x_i)
// Per block: 64 points x 64 samples; per chunk of 32 frequencies the block evaluates the
// 64 x 32 cos/sin features into shared memory (frequency-major), then every thread
// accumulates a 4 x 4 register tile (4 points x 4 samples) over the chunk.  Shared-memory
// layouts avoid bank conflicts: point rows have an odd stride, and the weights (written
// transposed) have their 4-sample groups XOR-swizzled by the frequency index.
template <typename T>
__global__ void __launch_bounds__(256) rff_kernel(const KP<T> kp, const T *X, int64_t n, int m,
                                                  const T *omega_hat, const T *chi2, const T *W, int s, T *F,
                                                  int64_t ldf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = kp.d, h = m / 2;
    T *Cs = reinterpret_cast<T *>(smem_raw);  // RFC x RP   cos features
    T *Sn = Cs + RFC * RP;                     // RFC x RP   sin features
    T *Wc = Sn + RFC * RP;                     // RFC x RS   cos weights
    T *Ws = Wc + RFC * RS;                     // RFC x RS   sin weights
    T *Xs = Ws + RFC * RS;                     // RP x xd
    const int xd = d | 1;
    T *Om = Xs + RP * xd;                      // RFC x d    frequencies
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t p0 = (int64_t)blockIdx.x * RP;
    const int j0 = blockIdx.y * RS;
    for (int e = tid; e < RP * d; e += 256) {
        const int r = e / d, k = e - r * d;
        Xs[r * xd + k] = (p0 + r < n) ? X[(p0 + r) * d + k] : T(0);
    }
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int l0 = 0; l0 < h; l0 += RFC) {
        __syncthreads();
        for (int e = tid; e < RFC * d; e += 256) {
            const int l = e / d, k = e - l * d;
            T w = T(0);
            if (l0 + l < h) {
                const T t = (kp.kind == GP_MATERN32) ? sqrt(T(3) / chi2[l0 + l]) : T(1);
                w = omega_hat[(int64_t)(l0 + l) * d + k] * kp.inv_ell[k] * t;
            }
            Om[e] = w;
        }
        for (int e = tid; e < RS * RFC; e += 256) {
            const int j = e / RFC, l = e - j * RFC;
            const bool ok = (j0 + j < s) && (l0 + l < h);
            const int js = j ^ ((l & 7) << 2);
            Wc[l * RS + js] = ok ? W[(int64_t)(j0 + j) * m + l0 + l] : T(0);
            Ws[l * RS + js] = ok ? W[(int64_t)(j0 + j) * m + h + l0 + l] : T(0);
        }
        __syncthreads();
        for (int e = tid; e < RP * RFC; e += 256) {
            const int l = e / RP, pnt = e - l * RP;
            T arg = T(0);
            for (int k = 0; k < d; ++k) arg += Om[l * d + k] * Xs[pnt * xd + k];
            T sv, cv;
            sc(arg, &sv, &cv);
            Cs[l * RP + pnt] = cv;
            Sn[l * RP + pnt] = sv;
        }
        __syncthreads();
#pragma unroll 8
        for (int l = 0; l < RFC; ++l) {
            T cv[4], sv[4], wc[4], ws[4];
            ld4(Cs + l * RP + 4 * tx, cv);
            ld4(Sn + l * RP + 4 * tx, sv);
            const int jo = (4 * ty) ^ ((l & 7) << 2);
            ld4(Wc + l * RS + jo, wc);
            ld4(Ws + l * RS + jo, ws);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += cv[a] * wc[b] + sv[a] * ws[b];
        }
    }
    const T amp = kp.sf * sqrt(T(2) / T(m));
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = j0 + 4 * ty + b;
        if (j >= s) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t i = p0 + 4 * tx + a;
            if (i < n) F[(int64_t)j * ldf + i] = amp * acc[a][b];
        }
    }
}

template <typename T>
int launch_rff(const KP<T> &kp, const T *X, int64_t n, int m, const T *omega_hat, const T *chi2, const T *W,
               int s, T *F, int64_t ldf, cudaStream_t st) {
    const int d = kp.d;
    size_t smem = sizeof(T) * (size_t)(2 * RFC * RP + 2 * RFC * RS + RP * (d | 1) + RFC * d);
    if (smem > kMaxDynSmem) {
        set_error("rff: d=%d too large", d);
        return GP_ERR_UNSUPPORTED;
    }
    GP_TRY(ensure_max_dyn_smem((const void *)rff_kernel<T>));
    dim3 grid((unsigned)cdiv(n, RP), (unsigned)cdiv(s, RS));
    rff_kernel<T><<<grid, 256, smem, st>>>(kp, X, n, m, omega_hat, chi2, W, s, F, ldf);
    return check_launch("rff_kernel");
}

}  // namespace

template <typename T>
int rff_prior(const KP<T> &kp, const T *X, int64_t n, int m, const T *omega_hat, const T *chi2, const T *W,
              int s, T *F, int64_t ldf, cudaStream_t st) {
    return launch_rff<T>(kp, X, n, m, omega_hat, chi2, W, s, F, ldf, st);
}
template int rff_prior<float>(const KP<float> &, const float *, int64_t, int, const float *, const float *,
                              const float *, int, float *, int64_t, cudaStream_t);

size_t rff_workspace(int d, int m, int s, int prec) {
    return (prec == GP_PREC_TC16 && tc_rff_fits(d, m, s)) ? tc_rff_workspace(d, m, s) : 0;
}

int rff_prior_ws(const KP<float> &kp, const float *X, int64_t n, int m, const float *omega_hat, const float *chi2,
                 const float *W, int s, float *F, int64_t ldf, int prec, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (prec == GP_PREC_TC16 && tc_rff_fits(kp.d, m, s))
        return tc_rff(kp, X, n, m, omega_hat, chi2, W, s, F, ldf, ws, ws_bytes, st);
    return launch_rff<float>(kp, X, n, m, omega_hat, chi2, W, s, F, ldf, st);
}
template int rff_prior<double>(const KP<double> &, const double *, int64_t, int, const double *, const double *,
                               const double *, int, double *, int64_t, cudaStream_t);

// ===========================================================================
// Pathwise right-hand sides: B = [y, F_j + sigma w_j]  (App. B)
// ===========================================================================
namespace {
__global__ void pathwise_rhs_kernel(float sigma, const float *y, const float *F, const float *w, int64_t n,
                                    int s, float *B) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (i >= n) return;
    B[(int64_t)c * n + i] = (c == 0) ? y[i] : F[(int64_t)(c - 1) * n + i] + sigma * w[(int64_t)(c - 1) * n + i];
}

// Wd[j][i] = Vsol[0][i] - Vsol[j+1][i]
__global__ void cond_weights_kernel(const float *Vsol, int64_t n, int s, float *Wd) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i < n) Wd[(int64_t)j * n + i] = Vsol[i] - Vsol[(int64_t)(j + 1) * n + i];
}
// out[j][i] += Fstar[j][i]
__global__ void add_prior_kernel(const float *Fstar, float *out, int64_t count) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        out[e] += Fstar[e];
}
}  // namespace

int pathwise_rhs(float sigma, const float *y, const float *F, const float *w, int64_t n, int s, float *B,
                 cudaStream_t st) {
    dim3 grid((unsigned)cdiv(n, 256), (unsigned)(s + 1));
    pathwise_rhs_kernel<<<grid, 256, 0, st>>>(sigma, y, F, w, n, s, B);
    return check_launch("pathwise_rhs_kernel");
}

// ===========================================================================
// Posterior samples (Eq. pathwise_conditioning; Sec. 3):
//   out_j = Fstar_j + K(X*, X) (v_y - zhat_j)
// ===========================================================================
size_t posterior_workspace(int64_t nstar, int64_t n, int d, int s, int prec) {
    Carver c(nullptr);
    c.take<float>((size_t)s * (size_t)n);
    c.take<char>(mvm_workspace<float>(nstar, n, d, s, prec));
    return c.bytes();
}

int posterior_samples(const KP<float> &kp, const float *Xstar, int64_t nstar, const float *X, int64_t n,
                      const float *Vsol, int s, const float *Fstar, float *out, int prec, void *ws,
                      size_t ws_bytes, cudaStream_t st) {
    Carver c(ws);
    float *Wd = c.take<float>((size_t)s * (size_t)n);
    size_t mw = mvm_workspace<float>(nstar, n, kp.d, s, prec);
    void *mws = c.take<char>(mw);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    dim3 g1((unsigned)cdiv(n, 256), (unsigned)s);
    cond_weights_kernel<<<g1, 256, 0, st>>>(Vsol, n, s, Wd);
    GP_TRY(check_launch("cond_weights_kernel"));
    GP_TRY(apply_mvm<float>(kp, Xstar, nstar, X, n, Wd, n, s, out, nstar, 0, prec, mws, mw, st));
    const int64_t cnt = (int64_t)s * nstar;
    add_prior_kernel<<<(unsigned)std::min<int64_t>(cdiv(cnt, 256), 4096), 256, 0, st>>>(Fstar, out, cnt);
    return check_launch("add_prior_kernel");
}

// ===========================================================================
// Predictions from the pathwise solutions (Sec. 3 "Amortising Linear Solves for
// Optimisation and Prediction"): mean = k(x*, X) v_y, predictive variance = the s
// posterior samples' spread around that mean plus sigma^2, RMSE and mean test
// log-likelihood of ystar.
// ===========================================================================
namespace {

constexpr int PRED_BLOCKS = 256;

// M = K(X*, X) [v_y, zhat_1..] (R x nstar); per point: mean, variance; per block:
// partial sums of squared errors and log-densities (FP64) when ystar is given.
__global__ void predict_kernel(const float *M, const float *Fstar, const float *ystar, int64_t nstar, int s,
                               double sigma2, float *mean, float *var, double *part) {
    double se = 0.0, ll = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nstar; i += (int64_t)gridDim.x * blockDim.x) {
        const double mu = (double)M[i];
        double acc = 0.0;
        for (int j = 0; j < s; ++j) {
            const double dev = (double)Fstar[(int64_t)j * nstar + i] - (double)M[(int64_t)(j + 1) * nstar + i];
            acc += dev * dev;
        }
        const double v = acc / (double)s + sigma2;
        mean[i] = (float)mu;
        var[i] = (float)v;
        if (ystar) {
            const double e = (double)ystar[i] - mu;
            se += e * e;
            ll += -0.5 * log(2.0 * 3.14159265358979323846 * v) - 0.5 * e * e / v;
        }
    }
    if (!part) return;
    __shared__ double r1[32], r2[32];
    se = warp_sum(se);
    ll = warp_sum(ll);
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = se;
        r2[threadIdx.x >> 5] = ll;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += r1[w];
            b += r2[w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void predict_metrics_kernel(const double *part, int nblocks, int64_t nstar, double *metrics) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblocks; ++k) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    metrics[0] = sqrt(a / (double)nstar);
    metrics[1] = b / (double)nstar;
}

}  // namespace

size_t predict_workspace(int64_t nstar, int64_t n, int d, int s, int prec) {
    Carver c(nullptr);
    c.take<float>((size_t)(s + 1) * (size_t)nstar);
    c.take<double>(2 * PRED_BLOCKS);
    c.take<char>(mvm_workspace<float>(nstar, n, d, s + 1, prec));
    return c.bytes();
}

int predict(const KP<float> &kp, const float *Xstar, int64_t nstar, const float *X, int64_t n, const float *Vsol,
            int s, const float *Fstar, const float *ystar, float *mean, float *var, double *metrics, int prec,
            void *ws, size_t ws_bytes, cudaStream_t st) {
    Carver c(ws);
    float *M = c.take<float>((size_t)(s + 1) * (size_t)nstar);
    double *part = c.take<double>(2 * PRED_BLOCKS);
    const size_t mw = mvm_workspace<float>(nstar, n, kp.d, s + 1, prec);
    void *mws = c.take<char>(mw);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    GP_TRY(apply_mvm<float>(kp, Xstar, nstar, X, n, Vsol, n, s + 1, M, nstar, 0, prec, mws, mw, st));
    const bool metr = ystar && metrics;
    const int nb = (int)std::min<int64_t>(PRED_BLOCKS, cdiv(nstar, 256));
    predict_kernel<<<nb, 256, 0, st>>>(M, Fstar, ystar, nstar, s, (double)kp.sigma2, mean, var,
                                       metr ? part : nullptr);
    GP_TRY(check_launch("predict_kernel"));
    if (metr) {
        predict_metrics_kernel<<<1, 32, 0, st>>>(part, nb, nstar, metrics);
        GP_TRY(check_launch("predict_metrics_kernel"));
    }
    return GP_OK;
}

// ===========================================================================
// Solver diagnostic: RKHS squared distance between an initialisation and a
// solution (Sec. 3, "Initial Distance to the Linear System Solution", Eq.
// RKHS_distance): dist[c] = e_c^T H e_c with e_c = U[c] - Uinit[c] (the sign of e
// does not matter).  One product H E in the requested form, then per-column FP64
// dot products summed over fixed blocks in a fixed order.
// ===========================================================================
namespace {

constexpr int RK_PARTS = 64;

template <typename T>
__global__ void rkhs_diff_kernel(const T *U, const T *U0, T *E, int64_t cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        E[i] = U[i] - U0[i];
}

// grid (RK_PARTS, R): block p of column c sums e_i y_i over rows i = p*256 + t (mod RK_PARTS*256).
template <typename T>
__global__ void rkhs_dot_kernel(const T *E, const T *Y, int64_t n, double *part) {
    const int c = blockIdx.y;
    const T *e = E + (int64_t)c * n;
    const T *y = Y + (int64_t)c * n;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)e[i] * (double)y[i];
    __shared__ double red[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[(int64_t)c * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void rkhs_finish_kernel(const double *part, int nparts, int R, double *dist) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= R) return;
    double t = 0.0;
    for (int p = 0; p < nparts; ++p) t += part[(int64_t)c * nparts + p];
    dist[c] = t;
}

}  // namespace

template <typename T>
size_t rkhs_workspace(int64_t n, int d, int R, int prec) {
    Carver c(nullptr);
    c.take<T>((size_t)R * (size_t)n);  // E
    c.take<T>((size_t)R * (size_t)n);  // H E
    c.take<double>((size_t)R * RK_PARTS);
    c.take<char>(mvm_workspace<T>(n, n, d, R, prec));
    return c.bytes();
}

template <typename T>
int rkhs_sqdist(const KP<T> &kp, const T *X, int64_t n, const T *U0, const T *U, int R, double *dist, int prec,
                void *ws, size_t ws_bytes, cudaStream_t st) {
    Carver c(ws);
    T *E = c.take<T>((size_t)R * (size_t)n);
    T *Y = c.take<T>((size_t)R * (size_t)n);
    double *part = c.take<double>((size_t)R * RK_PARTS);
    const size_t mw = mvm_workspace<T>(n, n, kp.d, R, prec);
    void *mws = c.take<char>(mw);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    const T *Ed = U;
    if (U0) {
        const int64_t cnt = (int64_t)R * n;
        rkhs_diff_kernel<T><<<(unsigned)std::min<int64_t>(cdiv(cnt, 256), 4096), 256, 0, st>>>(U, U0, E, cnt);
        GP_TRY(check_launch("rkhs_diff_kernel"));
        Ed = E;
    }
    GP_TRY(apply_mvm<T>(kp, X, n, X, n, Ed, n, R, Y, n, 1, prec, mws, mw, st));
    rkhs_dot_kernel<T><<<dim3(RK_PARTS, (unsigned)R), 256, 0, st>>>(Ed, Y, n, part);
    GP_TRY(check_launch("rkhs_dot_kernel"));
    rkhs_finish_kernel<<<(unsigned)cdiv(R, 128), 128, 0, st>>>(part, RK_PARTS, R, dist);
    return check_launch("rkhs_finish_kernel");
}

template size_t rkhs_workspace<float>(int64_t, int, int, int);
template size_t rkhs_workspace<double>(int64_t, int, int, int);
template int rkhs_sqdist<float>(const KP<float> &, const float *, int64_t, const float *, const float *, int,
                                double *, int, void *, size_t, cudaStream_t);
template int rkhs_sqdist<double>(const KP<double> &, const double *, int64_t, const double *, const double *, int,
                                 double *, int, void *, size_t, cudaStream_t);

}  // namespace gp
