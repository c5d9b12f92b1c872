// Internal helpers shared by the solver translation units (CG/SGD, AP).
#pragma once

#include "solvers.cuh"

#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

namespace gp {

namespace {

constexpr double kNormEps = 1e-12;   // eps of the normalisation b / (||b|| + eps)
constexpr double kFreeze = 1e-30;    // CG column frozen once gamma <= this
// x (float) -> y (double), count elements
__global__ void widen_kernel(const float *x, double *y, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (double)x[i];
}

// Row partitions of the per-column partial sums: enough blocks (partitions x columns)
// to fill the GPU for the vector updates, at most 64 partials per column.  A partition
// covers a multiple of 4 rows, so that float vectors can be read as float4 when n % 4 == 0.
int nparts_for(int64_t n) { return (int)std::min<int64_t>(64, std::max<int64_t>(1, cdiv(n, 2048))); }
__host__ __device__ inline int64_t part_len(int64_t n, int P) { return rup(cdiv(n, P), 4); }

// Sum of a[i] b[i] over [i0, i1) by the threads of a block, FP64 accumulation.  For float
// with 16-byte aligned rows (n % 4 == 0) four products are summed in FP32 (FMA) before each
// FP64 addition: FP64 runs at a small fraction of the FP32 rate on this GPU, and the FP32
// rounding of a four-term sum is below that of the FP32 inputs themselves.
template <typename T>
__device__ __forceinline__ double block_dot(const T *a, const T *b, int64_t i0, int64_t i1, bool vec4) {
    double s = 0.0;
    if constexpr (std::is_same<T, float>::value) {
        if (vec4) {
            const float4 *a4 = reinterpret_cast<const float4 *>(a), *b4 = reinterpret_cast<const float4 *>(b);
            for (int64_t q = (i0 >> 2) + threadIdx.x; q < (i1 >> 2); q += blockDim.x) {
                const float4 x = a4[q], y = b4[q];
                s += (double)fmaf(x.w, y.w, fmaf(x.z, y.z, fmaf(x.y, y.y, x.x * y.x)));
            }
            return s;
        }
    }
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s += (double)a[i] * (double)b[i];
    return s;
}

// part[c*P + p] = sum_{i in chunk p} A[c][i] * B[c][i]   (grid P x R)
template <typename T>
__global__ void coldot_kernel(const T *A, const T *B, int64_t n, int P, double *part, const int *done) {
    if (done && *done) return;
    const int p = blockIdx.x, c = blockIdx.y;
    const int64_t per = part_len(n, P);
    const int64_t i0 = min(n, (int64_t)p * per), i1 = min(n, i0 + per);
    const T *a = A + (int64_t)c * n, *b = B + (int64_t)c * n;
    double s = block_dot<T>(a, b, i0, i1, (n & 3) == 0);
    __shared__ double red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[(int64_t)c * P + p] = t;
    }
}

// The same sum taken by one whole warp (lane l adds partials l, l + 32, ... in order, then a
// fixed butterfly): one round of loads instead of P dependent ones; deterministic.
__device__ __forceinline__ double sum_parts_warp(const double *part, int c, int P) {
    double s = 0.0;
    for (int p = (int)(threadIdx.x & 31); p < P; p += 32) s += part[(int64_t)c * P + p];
    return warp_sum(s);
}

__device__ __forceinline__ double sum_parts(const double *part, int c, int P) {
    double s = 0.0;
    for (int p = 0; p < P; ++p) s += part[(int64_t)c * P + p];
    return s;
}

// A block's column factor f = (inv ? 1 / scale[c] : scale[c]) in FP64 and as a sum of two floats
// fh + fl (f to about 2^-48), computed once by thread 0: FP64 division and float <-> double
// conversions run at a small fraction of the FP32 rate on this GPU, so taking them in every
// thread would dominate these memory-bound kernels.  Called by every thread of the block (it
// synchronises); repeated calls in one kernel are safe.
struct ColFactor {
    double d;
    float h, l;
};
__device__ __forceinline__ ColFactor block_factor(const double *scale, int c, int inv) {
    __shared__ double s_d;
    __shared__ float s_h, s_l;
    __syncthreads();  // a previous call's values are no longer read
    if (threadIdx.x == 0) {
        const double f = inv ? 1.0 / scale[c] : scale[c];
        s_d = f;
        s_h = (float)f;
        s_l = (float)(f - (double)s_h);
    }
    __syncthreads();
    return ColFactor{s_d, s_h, s_l};
}

// scale[c] = sqrt(sum parts) + eps
__global__ void norm_scale_kernel(int R, int P, const double *part, double *scale) {
    for (int c = threadIdx.x; c < R; c += blockDim.x) scale[c] = sqrt(sum_parts(part, c, P)) + kNormEps;
}

// V[c] *= (inv ? 1/scale[c] : scale[c]).  For float the FP64 factor is carried as fh + fl, and
// v f = fma(v, fh, v fl) is the FP64 product rounded about once, in FP32 arithmetic only.
template <typename T>
__global__ void scale_cols_kernel(T *V, int64_t n, const double *scale, int inv) {
    const int c = blockIdx.y;
    const ColFactor cf = block_factor(scale, c, inv);
    if constexpr (std::is_same<T, float>::value) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const float v = V[(int64_t)c * n + i];
            V[(int64_t)c * n + i] = fmaf(v, cf.h, v * cf.l);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            V[(int64_t)c * n + i] *= cf.d;
    }
}

// r = B / scale - HV ; d = r.  For float, b / scale is B fh + B fl (the FP64 factor as a sum of
// two floats), so the difference sees b / scale to about 2^-48.
template <typename T>
__global__ void init_residual_kernel(const T *B, const T *HV, T *r, T *d, int64_t n, const double *scale) {
    const int c = blockIdx.y;
    const ColFactor cf = block_factor(scale, c, 1);
    T fh, fl;
    if constexpr (std::is_same<T, float>::value) {
        fh = cf.h;
        fl = cf.l;
    } else {
        fh = cf.d;
        fl = 0.0;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = (int64_t)c * n + i;
        T v = fma(B[e], fh, fma(B[e], fl, -HV[e]));
        r[e] = v;
        if (d) d[e] = v;
    }
}

// Split norms and the loop condition (App. B): res_y = ||r_y||, res_z = mean_j ||r_j||,
// from rt[c] = ||r_c|| (the column norms, square roots already taken).
__device__ void finish_state(SolverState *st, const double *rt, int R, long long t, long long max_iters, double tol,
                             int stop_rule) {
    double ry = rt[0];
    double rz = 0.0;
    for (int c = 1; c < R; ++c) rz += rt[c];
    rz = (R > 1) ? rz / (double)(R - 1) : 0.0;
    st->res_y = ry;
    st->res_z = rz;
    st->iter = t;
    st->certified = 0;
    bool finite = isfinite(ry) && isfinite(rz);
    bool conv = (stop_rule == GP_STOP_EITHER) ? (ry <= tol || rz <= tol) : (ry <= tol && rz <= tol);
    st->converged = conv ? 1 : 0;
    if (!finite) {
        st->status = GP_ERR_BREAKDOWN;
        st->done = 1;
    } else if (conv || t >= max_iters) {
        st->done = 1;
    }
}

// Single-thread form: sq[c] = ||r_c||^2.
__device__ void finish_norms(SolverState *st, const double *sq, int R, long long t, long long max_iters,
                             double tol, int stop_rule) {
    double rt[512];
    for (int c = 0; c < R; ++c) rt[c] = sqrt(sq[c]);
    finish_state(st, rt, R, t, max_iters, tol, stop_rule);
}

// Block form, called by every thread of the block: sq (shared, R values) holds
// ||r_c||^2 on entry and is overwritten with the norms.
__device__ void finish_norms_block(SolverState *st, double *sq, int R, long long t, long long max_iters, double tol,
                                   int stop_rule) {
    for (int c = threadIdx.x; c < R; c += blockDim.x) sq[c] = sqrt(sq[c]);
    __syncthreads();
    if (threadIdx.x == 0) finish_state(st, sq, R, t, max_iters, tol, stop_rule);
}

// True residual (App. B "Linear System Solver": r = b - H u, here of the normalised system):
// r = b~ - H v with b~ = b / scale.  With an FP64 product (TH = double) the difference is taken
// in FP64 and stored in T.  With an FP32 product it is two FP32 fused multiply-adds with the FP64
// factor 1 / scale carried as a sum of two floats (b~ to about 2^-48, the difference rounded
// about once), and four squares are summed in FP32 per FP64 addition.  The partial sums of
// ||r||^2 go to partN.  Skipped while *skip != 0.  grid P x R
template <typename T, typename TH>
__global__ void true_residual_kernel(const T *B, const TH *Hv, T *r, int64_t n, int P, const double *scale,
                                     double *partN, const int *skip) {
    if (skip && *skip) return;
    const int p = blockIdx.x, c = blockIdx.y;
    const int64_t per = part_len(n, P);
    const int64_t i0 = min(n, (int64_t)p * per), i1 = min(n, i0 + per);
    const ColFactor cf = block_factor(scale, c, 1);
    const int64_t off = (int64_t)c * n;
    double sum = 0.0;
    if constexpr (std::is_same<T, float>::value && std::is_same<TH, float>::value) {
        float acc = 0.0f;
        int k = 0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const float v = fmaf(B[off + i], cf.h, fmaf(B[off + i], cf.l, -Hv[off + i]));
            r[off + i] = v;
            acc = fmaf(v, v, acc);
            if (++k == 4) {
                sum += (double)acc;
                acc = 0.0f;
                k = 0;
            }
        }
        sum += (double)acc;
    } else {
        const double f = cf.d;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const double v = (double)B[off + i] * f - (double)Hv[off + i];
            r[off + i] = (T)v;
            sum += v * v;
        }
    }
    __shared__ double red[32];
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partN[(int64_t)c * P + p] = t;
    }
}

// State after a true-residual recomputation: (CG) gamma <- r^T P^-1 r (partG; = ||r||^2 without
// a preconditioner) for the next iteration, when gamma is given, and the restart direction's
// bound ||r|| when dbound is given; the split norms from partN and the loop condition at the
// current iteration count, marked certified.  reopen = 0: a recomputation during the solve
// (skipped once done is latched).  reopen = 1: the check after the loop stopped; done is
// re-evaluated from the true norms, so a solve whose recursive residual met the tolerance
// while its true residual does not is resumed.  One block, R <= 512.
__global__ void true_state_kernel(int R, int P, const double *partG, const double *partN, double *gamma,
                                  SolverState *st, long long max_iters, double tol, int stop_rule, int reopen,
                                  double *dbound = nullptr) {
    if (!reopen && st->done) return;
    __shared__ double sq[512];
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        sq[c] = sum_parts(partN, c, P);
        if (gamma) gamma[c] = sum_parts(partG, c, P);
        if (dbound) dbound[c] = sqrt(sq[c]) * (1.0 + 1e-6);
    }
    __syncthreads();
    if (threadIdx.x == 0 && reopen && st->status == GP_OK) st->done = 0;
    finish_norms_block(st, sq, R, st->iter, max_iters, tol, stop_rule);
    if (threadIdx.x == 0) st->certified = 1;
}

}  // namespace

// Host-side polling of the device state.
static inline int poll_state(const SolverState *dev, SolverState *host, cudaStream_t st) {
    GP_TRY_CUDA(cudaMemcpyAsync(host, dev, sizeof(SolverState), cudaMemcpyDeviceToHost, st));
    GP_TRY_CUDA(cudaStreamSynchronize(st));
    return GP_OK;
}

// The same poll, also reading the tensor-core kernels' time-out word (cleared when set, so the
// caller reports GP_ERR_TIMEOUT once): one synchronisation for both.
static inline int poll_state_tc(const SolverState *dev, SolverState *host, int *timed_out, cudaStream_t st) {
    int *w = tc_timeout_word();
    int h = 0;
    GP_TRY_CUDA(cudaMemcpyAsync(host, dev, sizeof(SolverState), cudaMemcpyDeviceToHost, st));
    if (w) GP_TRY_CUDA(cudaMemcpyAsync(&h, w, sizeof(int), cudaMemcpyDeviceToHost, st));
    GP_TRY_CUDA(cudaStreamSynchronize(st));
    if (h) {
        *timed_out = 1;
        GP_TRY_CUDA(cudaMemsetAsync(w, 0, sizeof(int), st));
    }
    return GP_OK;
}

static inline void fill_info(const SolverState &s, gp_solve_info_t *info) {
    info->iters = s.iter;
    info->converged = s.converged;
    info->status = s.status;
    info->res_y = s.res_y;
    info->res_z = s.res_z;
}


}  // namespace gp
