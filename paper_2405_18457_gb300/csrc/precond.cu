// Pivoted Cholesky preconditioner for conjugate gradients (App. B "Conjugate Gradients": a
// rank-100 pivoted Cholesky preconditioner in every CG run; the greedy factorisation of
// Harbrecht, Peters and Schneider 2012 as used by Gardner et al. 2018).
//
//   K ~ L^T L with L (k x n) built greedily: step m picks the point p with the largest remaining
//   diagonal (ties: lowest index), row m of L is (k(x_j, x_p) - sum_{l<m} L[l][j] L[l][p]) /
//   sqrt(diag_p), and its square leaves the remaining diagonal.
//   P = L^T L + sigma^2 I, applied through the Woodbury identity
//   P^-1 r = (r - L^T (sigma^2 I_k + L L^T)^-1 L r) / sigma^2,
// with the k x k matrix C = sigma^2 I + L L^T factorised once per solve in FP64.
#include "solvers.cuh"

#include <algorithm>

namespace gp {

namespace {

constexpr int PT = 128;    // points per tile of the L r / L^T w kernels
constexpr int PC_MAXK = 128;

__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(double x) { return x; }

// diag_j = k(x_j, x_j) = s_f^2 (stationary kernels)
template <typename T>
__global__ void pc_init_kernel(T *dg, int64_t n, T sf2, int *rank) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        dg[j] = sf2;
    if (blockIdx.x == 0 && threadIdx.x == 0) *rank = 0;
}

// Pivot of step m: the largest remaining diagonal, lowest index on ties (used points are
// marked -1).  One block.  Stops the factorisation (rank = m) when it is not positive.
template <typename T>
__global__ void pc_pivot_kernel(const T *dg, int64_t n, int m, int64_t *piv, T *lpp, int *rank) {
    __shared__ T bv[1024];
    __shared__ int64_t bi[1024];
    T best = T(-2);
    int64_t bidx = -1;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const T v = dg[j];
        if (v > best) {  // strictly greater: the lowest index wins within a thread
            best = v;
            bidx = j;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bidx;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            const T v2 = bv[threadIdx.x + off];
            const int64_t i2 = bi[threadIdx.x + off];
            if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 >= 0 && (bi[threadIdx.x] < 0 || i2 < bi[threadIdx.x]))) {
                bv[threadIdx.x] = v2;
                bi[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const bool go = (*rank == m) && bi[0] >= 0 && bv[0] > T(0);
        piv[m] = go ? bi[0] : -1;
        *lpp = go ? sqrt(bv[0]) : T(0);
        if (go) *rank = m + 1;
    }
}

// Row m of L and the diagonal update; zero row once the factorisation has stopped.
template <typename T>
__global__ void pc_row_kernel(const KP<T> kp, const T *X, int64_t n, int m, const int64_t *piv, const T *lpp,
                              T *L, T *dg) {
    const int64_t p = piv[m];
    const int d = kp.d;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if (p < 0) {
            L[(int64_t)m * n + j] = T(0);
            continue;
        }
        T r2 = T(0);
        for (int k = 0; k < d; ++k) {
            const T t = (X[j * d + k] - X[p * d + k]) * kp.inv_ell[k];
            r2 += t * t;
        }
        T v = kval(kp.kind, kp.sf2, r2);
        for (int l = 0; l < m; ++l) v -= L[(int64_t)l * n + j] * L[(int64_t)l * n + p];
        const T lm = v / *lpp;
        L[(int64_t)m * n + j] = lm;
        dg[j] = (j == p) ? T(-1) : dg[j] - lm * lm;
    }
}

// C = sigma^2 I + L L^T (k x k): one 32 x 32 tile per block, points streamed in 64s, products
// in the element type within a chunk and FP64 across chunks (FP64 arithmetic is slow on
// this GPU; the FP64 form keeps it throughout).
template <typename T>
__global__ void pc_gram_kernel(const T *L, int64_t n, int k, double sigma2, double *C) {
    __shared__ T Ta[32][65], Tb[32][65];
    const int a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads, 4 rows each
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t j0 = 0; j0 < n; j0 += 64) {
        for (int e = threadIdx.x; e < 32 * 64; e += 256) {
            const int r = e / 64, c = e % 64;
            const int64_t j = j0 + c;
            Ta[r][c] = (a0 + r < k && j < n) ? L[(int64_t)(a0 + r) * n + j] : T(0);
            Tb[r][c] = (b0 + r < k && j < n) ? L[(int64_t)(b0 + r) * n + j] : T(0);
        }
        __syncthreads();
        for (int q = 0; q < 4; ++q) {
            const int ar = ty + 8 * q;
            T s = T(0);
            for (int c = 0; c < 64; ++c) s += Ta[ar][c] * Tb[tx][c];
            acc[q] += to_d(s);
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        const int a = a0 + ty + 8 * q, b = b0 + tx;
        if (a < k && b < k) C[(int64_t)a * k + b] = acc[q] + (a == b ? sigma2 : 0.0);
    }
}

// In-place Cholesky C = G G^T (lower triangle, FP64), one block, right-looking.
__global__ void pc_chol_kernel(double *C, int k, int *fail) {
    for (int j = 0; j < k; ++j) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const double v = C[(int64_t)j * k + j];
            if (!(v > 0.0)) *fail = 1;
            C[(int64_t)j * k + j] = v > 0.0 ? sqrt(v) : 1.0;
        }
        __syncthreads();
        const double g = C[(int64_t)j * k + j];
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) C[(int64_t)i * k + j] /= g;
        __syncthreads();
        for (int e = threadIdx.x; e < (k - j - 1) * (k - j - 1); e += blockDim.x) {
            const int i = j + 1 + e / (k - j - 1), c = j + 1 + e % (k - j - 1);
            if (c <= i) C[(int64_t)i * k + c] -= C[(int64_t)i * k + j] * C[(int64_t)c * k + j];
        }
    }
}

// part[tile][m][c] = sum over the tile's points of L[m][i] r[c][i] (element type within the
// tile, FP64 across tiles).  Rows are padded to an odd stride (no bank conflicts).
constexpr int PTS = PT + 1;
template <typename T>
__global__ void __launch_bounds__(256) pc_lr_kernel(const T *L, const T *r, int64_t n, int k, int R, double *part,
                                                    const int *done) {
    if (done && *done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ls = reinterpret_cast<T *>(smem_raw);  // k x PTS
    T *Rs = Ls + (size_t)k * PTS;             // R x PTS
    const int64_t i0 = (int64_t)blockIdx.x * PT;
    for (int e = threadIdx.x; e < k * PT; e += blockDim.x) {
        const int m = e / PT, q = e % PT;
        Ls[m * PTS + q] = (i0 + q < n) ? L[(int64_t)m * n + i0 + q] : T(0);
    }
    for (int e = threadIdx.x; e < R * PT; e += blockDim.x) {
        const int c = e / PT, q = e % PT;
        Rs[c * PTS + q] = (i0 + q < n) ? r[(int64_t)c * n + i0 + q] : T(0);
    }
    __syncthreads();
    double *out = part + (int64_t)blockIdx.x * k * R;
    for (int e = threadIdx.x; e < k * R; e += blockDim.x) {
        const int m = e / R, c = e % R;
        const T *lm = Ls + (size_t)m * PTS;
        const T *rc = Rs + (size_t)c * PTS;
        T s = T(0);
        for (int q = 0; q < PT; ++q) s += lm[q] * rc[q];
        out[e] = to_d(s);
    }
}

// w[m][c] = (C^-1 (L r))[m][c]: sums the tiles' partials, then forward and back substitution
// with the Cholesky factor of C.  One block per right-hand side.
__global__ void pc_solve_kernel(const double *part, int ntiles, const double *G, int k, int R, double *w,
                                const int *done) {
    if (done && *done) return;
    __shared__ double y[PC_MAXK];
    const int c = blockIdx.x;
    for (int m = threadIdx.x; m < k; m += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < ntiles; ++t) s += part[((int64_t)t * k + m) * R + c];
        y[m] = s;
    }
    __syncthreads();
    // G z = y
    for (int m = 0; m < k; ++m) {
        if (threadIdx.x == 0) y[m] /= G[(int64_t)m * k + m];
        __syncthreads();
        for (int i = m + 1 + threadIdx.x; i < k; i += blockDim.x) y[i] -= G[(int64_t)i * k + m] * y[m];
        __syncthreads();
    }
    // G^T w = z
    for (int m = k - 1; m >= 0; --m) {
        if (threadIdx.x == 0) y[m] /= G[(int64_t)m * k + m];
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] -= G[(int64_t)m * k + i] * y[m];
        __syncthreads();
    }
    for (int m = threadIdx.x; m < k; m += blockDim.x) w[(int64_t)m * R + c] = y[m];
}

// p[c][i] = (r[c][i] - sum_m L[m][i] w[m][c]) / sigma^2; 16 right-hand sides per thread.
template <typename T>
__global__ void __launch_bounds__(256) pc_out_kernel(const T *L, const T *r, const double *w, int64_t n, int k,
                                                     int R, double inv_sigma2, T *p, const int *done) {
    if (done && *done) return;
    __shared__ T Ws[PC_MAXK * 16];
    const int c0 = blockIdx.y * 16;
    const int nc = min(16, R - c0);
    for (int e = threadIdx.x; e < k * 16; e += blockDim.x) {
        const int m = e / 16, cc = e % 16;
        Ws[e] = cc < nc ? (T)w[(int64_t)m * R + c0 + cc] : T(0);
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc[16];
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) acc[cc] = T(0);
    for (int m = 0; m < k; ++m) {
        const T l = L[(int64_t)m * n + i];
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) acc[cc] += l * Ws[m * 16 + cc];
    }
#pragma unroll
    for (int cc = 0; cc < 16; ++cc)
        if (cc < nc) {
            const int64_t e = (int64_t)(c0 + cc) * n + i;
            p[e] = (T)((to_d(r[e]) - to_d(acc[cc])) * inv_sigma2);
        }
}

size_t lr_smem(int k, int R, size_t tsz) { return tsz * (size_t)(k + R) * PTS; }

}  // namespace

template <typename T>
size_t precond_workspace(int64_t n, int R, int k) {
    if (k <= 0) return 0;
    const int64_t tiles = cdiv(n, PT);
    Carver c(nullptr);
    c.take<T>((size_t)k * n);           // L
    c.take<T>((size_t)n);               // remaining diagonal
    c.take<int64_t>((size_t)k);         // pivots
    c.take<T>(1);                       // sqrt of the pivot's diagonal
    c.take<int>(2);                     // rank, failure flag
    c.take<double>((size_t)k * k);      // C and its factor
    c.take<double>((size_t)tiles * k * R);  // L r partials
    c.take<double>((size_t)k * R);      // w
    return c.bytes();
}

template <typename T>
int precond_build(const KP<T> &kp, const T *X, int64_t n, int R, int k, void *ws, size_t ws_bytes, Precond<T> *out,
                  cudaStream_t st) {
    if (k > PC_MAXK) {
        set_error("preconditioner rank must be <= %d", PC_MAXK);
        return GP_ERR_INVALID_ARG;
    }
    if (lr_smem(k, std::min(R, 128), sizeof(T)) > (size_t)kMaxDynSmem) {
        set_error("preconditioner rank %d with %d right-hand sides exceeds shared memory", k, R);
        return GP_ERR_UNSUPPORTED;
    }
    const int64_t tiles = cdiv(n, PT);
    Carver c(ws);
    Precond<T> P{};
    P.k = k;
    P.n = n;
    P.R = R;
    P.L = c.take<T>((size_t)k * n);
    T *dg = c.take<T>((size_t)n);
    int64_t *piv = c.take<int64_t>((size_t)k);
    T *lpp = c.take<T>(1);
    int *flags = c.take<int>(2);
    P.G = c.take<double>((size_t)k * k);
    P.part = c.take<double>((size_t)tiles * k * R);
    P.w = c.take<double>((size_t)k * R);
    P.inv_sigma2 = 1.0 / ((double)kp.sigma * (double)kp.sigma);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    GP_TRY(ensure_max_dyn_smem((const void *)pc_lr_kernel<T>));
    const unsigned nb = (unsigned)std::min<int64_t>(cdiv(n, 256), 2048);
    pc_init_kernel<T><<<nb, 256, 0, st>>>(dg, n, kp.sf2, flags);
    GP_TRY_CUDA(cudaMemsetAsync(flags + 1, 0, sizeof(int), st));
    for (int m = 0; m < k; ++m) {
        pc_pivot_kernel<T><<<1, 1024, 0, st>>>(dg, n, m, piv, lpp, flags);
        pc_row_kernel<T><<<nb, 256, 0, st>>>(kp, X, n, m, piv, lpp, P.L, dg);
    }
    GP_TRY(check_launch("pivoted cholesky", 1 + 2 * k));
    const unsigned kt = (unsigned)cdiv(k, 32);
    pc_gram_kernel<T><<<dim3(kt, kt), 256, 0, st>>>(P.L, n, k, (double)kp.sigma * (double)kp.sigma, P.G);
    pc_chol_kernel<<<1, 256, 0, st>>>(P.G, k, flags + 1);
    GP_TRY(check_launch("preconditioner factor", 2));
    *out = P;
    return GP_OK;
}

template <typename T>
int precond_apply(const Precond<T> &P, const T *r, T *p, const int *done, cudaStream_t st) {
    const int64_t tiles = cdiv(P.n, PT);
    // right-hand sides in passes of at most 128 (shared memory of the L r tiles)
    for (int c0 = 0; c0 < P.R; c0 += 128) {
        const int R = std::min(128, P.R - c0);
        const T *rc = r + (int64_t)c0 * P.n;
        T *pc = p + (int64_t)c0 * P.n;
        pc_lr_kernel<T><<<(unsigned)tiles, 256, lr_smem(P.k, R, sizeof(T)), st>>>(P.L, rc, P.n, P.k, R, P.part, done);
        pc_solve_kernel<<<R, 128, 0, st>>>(P.part, (int)tiles, P.G, P.k, R, P.w, done);
        pc_out_kernel<T><<<dim3((unsigned)cdiv(P.n, 256), (unsigned)cdiv(R, 16)), 256, 0, st>>>(
            P.L, rc, P.w, P.n, P.k, R, P.inv_sigma2, pc, done);
        GP_TRY(check_launch("preconditioner apply", 3));
    }
    return GP_OK;
}

template size_t precond_workspace<float>(int64_t, int, int);
template size_t precond_workspace<double>(int64_t, int, int);
template int precond_build<float>(const KP<float> &, const float *, int64_t, int, int, void *, size_t,
                                  Precond<float> *, cudaStream_t);
template int precond_build<double>(const KP<double> &, const double *, int64_t, int, int, void *, size_t,
                                   Precond<double> *, cudaStream_t);
template int precond_apply<float>(const Precond<float> &, const float *, float *, const int *, cudaStream_t);
template int precond_apply<double>(const Precond<double> &, const double *, double *, const int *, cudaStream_t);

}  // namespace gp
