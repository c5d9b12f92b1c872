// Reverse-mode derivatives of the bilinear form
//   f(theta, X, U, W) = sum_c lam_c u_c^T H(theta, X) w_c,   H = K + sigma^2 I (Sec. 2),
// the quantity whose theta-gradient is the marginal-likelihood estimator (Eq. mll_grad
// with Eq. trace or Eq. pathwise_estimator) and whose vector-Jacobian products give the
// backward pass of Y = H V (upstream G: f = sum_c g_c^T H v_c).
//
// The theta-gradient is the fused estimator reduction (simt.cu, tc.cu).  This file adds
// the point gradient
//   df/dx_i = -diag(1/l^2) sum_j S_ij psi_ij (x_i - x_j),   S = M + M^T,
//   M_ij = sum_c lam_c u_ci w_cj,
// where dk(x, x')/dx = -psi(r) (x - x') / l^2 with psi = k (RBF) or 3 s_f^2 exp(-sqrt3 r)
// (Matern-3/2): the same radial factor as dk/dl.  Kernel tiles are recomputed, never
// stored; per-row sums run over column splits into FP64 partials that a second kernel
// adds in a fixed order (deterministic), then scales by -1/l_k.
#include "solvers.cuh"

#include <algorithm>

namespace gp {

namespace {

constexpr int XB = 64;   // tile edge (rows and columns)
constexpr int XT = 256;  // threads per block

int sm_count() { return device_sm_count(); }

struct DxPlan {
    int row_tiles, jsplit;
};

DxPlan plan_dx(int64_t n) {
    DxPlan p;
    p.row_tiles = (int)cdiv(n, XB);
    int64_t col_tiles = cdiv(n, XB);
    int64_t want = 4LL * sm_count();
    p.jsplit = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(want, p.row_tiles), col_tiles));
    return p;
}

template <typename T>
size_t dx_smem(int d, int R, int sym) {
    const int dp = d + 1, rp = R | 1;
    return sizeof(T) * (size_t)(2 * XB * dp + (sym ? 2 : 4) * XB * rp + XB * (XB + 1));
}

// partial[y][i][k] = sum over the column tiles of split y of S_ij psi_ij (a_ik - a_jk),
// a = x / l.  KPT = outputs per thread per row (4 threads share a row).
template <typename T, int KPT>
__global__ void __launch_bounds__(XT) dx_simt_kernel(const GradArgs<T> a, int sym, int jsplit, double *partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = a.kp.d, dp = d + 1, R = a.R, rp = R | 1;
    T *As = reinterpret_cast<T *>(smem_raw);  // rows: x / l
    T *Bs = As + XB * dp;                     // columns: x / l
    T *UI = Bs + XB * dp;                     // rows: lam_c u_ci
    T *WJ = UI + XB * rp;                     // columns: w_cj
    T *WI = WJ + XB * rp;                     // rows: lam_c w_ci     (unused when sym)
    T *UJ = WI + (sym ? 0 : XB * rp);         // columns: u_cj        (unused when sym)
    T *W1 = UJ + (sym ? 0 : XB * rp);         // S_ij psi_ij
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t n = a.n;
    const int64_t row0 = (int64_t)blockIdx.x * XB;
    const int64_t col_tiles = cdiv(n, XB);
    const int64_t per = cdiv(col_tiles, jsplit);
    const int64_t jt0 = (int64_t)blockIdx.y * per, jt1 = min(col_tiles, jt0 + per);

    auto ucol = [&](int c, int64_t g) -> T { return c == 0 ? a.U0[g] : a.U[(int64_t)(c - 1) * a.ldu + g]; };
    auto wcol = [&](int c, int64_t g) -> T { return c == 0 ? a.W0[g] : a.W[(int64_t)(c - 1) * a.ldw + g]; };
    auto lam = [&](int c) -> T { return c == 0 ? T(a.lam0) : T(a.lam_rest); };

    for (int e = tid; e < XB * d; e += XT) {
        int r = e / d, k = e - r * d;
        int64_t gi = row0 + r;
        As[r * dp + k] = gi < n ? a.X[gi * d + k] * a.kp.inv_ell[k] : T(0);
    }
    for (int e = tid; e < XB * R; e += XT) {
        int c = e / XB, r = e - c * XB;
        int64_t gi = row0 + r;
        UI[r * rp + c] = gi < n ? lam(c) * ucol(c, gi) : T(0);
        if (!sym) WI[r * rp + c] = gi < n ? lam(c) * wcol(c, gi) : T(0);
    }

    // output ownership in the accumulation phase: row orow, dimensions kq + 4 q
    const int orow = tid >> 2, kq = tid & 3;
    double acc[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) acc[q] = 0.0;

    for (int64_t jt = jt0; jt < jt1; ++jt) {
        const int64_t col0 = jt * XB;
        __syncthreads();
        for (int e = tid; e < XB * d; e += XT) {
            int r = e / d, k = e - r * d;
            int64_t gj = col0 + r;
            Bs[r * dp + k] = gj < n ? a.X[gj * d + k] * a.kp.inv_ell[k] : T(0);
        }
        for (int e = tid; e < XB * R; e += XT) {
            int c = e / XB, r = e - c * XB;
            int64_t gj = col0 + r;
            WJ[r * rp + c] = gj < n ? wcol(c, gj) : T(0);
            if (!sym) UJ[r * rp + c] = gj < n ? ucol(c, gj) : T(0);
        }
        __syncthreads();
        // W1_ij = S_ij psi_ij on the 64 x 64 tile (zero outside the matrix)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = ty + 16 * p;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = tx + 16 * q;
                T w = T(0);
                if (row0 + i < n && col0 + j < n) {
                    T m = T(0);
                    for (int c = 0; c < R; ++c) m += UI[i * rp + c] * WJ[j * rp + c];
                    if (sym) {
                        m += m;
                    } else {
                        for (int c = 0; c < R; ++c) m += WI[i * rp + c] * UJ[j * rp + c];
                    }
                    T r2 = T(0);
                    for (int k = 0; k < d; ++k) {
                        T t = As[i * dp + k] - Bs[j * dp + k];
                        r2 += t * t;
                    }
                    T kv;
                    w = m * kphi(a.kp.kind, a.kp.sf2, r2, &kv);
                }
                W1[i * (XB + 1) + j] = w;
            }
        }
        __syncthreads();
        // acc[q] += sum_j W1_ij (a_ik - a_jk), k = kq + 4 q
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
            const int k = kq + 4 * q;
            if (k < d) {
                const T ai = As[orow * dp + k];
                T s = T(0);
                for (int j = 0; j < XB; ++j) s += W1[orow * (XB + 1) + j] * (ai - Bs[j * dp + k]);
                acc[q] += (double)s;
            }
        }
    }
    const int64_t gi = row0 + orow;
    if (gi < n) {
        double *out = partial + ((int64_t)blockIdx.y * n + gi) * d;
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
            const int k = kq + 4 * q;
            if (k < d) out[k] = acc[q];
        }
    }
}

// dX[i][k] = -(1/l_k) sum_y partial[y][i][k]  (fixed order over splits)
template <typename T>
__global__ void dx_finalize_kernel(const KP<T> kp, int64_t n, int jsplit, const double *partial, T *dX) {
    const int d = kp.d;
    const int64_t total = n * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % d);
        double s = 0.0;
        for (int y = 0; y < jsplit; ++y) s += partial[(int64_t)y * total + e];
        dX[e] = (T)(-s / (double)kp.ell[k]);
    }
}

// value = sum_c lam_c u_c^T K w_c + sigma^2 sum_c lam_c u_c^T w_c
//       = (s_f / 2) df/ds_f + (sigma / 2) df/dsigma   (both parts homogeneous of degree 2)
template <typename T>
__global__ void bilinear_value_kernel(const KP<T> kp, const double *g, double *value) {
    if (threadIdx.x == 0 && blockIdx.x == 0)
        *value = 0.5 * ((double)kp.sf * g[kp.d] + (double)kp.sigma * g[kp.d + 1]);
}

template <typename T, int KPT>
int launch_dx(const GradArgs<T> &a, int sym, const DxPlan &pl, double *partial, T *dX, cudaStream_t st) {
    GP_TRY(ensure_max_dyn_smem((const void *)dx_simt_kernel<T, KPT>));
    dim3 grid((unsigned)pl.row_tiles, (unsigned)pl.jsplit);
    dx_simt_kernel<T, KPT><<<grid, XT, dx_smem<T>(a.kp.d, a.R, sym), st>>>(a, sym, pl.jsplit, partial);
    GP_TRY(check_launch("dx_simt_kernel"));
    const int64_t total = a.n * a.kp.d;
    const int blocks = (int)std::min<int64_t>(cdiv(total, 256), 4LL * sm_count());
    dx_finalize_kernel<T><<<blocks, 256, 0, st>>>(a.kp, a.n, pl.jsplit, partial, dX);
    return check_launch("dx_finalize_kernel");
}

}  // namespace

template <typename T>
size_t bilinear_dx_workspace(int64_t n, int d) {
    DxPlan pl = plan_dx(n);
    Carver c(nullptr);
    c.take<double>((size_t)pl.jsplit * (size_t)n * (size_t)d);
    return c.bytes();
}

template <typename T>
int bilinear_dx(const GradArgs<T> &a, int sym, T *dX, void *ws, size_t ws_bytes, cudaStream_t st) {
    const int d = a.kp.d;
    if (dx_smem<T>(d, a.R, sym) > (size_t)kMaxDynSmem) {
        set_error("bilinear_grad: d=%d with %d vectors exceeds the point-gradient tile", d, a.R);
        return GP_ERR_UNSUPPORTED;
    }
    DxPlan pl = plan_dx(a.n);
    Carver c(ws);
    double *partial = c.take<double>((size_t)pl.jsplit * (size_t)a.n * (size_t)d);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    if (d <= 16) return launch_dx<T, 4>(a, sym, pl, partial, dX, st);
    if (d <= 32) return launch_dx<T, 8>(a, sym, pl, partial, dX, st);
    return launch_dx<T, GP_MAX_D / 4>(a, sym, pl, partial, dX, st);
}

template <typename T>
int bilinear_value(const KP<T> &kp, const double *g, double *value, cudaStream_t st) {
    bilinear_value_kernel<T><<<1, 32, 0, st>>>(kp, g, value);
    return check_launch("bilinear_value_kernel");
}

template size_t bilinear_dx_workspace<float>(int64_t, int);
template size_t bilinear_dx_workspace<double>(int64_t, int);
template int bilinear_dx<float>(const GradArgs<float> &, int, float *, void *, size_t, cudaStream_t);
template int bilinear_dx<double>(const GradArgs<double> &, int, double *, void *, size_t, cudaStream_t);
template int bilinear_value<float>(const KP<float> &, const double *, double *, cudaStream_t);
template int bilinear_value<double>(const KP<double> &, const double *, double *, cudaStream_t);

}  // namespace gp
