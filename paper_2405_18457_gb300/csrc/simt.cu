// CUDA-core (SIMT) kernel-matrix products and the fused gradient reduction, in
// FP32 and FP64.  These serve GP_PREC_FP32 and the plain FP64 form (*_f64
// entry points).  Tiles of 64 x 64 kernel entries are evaluated with direct
// coordinate differences (no norm split, so no cancellation) into shared
// memory and immediately contracted with the right-hand sides; the kernel
// matrix never reaches global memory.
#include "gp_internal.cuh"

#include <algorithm>

namespace gp {

namespace {

constexpr int BM = 64;   // rows of a tile
constexpr int BN = 64;   // columns of a tile
constexpr int NT = 256;  // threads per block (16 x 16)

int num_sms() { return device_sm_count(); }

template <typename T>
struct SplitPlan {
    int nsplit;
    int zchunks;
    int cpt;
};

int pick_cpt(int R) {
    if (R <= 16) return 1;
    if (R <= 32) return 2;
    if (R <= 64) return 4;
    if (R <= 80) return 5;
    return 8;
}

template <typename T>
SplitPlan<T> plan_mvm(int64_t n1, int64_t n2, int R) {
    SplitPlan<T> p;
    p.cpt = pick_cpt(R);
    p.zchunks = (int)cdiv(R, 16 * p.cpt);
    int64_t row_tiles = cdiv(std::max<int64_t>(n1, 1), BM);
    int64_t col_tiles = cdiv(std::max<int64_t>(n2, 1), BN);
    int64_t want = 2LL * num_sms();
    int64_t have = row_tiles * p.zchunks;
    int64_t ns = 1;
    if (have < want) ns = std::min<int64_t>(cdiv(want, have), std::max<int64_t>(col_tiles / 4, 1));
    p.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(ns, 1024));
    return p;
}

template <typename T>
size_t mvm_smem(int d, int cpt) {
    int dp = d + 1;
    return sizeof(T) * (size_t)(2 * BM * dp + BM * (BN + 1) + BN * (16 * cpt + 1));
}

template <typename T, int CPT>
__global__ void __launch_bounds__(NT) mvm_simt_kernel(const MvmArgs<T> a, int nsplit, T *partial) {
    if (a.done && *a.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = a.kp.d, dp = d + 1;
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Bs = As + BM * dp;
    T *Ks = Bs + BN * dp;
    T *Vs = Ks + BM * (BN + 1);
    constexpr int VP = 16 * CPT + 1;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int split = blockIdx.y;
    const int cbase = blockIdx.z * 16 * CPT;
    const int64_t col0 = a.col0_dev ? *a.col0_dev : 0;
    int64_t n2 = a.n2;
    if (a.col0_dev) n2 = min(n2, a.n2_total - col0);
    if (n2 < 0) n2 = 0;
    const int64_t per = cdiv(cdiv(n2, BN), nsplit) * BN;
    const int64_t jbeg = (int64_t)split * per;
    const int64_t jend = min(n2, jbeg + per);

    for (int e = tid; e < BM * d; e += NT) {
        int r = e / d, k = e - r * d;
        int64_t gi = row0 + r;
        As[r * dp + k] = gi < a.n1 ? a.X1[gi * d + k] * a.kp.inv_ell[k] : T(0);
    }
    T acc[4][CPT];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[p][q] = T(0);

    for (int64_t jt = jbeg; jt < jend; jt += BN) {
        __syncthreads();
        for (int e = tid; e < BN * d; e += NT) {
            int r = e / d, k = e - r * d;
            int64_t gj = jt + r;
            Bs[r * dp + k] = gj < jend ? a.X2[(col0 + gj) * d + k] * a.kp.inv_ell[k] : T(0);
        }
        for (int e = tid; e < BN * 16 * CPT; e += NT) {
            int cc = e / BN, jj = e - cc * BN;
            int64_t gj = jt + jj;
            int c = cbase + cc;
            Vs[jj * VP + cc] = (gj < jend && c < a.R) ? a.V[(int64_t)c * a.ldv + gj] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = ty + 16 * p;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = tx + 16 * q;
                T r2 = T(0);
                for (int k = 0; k < d; ++k) {
                    T t = As[i * dp + k] - Bs[j * dp + k];
                    r2 += t * t;
                }
                Ks[i * (BN + 1) + j] = (jt + j < jend) ? kval(a.kp.kind, a.kp.sf2, r2) : T(0);
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int j = 0; j < BN; ++j) {
            T kv[4], vv[CPT];
#pragma unroll
            for (int p = 0; p < 4; ++p) kv[p] = Ks[(tx + 16 * p) * (BN + 1) + j];
#pragma unroll
            for (int q = 0; q < CPT; ++q) vv[q] = Vs[j * VP + ty + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < CPT; ++q) acc[p][q] += kv[p] * vv[q];
        }
    }

    const int64_t drow0 = a.diag_from_col0 ? col0 : a.drow0;
    const int64_t ndiag = a.diag_from_col0 ? n2 : a.ndiag;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int64_t i = row0 + tx + 16 * p;
        if (i >= a.n1) continue;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = cbase + ty + 16 * q;
            if (c >= a.R) continue;
            if (nsplit > 1) {
                partial[((int64_t)split * a.R + c) * a.n1 + i] = acc[p][q];
            } else {
                T y = a.alpha * acc[p][q];
                if (a.beta != T(0)) y += a.beta * a.Y[(int64_t)c * a.ldy + i];
                if (a.diag_coef != T(0) && i >= drow0 && i < drow0 + ndiag)
                    y += a.diag_coef * a.Vd[(int64_t)c * a.ldvd + (i - drow0)];
                a.Y[(int64_t)c * a.ldy + i] = y;
            }
        }
    }
}

// Sums the split partials in a fixed order and applies the epilogue.
template <typename T>
__global__ void mvm_reduce_kernel(const MvmArgs<T> a, int nsplit, const T *partial) {
    if (a.done && *a.done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= a.n1) return;
    const int64_t col0 = a.col0_dev ? *a.col0_dev : 0;
    int64_t n2 = a.n2;
    if (a.col0_dev) n2 = min(n2, a.n2_total - col0);
    T s = T(0);
    for (int sp = 0; sp < nsplit; ++sp) s += partial[((int64_t)sp * a.R + c) * a.n1 + i];
    T y = a.alpha * s;
    if (a.beta != T(0)) y += a.beta * a.Y[(int64_t)c * a.ldy + i];
    const int64_t drow0 = a.diag_from_col0 ? col0 : a.drow0;
    const int64_t ndiag = a.diag_from_col0 ? n2 : a.ndiag;
    if (a.diag_coef != T(0) && i >= drow0 && i < drow0 + ndiag)
        y += a.diag_coef * a.Vd[(int64_t)c * a.ldvd + (i - drow0)];
    a.Y[(int64_t)c * a.ldy + i] = y;
}

template <typename T, int CPT>
int launch_mvm(const MvmArgs<T> &a, const SplitPlan<T> &pl, T *partial, cudaStream_t st) {
    size_t smem = mvm_smem<T>(a.kp.d, CPT);
    GP_TRY(ensure_max_dyn_smem((const void *)mvm_simt_kernel<T, CPT>));
    dim3 grid((unsigned)cdiv(a.n1, BM), (unsigned)pl.nsplit, (unsigned)pl.zchunks);
    prof_begin(st);
    mvm_simt_kernel<T, CPT><<<grid, NT, smem, st>>>(a, pl.nsplit, partial);
    prof_end(st);
    GP_TRY(check_launch("mvm_simt_kernel"));
    if (pl.nsplit > 1) {
        dim3 g2((unsigned)cdiv(a.n1, 256), (unsigned)a.R);
        mvm_reduce_kernel<T><<<g2, 256, 0, st>>>(a, pl.nsplit, partial);
        GP_TRY(check_launch("mvm_reduce_kernel"));
    }
    return GP_OK;
}

}  // namespace

template <typename T>
size_t mvm_simt_workspace(int64_t n1, int64_t n2, int R) {
    SplitPlan<T> pl = plan_mvm<T>(n1, n2, R);
    Carver c(nullptr);
    if (pl.nsplit > 1) c.take<T>((size_t)pl.nsplit * (size_t)R * (size_t)n1);
    return c.bytes();
}

template <typename T>
int mvm_simt(const MvmArgs<T> &a, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (a.n1 == 0 || a.R == 0) return GP_OK;
    SplitPlan<T> pl = plan_mvm<T>(a.n1, a.n2, a.R);
    if (mvm_smem<T>(a.kp.d, pl.cpt) > kMaxDynSmem) {
        set_error("mvm: d=%d too large for the CUDA-core tile in this precision", a.kp.d);
        return GP_ERR_UNSUPPORTED;
    }
    Carver c(ws);
    T *partial = nullptr;
    if (pl.nsplit > 1) partial = c.take<T>((size_t)pl.nsplit * (size_t)a.R * (size_t)a.n1);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    switch (pl.cpt) {
        case 1: return launch_mvm<T, 1>(a, pl, partial, st);
        case 2: return launch_mvm<T, 2>(a, pl, partial, st);
        case 4: return launch_mvm<T, 4>(a, pl, partial, st);
        case 5: return launch_mvm<T, 5>(a, pl, partial, st);
        default: return launch_mvm<T, 8>(a, pl, partial, st);
    }
}

template size_t mvm_simt_workspace<float>(int64_t, int64_t, int);
template size_t mvm_simt_workspace<double>(int64_t, int64_t, int);
template int mvm_simt<float>(const MvmArgs<float> &, void *, size_t, cudaStream_t);
template int mvm_simt<double>(const MvmArgs<double> &, void *, size_t, cudaStream_t);

// ===========================================================================
// Fused gradient reduction (CUDA cores)
// ===========================================================================
namespace {

constexpr int GB = 64;  // tile edge

template <typename T>
struct GradPlan {
    int row_tiles, jsplit, nblocks;
};

template <typename T>
GradPlan<T> plan_grad(int64_t n) {
    GradPlan<T> p;
    p.row_tiles = (int)cdiv(n, GB);
    int64_t col_tiles = cdiv(n, GB);
    int64_t want = 4LL * num_sms();
    int64_t js = std::max<int64_t>(1, std::min<int64_t>(cdiv(want, p.row_tiles), col_tiles));
    p.jsplit = (int)js;
    p.nblocks = p.row_tiles * p.jsplit;
    return p;
}

template <typename T>
size_t grad_smem(int d, int R) {
    int dp = d + 1, rp = R | 1;
    return sizeof(T) * (size_t)(2 * GB * dp + 2 * GB * rp + GB * (GB + 1));
}

// Per block: partial[block][k] for k < d (length-scale sums before the 1/l_k
// factor) and partial[block][d] (signal sum before the 2/s_f factor).
template <typename T, int DMAX>
__global__ void __launch_bounds__(NT) grad_simt_kernel(const GradArgs<T> a, int jsplit, double *partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = a.kp.d, dp = d + 1, R = a.R, rp = R | 1;
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Bs = As + GB * dp;
    T *Us = Bs + GB * dp;
    T *Ws = Us + GB * rp;
    T *Ms = Ws + GB * rp;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t n = a.n;
    const int64_t row0 = (int64_t)blockIdx.x * GB;
    const int64_t col_tiles = cdiv(n, GB);
    const int64_t per = cdiv(col_tiles, jsplit);
    const int64_t jt0 = (int64_t)blockIdx.y * per, jt1 = min(col_tiles, jt0 + per);

    for (int e = tid; e < GB * d; e += NT) {
        int r = e / d, k = e - r * d;
        int64_t gi = row0 + r;
        As[r * dp + k] = gi < n ? a.X[gi * d + k] * a.kp.inv_ell[k] : T(0);
    }
    for (int e = tid; e < GB * R; e += NT) {
        int c = e / GB, r = e - c * GB;
        int64_t gi = row0 + r;
        T u = T(0);
        if (gi < n) u = (c == 0) ? a.U0[gi] * T(a.lam0) : a.U[(int64_t)(c - 1) * a.ldu + gi] * T(a.lam_rest);
        Us[r * rp + c] = u;
    }
    double gacc[DMAX];
    double sacc = 0.0;
#pragma unroll
    for (int k = 0; k < DMAX; ++k) gacc[k] = 0.0;

    for (int64_t jt = jt0; jt < jt1; ++jt) {
        const int64_t col0 = jt * GB;
        __syncthreads();
        for (int e = tid; e < GB * d; e += NT) {
            int r = e / d, k = e - r * d;
            int64_t gj = col0 + r;
            Bs[r * dp + k] = gj < n ? a.X[gj * d + k] * a.kp.inv_ell[k] : T(0);
        }
        for (int e = tid; e < GB * R; e += NT) {
            int c = e / GB, r = e - c * GB;
            int64_t gj = col0 + r;
            T w = T(0);
            if (gj < n) w = (c == 0) ? a.W0[gj] : a.W[(int64_t)(c - 1) * a.ldw + gj];
            Ws[r * rp + c] = w;
        }
        __syncthreads();
        // M_ij = sum_c lam_c U_ci W_cj
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int i = ty + 16 * p;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = tx + 16 * q;
                T m = T(0);
                for (int c = 0; c < R; ++c) m += Us[i * rp + c] * Ws[j * rp + c];
                Ms[i * (GB + 1) + j] = m;
            }
        }
        __syncthreads();
        T gl[DMAX];
        T sl = T(0);
#pragma unroll
        for (int k = 0; k < DMAX; ++k) gl[k] = T(0);
        for (int p = 0; p < 4; ++p) {
            const int i = ty + 16 * p;
            if (row0 + i >= n) continue;
            for (int q = 0; q < 4; ++q) {
                const int j = tx + 16 * q;
                if (col0 + j >= n) continue;
                T r2 = T(0);
                for (int k = 0; k < d; ++k) {
                    T t = As[i * dp + k] - Bs[j * dp + k];
                    r2 += t * t;
                }
                T kv;
                T phi = kphi(a.kp.kind, a.kp.sf2, r2, &kv);
                T m = Ms[i * (GB + 1) + j];
                T w = phi * m;
                sl += kv * m;
                if (DMAX <= 32) {
#pragma unroll
                    for (int k = 0; k < DMAX; ++k) {
                        if (k < d) {
                            T t = As[i * dp + k] - Bs[j * dp + k];
                            gl[k] += w * t * t;
                        }
                    }
                } else {
                    for (int k = 0; k < d; ++k) {
                        T t = As[i * dp + k] - Bs[j * dp + k];
                        gl[k] += w * t * t;
                    }
                }
            }
        }
        if (DMAX <= 32) {
#pragma unroll
            for (int k = 0; k < DMAX; ++k) gacc[k] += (double)gl[k];
        } else {
            for (int k = 0; k < d; ++k) gacc[k] += (double)gl[k];
        }
        sacc += (double)sl;
    }

    // block reduction, fixed order
    __shared__ double red[NT / 32];
    const int lane = tid & 31, warp = tid >> 5;
    double *out = partial + (int64_t)(blockIdx.y * gridDim.x + blockIdx.x) * (d + 1);
    for (int k = 0; k <= d; ++k) {
        double v = (k < d) ? 0.0 : sacc;
        if (DMAX <= 32) {
#pragma unroll
            for (int kk = 0; kk < DMAX; ++kk)
                if (kk == k && k < d) v = gacc[kk];
        } else if (k < d) {
            v = gacc[k];
        }
        v = warp_sum(v);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; ++w) s += red[w];
            out[k] = s;
        }
    }
}

// sum_c lam_c U_c . W_c, per-block partials (the sigma term: dH/dsigma = 2 sigma I).  Blocks
// walk groups of 32 rows (lane = row, so every column read is coalesced); warp w of a block
// takes the columns c = w, w + 8, ...  The products of a row group and their sum over the
// warp's columns are taken in T, with one FP64 addition per group (FP64 arithmetic and
// conversions run at a small fraction of the FP32 rate on this GPU).
template <typename T>
__global__ void diag_dot_kernel(const GradArgs<T> a, double *partial) {
    const int64_t n = a.n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 32 + lane; i - lane < n; i += (int64_t)gridDim.x * 32) {
        if (i >= n) continue;
        T g0 = T(0), gr = T(0);
        for (int c = warp; c < a.R; c += nw) {
            if (c == 0)
                g0 = a.U0[i] * a.W0[i];
            else
                gr = fma(a.U[(int64_t)(c - 1) * a.ldu + i], a.W[(int64_t)(c - 1) * a.ldw + i], gr);
        }
        s += a.lam0 * (double)g0 + a.lam_rest * (double)gr;
    }
    __shared__ double red[32];
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// grad[k] = (sum_b partial[b][k]) / l_k for k < d; grad[d] = 2/s_f * sum_b partial[b][d];
// grad[d+1] = 2 sigma * sum_b dpart[b].
template <typename T>
__global__ void grad_finalize_kernel(const KP<T> kp, int nblocks, const double *partial, int ndiag,
                                     const double *dpart, double *grad, const double *theta_dev) {
    const int d = kp.d;
    const int k = blockIdx.x;  // one block per output
    double s = 0.0;
    if (k <= d) {
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(int64_t)b * (d + 1) + k];
    } else {
        for (int b = threadIdx.x; b < ndiag; b += blockDim.x) s += dpart[b];
    }
    __shared__ double red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double ell = theta_dev ? theta_dev[k < d ? k : 0] : (k < d ? (double)kp.ell[k] : 0.0);
        const double sf = theta_dev ? theta_dev[d] : (double)kp.sf;
        const double sigma = theta_dev ? theta_dev[d + 1] : (double)kp.sigma;
        if (k < d) grad[k] = t / ell;
        else if (k == d) grad[k] = 2.0 * t / sf;
        else grad[k] = 2.0 * sigma * t;
    }
}

constexpr int DIAG_BLOCKS = 256;

template <typename T, int DMAX>
int launch_grad(const GradArgs<T> &a, const GradPlan<T> &pl, double *partial, double *dpart,
                cudaStream_t st) {
    GP_TRY(ensure_max_dyn_smem((const void *)grad_simt_kernel<T, DMAX>));
    size_t smem = grad_smem<T>(a.kp.d, a.R);
    dim3 grid((unsigned)pl.row_tiles, (unsigned)pl.jsplit);
    grad_simt_kernel<T, DMAX><<<grid, NT, smem, st>>>(a, pl.jsplit, partial);
    GP_TRY(check_launch("grad_simt_kernel"));
    diag_dot_kernel<T><<<DIAG_BLOCKS, 256, 0, st>>>(a, dpart);
    GP_TRY(check_launch("diag_dot_kernel"));
    grad_finalize_kernel<T><<<a.kp.d + 2, 256, 0, st>>>(a.kp, pl.nblocks, partial, DIAG_BLOCKS, dpart,
                                                        a.grad, nullptr);
    GP_TRY(check_launch("grad_finalize_kernel"));
    return GP_OK;
}

}  // namespace

// sigma term and final assembly shared with the tensor-core estimator:
// partial[b][k] (k < d: length-scale sums before 1/l_k; k = d: signal sum
// before 2/s_f) over nblocks blocks -> grad (d+2).
template <typename T>
int grad_tail(const GradArgs<T> &a, int nblocks, const double *partial, double *dpart, cudaStream_t st) {
    diag_dot_kernel<T><<<DIAG_BLOCKS, 256, 0, st>>>(a, dpart);
    GP_TRY(check_launch("diag_dot_kernel"));
    grad_finalize_kernel<T><<<a.kp.d + 2, 256, 0, st>>>(a.kp, nblocks, partial, DIAG_BLOCKS, dpart, a.grad,
                                                        a.dev_theta);
    return check_launch("grad_finalize_kernel");
}
template int grad_tail<float>(const GradArgs<float> &, int, const double *, double *, cudaStream_t);

template <typename T>
size_t grad_simt_workspace(int64_t n, int d, int R) {
    GradPlan<T> pl = plan_grad<T>(n);
    Carver c(nullptr);
    c.take<double>((size_t)pl.nblocks * (size_t)(d + 1));
    c.take<double>(DIAG_BLOCKS);
    return c.bytes();
}

template <typename T>
int grad_simt(const GradArgs<T> &a, void *ws, size_t ws_bytes, cudaStream_t st) {
    const int d = a.kp.d;
    if (grad_smem<T>(d, a.R) > kMaxDynSmem) {
        set_error("mll_grad: d=%d with %d right-hand sides exceeds the CUDA-core tile", d, a.R);
        return GP_ERR_UNSUPPORTED;
    }
    GradPlan<T> pl = plan_grad<T>(a.n);
    Carver c(ws);
    double *partial = c.take<double>((size_t)pl.nblocks * (size_t)(d + 1));
    double *dpart = c.take<double>(DIAG_BLOCKS);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    if (d <= 16) return launch_grad<T, 16>(a, pl, partial, dpart, st);
    if (d <= 32) return launch_grad<T, 32>(a, pl, partial, dpart, st);
    return launch_grad<T, GP_MAX_D>(a, pl, partial, dpart, st);
}

template size_t grad_simt_workspace<float>(int64_t, int, int);
template size_t grad_simt_workspace<double>(int64_t, int, int);
template int grad_simt<float>(const GradArgs<float> &, void *, size_t, cudaStream_t);
template int grad_simt<double>(const GradArgs<double> &, void *, size_t, cudaStream_t);

}  // namespace gp
