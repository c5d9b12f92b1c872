// Linear system solvers of App. B: conjugate gradients (Alg. 1), stochastic
// gradient descent (Alg. 3); alternating projections (Alg. 2) is in ap.cu.
//
// All solvers run on the normalised systems H u~ = b / (||b|| + eps) and
// rescale on exit.  Vectors are stored column-blocked (vector c at base + c*n)
// in T; every inner product, norm and step size is FP64.  The loop condition
// is evaluated on the device each iteration and latched into a `done` flag
// that every later kernel of the solve checks first, so the host only polls
// the flag every few iterations and never waits per iteration.
#include "solver_common.cuh"

#include <algorithm>
#include <type_traits>

namespace gp {

namespace {

// ---------------------------------------------------------------- CG kernels
// gamma = r^T P^-1 r (partG; = ||r||^2 without a preconditioner) after the initial residual,
// split norms from ||r||^2 (partN); sets done if already converged.
// One block, one thread per column (R <= 512).
__global__ void cg_start_kernel(int R, int P, const double *partG, const double *partN, double *gamma,
                                SolverState *st, long long max_iters, double tol, int stop_rule, int certified,
                                double *dbound) {
    __shared__ double sq[512];
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        sq[c] = sum_parts(partN, c, P);
        gamma[c] = sum_parts(partG, c, P);
        if (dbound) dbound[c] = sqrt(sq[c]) * (1.0 + 1e-6);  // the first direction is r: bound ||r||
    }
    if (threadIdx.x == 0) {
        st->done = 0;
        st->status = GP_OK;
    }
    __syncthreads();
    finish_norms_block(st, sq, R, 0, max_iters, tol, stop_rule);
    if (threadIdx.x == 0) st->certified = certified;  // r = b~ - H v0 from an exact-class product
}

// alpha = gamma / d^T H d, frozen columns get 0.
__global__ void cg_alpha_kernel(int R, int P, const double *part, const double *gamma, double *alpha,
                                SolverState *st) {
    if (st->done) return;
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        double dHd = sum_parts(part, c, P);
        double g = gamma[c];
        alpha[c] = (g > kFreeze && dHd > 0.0 && isfinite(dHd)) ? g / dHd : 0.0;
    }
}

// v += alpha d ; r -= alpha Hd ; part = ||r||^2 partial sums   (grid P x R)
template <typename T>
__global__ void cg_update_kernel(T *v, T *r, const T *d, const T *Hd, int64_t n, int P, const double *alpha,
                                 double *part, const SolverState *st) {
    if (st->done) return;
    const int p = blockIdx.x, c = blockIdx.y;
    const int64_t per = cdiv(n, P);
    const int64_t i0 = (int64_t)p * per, i1 = min(n, i0 + per);
    const T a = (T)alpha[c];
    const int64_t off = (int64_t)c * n;
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        v[off + i] += a * d[off + i];
        T rv = r[off + i] - a * Hd[off + i];
        r[off + i] = rv;
        s += (double)rv * (double)rv;
    }
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

// beta = gamma_new / gamma ; gamma = gamma_new (partG: r^T P^-1 r) ; split norms from ||r||^2
// (partN, current for frozen columns too) ; t++ ; loop condition.  One block, one thread per
// column.  Without a preconditioner partG == partN.
__global__ void cg_beta_kernel(int R, int P, const double *partG, const double *partN, double *gamma,
                               const double *alpha, double *beta, SolverState *st, long long max_iters, double tol,
                               int stop_rule) {
    if (st->done) return;
    __shared__ double sq[512];
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        double gn = sum_parts(partG, c, P);
        bool active = alpha[c] != 0.0;
        beta[c] = active ? gn / gamma[c] : 0.0;
        if (active) gamma[c] = gn;
        sq[c] = sum_parts(partN, c, P);
    }
    const long long t = st->iter + 1;
    __syncthreads();
    finish_norms_block(st, sq, R, t, max_iters, tol, stop_rule);
}

// d = r + beta d
template <typename T>
__global__ void cg_dir_kernel(T *d, const T *r, int64_t n, const double *beta, const SolverState *st) {
    if (st->done) return;
    const int c = blockIdx.y;
    const T b = (T)beta[c];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = (int64_t)c * n + i;
        d[e] = r[e] + b * d[e];
    }
}

// Fused forms of one iteration without a preconditioner (two launches instead of four).
// alpha_c = gamma_c / d_c^T H d_c from the PD partials of d^T H d per column (summed in a fixed
// order by every block; block 0 of column c records alpha_c), then v += alpha d, r -= alpha Hd
// and the partial sums of ||r||^2 into partN.  grid P x R
template <typename T>
__global__ void cg_update_fused_kernel(T *v, T *r, const T *d, const T *Hd, int64_t n, int P, const double *partD,
                                       int PD, const double *gcur, double *alpha, double *partN,
                                       const SolverState *st) {
    if (st->done) return;
    const int p = blockIdx.x, c = blockIdx.y;
    __shared__ double s_al;
    if (threadIdx.x < 32) {
        const double dHd = sum_parts_warp(partD, c, PD);
        if (threadIdx.x == 0) {
            const double g = gcur[c];
            const double al = (g > kFreeze && dHd > 0.0 && isfinite(dHd)) ? g / dHd : 0.0;
            s_al = al;
            if (p == 0) alpha[c] = al;
        }
    }
    __syncthreads();
    const int64_t per = part_len(n, P);
    const int64_t i0 = min(n, (int64_t)p * per), i1 = min(n, i0 + per);
    const T a = (T)s_al;
    const int64_t off = (int64_t)c * n;
    double sum = 0.0;
    bool done4 = false;
    if constexpr (std::is_same<T, float>::value) {
        if ((n & 3) == 0) {
            // float4 rows; the squares of four residual entries summed in FP32 per FP64 add
            float4 *v4 = reinterpret_cast<float4 *>(v + off), *r4 = reinterpret_cast<float4 *>(r + off);
            const float4 *d4 = reinterpret_cast<const float4 *>(d + off), *h4 = reinterpret_cast<const float4 *>(Hd + off);
            for (int64_t q = (i0 >> 2) + threadIdx.x; q < (i1 >> 2); q += blockDim.x) {
                float4 vv = v4[q], rr = r4[q];
                const float4 dv = d4[q], hv = h4[q];
                vv.x += a * dv.x;
                vv.y += a * dv.y;
                vv.z += a * dv.z;
                vv.w += a * dv.w;
                rr.x -= a * hv.x;
                rr.y -= a * hv.y;
                rr.z -= a * hv.z;
                rr.w -= a * hv.w;
                v4[q] = vv;
                r4[q] = rr;
                sum += (double)fmaf(rr.w, rr.w, fmaf(rr.z, rr.z, fmaf(rr.y, rr.y, rr.x * rr.x)));
            }
            done4 = true;
        }
    }
    if (!done4) {
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            v[off + i] += a * d[off + i];
            T rv = r[off + i] - a * Hd[off + i];
            r[off + i] = rv;
            sum += (double)rv * (double)rv;
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

// beta_c = gamma_new / gamma_c (0 for a frozen column) from the ||r||^2 partials, d = r + beta d.
// gamma alternates between two arrays by iteration parity: block (0, c) writes the next one,
// every block reads the current one.  Block (0, c) also records ||r_c||^2 in sq[c]; the last of
// the R blocks (0, .) to do so (a counter, reset by that block) takes the split norms, the
// iteration count and the loop condition.  A block that starts after `done` is latched skips
// its part of d, which the finished solve no longer needs.  grid G x R
// The tensor-core operand of the next product, written by the direction kernel (tensor-core
// form): D16[c][i] = fp16(d_c[i] * 2^(1-e_c)) with a power-of-two scale from a bound on
// max_i |d_c[i]| known before d is formed, |r_i| + |beta| |d_old,i| <= ||r|| + |beta| B_old (B
// the previous direction's bound; the first direction is r, B = ||r||), so no column-max pass
// is needed; vinv[c] = 2^(e_c - 1) undoes the scale.  Rows are p2 halves (columns padded with
// zeros, zeroed once per solve).
struct DirOperand {
    __half *D16;
    int64_t p2;
    float *vinv;
    const double *bcur;
    double *bnext;
};

template <typename T>
__global__ void cg_dir_fused_kernel(T *d, const T *r, int64_t n, int P, const double *partN, const double *gcur,
                                    double *gnext, const double *alpha, SolverState *st, long long max_iters,
                                    double tol, int stop_rule, int R, double *sq, int *counter, DirOperand op16) {
    if (st->done) return;
    const int c = blockIdx.y;
    __shared__ double s_b;
    __shared__ float s_scale;
    __shared__ int s_last;
    if (threadIdx.x < 32) {
        const double gn = sum_parts_warp(partN, c, P);
        if (threadIdx.x == 0) {
            const bool active = alpha[c] != 0.0;
            s_b = active ? gn / gcur[c] : 0.0;
            s_last = 0;
            if (op16.D16) {
                const double bnew = sqrt(gn) * (1.0 + 1e-6) + fabs(s_b) * op16.bcur[c];
                int e = 0;
                float scale = 1.0f, inv = 1.0f;
                if (bnew > 0.0 && isfinite(bnew)) {
                    frexp(bnew, &e);  // bnew = f 2^e, f in [0.5, 1): |d| * 2^(1-e) < 2
                    scale = ldexpf(1.0f, 1 - e);
                    inv = ldexpf(1.0f, e - 1);
                }
                s_scale = scale;
                if (blockIdx.x == 0) {
                    op16.bnext[c] = bnew;
                    op16.vinv[c] = inv;
                }
            }
            if (blockIdx.x == 0) {
                gnext[c] = active ? gn : gcur[c];
                sq[c] = gn;
                __threadfence();
                s_last = (atomicAdd(counter, 1) == R - 1) ? 1 : 0;
            }
        }
    }
    __syncthreads();
    if (s_last) {
        // every column's ||r||^2 is in sq: norms (the block in parallel), then the iteration
        // count and the loop condition
        __shared__ double rt[512];
        __threadfence();
        const volatile double *vs = sq;
        for (int cc = threadIdx.x; cc < R; cc += blockDim.x) rt[cc] = sqrt(vs[cc]);
        __syncthreads();
        if (threadIdx.x == 0) {
            *counter = 0;
            finish_state(st, rt, R, st->iter + 1, max_iters, tol, stop_rule);
        }
    }
    const T b = (T)s_b;
    bool done4 = false;
    if constexpr (std::is_same<T, float>::value) {
        const float sc = op16.D16 ? s_scale : 0.0f;
        __half *h16 = op16.D16 ? op16.D16 + (int64_t)c * op16.p2 : nullptr;
        if ((n & 3) == 0) {
            float4 *d4 = reinterpret_cast<float4 *>(d + (int64_t)c * n);
            const float4 *r4 = reinterpret_cast<const float4 *>(r + (int64_t)c * n);
            for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (n >> 2);
                 q += (int64_t)gridDim.x * blockDim.x) {
                float4 dv = d4[q];
                const float4 rv = r4[q];
                dv.x = rv.x + b * dv.x;
                dv.y = rv.y + b * dv.y;
                dv.z = rv.z + b * dv.z;
                dv.w = rv.w + b * dv.w;
                d4[q] = dv;
                if (h16) {
                    __half2 lo = __floats2half2_rn(dv.x * sc, dv.y * sc), hi = __floats2half2_rn(dv.z * sc, dv.w * sc);
                    uint2 u;
                    u.x = *reinterpret_cast<uint32_t *>(&lo);
                    u.y = *reinterpret_cast<uint32_t *>(&hi);
                    reinterpret_cast<uint2 *>(h16)[q] = u;
                }
            }
            done4 = true;
        }
        if (!done4) {
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
                 i += (int64_t)gridDim.x * blockDim.x) {
                const int64_t e = (int64_t)c * n + i;
                const float v = r[e] + b * d[e];
                d[e] = v;
                if (h16) h16[i] = __float2half_rn(v * sc);
            }
            done4 = true;
        }
    }
    if (!done4) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t e = (int64_t)c * n + i;
            d[e] = r[e] + b * d[e];
        }
    }
}

}  // namespace

// ===========================================================================
// Operator: H applied to R column-blocked vectors of stride n, skipping when done
// ===========================================================================
template <typename T>
struct HOp {
    KP<T> kp;
    const T *X;
    int64_t n;
    int R;
    int prec;
    void *ws;
    size_t wsb;
    TcPoints pts{};
    bool tc = false;

    static size_t workspace(int64_t n, int d, int R, int prec) {
        Carver c(nullptr);
        if (std::is_same<T, float>::value && prec == GP_PREC_TC16) {
            c.take<char>(tc_points_bytes(n, d));
            c.take<char>(tc_mvm_workspace(n, n, R));
        } else {
            c.take<char>(mvm_simt_workspace<T>(n, n, R));
        }
        return c.bytes();
    }
    int init(const KP<T> &k, const T *Xp, int64_t np, int Rp, int pr, void *w, size_t wb, cudaStream_t st) {
        kp = k;
        X = Xp;
        n = np;
        R = Rp;
        prec = pr;
        if constexpr (std::is_same<T, float>::value) {
            if (prec == GP_PREC_TC16) {
                tc = true;
                Carver c(w);
                void *pbuf = c.take<char>(tc_points_bytes(n, kp.d));
                wsb = tc_mvm_workspace(n, n, R);
                ws = c.take<char>(wsb);
                GP_TRY(check_ws(w, wb, c.bytes()));
                return tc_prepare_points(kp, X, n, pbuf, &pts, st);
            }
        }
        ws = w;
        wsb = wb;
        return GP_OK;
    }
    // Y = alpha * K V + beta * Y + diag (sigma^2 V unless overridden); split: the tensor-core
    // form's split products (FP32-class), for true residuals
    // dotpart / nparts (tensor-core form): the product also takes the per-CTA partial sums of
    // V^T Y per column when its schedule allows (*nparts = their count per column, else 0).
    int apply(const T *V, T *Y, const int *done, cudaStream_t st, bool split = false, const void *V16pre = nullptr,
              const float *vinv_pre = nullptr, double *dotpart = nullptr, int *nparts = nullptr) {
        if (nparts) *nparts = 0;
        if constexpr (std::is_same<T, float>::value) {
            if (tc) {
                TcMvmArgs a{};
                a.kind = kp.kind;
                a.rows = pts;
                a.cols = pts;
                a.V = V;
                a.ldv = n;
                a.R = R;
                a.Y = Y;
                a.ldy = n;
                a.sf2 = kp.sf2;
                a.alpha = 1.0f;
                a.beta = 0.0f;
                a.diag_coef = kp.sigma2;
                a.Vd = V;
                a.ldvd = n;
                a.drow0 = 0;
                a.ndiag = n;
                a.done = done;
                a.split = split ? 1 : 0;
                a.V16pre = V16pre;
                a.vinv_pre = vinv_pre;
                a.dotv = V;
                a.lddv = n;
                a.dotpart = dotpart;
                a.dot_parts = nparts;
                return tc_mvm(a, ws, wsb, st);
            }
        }
        MvmArgs<T> a{};
        a.kp = kp;
        a.X1 = X;
        a.n1 = n;
        a.X2 = X;
        a.n2 = n;
        a.n2_total = n;
        a.V = V;
        a.ldv = n;
        a.R = R;
        a.Y = Y;
        a.ldy = n;
        a.alpha = T(1);
        a.beta = T(0);
        a.diag_coef = kp.sigma2;
        a.Vd = V;
        a.ldvd = n;
        a.ndiag = n;
        a.done = done;
        return mvm_simt<T>(a, ws, wsb, st);
    }
};

// ===========================================================================
// True residual with the FP64 product (FP32 form's check)
// ===========================================================================
size_t f64_residual_workspace(int64_t n, int d, int R) {
    Carver c(nullptr);
    c.take<double>((size_t)n * d);
    c.take<double>((size_t)R * n);
    c.take<double>((size_t)R * n);
    c.take<char>(mvm_simt_workspace<double>(n, n, R));
    return c.bytes();
}

int f64_residual(const KP<float> &kp, const float *X, int64_t n, const float *B, const float *V, int R,
                 const double *scale, float *r, double *partN, int P, void *ws, size_t ws_bytes, cudaStream_t st) {
    Carver c(ws);
    double *X64 = c.take<double>((size_t)n * kp.d);
    double *V64 = c.take<double>((size_t)R * n);
    double *HV64 = c.take<double>((size_t)R * n);
    const size_t mb = mvm_simt_workspace<double>(n, n, R);
    void *mw = c.take<char>(mb);
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));
    KP<double> k64;
    k64.kind = kp.kind;
    k64.d = kp.d;
    for (int k = 0; k < kp.d; ++k) {
        k64.ell[k] = (double)kp.ell[k];
        k64.inv_ell[k] = 1.0 / (double)kp.ell[k];
    }
    k64.sf = (double)kp.sf;
    k64.sf2 = k64.sf * k64.sf;
    k64.sigma = (double)kp.sigma;
    k64.sigma2 = k64.sigma * k64.sigma;
    const unsigned nb = (unsigned)std::min<int64_t>(cdiv((int64_t)R * n, 256), 4096);
    widen_kernel<<<nb, 256, 0, st>>>(X, X64, n * kp.d);
    widen_kernel<<<nb, 256, 0, st>>>(V, V64, (int64_t)R * n);
    GP_TRY(check_launch("widen_kernel", 2));
    MvmArgs<double> a{};
    a.kp = k64;
    a.X1 = X64;
    a.n1 = n;
    a.X2 = X64;
    a.n2 = n;
    a.n2_total = n;
    a.V = V64;
    a.ldv = n;
    a.R = R;
    a.Y = HV64;
    a.ldy = n;
    a.alpha = 1.0;
    a.beta = 0.0;
    a.diag_coef = k64.sigma2;
    a.Vd = V64;
    a.ldvd = n;
    a.ndiag = n;
    GP_TRY(mvm_simt<double>(a, mw, mb, st));
    true_residual_kernel<float, double><<<dim3((unsigned)P, (unsigned)R), 256, 0, st>>>(B, HV64, r, n, P, scale,
                                                                                         partN, nullptr);
    return check_launch("true_residual_kernel");
}

// ===========================================================================
// Conjugate gradients, Alg. 1 (P = identity)
// ===========================================================================
template <typename T>
size_t cg_workspace(int64_t n, int d, int R, int prec, int pc_rank) {
    const int P = nparts_for(n);
    Carver c(nullptr);
    for (int k = 0; k < 3; ++k) c.take<T>((size_t)R * n);  // r, d, Hd
    c.take<double>((size_t)R * P);                          // partial sums
    c.take<double>((size_t)R * P);                          // ||r||^2 partial sums
    for (int k = 0; k < 6; ++k) c.take<double>(R);          // scale, gamma (x2), alpha, beta, ||r||^2
    c.take<int>(1);                                         // block counter of the direction kernel
    c.take<SolverState>(1);
    c.take<char>(HOp<T>::workspace(n, d, R, prec));
    if (std::is_same<T, float>::value && prec == GP_PREC_FP32) c.take<char>(f64_residual_workspace(n, d, R));
    if (std::is_same<T, float>::value && prec == GP_PREC_TC16 && pc_rank == 0 && R <= 128) {
        c.take<__half>((size_t)tc_rhs_pad(R) * tc_cols_pad(n));  // the directions' fp16 operand
        c.take<float>(256);
        c.take<double>(2 * (size_t)R);
        c.take<double>((size_t)R * 256);                   // d^T H d partials of the product's CTAs
    }
    if (pc_rank > 0) {
        c.take<T>((size_t)R * n);                           // p = P^-1 r
        c.take<double>((size_t)R * P);                      // r^T p partial sums
        c.take<char>(precond_workspace<T>(n, R, pc_rank));
    }
    return c.bytes();
}

template <typename T>
int cg_solve(const KP<T> &kp, const T *X, int64_t n, const T *B, int R, T *V, int64_t max_iters, double tol,
             int stop_rule, int prec, gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t st,
             int pc_rank) {
    if (R > 512) {
        set_error("nrhs must be <= 512");
        return GP_ERR_INVALID_ARG;
    }
    const bool pc = pc_rank > 0;
    const int P = nparts_for(n);
    Carver c(ws);
    T *r = c.take<T>((size_t)R * n);
    T *dd = c.take<T>((size_t)R * n);
    T *Hd = c.take<T>((size_t)R * n);
    double *part = c.take<double>((size_t)R * P);
    double *partN = c.take<double>((size_t)R * P);
    double *scale = c.take<double>(R);
    double *gamma = c.take<double>(2 * (size_t)R);  // two arrays, alternating by iteration parity
    double *alpha = c.take<double>(R);
    double *sqn = c.take<double>(R);
    int *dcount = c.take<int>(1);
    double *beta = c.take<double>(R);
    SolverState *sd = c.take<SolverState>(1);
    size_t opb = HOp<T>::workspace(n, kp.d, R, prec);
    void *opw = c.take<char>(opb);
    const bool check64 = std::is_same<T, float>::value && prec == GP_PREC_FP32;
    const size_t c64b = check64 ? f64_residual_workspace(n, kp.d, R) : 0;
    void *c64w = check64 ? c.take<char>(c64b) : nullptr;
    // tensor-core form without a preconditioner: the direction kernel writes the next product's
    // fp16 operand itself (no column-max and conversion launches per iteration)
    const bool d16 = std::is_same<T, float>::value && prec == GP_PREC_TC16 && !pc && R <= 128;
    const int64_t p2 = tc_cols_pad(n);
    __half *D16 = d16 ? c.take<__half>((size_t)tc_rhs_pad(R) * p2) : nullptr;
    float *vinv16 = d16 ? c.take<float>(256) : nullptr;
    double *dbnd = d16 ? c.take<double>(2 * (size_t)R) : nullptr;
    double *dotp = d16 ? c.take<double>((size_t)R * 256) : nullptr;
    T *pz = pc ? c.take<T>((size_t)R * n) : nullptr;
    double *partG = pc ? c.take<double>((size_t)R * P) : part;
    const size_t pcb = pc ? precond_workspace<T>(n, R, pc_rank) : 0;
    void *pcw = pc ? c.take<char>(pcb) : nullptr;
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));

    HOp<T> op;
    GP_TRY(op.init(kp, X, n, R, prec, opw, opb, st));
    Precond<T> pcd{};
    if (pc) GP_TRY(precond_build<T>(kp, X, n, R, pc_rank, pcw, pcb, &pcd, st));
    const dim3 gv((unsigned)std::min<int64_t>(cdiv(n, 2048), 1024), (unsigned)R);  // about 8 rows per thread
    const dim3 gp_((unsigned)P, (unsigned)R);
    // direction update: about four float4 per thread
    const dim3 gd((unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 4096), 1024)), (unsigned)R);
    const int *done = &sd->done;

    GP_TRY_CUDA(cudaMemsetAsync(dcount, 0, sizeof(int), st));
    if (d16) GP_TRY_CUDA(cudaMemsetAsync(D16, 0, sizeof(__half) * (size_t)tc_rhs_pad(R) * p2, st));
    // normalisation (App. B): scale_c = ||b_c|| + eps, v <- v / scale
    coldot_kernel<T><<<gp_, 256, 0, st>>>(B, B, n, P, part, nullptr);
    norm_scale_kernel<<<1, 256, 0, st>>>(R, P, part, scale);
    scale_cols_kernel<T><<<gv, 256, 0, st>>>(V, n, scale, 1);
    GP_TRY(check_launch("cg setup", 3));
    // r = b~ - H v ; p = P^-1 r ; d = p ; gamma = r^T p  (with the form's own product: its error
    // is caught by the check when the loop stops)
    GP_TRY(op.apply(V, Hd, nullptr, st));
    init_residual_kernel<T><<<gv, 256, 0, st>>>(B, Hd, r, dd, n, scale);
    GP_TRY(check_launch("cg residual"));
    if (pc) {
        GP_TRY(precond_apply<T>(pcd, r, pz, nullptr, st));
        GP_TRY_CUDA(cudaMemcpyAsync(dd, pz, sizeof(T) * (size_t)R * n, cudaMemcpyDeviceToDevice, st));
        coldot_kernel<T><<<gp_, 256, 0, st>>>(r, pz, n, P, partG, nullptr);
    }
    coldot_kernel<T><<<gp_, 256, 0, st>>>(r, r, n, P, part, nullptr);
    // the FP32 form's initial residual is not of the check's (FP64) class either
    cg_start_kernel<<<1, 256, 0, st>>>(R, P, partG, part, gamma, sd, (long long)max_iters, tol, stop_rule,
                                       (op.tc || check64) ? 0 : 1, dbnd);
    GP_TRY(check_launch("cg start", pc ? 3 : 2));

    // Iterations are enqueued speculatively in chunks without waiting for the start-up
    // kernels: once the device-side loop condition latches `done`, the remaining kernels
    // of a chunk return immediately, so a chunk overshoot costs only empty launches.
    // Chunks of 8, 4, 4, 4, 8, 16, 32, 32, ... iterations between polls: a warm-started solve
    // typically needs about ten, so few empty iterations are enqueued past convergence.
    //
    // The iterations carry Alg. 1's recursive residual, which drifts from b~ - H v under the
    // products' rounding.  When the loop stops on it (unless the state already comes from a
    // true residual), the true residual is recomputed once (differences rounded once, FP64 norms) and
    // the tolerance is judged on it; if it misses, CG restarts from it (d = r, or P^-1 r)
    // within the budget.  The FP32 form recomputes it with the FP64 product: a product of H
    // with the whole iterate carries an error of about u ||H|| ||v||, which in FP32 on an
    // ill-conditioned system lies far above the residuals CG reaches (measured: replacing the
    // recursive residual by an FP32 true residual every 10 iterations made CG diverge on the
    // small workload); the tensor-core form uses its split products (FP32-class), since its
    // plain fp16 product is off by about 2^-11 ||H|| ||v||.  The reported norms are therefore
    // always true-residual norms.
    SolverState hs{};
    // The first chunk follows the previous solve on this thread (warm-started solves of one
    // optimisation take similar counts), so that most solves poll once.
    static thread_local int64_t last_iters = 0;
    int64_t chunk = last_iters > 0 ? std::min<int64_t>(std::max<int64_t>(last_iters + 1, 4), 64) : 8;
    int64_t ti = 0;  // host index of the next enqueued iteration (selects gamma's parity array)
    int polls = 0, timed_out = 0;
    // gamma array the iteration with host index i reads as its current gamma
    auto gamma_at = [&](int64_t i) { return pc ? gamma : gamma + (i & 1) * R; };
    auto poll = [&]() -> int { return op.tc ? poll_state_tc(sd, &hs, &timed_out, st) : poll_state(sd, &hs, st); };
    bool d16_valid = false;  // D16 holds the current direction (written by the last direction kernel)
    int64_t dev_iters = 0;  // iterations the device has performed, as of the last poll
    int checks = 0;         // failed true-residual checks so far (restarts)
    double prev_y = 0.0, prev_z = 0.0;
    for (;;) {
        const int64_t left = max_iters - dev_iters;
        int64_t phase = 0;
        while (phase < left) {
            const int64_t k = std::min<int64_t>(chunk, left - phase);
            for (int64_t it = 0; it < k; ++it, ++ti) {
                // d^T H d: partial sums from the product itself where it takes them
                int nd = 0;
                GP_TRY(op.apply(dd, Hd, done, st, false, d16_valid ? D16 : nullptr, d16_valid ? vinv16 : nullptr,
                                pc ? nullptr : dotp, &nd));
                if (nd == 0) coldot_kernel<T><<<gp_, 256, 0, st>>>(dd, Hd, n, P, part, done);
                const double *pdot = nd > 0 ? dotp : part;
                const int ndot = nd > 0 ? nd : P;
                if (!pc) {
                    const double *gcur = gamma_at(ti);
                    double *gnext = gamma_at(ti + 1);
                    const DirOperand o16{D16, p2, vinv16, d16 ? dbnd + (ti & 1) * R : nullptr,
                                         d16 ? dbnd + ((ti + 1) & 1) * R : nullptr};
                    cg_update_fused_kernel<T><<<gp_, 256, 0, st>>>(V, r, dd, Hd, n, P, pdot, ndot, gcur, alpha, partN,
                                                                    sd);
                    cg_dir_fused_kernel<T><<<gd, 256, 0, st>>>(dd, r, n, P, partN, gcur, gnext, alpha, sd,
                                                               (long long)max_iters, tol, stop_rule, R, sqn, dcount,
                                                               o16);
                    GP_TRY(check_launch("cg iteration", nd > 0 ? 2 : 3));
                    d16_valid = d16;
                } else {
                    cg_alpha_kernel<<<1, 256, 0, st>>>(R, P, part, gamma, alpha, sd);
                    cg_update_kernel<T><<<gp_, 256, 0, st>>>(V, r, dd, Hd, n, P, alpha, part, sd);
                    GP_TRY(precond_apply<T>(pcd, r, pz, done, st));
                    coldot_kernel<T><<<gp_, 256, 0, st>>>(r, pz, n, P, partG, done);
                    cg_beta_kernel<<<1, 256, 0, st>>>(R, P, partG, part, gamma, alpha, beta, sd, (long long)max_iters,
                                                      tol, stop_rule);
                    cg_dir_kernel<T><<<gv, 256, 0, st>>>(dd, pz, n, beta, sd);
                    GP_TRY(check_launch("cg iteration", 6));
                }
            }
            phase += k;
            ++polls;
            chunk = polls < 4 ? 4 : std::min<int64_t>(polls == 4 ? 8 : chunk * 2, 32);
            GP_TRY(poll());
            if (hs.done) break;
        }
        if (phase == 0) GP_TRY(poll());
        dev_iters = hs.iter;
        if (timed_out || hs.status != GP_OK || hs.certified) break;
        // the loop stopped on the recursive residual: recompute the true one and judge it
        if (check64) {
            if constexpr (std::is_same<T, float>::value)
                GP_TRY(f64_residual(kp, X, n, B, V, R, scale, r, partN, P, c64w, c64b, st));
        } else {
            GP_TRY(op.apply(V, Hd, nullptr, st, true));
            true_residual_kernel<T, T><<<gp_, 256, 0, st>>>(B, Hd, r, n, P, scale, partN, nullptr);
            GP_TRY(check_launch("cg true residual"));
        }
        // restart direction (used only if the check fails): d = r, or P^-1 r with gamma = r^T P^-1 r
        if (pc) {
            GP_TRY(precond_apply<T>(pcd, r, pz, nullptr, st));
            coldot_kernel<T><<<gp_, 256, 0, st>>>(r, pz, n, P, partG, nullptr);
            GP_TRY(check_launch("cg restart (preconditioned)"));
        }
        GP_TRY_CUDA(cudaMemcpyAsync(dd, pc ? pz : r, sizeof(T) * (size_t)R * n, cudaMemcpyDeviceToDevice, st));
        true_state_kernel<<<1, 256, 0, st>>>(R, P, pc ? partG : partN, partN, gamma_at(ti), sd, (long long)max_iters,
                                             tol, stop_rule, 1, d16 ? dbnd + (ti & 1) * R : nullptr);
        d16_valid = false;  // the restart direction is converted by the product itself
        GP_TRY(check_launch("cg true-residual state"));
        GP_TRY(poll());
        dev_iters = hs.iter;
        if (timed_out || hs.done) break;
        // A restart that did not lower the true residual (by 10%) since the previous check means
        // the form's arithmetic has reached the accuracy it can attain on this system: stop
        // there, not converged, rather than spend the budget on further restarts.
        if (checks > 0 && std::max(hs.res_y / prev_y, hs.res_z / prev_z) > 0.9) break;
        prev_y = hs.res_y;
        prev_z = hs.res_z;
        ++checks;
        chunk = 4;  // restarted from a residual close to the tolerance
    }
    // the loop ends on a poll (the state no longer changes), so the rescale is not waited for
    scale_cols_kernel<T><<<gv, 256, 0, st>>>(V, n, scale, 0);
    GP_TRY(check_launch("cg rescale"));
    fill_info(hs, info);
    last_iters = hs.iter;
    if (timed_out) {
        set_error("a bounded wait in a tensor-core kernel gave up (its results are not valid)");
        return GP_ERR_TIMEOUT;
    }
    if (hs.status != GP_OK) {
        set_error("CG breakdown: residual became non-finite at iteration %lld", hs.iter);
        return hs.status;
    }
    return GP_OK;
}

template size_t cg_workspace<float>(int64_t, int, int, int, int);
template size_t cg_workspace<double>(int64_t, int, int, int, int);
template int cg_solve<float>(const KP<float> &, const float *, int64_t, const float *, int, float *, int64_t,
                             double, int, int, gp_solve_info_t *, void *, size_t, cudaStream_t, int);
template int cg_solve<double>(const KP<double> &, const double *, int64_t, const double *, int, double *,
                              int64_t, double, int, int, gp_solve_info_t *, void *, size_t, cudaStream_t, int);

// ===========================================================================
// Stochastic gradient descent, Alg. 3
// ===========================================================================
namespace {

// Gather the batch rows of X into Xb (batch x d) and mark them in slot[].
template <typename T>
__global__ void sgd_gather_kernel(const T *X, int d, const int32_t *idx, int64_t batch, T *Xb, int *slot,
                                  const SolverState *st) {
    if (st->done) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < batch * d; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = e / d, k = e - q * d;
        int64_t i = idx[q];
        Xb[e] = X[i * d + k];
        if (k == 0) slot[i] = (int)q;
    }
}

// g[c][q] = (K V)[c][q] + sigma^2 v[c][idx q] - b~[c][idx q]  (in place in G)
// and the residual estimate update r[c][idx q] <- g, maintaining sum r^2 per
// column incrementally in FP64: rsq[c] += g^2 - r_old^2.
// With gmax (tensor-core form): also the batch gradient's column maxima (atomicMax on float bits)
// for the step's operand bound, and the next step's maxima buffers zeroed.
template <typename T>
__global__ void sgd_grad_kernel(T *G, const T *V, const T *Bn, T *r, int64_t n, const int32_t *idx,
                                int64_t batch, T sigma2, const int *slot, double *rsq_delta_part,
                                const SolverState *st, unsigned *gmax, const float *pv, const float *pm, int nblk,
                                float *vmax, float *mmax) {
    if (st->done) return;
    const int c = blockIdx.y;
    double s = 0.0;
    float gm = 0.0f;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < batch; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx[q];
        int64_t e = (int64_t)c * n + i;
        T g = G[(int64_t)c * batch + q] + sigma2 * V[e] - Bn[e];
        G[(int64_t)c * batch + q] = g;
        gm = fmaxf(gm, fabsf((float)g));
        if (slot[i] == (int)q) {  // one writer per row even if an index repeats
            T old = r[e];
            s += (double)g * (double)g - (double)old * (double)old;
        }
    }
    if (gmax) {
        for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&gmax[c], __float_as_uint(gm));
        if (pv && blockIdx.x == 0) {
            // the previous step's maxima of v and m from its blocks' partial maxima
            float a = 0.0f, b = 0.0f;
            for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
                a = fmaxf(a, pv[(int64_t)c * nblk + k]);
                b = fmaxf(b, pm[(int64_t)c * nblk + k]);
            }
            for (int o = 16; o > 0; o >>= 1) {
                a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
                b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
            }
            __shared__ float s_a[32], s_b[32];
            if ((threadIdx.x & 31) == 0) {
                s_a[threadIdx.x >> 5] = a;
                s_b[threadIdx.x >> 5] = b;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                    a = fmaxf(a, s_a[w]);
                    b = fmaxf(b, s_b[w]);
                }
                vmax[c] = a;
                mmax[c] = b;
            }
        }
    }
    __shared__ double red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        rsq_delta_part[(int64_t)c * gridDim.x + blockIdx.x] = t;
    }
}

// The next row panel's fp16 operand, written by the step kernel (tensor-core form): V16[c][i] =
// fp16(v_c[i] 2^(1-e_c)) with a power-of-two scale from a bound on max_i |v_c[i]| known before
// the step, B = max|v_old| + rho max|m_old| + (lr/b) max|g| >= max|v_old + m_new| (the maxima
// exact: the previous step's, from its per-block partial maxima reduced by the next gradient
// kernel, and the batch gradient's); vinv[c] = 2^(e_c - 1).
struct SgdOperand {
    __half *V16;
    int64_t p2;
    float *vinv;
    const float *vmax, *mmax;  // maxima of this step's inputs v, m (per column)
    float *pv, *pm;            // this step's per-block maxima of its outputs (R x nblk)
    int nblk;
    const unsigned *gmax;      // the batch gradient's maxima (this iteration, float bits)
    unsigned *gmax_next;       // zeroed here for the next iteration's gradient
};

// W consecutive elements as one 16-byte access (W = 1: scalar).
template <typename T, int W>
struct SgdVec {
    using type = T;
};
template <>
struct SgdVec<float, 4> {
    using type = float4;
};
template <>
struct SgdVec<double, 2> {
    using type = double2;
};
constexpr int kSgdUnroll = 2;  // row groups per thread with their loads in flight together

// Dense step over all rows: m = rho m - (lr/b) g ; v += m ; r[i] = g on batch rows.  grid
// (blocks, R): one column per blockIdx.y; each thread takes W consecutive rows (one 16-byte load
// of m and of v) in kSgdUnroll grid-strided groups whose loads are issued before any arithmetic,
// so that enough bytes are in flight for HBM.  Requires n % W == 0 and 16-byte aligned columns
// for W > 1.  With the fp16 operand each thread keeps running maxima of |v| and |m|, and each
// block writes its maxima (no atomics).
template <typename T, int W>
__global__ void __launch_bounds__(256) sgd_step_kernel(T *__restrict__ Vv, T *__restrict__ M, T *__restrict__ r,
                                                       const T *__restrict__ G, int64_t n, int64_t batch,
                                                       const int *__restrict__ slot, T rho, T lrb,
                                                       const SolverState *st, SgdOperand op16) {
    using VT = typename SgdVec<T, W>::type;
    if (st->done) return;
    const int c = blockIdx.y;
    const bool f16 = op16.V16 != nullptr;
    float scale = 1.0f;
    if (f16) {
        // the column's scale, once per block (FP64 arithmetic is slow on this GPU)
        __shared__ float s_scale;
        if (threadIdx.x == 0) {
            const double bnd =
                (double)op16.vmax[c] + (double)rho * op16.mmax[c] + (double)lrb * __uint_as_float(op16.gmax[c]);
            int e = 0;
            float sc = 1.0f;
            if (bnd > 0.0 && isfinite(bnd)) {
                frexp(bnd * (1.0 + 1e-6), &e);  // |v| 2^(1-e) < 2
                sc = ldexpf(1.0f, 1 - e);
            }
            s_scale = sc;
            if (blockIdx.x == 0) {
                op16.vinv[c] = 1.0f / sc;
                op16.gmax_next[c] = 0u;
            }
        }
        __syncthreads();
        scale = s_scale;
    }
    VT *Vc = reinterpret_cast<VT *>(Vv + (int64_t)c * n);
    VT *Mc = reinterpret_cast<VT *>(M + (int64_t)c * n);
    T *rc = r + (int64_t)c * n;
    const T *Gc = G + (int64_t)c * batch;
    const int64_t nv = n / W, stride = (int64_t)gridDim.x * blockDim.x;
    float vm = 0.0f, mm = 0.0f;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j0 < nv; j0 += kSgdUnroll * stride) {
        VT mv[kSgdUnroll], vv[kSgdUnroll];
#pragma unroll
        for (int u = 0; u < kSgdUnroll; ++u) {
            const int64_t j = j0 + u * stride;
            if (j < nv) {
                mv[u] = Mc[j];
                vv[u] = Vc[j];
            }
        }
#pragma unroll
        for (int u = 0; u < kSgdUnroll; ++u) {
            const int64_t j = j0 + u * stride;
            if (j >= nv) break;
            T *m = reinterpret_cast<T *>(&mv[u]);
            T *v = reinterpret_cast<T *>(&vv[u]);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const int64_t i = j * W + k;
                const int q = slot[i];
                const T g = (q >= 0) ? Gc[q] : T(0);
                m[k] = rho * m[k] - lrb * g;
                v[k] += m[k];
                if (q >= 0) rc[i] = g;
            }
            Mc[j] = mv[u];
            Vc[j] = vv[u];
            if constexpr (std::is_same<T, float>::value) {
                if (f16) {
                    alignas(8) __half h[W];
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        h[k] = __float2half_rn(v[k] * scale);
                        vm = fmaxf(vm, fabsf(v[k]));
                        mm = fmaxf(mm, fabsf(m[k]));
                    }
                    __half *dst = op16.V16 + (int64_t)c * op16.p2 + j * W;
                    if constexpr (W == 4) {
                        *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(h);
                    } else {
#pragma unroll
                        for (int k = 0; k < W; ++k) dst[k] = h[k];
                    }
                }
            }
        }
    }
    if (f16) {
        __shared__ float s_v[8], s_m[8];
        for (int o = 16; o > 0; o >>= 1) {
            vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
            mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
        }
        if ((threadIdx.x & 31) == 0) {
            s_v[threadIdx.x >> 5] = vm;
            s_m[threadIdx.x >> 5] = mm;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                vm = fmaxf(vm, s_v[w]);
                mm = fmaxf(mm, s_m[w]);
            }
            op16.pv[(int64_t)c * op16.nblk + blockIdx.x] = vm;
            op16.pm[(int64_t)c * op16.nblk + blockIdx.x] = mm;
        }
    }
}

__global__ void sgd_clear_slots_kernel(const int32_t *idx, int64_t batch, int *slot, const SolverState *st) {
    if (st->done) return;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < batch; q += (int64_t)gridDim.x * blockDim.x)
        slot[idx[q]] = -1;
}

// out[c] = max_i |V[c][i]| as float bits (atomicMax; out zeroed by the caller).  grid (blocks, R)
__global__ void absmax_cols_kernel(const float *V, int64_t n, unsigned *out) {
    const int c = blockIdx.y;
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(V[(int64_t)c * n + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&out[c], __float_as_uint(m));
}

__global__ void fill_int_kernel(int *p, int64_t cnt, int v) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = v;
}

// rsq[c] = sum parts (initial, exact) and loop condition.
__global__ void sgd_start_kernel(int R, int P, const double *part, double *rsq, SolverState *st,
                                 long long max_iters, double tol, int stop_rule) {
    if (threadIdx.x != 0) return;
    double sq[512];
    for (int c = 0; c < R; ++c) {
        sq[c] = sum_parts(part, c, P);
        rsq[c] = sq[c];
    }
    st->done = 0;
    st->status = GP_OK;
    double r0 = 0.0;
    for (int c = 0; c < R; ++c) r0 += sq[c];
    st->res0 = r0;
    finish_norms(st, sq, R, 0, max_iters, tol, stop_rule);
}

__global__ void sgd_norm_kernel(int R, int nb, const double *dpart, double *rsq, SolverState *st,
                                long long max_iters, double tol, int stop_rule) {
    if (st->done) return;
    if (threadIdx.x != 0) return;
    double sq[512];
    double tot = 0.0;
    for (int c = 0; c < R; ++c) {
        double s = rsq[c];
        for (int b = 0; b < nb; ++b) s += dpart[(int64_t)c * nb + b];
        s = fmax(s, 0.0);
        rsq[c] = s;
        sq[c] = s;
        tot += s;
    }
    finish_norms(st, sq, R, st->iter + 1, max_iters, tol, stop_rule);
    if (!(tot <= 1e12 * fmax(st->res0, 1e-300))) {
        st->status = GP_ERR_DIVERGED;
        st->done = 1;
    }
}

}  // namespace

template <typename T>
static size_t sgd_panel_ws(int64_t batch, int64_t n, int d, int R, int prec) {
    if (std::is_same<T, float>::value && prec == GP_PREC_TC16) {
        // tensor-core panel: all points as columns (prepared once per solve), the batch rows
        // (prepared every iteration with the same scale), the product's own scratch
        Carver c(nullptr);
        c.take<char>(tc_points_bytes(n, d));
        c.take<char>(tc_points_bytes(batch, d));
        c.take<char>(tc_mvm_workspace(batch, n, R));
        return c.bytes();
    }
    return mvm_workspace<T>(batch, n, d, R, prec);
}

template <typename T>
size_t sgd_workspace(int64_t n, int d, int R, int64_t batch, int prec) {
    const int P = nparts_for(n);
    Carver c(nullptr);
    for (int k = 0; k < 3; ++k) c.take<T>((size_t)R * n);  // normalised b, momentum, residual estimate
    c.take<T>((size_t)R * batch);                           // batch gradient
    c.take<T>((size_t)batch * d);                           // gathered batch points
    c.take<int>((size_t)n);                                 // row -> batch slot
    c.take<double>((size_t)R * P);
    c.take<double>((size_t)R * 64);
    for (int k = 0; k < 2; ++k) c.take<double>(R);
    c.take<SolverState>(1);
    c.take<char>(sgd_panel_ws<T>(batch, n, d, R, prec));
    if (std::is_same<T, float>::value && prec == GP_PREC_TC16 && R <= 128) {
        c.take<__half>((size_t)tc_rhs_pad(R) * tc_cols_pad(n));  // the step's fp16 operand of v
        c.take<float>(256);
        c.take<float>(2 * (size_t)R);                            // maxima of v, m
        c.take<unsigned>(2 * (size_t)R);                         // maxima of g (x 2)
        c.take<float>(2 * (size_t)R * 2048);                     // the step's per-block maxima
    }
    return c.bytes();
}

template <typename T>
int sgd_solve(const KP<T> &kp, const T *X, int64_t n, const T *B, int R, T *V, int64_t batch,
              const int32_t *idx, double lr, double rho, int64_t max_iters, double tol, int stop_rule, int prec,
              gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (R > 512) {
        set_error("nrhs must be <= 512");
        return GP_ERR_INVALID_ARG;
    }
    const int d = kp.d;
    const int P = nparts_for(n);
    Carver c(ws);
    T *Bn = c.take<T>((size_t)R * n);
    T *M = c.take<T>((size_t)R * n);
    T *r = c.take<T>((size_t)R * n);
    T *G = c.take<T>((size_t)R * batch);
    T *Xb = c.take<T>((size_t)batch * d);
    int *slot = c.take<int>((size_t)n);
    double *part = c.take<double>((size_t)R * P);
    double *dpart = c.take<double>((size_t)R * 64);
    double *scale = c.take<double>(R);
    double *rsq = c.take<double>(R);
    SolverState *sd = c.take<SolverState>(1);
    size_t pwb = sgd_panel_ws<T>(batch, n, d, R, prec);
    void *pw = c.take<char>(pwb);
    // tensor-core form: the step writes the next panel's fp16 operand of v itself
    const bool v16 = std::is_same<T, float>::value && prec == GP_PREC_TC16 && R <= 128;
    const int64_t p2 = tc_cols_pad(n);
    __half *V16 = v16 ? c.take<__half>((size_t)tc_rhs_pad(R) * p2) : nullptr;
    float *vinv16 = v16 ? c.take<float>(256) : nullptr;
    float *vmm = v16 ? c.take<float>(2 * (size_t)R) : nullptr;          // vmax, mmax
    unsigned *gmx = v16 ? c.take<unsigned>(2 * (size_t)R) : nullptr;    // gmax[2]
    float *pvm = v16 ? c.take<float>(2 * (size_t)R * 2048) : nullptr;   // per-block maxima of v, m
    GP_TRY(check_ws(ws, ws_bytes, c.bytes()));

    const dim3 gv((unsigned)std::min<int64_t>(cdiv(n, 2048), 1024), (unsigned)R);  // about 8 rows per thread
    const dim3 gp_((unsigned)P, (unsigned)R);
    const int nbg = (int)std::min<int64_t>(64, std::max<int64_t>(1, cdiv(batch, 256)));
    // b~ = b / (||b|| + eps), v <- v / scale, m = 0, r = b~
    coldot_kernel<T><<<gp_, 256, 0, st>>>(B, B, n, P, part, nullptr);
    norm_scale_kernel<<<1, 256, 0, st>>>(R, P, part, scale);
    GP_TRY_CUDA(cudaMemcpyAsync(Bn, B, sizeof(T) * R * n, cudaMemcpyDeviceToDevice, st));
    scale_cols_kernel<T><<<gv, 256, 0, st>>>(Bn, n, scale, 1);
    scale_cols_kernel<T><<<gv, 256, 0, st>>>(V, n, scale, 1);
    GP_TRY_CUDA(cudaMemsetAsync(M, 0, sizeof(T) * R * n, st));
    GP_TRY_CUDA(cudaMemcpyAsync(r, Bn, sizeof(T) * R * n, cudaMemcpyDeviceToDevice, st));
    fill_int_kernel<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 4096), 256, 0, st>>>(slot, n, -1);
    if (v16) {
        GP_TRY_CUDA(cudaMemsetAsync(V16, 0, sizeof(__half) * (size_t)tc_rhs_pad(R) * p2, st));
        GP_TRY_CUDA(cudaMemsetAsync(vmm, 0, sizeof(float) * 2 * (size_t)R, st));
        GP_TRY_CUDA(cudaMemsetAsync(gmx, 0, sizeof(unsigned) * 2 * (size_t)R, st));
        if constexpr (std::is_same<T, float>::value)
            absmax_cols_kernel<<<dim3((unsigned)std::min<int64_t>(cdiv(n, 256), 256), (unsigned)R), 256, 0, st>>>(
                V, n, reinterpret_cast<unsigned *>(vmm));  // max |v0| (non-negative float bits = the float)
    }
    coldot_kernel<T><<<gp_, 256, 0, st>>>(r, r, n, P, part, nullptr);
    sgd_start_kernel<<<1, 32, 0, st>>>(R, P, part, rsq, sd, (long long)max_iters, tol, stop_rule);
    GP_TRY(check_launch("sgd setup", 7));

    SolverState hs{};
    GP_TRY(poll_state(sd, &hs, st));
    // Tensor-core row panel G = K(X_b, X) V: columns prepared once per solve, rows per iteration.
    TcMvmArgs ta{};
    void *rbuf = nullptr, *tw = nullptr;
    size_t twb = 0;
    if constexpr (std::is_same<T, float>::value) {
        if (prec == GP_PREC_TC16) {
            Carver pc(pw);
            void *cbuf = pc.take<char>(tc_points_bytes(n, d));
            rbuf = pc.take<char>(tc_points_bytes(batch, d));
            twb = tc_mvm_workspace(batch, n, R);
            tw = pc.take<char>(twb);
            GP_TRY(tc_prepare_points(kp, X, n, cbuf, &ta.cols, st));
            ta.kind = kp.kind;
            ta.V = V;
            ta.ldv = n;
            ta.R = R;
            ta.Y = G;
            ta.ldy = batch;
            ta.sf2 = kp.sf2;
            ta.alpha = 1.0f;
            ta.beta = 0.0f;
            ta.diag_coef = 0.0f;
            ta.done = &sd->done;
        }
    }
    int64_t t = 0, chunk = 8;
    const T lrb = (T)(lr / (double)batch);
    float *vmax = vmm, *mmax = vmm ? vmm + R : nullptr;
    float *pv = pvm, *pm = pvm ? pvm + (size_t)R * 2048 : nullptr;
    // the step kernel's launch: 16-byte accesses where every column starts 16-byte aligned
    constexpr int kW = 16 / sizeof(T);
    const bool vec = (n % kW == 0) && ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(M) |
                                        reinterpret_cast<uintptr_t>(r)) % 16 == 0);
    const dim3 gs((unsigned)std::min<int64_t>(cdiv(vec ? n / kW : n, 256 * kSgdUnroll), 2048), (unsigned)R);
    const int nblk = (int)gs.x;  // <= 2048, the per-block maxima's row length
    while (!hs.done && t < max_iters) {
        int64_t k = std::min<int64_t>(chunk, max_iters - t);
        for (int64_t it = 0; it < k; ++it, ++t) {
            const int32_t *bi = idx + t * batch;
            sgd_gather_kernel<T><<<(unsigned)cdiv(batch * d, 256), 256, 0, st>>>(X, d, bi, batch, Xb, slot, sd);
            GP_TRY(check_launch("sgd gather"));
            // G = K(X_b, X) V   (row panel H[i, :] v without the noise term)
            if constexpr (std::is_same<T, float>::value) {
                if (prec == GP_PREC_TC16) {
                    GP_TRY(tc_prepare_rows(kp, Xb, batch, ta.cols, rbuf, &ta.rows, st));
                    ta.V16pre = (v16 && t > 0) ? V16 : nullptr;  // written by the previous step
                    ta.vinv_pre = vinv16;
                    GP_TRY(tc_mvm(ta, tw, twb, st));
                } else {
                    MvmArgs<T> a{};
                    a.kp = kp; a.X1 = Xb; a.n1 = batch; a.X2 = X; a.n2 = n; a.n2_total = n;
                    a.V = V; a.ldv = n; a.R = R; a.Y = G; a.ldy = batch;
                    a.alpha = T(1); a.beta = T(0); a.diag_coef = T(0); a.done = &sd->done;
                    GP_TRY(mvm_simt<T>(a, pw, pwb, st));
                }
            } else {
                MvmArgs<T> a{};
                a.kp = kp; a.X1 = Xb; a.n1 = batch; a.X2 = X; a.n2 = n; a.n2_total = n;
                a.V = V; a.ldv = n; a.R = R; a.Y = G; a.ldy = batch;
                a.alpha = T(1); a.beta = T(0); a.diag_coef = T(0); a.done = &sd->done;
                GP_TRY(mvm_simt<T>(a, pw, pwb, st));
            }
            const int pc = (int)(t & 1), pn = (int)((t + 1) & 1);
            sgd_grad_kernel<T><<<dim3(nbg, R), 256, 0, st>>>(G, V, Bn, r, n, bi, batch, kp.sigma2, slot, dpart, sd,
                                                            v16 ? gmx + pc * R : nullptr, (v16 && t > 0) ? pv : nullptr,
                                                            pm, nblk, vmax, mmax);
            const SgdOperand o16{V16, p2, vinv16, vmax, mmax, pv, pm, nblk, v16 ? gmx + pc * R : nullptr,
                                 v16 ? gmx + pn * R : nullptr};
            if (vec)
                sgd_step_kernel<T, kW><<<gs, 256, 0, st>>>(V, M, r, G, n, batch, slot, (T)rho, lrb, sd, o16);
            else
                sgd_step_kernel<T, 1><<<gs, 256, 0, st>>>(V, M, r, G, n, batch, slot, (T)rho, lrb, sd, o16);
            sgd_clear_slots_kernel<<<(unsigned)cdiv(batch, 256), 256, 0, st>>>(bi, batch, slot, sd);
            sgd_norm_kernel<<<1, 32, 0, st>>>(R, nbg, dpart, rsq, sd, (long long)max_iters, tol, stop_rule);
            GP_TRY(check_launch("sgd iteration", 4));
        }
        chunk = std::min<int64_t>(chunk * 2, 64);
        GP_TRY(poll_state(sd, &hs, st));
    }
    scale_cols_kernel<T><<<gv, 256, 0, st>>>(V, n, scale, 0);
    GP_TRY(check_launch("sgd rescale"));
    GP_TRY(poll_state(sd, &hs, st));
    fill_info(hs, info);
    if (hs.status == GP_ERR_DIVERGED) {
        set_error("SGD diverged at iteration %lld (residual estimate grew beyond 1e6 x its start)", hs.iter);
        return hs.status;
    }
    if (hs.status != GP_OK) {
        set_error("SGD breakdown at iteration %lld", hs.iter);
        return hs.status;
    }
    return GP_OK;
}

template size_t sgd_workspace<float>(int64_t, int, int, int64_t, int);
template size_t sgd_workspace<double>(int64_t, int, int, int64_t, int);
template int sgd_solve<float>(const KP<float> &, const float *, int64_t, const float *, int, float *, int64_t,
                              const int32_t *, double, double, int64_t, double, int, int, gp_solve_info_t *,
                              void *, size_t, cudaStream_t);
template int sgd_solve<double>(const KP<double> &, const double *, int64_t, const double *, int, double *,
                               int64_t, const int32_t *, double, double, int64_t, double, int, int,
                               gp_solve_info_t *, void *, size_t, cudaStream_t);

}  // namespace gp
