// Batches of independent GPs of uneven size: one marginal-likelihood step (operands
// from theta, warm-started CG of Alg. 1, the gradient estimator of Eq. mll_grad and the
// softplus/Adam update) for every member at once, with all state on the device.
//
// Members are packed one after another (points, vector blocks, hyperparameters).  Each
// per-point kernel walks a table of 1024-row chunks, each reduction sums a member's own
// chunks in a fixed order (deterministic), and the product is the grouped tcgen05
// kernel of tc.cu (one CTA per 128-row work item, longest first).  After
// gp_batch_bind() no call synchronises, allocates or copies from the host, so a whole
// step can be captured into a CUDA graph and replayed; a member whose CG has met the
// tolerance is skipped by every later kernel of the solve (device flag per member).
#include "solver_common.cuh"

#include <algorithm>
#include <cstring>
#include <exception>
#include <new>
#include <vector>

using namespace gp;

namespace gp {
namespace bt {

constexpr int GT = 64;          // gradient tile edge
constexpr int GL = 32;          // gradient column tiles per work item
constexpr int GSTRIDE = kBatchMaxD + 1;  // partial sums per gradient item
constexpr int kMaxBatchR = 128;
// Members with at least this many points take the tensor-core gradient (16-bit operands; with
// fewer points the CUDA-core FP32 estimator is both cheap and tighter).
constexpr int64_t kTcGradMinN = 1024;

struct BGItem {
    int member, row_tile, ct0, ct1;
};

}  // namespace bt
}  // namespace gp

using gp::bt::BGItem;

struct gp_batch {
    int kind = 0, G = 0, s = 0, R = 0, R_pad = 0;
    std::vector<BMember> mem;
    std::vector<BChunk> chunks;
    std::vector<BItem> items[3];
    std::vector<BGItem> gitems;
    int64_t class_rows[3] = {0, 0, 0};
    int KD[3] = {64, 128, 192};
    int64_t N = 0, x_len = 0, theta_len = 0, v_cols = 0;
    struct Ptrs {
        BMember *mem;
        BChunk *chunks;
        BItem *items[3];
        BGItem *gitems;
        void *PA[3], *PB[3];
        void *V16;
        float *vinv;
        unsigned *colmax;
        float *r, *dd, *Hd;
        double *part, *scale, *gamma, *alpha, *beta;
        SolverState *state;
        int *done;
        int *cdone;  // member done with a state from a true residual (skipped by its recomputation)
        int *cskip;  // members a true-residual check leaves alone: certified, or still iterating
        double *gpart, *spart;
        int *err;
        void *tcg;         // workspace of the tensor-core gradient, reused member by member
        size_t tcg_bytes;  // 0: the batch's gradient runs on the CUDA cores
    } p{};
    void *ws = nullptr;
    bool bound = false;

    // Carves the workspace (base == nullptr: size query).  Same code for both.
    size_t carve(void *base, Ptrs *o) const {
        Carver c(base);
        const size_t nch = chunks.size();
        o->mem = c.take<BMember>(mem.size());
        o->chunks = c.take<BChunk>(std::max<size_t>(nch, 1));
        for (int k = 0; k < 3; ++k) o->items[k] = c.take<BItem>(std::max<size_t>(items[k].size(), 1));
        o->gitems = c.take<BGItem>(std::max<size_t>(gitems.size(), 1));
        for (int k = 0; k < 3; ++k) {
            o->PA[k] = c.take<uint16_t>((size_t)std::max<int64_t>(class_rows[k], 1) * KD[k]);
            o->PB[k] = c.take<uint16_t>((size_t)std::max<int64_t>(class_rows[k], 1) * KD[k]);
        }
        // high parts, then the split form's low parts
        o->V16 = c.take<uint16_t>((size_t)2 * R_pad * (size_t)std::max<int64_t>(v_cols, 1));
        o->vinv = c.take<float>((size_t)G * R_pad);
        o->colmax = c.take<unsigned>((size_t)G * R_pad);
        o->r = c.take<float>((size_t)R * N);
        o->dd = c.take<float>((size_t)R * N);
        o->Hd = c.take<float>((size_t)R * N);
        o->part = c.take<double>((size_t)R * std::max<size_t>(nch, 1));
        o->scale = c.take<double>((size_t)G * R);
        o->gamma = c.take<double>((size_t)G * R);
        o->alpha = c.take<double>((size_t)G * R);
        o->beta = c.take<double>((size_t)G * R);
        o->state = c.take<SolverState>(G);
        o->done = c.take<int>(G);
        o->cdone = c.take<int>(G);
        o->cskip = c.take<int>(G);
        o->gpart = c.take<double>((size_t)gp::bt::GSTRIDE * std::max<size_t>(gitems.size(), 1));
        o->spart = c.take<double>(std::max<size_t>(nch, 1));
        o->err = c.take<int>(1);
        o->tcg_bytes = tc_grad_bytes();
        o->tcg = o->tcg_bytes ? c.take<char>(o->tcg_bytes) : nullptr;
        return c.bytes();
    }
    // Largest tensor-core gradient workspace over the members that take that estimator.
    size_t tc_grad_bytes() const {
        size_t mx = 0;
        for (const BMember &m : mem)
            if (m.tcg) mx = std::max(mx, gp::tc_grad_workspace(m.n, m.d, R));
        return mx;
    }
};

namespace gp {
namespace bt {

int nsms() { return device_sm_count(); }

// ---------------------------------------------------------------- parameters
// Member parameters from the packed device theta [l_1..l_d, s_f, sigma] per member.
__global__ void bt_params_kernel(BMember *mem, int G, const double *theta, int *err) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    BMember &m = mem[g];
    const double *th = theta + m.to;
    bool ok = true;
    for (int k = 0; k < m.d + 2; ++k) ok = ok && isfinite(th[k]) && th[k] > 0.0;
    if (!ok) atomicExch(err, 1);
    for (int k = 0; k < m.d; ++k) m.inv_ell[k] = ok ? (float)(1.0 / th[k]) : 1.0f;
    const double sf = ok ? th[m.d] : 1.0, sg = ok ? th[m.d + 1] : 1.0;
    m.sf = (float)sf;
    m.sf2 = (float)(sf * sf);
    m.sigma = (float)sg;
    m.sigma2 = (float)(sg * sg);
    m.bound = 0u;
}

// ---------------------------------------------------------------- per-chunk vector kernels
__device__ __forceinline__ double block_sum(double s, double *red) {
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// part[c * nch + q] = sum over the rows of chunk q of A_c . B_c
__global__ void bt_dot_kernel(const BMember *mem, const BChunk *chunks, int nch, const float *A, const float *B,
                              double *part, const int *mdone) {
    __shared__ double red[32];
    const int c = blockIdx.y;
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const BChunk k = chunks[q];
        if (mdone && mdone[k.member]) continue;
        const BMember &m = mem[k.member];
        const int64_t base = m.vo + (int64_t)c * m.n;
        // a thread's few products of the chunk summed in FP32 (FMA), one FP64 addition per
        // chunk and thread: FP64 is slow on this GPU
        float sf = 0.0f;
        for (int r = threadIdx.x; r < kBatchChunk; r += blockDim.x) {
            const int64_t i = (int64_t)k.start + r;
            if (i >= m.n) break;
            sf = fmaf(A[base + i], B[base + i], sf);
        }
        double s = (double)sf;
        s = block_sum(s, red);
        if (threadIdx.x == 0) part[(int64_t)c * nch + q] = s;
    }
}

__device__ __forceinline__ double member_sum(const double *part, int nch, int c, const BMember &m) {
    double s = 0.0;
    for (int q = m.ch0; q < m.ch0 + m.nch; ++q) s += part[(int64_t)c * nch + q];
    return s;
}
// The same sum by a whole warp (lane l adds chunks l, l + 32, ... in order, then a fixed
// butterfly): one round of loads instead of one per chunk.
__device__ __forceinline__ double member_sum_warp(const double *part, int nch, int c, const BMember &m) {
    double s = 0.0;
    for (int q = m.ch0 + (int)(threadIdx.x & 31); q < m.ch0 + m.nch; q += 32) s += part[(int64_t)c * nch + q];
    return warp_sum(s);
}

// scale[g][c] = ||b_gc|| + eps  (App. B normalisation)
__global__ void bt_norm_scale_kernel(const BMember *mem, int G, int R, int nch, const double *part, double *scale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= G * R) return;
    const int g = e / R, c = e - g * R;
    scale[e] = sqrt(member_sum(part, nch, c, mem[g])) + kNormEps;
}

// V_gc *= (inv ? 1 / scale : scale)
__global__ void bt_scale_cols_kernel(const BMember *mem, const BChunk *chunks, int nch, float *V, int R,
                                     const double *scale, int inv) {
    const int c = blockIdx.y;
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const BChunk k = chunks[q];
        const BMember &m = mem[k.member];
        const ColFactor f = block_factor(scale + (int64_t)k.member * R, c, inv);
        float *v = V + m.vo + (int64_t)c * m.n;
        for (int r = threadIdx.x; r < kBatchChunk; r += blockDim.x) {
            const int64_t i = (int64_t)k.start + r;
            if (i >= m.n) break;
            v[i] = fmaf(v[i], f.h, v[i] * f.l);
        }
    }
}

// r = b / scale - H v ; d = r
__global__ void bt_init_residual_kernel(const BMember *mem, const BChunk *chunks, int nch, const float *B,
                                        const float *HV, float *r, float *d, int R, const double *scale) {
    const int c = blockIdx.y;
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const BChunk k = chunks[q];
        const BMember &m = mem[k.member];
        const ColFactor f = block_factor(scale + (int64_t)k.member * R, c, 1);
        const int64_t base = m.vo + (int64_t)c * m.n;
        for (int rr = threadIdx.x; rr < kBatchChunk; rr += blockDim.x) {
            const int64_t i = (int64_t)k.start + rr;
            if (i >= m.n) break;
            const float v = fmaf(B[base + i], f.h, fmaf(B[base + i], f.l, -HV[base + i]));
            r[base + i] = v;
            d[base + i] = v;
        }
    }
}

// ---------------------------------------------------------------- CG (Alg. 1) per member
// one block per member: warps over the columns, lanes over the member's chunks
__global__ void bt_cg_start_kernel(const BMember *mem, int G, int R, int nch, const double *part, double *gamma,
                                   SolverState *state, int *done, int *cdone, long long max_iters, double tol,
                                   int stop_rule) {
    const int g = blockIdx.x;
    if (g >= G) return;
    __shared__ double sq[kMaxBatchR];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = w; c < R; c += nw) {
        const double v = member_sum_warp(part, nch, c, mem[g]);
        if ((threadIdx.x & 31) == 0) {
            sq[c] = v;
            gamma[(int64_t)g * R + c] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        SolverState *st = state + g;
        st->done = 0;
        st->status = GP_OK;
        st->res0 = 0.0;
        finish_norms(st, sq, R, 0, max_iters, tol, stop_rule);
        st->certified = 0;  // the initial residual came from the plain product
        done[g] = st->done;
        cdone[g] = 0;
    }
}

// one warp per (member, column)
__global__ void bt_cg_alpha_kernel(const BMember *mem, int G, int R, int nch, const double *part,
                                   const double *gamma, double *alpha, const int *done) {
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (e >= (int64_t)G * R) return;
    const int g = (int)(e / R), c = (int)(e - (int64_t)g * R);
    if (done[g]) return;
    const double dHd = member_sum_warp(part, nch, c, mem[g]);
    if ((threadIdx.x & 31) == 0) {
        const double gm = gamma[e];
        alpha[e] = (gm > kFreeze && dHd > 0.0 && isfinite(dHd)) ? gm / dHd : 0.0;
    }
}

// v += alpha d ; r -= alpha Hd ; part = ||r||^2 partial sums
__global__ void bt_cg_update_kernel(const BMember *mem, const BChunk *chunks, int nch, float *V, float *r,
                                    const float *d, const float *Hd, int R, const double *alpha, double *part,
                                    const int *done) {
    __shared__ double red[32];
    const int c = blockIdx.y;
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const BChunk k = chunks[q];
        if (done[k.member]) continue;
        const BMember &m = mem[k.member];
        const float a = (float)alpha[(int64_t)k.member * R + c];
        const int64_t base = m.vo + (int64_t)c * m.n;
        float sf = 0.0f;
        for (int rr = threadIdx.x; rr < kBatchChunk; rr += blockDim.x) {
            const int64_t i = (int64_t)k.start + rr;
            if (i >= m.n) break;
            V[base + i] += a * d[base + i];
            const float rv = r[base + i] - a * Hd[base + i];
            r[base + i] = rv;
            sf = fmaf(rv, rv, sf);
        }
        double s = (double)sf;
        s = block_sum(s, red);
        if (threadIdx.x == 0) part[(int64_t)c * nch + q] = s;
    }
}

// one block per member: warps over the columns, lanes over the member's chunks
__global__ void bt_cg_beta_kernel(const BMember *mem, int G, int R, int nch, const double *part, double *gamma,
                                  const double *alpha, double *beta, SolverState *state, int *done,
                                  long long max_iters, double tol, int stop_rule) {
    const int g = blockIdx.x;
    if (g >= G || done[g]) return;
    __shared__ double sq[kMaxBatchR];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = w; c < R; c += nw) {
        const double gn = member_sum_warp(part, nch, c, mem[g]);
        if ((threadIdx.x & 31) == 0) {
            const int64_t e = (int64_t)g * R + c;
            const bool active = alpha[e] != 0.0;
            beta[e] = active ? gn / gamma[e] : 0.0;
            if (active) gamma[e] = gn;
            sq[c] = active ? gn : gamma[e];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        SolverState *st = state + g;
        finish_norms(st, sq, R, st->iter + 1, max_iters, tol, stop_rule);
        done[g] = st->done;
    }
}

// Members a true-residual check covers: done on their recursive residual (or by the budget)
// and not yet certified.
__global__ void bt_check_flags_kernel(int G, const int *done, const int *cdone, int *cskip) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G) cskip[g] = (cdone[g] || !done[g]) ? 1 : 0;
}

// True residual r = b~ - H v of each member not flagged in skip (App. B "Linear System Solver"),
// each difference two FP32 fused multiply-adds (1 / scale as a sum of two floats), stored as r
// and as the restart direction d (used only if the member misses the tolerance and resumes);
// partial sums of ||r||^2 with four FP32 squares per FP64 addition.
__global__ void bt_true_residual_kernel(const BMember *mem, const BChunk *chunks, int nch, const float *B,
                                        const float *HV, float *r, float *d, int R, const double *scale,
                                        double *part, const int *skip) {
    __shared__ double red[32];
    const int c = blockIdx.y;
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const BChunk k = chunks[q];
        if (skip[k.member]) continue;
        const BMember &m = mem[k.member];
        const ColFactor f = block_factor(scale + (int64_t)k.member * R, c, 1);
        const int64_t base = m.vo + (int64_t)c * m.n;
        double s = 0.0;
        float acc = 0.0f;
        int nacc = 0;
        for (int rr = threadIdx.x; rr < kBatchChunk; rr += blockDim.x) {
            const int64_t i = (int64_t)k.start + rr;
            if (i >= m.n) break;
            const float v = fmaf(B[base + i], f.h, fmaf(B[base + i], f.l, -HV[base + i]));
            r[base + i] = v;
            d[base + i] = v;
            acc = fmaf(v, v, acc);
            if (++nacc == 4) {
                s += (double)acc;
                acc = 0.0f;
                nacc = 0;
            }
        }
        s += (double)acc;
        s = block_sum(s, red);
        if (threadIdx.x == 0) part[(int64_t)c * nch + q] = s;
    }
}

// Per member not flagged in skip (one block each), after its true residual: gamma <- ||r||^2,
// the split norms and the loop condition at the current iteration count from the true norms
// (a member stopped by its recursive residual restarts from the true one when it misses the
// tolerance), marked certified; cdone set when the member is done.
__global__ void bt_true_state_kernel(const BMember *mem, int G, int R, int nch, const double *part, double *gamma,
                                     SolverState *state, int *done, int *cdone, const int *skip, long long max_iters,
                                     double tol, int stop_rule) {
    const int g = blockIdx.x;
    if (g >= G || skip[g]) return;
    __shared__ double sq[kMaxBatchR];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = w; c < R; c += nw) {
        const double v = member_sum_warp(part, nch, c, mem[g]);
        if ((threadIdx.x & 31) == 0) {
            sq[c] = v;
            gamma[(int64_t)g * R + c] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        SolverState *st = state + g;
        if (st->status == GP_OK) st->done = 0;
        finish_norms(st, sq, R, st->iter, max_iters, tol, stop_rule);
        st->certified = 1;
        done[g] = st->done;
        cdone[g] = st->done;
    }
}

// d = r + beta d
__global__ void bt_cg_dir_kernel(const BMember *mem, const BChunk *chunks, int nch, float *d, const float *r, int R,
                                 const double *beta, const int *done) {
    const int c = blockIdx.y;
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const BChunk k = chunks[q];
        if (done[k.member]) continue;
        const BMember &m = mem[k.member];
        const float b = (float)beta[(int64_t)k.member * R + c];
        const int64_t base = m.vo + (int64_t)c * m.n;
        for (int rr = threadIdx.x; rr < kBatchChunk; rr += blockDim.x) {
            const int64_t i = (int64_t)k.start + rr;
            if (i >= m.n) break;
            d[base + i] = r[base + i] + b * d[base + i];
        }
    }
}

__global__ void bt_cg_info_kernel(int G, const SolverState *state, gp_solve_info_t *info) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    info[g].iters = state[g].iter;
    info[g].converged = state[g].converged;
    info[g].status = state[g].status;
    info[g].res_y = state[g].res_y;
    info[g].res_z = state[g].res_z;
}

// ---------------------------------------------------------------- gradient (Eq. mll_grad)
// Per work item (64 rows of a member x up to GL column tiles of 64):
//   gpart[k]  = sum_ij phi_ij M_ij (a_ik - a_jk)^2   (k < d, before the 1/l_k factor)
//   gpart[d]  = sum_ij k_ij M_ij                     (before the 2/s_f factor)
// with M_ij = sum_c lam_c U_ci W_cj, U = the solutions, W = [v_y, probes] (standard,
// Eq. trace) or the solutions again (pathwise, Eq. pathwise_estimator).
// One work item with the coordinates padded to DM (4, 8, 16 or 32; zero beyond d).  Shared
// memory holds the tile's operands transposed (coordinate- and column-major: At[k][r],
// Bt[k][r], Ut[c][r], Wt[c][r]), and every thread keeps a 4 x 4 block of pairs (rows
// ty + 16p, columns tx + 16q) in registers: M by R outer-product steps, r^2 by DM steps, then
// w = phi M and the DM coordinate sums w (a_ik - a_jk)^2, so that each shared-memory value
// read feeds four FMAs.
template <int DM>
__device__ __forceinline__ void bt_grad_item(const BMember &m, const BGItem it, const float *X, const float *Vs,
                                             const float *B, int R, int pathwise, double lam0, double lamr,
                                             float *smem, double (&gacc)[kBatchMaxD], double &sacc) {
    const int d = m.d;
    float *At = smem;
    float *Bt = At + DM * GT;
    float *Ut = Bt + DM * GT;
    float *Wt = Ut + R * GT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t n = m.n;
    const float *Xm = X + m.xo;
    const float *Vm = Vs + m.vo;
    const float *Wm = pathwise ? Vm : B + m.vo;
    const int64_t row0 = (int64_t)it.row_tile * GT;
    const float sf2 = m.sf2;
    const int kind = m.kind;
    for (int e = tid; e < GT * DM; e += 256) {
        const int k = e / GT, r = e - k * GT;
        const int64_t i = row0 + r;
        At[e] = (i < n && k < d) ? Xm[i * d + k] * m.inv_ell[k] : 0.0f;
    }
    for (int e = tid; e < GT * R; e += 256) {
        const int c = e / GT, r = e - c * GT;
        const int64_t i = row0 + r;
        Ut[e] = i < n ? Vm[(int64_t)c * n + i] * (float)(c == 0 ? lam0 : lamr) : 0.0f;
    }
    bool rin[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) rin[p] = row0 + ty + 16 * p < n;
    for (int jt = it.ct0; jt < it.ct1; ++jt) {
        const int64_t col0 = (int64_t)jt * GT;
        __syncthreads();
        for (int e = tid; e < GT * DM; e += 256) {
            const int k = e / GT, r = e - k * GT;
            const int64_t j = col0 + r;
            Bt[e] = (j < n && k < d) ? Xm[j * d + k] * m.inv_ell[k] : 0.0f;
        }
        for (int e = tid; e < GT * R; e += 256) {
            const int c = e / GT, r = e - c * GT;
            const int64_t j = col0 + r;
            // W = [v_y, w_1..]: column 0 is always the y-solution
            Wt[e] = j < n ? (c == 0 ? Vm[j] : Wm[(int64_t)c * n + j]) : 0.0f;
        }
        __syncthreads();
        float M[4][4], r2[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) M[p][q] = r2[p][q] = 0.0f;
#pragma unroll 4
        for (int c = 0; c < R; ++c) {
            float u[4], w[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) u[p] = Ut[c * GT + ty + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q) w[q] = Wt[c * GT + tx + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) M[p][q] = fmaf(u[p], w[q], M[p][q]);
        }
#pragma unroll 4
        for (int k = 0; k < DM; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) a[p] = At[k * GT + ty + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bt[k * GT + tx + 16 * q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float t = a[p] - b[q];
                    r2[p][q] = fmaf(t, t, r2[p][q]);
                }
        }
        float sl = 0.0f;
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float kv;
                const float phi = kphi(kind, sf2, r2[p][q], &kv);
                const bool in = rin[p] && (col0 + tx + 16 * q < n);
                const float mm = in ? M[p][q] : 0.0f;
                sl = fmaf(kv, mm, sl);
                M[p][q] = phi * mm;  // w_ij, reusing M
            }
        sacc += (double)sl;
#pragma unroll 2
        for (int k = 0; k < DM; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) a[p] = At[k * GT + ty + 16 * p];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bt[k * GT + tx + 16 * q];
            float g = 0.0f;
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float t = a[p] - b[q];
                    g = fmaf(M[p][q] * t, t, g);
                }
            gacc[k] += (double)g;
        }
    }
}

// Per work item (64 rows of a member x up to GL column tiles of 64):
//   gpart[k]  = sum_ij phi_ij M_ij (a_ik - a_jk)^2   (k < d, before the 1/l_k factor)
//   gpart[d]  = sum_ij k_ij M_ij                     (before the 2/s_f factor)
// with M_ij = sum_c lam_c U_ci W_cj, U = the solutions, W = [v_y, probes] (standard,
// Eq. trace) or the solutions again (pathwise, Eq. pathwise_estimator).
__global__ void __launch_bounds__(256) bt_grad_kernel(const BMember *mem, const BGItem *gitems, int ngi,
                                                      const float *X, const float *Vs, const float *B, int R,
                                                      int pathwise, double lam0, double lamr, double *gpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gi = blockIdx.x;
    if (gi >= ngi) return;
    const BGItem it = gitems[gi];
    const BMember &m = mem[it.member];
    const int d = m.d;
    float *smem = reinterpret_cast<float *>(smem_raw);
    double gacc[kBatchMaxD];
#pragma unroll
    for (int k = 0; k < kBatchMaxD; ++k) gacc[k] = 0.0;
    double sacc = 0.0;
    if (d <= 4)
        bt_grad_item<4>(m, it, X, Vs, B, R, pathwise, lam0, lamr, smem, gacc, sacc);
    else if (d <= 8)
        bt_grad_item<8>(m, it, X, Vs, B, R, pathwise, lam0, lamr, smem, gacc, sacc);
    else if (d <= 16)
        bt_grad_item<16>(m, it, X, Vs, B, R, pathwise, lam0, lamr, smem, gacc, sacc);
    else
        bt_grad_item<32>(m, it, X, Vs, B, R, pathwise, lam0, lamr, smem, gacc, sacc);
    // block reduction in a fixed order
    __shared__ double red[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double *out = gpart + (int64_t)gi * GSTRIDE;
    for (int k = 0; k <= d; ++k) {
        double v = (k < d) ? 0.0 : sacc;
#pragma unroll
        for (int kk = 0; kk < kBatchMaxD; ++kk)
            if (kk == k && k < d) v = gacc[kk];
        v = warp_sum(v);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += red[w];
            out[k] = s;
        }
    }
}

// spart[q] = sum over the rows of chunk q of sum_c lam_c U_c W_c   (the sigma term)
__global__ void bt_sigma_dot_kernel(const BMember *mem, const BChunk *chunks, int nch, const float *Vs,
                                    const float *B, int R, int pathwise, double lam0, double lamr, double *spart) {
    __shared__ double red[32];
    for (int q = blockIdx.x; q < nch; q += gridDim.x) {
        const BChunk k = chunks[q];
        const BMember &m = mem[k.member];
        if (m.tcg) continue;  // block-uniform
        const float *Vm = Vs + m.vo;
        const float *Wm = pathwise ? Vm : B + m.vo;
        double s = 0.0;
        for (int rr = threadIdx.x; rr < kBatchChunk; rr += blockDim.x) {
            const int64_t i = (int64_t)k.start + rr;
            if (i >= m.n) break;
            double t = lam0 * (double)Vm[i] * (double)Vm[i];
            double u = 0.0;
            for (int c = 1; c < R; ++c) u += (double)Vm[(int64_t)c * m.n + i] * (double)Wm[(int64_t)c * m.n + i];
            s += t + lamr * u;
        }
        s = block_sum(s, red);
        if (threadIdx.x == 0) spart[q] = s;
    }
}

// grad[to + k] = sum_items gpart[k] / l_k ; grad[to + d] = 2/s_f sum gpart[d] ;
// grad[to + d + 1] = 2 sigma sum spart  (one block per member, fixed order)
__global__ void bt_grad_finalize_kernel(const BMember *mem, const double *gpart, const double *spart,
                                        const double *theta, double *grad) {
    const BMember &m = mem[blockIdx.x];
    if (m.tcg) return;  // written by the tensor-core estimator
    const int k = threadIdx.x;
    if (k > m.d + 1) return;
    double s = 0.0;
    if (k <= m.d) {
        for (int q = m.gi0; q < m.gi0 + m.ngi; ++q) s += gpart[(int64_t)q * GSTRIDE + k];
    } else {
        for (int q = m.ch0; q < m.ch0 + m.nch; ++q) s += spart[q];
    }
    const double *th = theta + m.to;
    double g;
    if (k < m.d) g = s / th[k];
    else if (k == m.d) g = 2.0 * s / th[m.d];
    else g = 2.0 * th[m.d + 1] * s;
    grad[m.to + k] = g;
}

// ---------------------------------------------------------------- Adam on softplus parameters
__global__ void bt_adam_init_kernel(int64_t P, const double *theta, double *nu, double *m, double *v,
                                    long long *t) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
        const double th = theta[e];
        nu[e] = th > 30.0 ? th : log(expm1(th));  // softplus^-1
        m[e] = 0.0;
        v[e] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *t = 0;
}

// Ascent step on nu with theta = softplus(nu) (chain rule: d theta / d nu = sigmoid(nu)).
__global__ void bt_adam_kernel(int64_t P, double *nu, double *m, double *v, const long long *t, const double *grad,
                               double lr, double b1, double b2, double eps, double *theta) {
    const double step = (double)(*t + 1);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
        const double sig = 1.0 / (1.0 + exp(-nu[e]));
        const double g = grad[e] * sig;
        m[e] = b1 * m[e] + (1.0 - b1) * g;
        v[e] = b2 * v[e] + (1.0 - b2) * g * g;
        const double mh = m[e] / (1.0 - pow(b1, step));
        const double vh = v[e] / (1.0 - pow(b2, step));
        nu[e] += lr * mh / (sqrt(vh) + eps);
        theta[e] = nu[e] > 30.0 ? nu[e] : log1p(exp(nu[e]));
    }
}

__global__ void bt_tick_kernel(long long *t) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *t += 1;
}

// ---------------------------------------------------------------- host helpers
int require_bound(const gp_batch *b) {
    if (!b) {
        set_error("batch is null");
        return GP_ERR_INVALID_ARG;
    }
    if (!b->bound) {
        set_error("gp_batch_bind() has not been called");
        return GP_ERR_INVALID_ARG;
    }
    return GP_OK;
}

dim3 chunk_grid(const gp_batch *b, int cols) {
    const int nch = (int)b->chunks.size();
    return dim3((unsigned)std::max(1, std::min(nch, 4 * nsms())), (unsigned)cols);
}

size_t grad_smem(int R) { return sizeof(float) * (size_t)(2 * GT * kBatchMaxD + 2 * GT * R); }

// Y = H V (diag = 1) or K V (diag = 0) for every member not flagged in mdone; split: the split
// tensor-core products (FP32-class, for true residuals).
int batch_apply(gp_batch *b, const float *V, float *Y, float diag, const int *mdone, cudaStream_t st,
                bool split = false) {
    auto &p = b->p;
    const int nch = (int)b->chunks.size();
    // batches of more than 80 right-hand sides per member take the plain form for true
    // residuals too (the split form's accumulators hold 80 columns)
    split = split && tc_split_fits_rpad(b->R_pad);
    GP_TRY(tc_group_convert(p.mem, b->G, p.chunks, nch, V, b->R, b->R_pad, p.colmax, p.V16, b->v_cols, p.vinv,
                            mdone, st, split));
    for (int k = 0; k < 3; ++k) {
        if (b->items[k].empty()) continue;
        TcGroupArgs a{};
        a.kind = b->kind;
        a.KD = b->KD[k];
        a.R = b->R;
        a.R_pad = b->R_pad;
        a.PA = p.PA[k];
        a.PB = p.PB[k];
        a.class_rows = b->class_rows[k];
        a.V16 = p.V16;
        a.v_cols = b->v_cols;
        a.vinv = p.vinv;
        a.items = p.items[k];
        a.nitems = (int)b->items[k].size();
        a.members = p.mem;
        a.mdone = mdone;
        a.Y = Y;
        a.Vd = V;
        a.diag = diag;
        a.err = p.err;
        a.split = split ? 1 : 0;
        GP_TRY(tc_group_mvm(a, st));
    }
    return GP_OK;
}

int batch_prepare(gp_batch *b, const double *theta, const float *X, cudaStream_t st) {
    auto &p = b->p;
    bt_params_kernel<<<(unsigned)cdiv(b->G, 128), 128, 0, st>>>(p.mem, b->G, theta, p.err);
    GP_TRY(check_launch("bt_params_kernel"));
    return tc_group_prepare(b->kind, p.mem, b->G, p.chunks, (int)b->chunks.size(), X, p.PA, p.PB, b->KD, st);
}

constexpr int64_t kCheckEvery = 10;  // iterations between the batched solver's true-residual checks

int batch_cg(gp_batch *b, const float *B, float *V, int64_t iters, double tol, int stop_rule,
             gp_solve_info_t *info, cudaStream_t st) {
    auto &p = b->p;
    const int G = b->G, R = b->R, nch = (int)b->chunks.size();
    const dim3 gc = chunk_grid(b, R);
    const unsigned gmr = (unsigned)cdiv((int64_t)G * R, 128), gmw = (unsigned)cdiv((int64_t)G * R * 32, 256);
    // normalisation (App. B): scale = ||b|| + eps per member and column, v <- v / scale
    bt_dot_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, B, B, p.part, nullptr);
    bt_norm_scale_kernel<<<gmr, 128, 0, st>>>(p.mem, G, R, nch, p.part, p.scale);
    bt_scale_cols_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, V, R, p.scale, 1);
    GP_TRY(check_launch("batched cg setup", 3));
    // r = b~ - H v ; d = r ; gamma = r^T r  (the plain product; the checks catch its error)
    GP_TRY(batch_apply(b, V, p.Hd, 1.0f, nullptr, st));
    bt_init_residual_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, B, p.Hd, p.r, p.dd, R, p.scale);
    bt_dot_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, p.r, p.r, p.part, nullptr);
    bt_cg_start_kernel<<<(unsigned)G, 256, 0, st>>>(p.mem, G, R, nch, p.part, p.gamma, p.state, p.done, p.cdone,
                                                    (long long)iters, tol, stop_rule);
    GP_TRY(check_launch("batched cg start", 3));
    // True residual b~ - H v of the members that stopped on their recursive residual and are
    // not yet certified: every kCheckEvery iterations (a member whose true residual misses the
    // tolerance restarts from it) and after the last iteration (the reported norms and flags).
    // Members still iterating keep their recursive residual: replacing it mid-solve with a
    // product of the whole iterate injects that product's rounding into the recurrence.
    auto true_residuals = [&]() -> int {
        bt_check_flags_kernel<<<(unsigned)cdiv(G, 128), 128, 0, st>>>(G, p.done, p.cdone, p.cskip);
        GP_TRY(batch_apply(b, V, p.Hd, 1.0f, p.cskip, st, true));
        bt_true_residual_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, B, p.Hd, p.r, p.dd, R, p.scale, p.part,
                                                    p.cskip);
        bt_true_state_kernel<<<(unsigned)G, 256, 0, st>>>(p.mem, G, R, nch, p.part, p.gamma, p.state, p.done, p.cdone,
                                                          p.cskip, (long long)iters, tol, stop_rule);
        return check_launch("batched cg true residual", 3);
    };
    for (int64_t it = 0; it < iters; ++it) {
        GP_TRY(batch_apply(b, p.dd, p.Hd, 1.0f, p.done, st));
        bt_dot_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, p.dd, p.Hd, p.part, p.done);
        bt_cg_alpha_kernel<<<gmw, 256, 0, st>>>(p.mem, G, R, nch, p.part, p.gamma, p.alpha, p.done);
        bt_cg_update_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, V, p.r, p.dd, p.Hd, R, p.alpha, p.part,
                                                p.done);
        bt_cg_beta_kernel<<<(unsigned)G, 256, 0, st>>>(p.mem, G, R, nch, p.part, p.gamma, p.alpha, p.beta, p.state, p.done,
                                             (long long)iters, tol, stop_rule);
        bt_cg_dir_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, p.dd, p.r, R, p.beta, p.done);
        GP_TRY(check_launch("batched cg iteration", 5));
        if ((it + 1) % kCheckEvery == 0 && it + 1 < iters) GP_TRY(true_residuals());
    }
    GP_TRY(true_residuals());
    bt_scale_cols_kernel<<<gc, 256, 0, st>>>(p.mem, p.chunks, nch, V, R, p.scale, 0);
    GP_TRY(check_launch("batched cg rescale"));
    if (info) {
        bt_cg_info_kernel<<<(unsigned)cdiv(G, 128), 128, 0, st>>>(G, p.state, info);
        GP_TRY(check_launch("bt_cg_info_kernel"));
    }
    return GP_OK;
}

int batch_grad(gp_batch *b, const double *theta, const float *X, const float *Vs, const float *B, int pathwise,
               double *grad, cudaStream_t st) {
    auto &p = b->p;
    const int ngi = (int)b->gitems.size(), nch = (int)b->chunks.size();
    const double lam0 = 0.5, lamr = -0.5 / (double)b->s;
    // Members with tcg set: the fused tensor-core estimator member by member (stream-ordered,
    // one workspace), with the hyperparameters read from the device (set from theta by the
    // preparation): no host copy of theta, so the step stays one CUDA graph.  The others: the
    // CUDA-core kernels below, which skip the tcg members.
    if (p.tcg) {
        for (int g = 0; g < b->G; ++g) {
            const BMember &hm = b->mem[g];
            if (!hm.tcg) continue;
            GradArgs<float> a{};
            a.kp.kind = b->kind;
            a.kp.d = hm.d;
            for (int k = 0; k < hm.d; ++k) a.kp.inv_ell[k] = a.kp.ell[k] = 1.0f;  // replaced on the device
            a.kp.sf = a.kp.sf2 = a.kp.sigma = a.kp.sigma2 = 1.0f;
            a.X = X + hm.xo;
            a.n = hm.n;
            a.U0 = Vs + hm.vo;
            a.U = Vs + hm.vo + hm.n;
            a.ldu = hm.n;
            a.W0 = Vs + hm.vo;  // column 0 is always the y-solution
            a.W = pathwise ? Vs + hm.vo + hm.n : B + hm.vo + hm.n;
            a.ldw = hm.n;
            a.R = b->R;
            a.lam0 = lam0;
            a.lam_rest = lamr;
            a.grad = grad + hm.to;
            a.dev_inv_ell = p.mem[g].inv_ell;
            a.dev_sf2 = &p.mem[g].sf2;
            a.dev_theta = theta + hm.to;
            GP_TRY(tc_grad(a, p.tcg, p.tcg_bytes, st));
        }
    }
    if (ngi == 0) return GP_OK;
    bt_grad_kernel<<<(unsigned)ngi, 256, grad_smem(b->R), st>>>(p.mem, p.gitems, ngi, X, Vs, B, b->R, pathwise,
                                                                lam0, lamr, p.gpart);
    bt_sigma_dot_kernel<<<chunk_grid(b, 1), 256, 0, st>>>(p.mem, p.chunks, nch, Vs, B, b->R, pathwise, lam0, lamr,
                                                          p.spart);
    bt_grad_finalize_kernel<<<(unsigned)b->G, 64, 0, st>>>(p.mem, p.gpart, p.spart, theta, grad);
    return check_launch("batched gradient", 3);
}

int batch_adam(gp_batch *b, double *nu, double *m, double *v, long long *t, const double *grad, double lr,
               double b1, double b2, double eps, double *theta, cudaStream_t st) {
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(b->theta_len, 256), 256));
    bt_adam_kernel<<<nb, 256, 0, st>>>(b->theta_len, nu, m, v, t, grad, lr, b1, b2, eps, theta);
    bt_tick_kernel<<<1, 32, 0, st>>>(t);
    return check_launch("batched adam", 2);
}

}  // namespace bt
}  // namespace gp

using namespace gp::bt;

#define BT_BEGIN   \
    clear_error(); \
    try {
#define BT_END                                      \
    }                                               \
    catch (const std::exception &ex) {              \
        set_error("internal error: %s", ex.what()); \
        return GP_ERR_CUDA;                         \
    }
#define BT_REQ(cond, ...)              \
    do {                               \
        if (!(cond)) {                 \
            set_error(__VA_ARGS__);    \
            return GP_ERR_INVALID_ARG; \
        }                              \
    } while (0)

extern "C" {

int gp_batch_create(int kind, int G, const int64_t *n, const int *d, int s, gp_batch_t **out) {
    BT_BEGIN
    BT_REQ(out != nullptr, "out is null");
    *out = nullptr;
    BT_REQ(kind == GP_RBF || kind == GP_MATERN32, "kind must be GP_RBF or GP_MATERN32");
    BT_REQ(G >= 1, "need at least one member");
    BT_REQ(n != nullptr && d != nullptr, "n and d must not be null");
    BT_REQ(s >= 1 && s + 1 <= kMaxBatchR, "s must be in [1, %d]", kMaxBatchR - 1);
    for (int g = 0; g < G; ++g) {
        BT_REQ(n[g] >= 1 && n[g] <= (int64_t)1 << 30, "member %d: n = %lld out of range", g, (long long)n[g]);
        BT_REQ(d[g] >= 1 && d[g] <= kBatchMaxD, "member %d: d = %d must be in [1, %d]", g, d[g], kBatchMaxD);
    }
    gp_batch *b = new (std::nothrow) gp_batch();
    if (!b) {
        set_error("out of host memory");
        return GP_ERR_CUDA;
    }
    b->kind = kind;
    b->G = G;
    b->s = s;
    b->R = s + 1;
    b->R_pad = (int)rup(b->R, 16);
    b->mem.resize(G);
    int64_t xo = 0, nacc = 0, to = 0;
    for (int g = 0; g < G; ++g) {
        BMember &m = b->mem[g];
        std::memset(&m, 0, sizeof m);
        m.n = n[g];
        m.d = d[g];
        m.kind = kind;
        m.xo = xo;
        m.vo = (int64_t)b->R * nacc;
        m.to = to;
        xo += n[g] * d[g];
        nacc += n[g];
        to += d[g] + 2;
        const int64_t n_pad = rup(n[g], 128);
        m.cb = b->v_cols;
        b->v_cols += n_pad;
        m.cls = (int)(rup(3 * d[g] + 4, 64) / 64) - 1;
        m.rb = b->class_rows[m.cls];
        b->class_rows[m.cls] += n_pad;
        m.ch0 = (int)b->chunks.size();
        for (int64_t st0 = 0; st0 < n_pad; st0 += kBatchChunk) b->chunks.push_back(BChunk{g, (int)st0});
        m.nch = (int)b->chunks.size() - m.ch0;
        const int tiles = (int)(n_pad / 128);
        for (int rt = 0; rt < tiles; ++rt)
            b->items[m.cls].push_back(
                BItem{(int)(m.rb / 128) + rt, (int)(m.rb / 128), (int)(m.cb / 128), tiles, g, 0, 0, 0});
        m.tcg = (n[g] >= kTcGradMinN && tc_available() && tc_grad_fits(n[g], d[g], b->R)) ? 1 : 0;
        m.gi0 = (int)b->gitems.size();
        const int gt = (int)cdiv(n[g], GT);
        if (!m.tcg)
            for (int rt = 0; rt < gt; ++rt)
                for (int c0 = 0; c0 < gt; c0 += GL) b->gitems.push_back(BGItem{g, rt, c0, std::min(gt, c0 + GL)});
        m.ngi = (int)b->gitems.size() - m.gi0;
    }
    b->N = nacc;
    b->x_len = xo;
    b->theta_len = to;
    for (int k = 0; k < 3; ++k)
        std::stable_sort(b->items[k].begin(), b->items[k].end(),
                         [](const BItem &a, const BItem &c) { return a.ntiles > c.ntiles; });
    *out = b;
    return GP_OK;
    BT_END
}

void gp_batch_destroy(gp_batch_t *b) { delete b; }

size_t gp_batch_workspace(const gp_batch_t *b) {
    if (!b) return 0;
    gp_batch::Ptrs tmp{};
    return b->carve(nullptr, &tmp);
}

int gp_batch_layout(const gp_batch_t *b, int64_t *x_len, int64_t *vec_len, int64_t *theta_len) {
    BT_BEGIN
    BT_REQ(b != nullptr, "batch is null");
    if (x_len) *x_len = b->x_len;
    if (vec_len) *vec_len = (int64_t)b->R * b->N;
    if (theta_len) *theta_len = b->theta_len;
    return GP_OK;
    BT_END
}

int gp_batch_member_offsets(const gp_batch_t *b, int64_t *x_off, int64_t *vec_off, int64_t *theta_off) {
    BT_BEGIN
    BT_REQ(b != nullptr, "batch is null");
    for (int g = 0; g < b->G; ++g) {
        if (x_off) x_off[g] = b->mem[g].xo;
        if (vec_off) vec_off[g] = b->mem[g].vo;
        if (theta_off) theta_off[g] = b->mem[g].to;
    }
    return GP_OK;
    BT_END
}

int gp_batch_bind(gp_batch_t *b, void *ws, size_t ws_bytes, cudaStream_t stream) {
    BT_BEGIN
    BT_REQ(b != nullptr, "batch is null");
    if (!tc_available()) {
        set_error("batched GPs need an sm_103 device with tcgen05");
        return GP_ERR_UNSUPPORTED;
    }
    gp_batch::Ptrs p{};
    const size_t need = b->carve(ws, &p);
    GP_TRY(check_ws(ws, ws_bytes, need));
    GP_TRY(tc_group_setup());
    GP_TRY(ensure_max_dyn_smem((const void *)bt_grad_kernel));
    if (grad_smem(b->R) > (size_t)kMaxDynSmem) {
        set_error("too many right-hand sides for the batched gradient tile");
        return GP_ERR_UNSUPPORTED;
    }
    GP_TRY_CUDA(cudaMemcpyAsync(p.mem, b->mem.data(), sizeof(BMember) * b->mem.size(), cudaMemcpyHostToDevice,
                                stream));
    GP_TRY_CUDA(cudaMemcpyAsync(p.chunks, b->chunks.data(), sizeof(BChunk) * b->chunks.size(),
                                cudaMemcpyHostToDevice, stream));
    for (int k = 0; k < 3; ++k)
        if (!b->items[k].empty())
            GP_TRY_CUDA(cudaMemcpyAsync(p.items[k], b->items[k].data(), sizeof(BItem) * b->items[k].size(),
                                        cudaMemcpyHostToDevice, stream));
    GP_TRY_CUDA(cudaMemcpyAsync(p.gitems, b->gitems.data(), sizeof(BGItem) * b->gitems.size(),
                                cudaMemcpyHostToDevice, stream));
    GP_TRY_CUDA(cudaMemsetAsync(p.done, 0, sizeof(int) * b->G, stream));
    GP_TRY_CUDA(cudaMemsetAsync(p.err, 0, sizeof(int), stream));
    GP_TRY_CUDA(cudaStreamSynchronize(stream));
    b->p = p;
    b->ws = ws;
    b->bound = true;
    return GP_OK;
    BT_END
}

int gp_batch_status(const gp_batch_t *b, cudaStream_t stream) {
    BT_BEGIN
    GP_TRY(require_bound(b));
    int h = 0;
    GP_TRY_CUDA(cudaMemcpyAsync(&h, b->p.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    GP_TRY_CUDA(cudaStreamSynchronize(stream));
    if (h) {
        set_error("a device check failed (non-positive or non-finite theta, or a timed-out wait)");
        return GP_ERR_INVALID_ARG;
    }
    return GP_OK;
    BT_END
}

int gp_batch_prepare(gp_batch_t *b, const double *theta, const float *X, cudaStream_t stream) {
    BT_BEGIN
    GP_TRY(require_bound(b));
    BT_REQ(theta && X, "null pointer argument");
    return batch_prepare(b, theta, X, stream);
    BT_END
}

int gp_batch_mvm(gp_batch_t *b, const float *V, float *Y, int add_noise, cudaStream_t stream) {
    BT_BEGIN
    GP_TRY(require_bound(b));
    BT_REQ(V && Y && V != Y, "V and Y must be distinct and not null");
    return batch_apply(b, V, Y, add_noise ? 1.0f : 0.0f, nullptr, stream);
    BT_END
}

int gp_batch_solve_cg(gp_batch_t *b, const float *B, float *V_inout, int64_t iters, double tol, int stop_rule,
                      gp_solve_info_t *info, cudaStream_t stream) {
    BT_BEGIN
    GP_TRY(require_bound(b));
    BT_REQ(B && V_inout, "null pointer argument");
    BT_REQ(iters >= 0, "iters must be >= 0");
    BT_REQ(tol >= 0.0 && std::isfinite(tol), "tol must be finite and >= 0");
    BT_REQ(stop_rule == GP_STOP_BOTH || stop_rule == GP_STOP_EITHER, "bad stop_rule");
    return batch_cg(b, B, V_inout, iters, tol, stop_rule, info, stream);
    BT_END
}

int gp_batch_mll_grad(gp_batch_t *b, const double *theta, const float *X, const float *Vsol, const float *B,
                      int pathwise, double *grad, cudaStream_t stream) {
    BT_BEGIN
    GP_TRY(require_bound(b));
    BT_REQ(theta && X && Vsol && grad && (pathwise || B), "null pointer argument");
    return batch_grad(b, theta, X, Vsol, B, pathwise ? 1 : 0, grad, stream);
    BT_END
}

int gp_batch_adam_init(gp_batch_t *b, const double *theta, double *nu, double *m, double *v, long long *t,
                       cudaStream_t stream) {
    BT_BEGIN
    BT_REQ(b && theta && nu && m && v && t, "null pointer argument");
    bt_adam_init_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(b->theta_len, 256), 256)), 256, 0,
                          stream>>>(b->theta_len, theta, nu, m, v, t);
    return check_launch("bt_adam_init_kernel");
    BT_END
}

int gp_batch_adam_step(gp_batch_t *b, double *nu, double *m, double *v, long long *t, const double *grad,
                       double lr, double beta1, double beta2, double eps, double *theta, cudaStream_t stream) {
    BT_BEGIN
    BT_REQ(b && nu && m && v && t && grad && theta, "null pointer argument");
    BT_REQ(lr > 0 && beta1 >= 0 && beta1 < 1 && beta2 >= 0 && beta2 < 1 && eps > 0, "bad Adam settings");
    return batch_adam(b, nu, m, v, t, grad, lr, beta1, beta2, eps, theta, stream);
    BT_END
}

int gp_batch_step(gp_batch_t *b, const float *X, double *theta, const float *B, float *V_inout, int64_t iters,
                  double tol, double *grad, double *nu, double *m, double *v, long long *t, double lr,
                  gp_solve_info_t *info, cudaStream_t stream) {
    BT_BEGIN
    GP_TRY(require_bound(b));
    BT_REQ(X && theta && B && V_inout && grad && nu && m && v && t, "null pointer argument");
    BT_REQ(iters >= 0 && tol >= 0.0 && std::isfinite(tol) && lr > 0.0, "bad iters, tol or lr");
    GP_TRY(batch_prepare(b, theta, X, stream));
    GP_TRY(batch_cg(b, B, V_inout, iters, tol, GP_STOP_BOTH, info, stream));
    GP_TRY(batch_grad(b, theta, X, V_inout, B, 0, grad, stream));
    return batch_adam(b, nu, m, v, t, grad, lr, 0.9, 0.999, 1e-8, theta, stream);
    BT_END
}

}  // extern "C"
