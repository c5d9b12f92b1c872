// Internal declarations shared by the translation units of libgp_gb300.so.
// Nothing here is part of the C ABI (include/gp.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <cmath>

#include "gp.h"

namespace gp {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();

#define GP_TRY_CUDA(call)                                                              \
    do {                                                                               \
        cudaError_t gp_e_ = (call);                                                    \
        if (gp_e_ != cudaSuccess) {                                                    \
            ::gp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(gp_e_), \
                            __FILE__, __LINE__);                                       \
            return GP_ERR_CUDA;                                                        \
        }                                                                              \
    } while (0)

#define GP_TRY(...)                   \
    do {                              \
        int gp_s_ = (__VA_ARGS__);    \
        if (gp_s_ != GP_OK)           \
            return gp_s_;             \
    } while (0)

// Checks the launch(es) just enqueued and counts them for gp_diag_launches().
int check_launch(const char *what, int count = 1);

// Optional CUDA-event timing of the kernel-matrix product kernels
// (gp_diag_reset(1) turns it on): events recorded on the launch stream around
// each product kernel.
// tag 0: kernel-matrix product kernels, tag 1: gradient-estimator kernels.
void prof_begin(cudaStream_t st, int tag = 0);
void prof_end(cudaStream_t st);

// Dynamic shared memory a kernel may opt into (227 KB per block on sm_103,
// minus headroom for the kernels' small static arrays).
constexpr int kMaxDynSmem = 220 * 1024;

// Per-device one-time set-up, safe to call from several host threads.  A kernel attribute
// applies to the device that is current when it is set, so the first launch of `kernel` on
// each device raises its dynamic shared-memory limit to kMaxDynSmem there.
int ensure_max_dyn_smem(const void *kernel);
// Streaming multiprocessors of the current device (queried once per device).
int device_sm_count();

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t rup(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// ---------------------------------------------------------------------------
// Kernel hyperparameters, pre-digested on the host (theta is a host array)
// ---------------------------------------------------------------------------
template <typename T>
struct KP {
    int kind;  // GP_RBF / GP_MATERN32
    int d;
    T inv_ell[GP_MAX_D];
    T ell[GP_MAX_D];
    T sf;      // signal amplitude s_f
    T sf2;     // s_f^2
    T sigma;   // noise std
    T sigma2;  // sigma^2
};

// Validates theta (finite, positive) and fills kp.  Returns GP_OK or
// GP_ERR_INVALID_ARG with the message set.
template <typename T>
int make_kp(int kind, const double *theta, int d, KP<T> *kp);

// ---------------------------------------------------------------------------
// Workspace carving: every buffer 256-byte aligned, sizes computed by the same
// code path that carves them (dry run with base == nullptr).
// ---------------------------------------------------------------------------
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename U>
    U *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        U *p = base ? reinterpret_cast<U *>(base + off) : nullptr;
        off += count * sizeof(U);
        return p;
    }
    size_t bytes() const { return (off + 255) & ~size_t(255); }
};

int check_ws(void *ws, size_t ws_bytes, size_t need);

// ---------------------------------------------------------------------------
// Kernel function (Sec. 2; App. B): value and the radial factor of dk/dl
// ---------------------------------------------------------------------------
__device__ __forceinline__ float kval(int kind, float sf2, float r2) {
    if (kind == GP_RBF) return sf2 * expf(-0.5f * r2);
    float r = sqrtf(r2);
    const float s3 = 1.7320508075688772f;
    return sf2 * (1.0f + s3 * r) * expf(-s3 * r);
}
__device__ __forceinline__ double kval(int kind, double sf2, double r2) {
    if (kind == GP_RBF) return sf2 * exp(-0.5 * r2);
    double r = sqrt(r2);
    const double s3 = 1.7320508075688772;
    return sf2 * (1.0 + s3 * r) * exp(-s3 * r);
}
// phi(r) with dk/dl_k = phi(r) * (x_k - x'_k)^2 / l_k^3:
//   RBF: phi = k ;  Matern-3/2: phi = 3 s_f^2 exp(-sqrt3 r).
// Returns k through *kout.
__device__ __forceinline__ float kphi(int kind, float sf2, float r2, float *kout) {
    if (kind == GP_RBF) {
        float k = sf2 * expf(-0.5f * r2);
        *kout = k;
        return k;
    }
    const float s3 = 1.7320508075688772f;
    float r = sqrtf(r2);
    float e = expf(-s3 * r);
    *kout = sf2 * (1.0f + s3 * r) * e;
    return 3.0f * sf2 * e;
}
__device__ __forceinline__ double kphi(int kind, double sf2, double r2, double *kout) {
    if (kind == GP_RBF) {
        double k = sf2 * exp(-0.5 * r2);
        *kout = k;
        return k;
    }
    const double s3 = 1.7320508075688772;
    double r = sqrt(r2);
    double e = exp(-s3 * r);
    *kout = sf2 * (1.0 + s3 * r) * e;
    return 3.0 * sf2 * e;
}

// ---------------------------------------------------------------------------
// CUDA-core (SIMT) products, T = float or double
// ---------------------------------------------------------------------------
// Y[c][i] = alpha * sum_j k(x1_i, x2_j) V[c][j] + beta * Y[c][i]
//           + diag_coef * Vd[c][i - drow0]   for drow0 <= i < drow0 + ndiag
// Columns may start at a device-resident offset col0 (points X2 + col0*d,
// clipped to n2_total); the diagonal rows then start at col0 as well.
template <typename T>
struct MvmArgs {
    KP<T> kp;
    const T *X1;
    int64_t n1;
    const T *X2;
    int64_t n2;           // number of columns (before clipping)
    int64_t n2_total;     // points available in X2 when col0_dev is used
    const int64_t *col0_dev;
    const T *V;
    int64_t ldv;
    int R;
    T *Y;
    int64_t ldy;
    T alpha, beta;
    T diag_coef;          // 0 disables the diagonal term
    const T *Vd;
    int64_t ldvd;
    int64_t drow0;        // ignored when diag_from_col0
    int64_t ndiag;
    int diag_from_col0;   // 1: diagonal rows are [col0, col0 + n2_eff)
    const int *done;      // optional device flag: skip all work when *done != 0
};

template <typename T>
size_t mvm_simt_workspace(int64_t n1, int64_t n2, int R);
template <typename T>
int mvm_simt(const MvmArgs<T> &a, void *ws, size_t ws_bytes, cudaStream_t st);

// Fused estimator reduction (Eq. mll_grad with Eq. trace / Eq. pathwise_estimator):
// grad_p = sum_c lam_c U_c^T dH_p W_c.  Column 0 of U/W is U0/W0, columns
// c >= 1 are U + (c-1)*ldu, W + (c-1)*ldw.
template <typename T>
struct GradArgs {
    KP<T> kp;
    const T *X;
    int64_t n;
    const T *U0, *U;
    int64_t ldu;
    const T *W0, *W;
    int64_t ldw;
    int R;
    double lam0, lam_rest;  // lambda_0 and lambda_c for c >= 1
    double *grad;           // device, d+2
    // Optional device-resident hyperparameters (a batch member whose theta lives on the device;
    // tensor-core form only): 1/l (d floats), s_f^2, and theta = [l, s_f, sigma] (d+2 doubles).
    // When set they replace kp's inv_ell, sf2, ell, sf and sigma.
    const float *dev_inv_ell = nullptr;
    const float *dev_sf2 = nullptr;
    const double *dev_theta = nullptr;
};
// The sigma term (dH/dsigma = 2 sigma I, an O(n R) dot product) and the final
// assembly of grad from per-block partial sums (256 doubles of scratch in dpart).
template <typename T>
int grad_tail(const GradArgs<T> &a, int nblocks, const double *partial, double *dpart, cudaStream_t st);
template <typename T>
size_t grad_simt_workspace(int64_t n, int d, int R);
template <typename T>
int grad_simt(const GradArgs<T> &a, void *ws, size_t ws_bytes, cudaStream_t st);

// ---------------------------------------------------------------------------
// tcgen05 path (fp16 operands, FP32 accumulation in tensor memory)
// ---------------------------------------------------------------------------
// Prepared operands for a point set under fixed theta.
struct TcPoints {
    const void *PA;          // n_pad x KD fp16, row operand (scaled, hi/lo split, norms)
    const void *PB;          // n_pad x KD fp16, column operand
    int64_t n, n_pad;
    int KD;                  // padded contraction length of the distance GEMM
    const float *dscale;     // device scalar: power-of-two scale of the tile values
    const unsigned *bound;   // device scalar: magnitude bound the scale was chosen from
};
size_t tc_points_bytes(int64_t n, int d);
// Rows and columns from one point set (H V).
int tc_prepare_points(const KP<float> &kp, const float *X, int64_t n, void *buf, TcPoints *out,
                      cudaStream_t st);
int tc_prepare_points_dev(const KP<float> &kp, const float *X, int64_t n, void *buf, TcPoints *out,
                          const float *inv_dev, cudaStream_t st);
// Fused tensor-core estimator (d <= 32, R <= 256; tc_grad falls back to the CUDA-core form
// outside tc_grad_fits).
bool tc_grad_fits(int64_t n, int d, int R);
size_t tc_grad_workspace(int64_t n, int d, int R);
int tc_grad(const GradArgs<float> &a, void *ws, size_t ws_bytes, cudaStream_t st);
// Rows from X1 and columns from X2 with one shared scale (cross products).
int tc_prepare_pair(const KP<float> &kp, const float *X1, int64_t n1, const float *X2, int64_t n2, void *buf1,
                    void *buf2, TcPoints *rows, TcPoints *cols, cudaStream_t st);

struct TcMvmArgs {
    int kind;
    TcPoints rows, cols;
    const float *V;    // R x n2 fp32 (stride ldv)
    int64_t ldv;
    int R;
    float *Y;
    int64_t ldy;
    float sf2;
    float alpha, beta, diag_coef;
    const float *Vd;
    int64_t ldvd;
    int64_t drow0, ndiag;
    const int *done;
    // Column panels (alternating projections): the product runs over ncols columns of
    // `cols` starting at the device-resident point offset *col0_dev (V has ncols entries
    // per right-hand side); with diag_from_col0 the diagonal rows start there as well
    // (clipped to cols.n).  ncols = 0 and col0_dev = null: all columns of `cols`.
    int64_t ncols;
    const int64_t *col0_dev;
    int diag_from_col0;
    // Split form: kernel values and V as fp16 high + low parts, Y += P_hi V_hi + P_hi V_lo +
    // P_lo V_hi (about 2^-22 relative per term instead of 2^-11; three GEMM2 passes per tile).
    int split;
    // V already converted by the caller (plain form, R <= 128): tc_rhs_pad(R) rows of
    // tc_cols_pad(n2) fp16 values (zero beyond n2 and R), V scaled per column by 1 / vinv_pre[c]
    // (a power of two); V is then only read for the diagonal term.
    const void *V16pre;
    const float *vinv_pre;
    // Optional (persistent schedule, one pass): per column c and CTA b, dotpart[c * G + b] =
    // the CTA's share of dotv_c^T y_c (dotv with stride lddv); dotpart holds R x 256 doubles.
    // *dot_parts (when set) receives G, or 0 when the product did not take the sums.
    const float *dotv;
    int64_t lddv;
    double *dotpart;
    int *dot_parts;
};
int tc_rhs_pad(int R);            // right-hand sides padded for the tensor-core product
int64_t tc_cols_pad(int64_t n);   // columns padded to whole tiles
size_t tc_mvm_workspace(int64_t n1, int64_t n2, int R);
// Row operand for points X1 that are a subset of an already prepared set `like` (same
// scale): the batch rows of the stochastic-gradient panel.
int tc_prepare_rows(const KP<float> &kp, const float *X1, int64_t n1, const TcPoints &like, void *buf, TcPoints *out,
                    cudaStream_t st);
int tc_mvm(const TcMvmArgs &a, void *ws, size_t ws_bytes, cudaStream_t st);
bool tc_available();
// Device word that a tensor-core kernel sets when one of its bounded waits gives up;
// tc_timeout_status synchronises the stream, reads and clears it (GP_ERR_TIMEOUT if set);
// tc_timeout_probe launches a wait that nothing completes, bounded by `limit` cycles.
int *tc_timeout_word();
int tc_timeout_status(cudaStream_t st);
int tc_timeout_probe(long long limit, cudaStream_t st);
// Random Fourier features on the tensor cores (fp16 hi/lo split of features and weights):
// d <= 32 and s <= 128; the workspace holds the scaled frequencies and the split weights.
bool tc_rff_fits(int d, int m, int s);
// 2-D fp16 tensor map (128-byte swizzle) of an inner x outer row-major array, box_inner x
// box_outer tiles (tc.cu).
int tc_make_map16(CUtensorMap *m, const void *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                  uint32_t box_outer);
size_t tc_rff_workspace(int d, int m, int s);
int tc_rff(const KP<float> &kp, const float *X, int64_t n, int m, const float *omega_hat, const float *chi2,
           const float *W, int s, float *F, int64_t ldf, void *ws, size_t ws_bytes, cudaStream_t st);
// Split-count autotuner of the product (rows == cols): times candidates, records the best
// for the shape in a process-wide table that later products of that shape use.
size_t tc_autotune_workspace(int64_t n, int R);
int tc_autotune(const TcMvmArgs &a, int reps, void *ws, size_t ws_bytes, cudaStream_t st, int *best_split,
                double *best_ms);
void tc_autotune_reset();
int tc_autotune_grad(const GradArgs<float> &a, int reps, void *ws, size_t ws_bytes, cudaStream_t st, int64_t *best_v,
                     double *best_ms);
int tc_autotune_save(const char *path);
int tc_autotune_load(const char *path);
int64_t tc_autotune_count();

// ---------------------------------------------------------------------------
// Batches of independent GPs (batched.cu): device tables shared with tc.cu
// ---------------------------------------------------------------------------
constexpr int kBatchMaxD = 32;

// One member GP of a batch.  Points, vectors and hyperparameters are packed
// member after member; the tensor-core operands of members with the same
// contraction depth share one row space (a "class").
struct BMember {
    int64_t n;      // points
    int64_t xo;     // offset of its points in the packed X (floats)
    int64_t vo;     // offset of its vector block in packed vectors (R vectors of n)
    int64_t to;     // offset of its hyperparameters in the packed theta (d + 2 doubles)
    int64_t cb;     // first column of its points in the packed fp16 V (multiple of 128)
    int64_t rb;     // first row of its points in its class's PA/PB (multiple of 128)
    int d, cls, kind;
    int ch0, nch;   // its point chunks in the batch's chunk table
    int gi0, ngi;   // its gradient work items (CUDA-core estimator)
    int tcg;        // 1: its gradient is taken by the tensor-core estimator instead
    // set from theta on the device before every use
    float inv_ell[kBatchMaxD];
    float sf, sf2, sigma, sigma2;
    float dscale;   // power-of-two scale of the distance operands
    unsigned bound; // magnitude bound it was chosen from (float bits)
};

// Rows [start, start + kBatchChunk) of a member (clipped to its 128-padded size): the
// unit of the batch's per-point kernels (operand preparation, vector updates, dots).
constexpr int kBatchChunk = 1024;
struct BChunk {
    int member;
    int start;
};

// A unit of work of the grouped product kernel: 128 rows of one member against a
// run of its 128-wide column tiles.
struct BItem {
    int row_tile;   // in the class row space (PA)
    int pb_tile;    // first column tile in the class row space (PB)
    int v_tile;     // first column tile in the packed fp16 V
    int ntiles;
    int member;
    int pad0, pad1, pad2;
};

// Grouped H V / K V over a batch (tc.cu).  PA/PB are the class's operand arrays,
// V16 the packed fp16 right-hand sides [R_pad][cols], vinv[member][R_pad] their
// scales.  Y, Vd (the diagonal term's vectors) are packed vector blocks.
struct TcGroupArgs {
    int kind, KD, R, R_pad;
    const void *PA, *PB;
    int64_t class_rows;  // rows of PA / PB
    const void *V16;
    int64_t v_cols;      // columns of V16
    const float *vinv;
    const BItem *items;
    int nitems;
    const BMember *members;
    const int *mdone;    // per member: skip when nonzero (may be null)
    float *Y;
    const float *Vd;
    float diag;          // 1: add sigma_g^2 Vd (H V), 0: K V
    int *err;
    int split;           // split form (V16 holds R_pad high rows, then R_pad low rows)
};
int tc_group_mvm(const TcGroupArgs &a, cudaStream_t st);
// Whether the split form of the grouped product takes R_pad right-hand sides in one pass.
bool tc_split_fits_rpad(int R_pad);
// Operands of every member from its device-side parameters (BMember inv_ell, bound):
// PA/PB rows of class c at PA[c], PB[c] (KD[c] halves per row).
int tc_group_prepare(int kind, BMember *members, int G, const BChunk *chunks, int nchunks, const float *X,
                     void *const *PA, void *const *PB, const int *KD, cudaStream_t st);
// fp16 right-hand sides: V16[c][cb_g + i] = V_g[c][i] * 2^-e_gc, vinv[g][c] = 2^e_gc; with
// split also the low parts at rows R_pad + c.
int tc_group_convert(const BMember *members, int G, const BChunk *chunks, int nchunks, const float *V, int R,
                     int R_pad, unsigned *colmax, void *V16, int64_t v_cols, float *vinv, const int *mdone,
                     cudaStream_t st, bool split = false);
int tc_group_setup();  // one-time kernel attributes (call before any stream capture)

// ---------------------------------------------------------------------------
// Small device helpers used by several files
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace gp
