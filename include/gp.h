/*
 * gp.h -- C ABI of the GB300 (sm_103a) iterative-GP library.
 *
 * The library implements the hot path of marginal-likelihood optimisation for
 * iterative Gaussian processes (Lin et al., NeurIPS 2024, "Improving Linear System
 * Solvers for Hyperparameter Optimisation in Iterative Gaussian Processes"):
 * the matrix-free batched product H V = (K(X, X; theta) + sigma^2 I) V over s+1
 * right-hand sides, the CG / alternating-projection / SGD solvers it drives
 * (warm start, iteration budget, tolerance), random-Fourier-feature prior samples,
 * the fused marginal-likelihood gradient estimators, pathwise-conditioned
 * posterior samples and the softplus/Adam outer step.
 *
 * Conventions shared by every entry point
 *   - Status: every function returns GP_OK (0) or a negative gp_status_t.  The
 *     message of the last failure on the calling thread is gp_last_error().
 *     No C++ exception crosses this boundary.
 *   - Hyperparameters: theta is a HOST array of d+2 doubles
 *     [l_1 .. l_d, s_f, sigma] in natural (positive) units.  l_k are the ARD
 *     length scales, s_f the signal amplitude (k(x, x) = s_f^2), sigma the noise
 *     standard deviation.  Non-positive or non-finite entries -> GP_ERR_INVALID_ARG.
 *   - kind: GP_RBF, k = s_f^2 exp(-r^2/2), or GP_MATERN32,
 *     k = s_f^2 (1 + sqrt3 r) exp(-sqrt3 r), with r^2 = sum_k (x_k - x'_k)^2 / l_k^2.
 *   - Points: X is n x d row-major in DEVICE memory (point i at X + i*d),
 *     1 <= d <= GP_MAX_D.
 *   - Blocks of vectors (right-hand sides, solutions, probes): "column-blocked",
 *     vector c of a block occupies DEVICE memory V + c*ldv, ldv >= n.  In torch
 *     terms a block is a contiguous (R, n) tensor.  Column 0 of a solver block
 *     is the y system, columns 1..s the probe systems.
 *   - Every pointer argument is borrowed: the caller owns all memory, the library
 *     never allocates, frees or retains a pointer after the call returns.
 *     Scratch memory is a caller-provided device buffer `ws` of at least the
 *     bytes reported by the matching *_workspace() query (256-byte aligned).
 *   - Work is stream-ordered on `stream`.  Functions that report solver
 *     information (gp_solve_*) synchronise `stream` before returning; the others
 *     return as soon as their work is enqueued.
 *   - prec selects the arithmetic of the kernel-matrix tiles:
 *       GP_PREC_FP32 : CUDA-core FP32 tiles (direct differences), FP32 vectors.
 *       GP_PREC_TC16 : tcgen05 tensor cores, IEEE fp16 operands with FP32
 *                      accumulation; the squared distance uses a three-term
 *                      hi/lo split so that cancellation stays below 1e-6;
 *                      FP32 vectors, FP64 solver scalars.  Products support
 *                      d <= 62 (GP_ERR_UNSUPPORTED beyond); the gradient
 *                      estimators use CUDA-core FP32 tiles when d > 32 or
 *                      s + 1 > 256 (or the tile plan does not fit).
 *     The *_f64 entry points are the plain FP64 GPU form (CUDA-core FP64 tiles
 *     and FP64 vectors) used as the comparison baseline.
 */
#ifndef GP_GB300_H
#define GP_GB300_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GP_MAX_D 128

typedef enum {
    GP_OK = 0,
    GP_ERR_INVALID_ARG = -1, /* a null pointer, a size out of range, a bad theta */
    GP_ERR_CUDA = -2,        /* a CUDA launch or runtime call failed            */
    GP_ERR_BREAKDOWN = -3,   /* solver hit a non-finite or non-positive pivot    */
    GP_ERR_DIVERGED = -4,    /* SGD residual estimate grew beyond 1e6 x start    */
    GP_ERR_TIMEOUT = -5,     /* a bounded device wait gave up                    */
    GP_ERR_UNSUPPORTED = -6, /* valid request this build cannot serve            */
    GP_ERR_WORKSPACE = -7    /* ws is null, misaligned or smaller than required  */
} gp_status_t;

typedef enum { GP_RBF = 0, GP_MATERN32 = 1 } gp_kernel_t;
/* Precision forms.  GP_PREC_FP32: CUDA-core FP32 tiles.  GP_PREC_TC16: tcgen05 fp16 operands
 * (kernel values, vectors and a hi/lo-split distance) with FP32 accumulation.
 * GP_PREC_TC16X3 (gp_kernel_mvm only; the solvers use it for their true residuals): the same
 * with the kernel values and the vectors split into fp16 high + low parts and
 * Y = P_hi V_hi + P_hi V_lo + P_lo V_hi, FP32-class products (relative error about 1e-6
 * instead of 1e-3) at a tensor-core rate. */
typedef enum { GP_PREC_FP32 = 1, GP_PREC_TC16 = 2, GP_PREC_TC16X3 = 3 } gp_prec_t;

/* Loop condition of Alg. 1-3.  GP_STOP_BOTH (default): iterate while
 * t < budget and (||r_y|| > tol or ||r_z|| > tol), i.e. stop once BOTH split
 * norms reach tol, as App. B "Linear System Solver" states.  GP_STOP_EITHER:
 * the listing's conjunction, stop as soon as either norm reaches tol. */
typedef enum { GP_STOP_BOTH = 0, GP_STOP_EITHER = 1 } gp_stop_t;

/* Solver report.  res_y = ||r_y|| and res_z = (1/s) sum_j ||r_j|| are the
 * relative residual norms of the normalised systems (App. B); for SGD they
 * are the residual estimate of Alg. 3.  converged = 1 when the stop rule was
 * met before the budget ran out (GP_OK with converged = 0 is not an error). */
typedef struct {
    int64_t iters;
    int converged;
    int status;
    double res_y;
    double res_z;
} gp_solve_info_t;

/* Message of the last failure on the calling thread ("" if none). */
const char *gp_last_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int gp_version(void);

/* Diagnostics (no counterpart in the paper; used by benchmarks).
 * gp_diag_reset(t) zeroes the launch counter and, when t != 0, starts timing
 * every kernel-matrix product kernel with CUDA events recorded on its launch
 * stream (t == 0 stops timing).  gp_diag_launches() returns the number of
 * library kernels launched since the reset.  gp_diag_kernel_time() waits for
 * the recorded events and returns the summed duration (ms) and the number of
 * timed launches of the kernel-matrix product kernels (which = 0) or of the
 * tensor-core gradient kernel (which = 1); gp_diag_product_time() is which = 0. */
void gp_diag_reset(int time_products);
long long gp_diag_launches(void);
int gp_diag_kernel_time(int which, double *total_ms, long long *count);
int gp_diag_product_time(double *total_ms, long long *count);

/* Device status.  Every wait of the tensor-core kernels on a barrier is bounded (about 2 s);
 * a wait that gives up makes its kernel skip the rest of its work, release its tensor memory,
 * return, and set a device status word.  gp_device_check() synchronises `stream`, reads and
 * clears the word: GP_ERR_TIMEOUT when a wait gave up since the last check (the results of
 * the calls in between are not valid), else GP_OK.  CG in the tensor-core form checks it
 * before returning.  gp_diag_timeout_probe() launches one wait that nothing completes,
 * bounded by wait_cycles (<= 4e9) SM cycles, to exercise that path. */
int gp_device_check(cudaStream_t stream);
int gp_diag_timeout_probe(long long wait_cycles, cudaStream_t stream);

/* Unit-rate probe (no counterpart in the paper; it gives the roofline of the kernel-matrix
 * kernels, which are bound by the special-function unit).  Measures, on the current device,
 * the throughput of ex2.approx, rsqrt.approx, sin.approx, cos.approx (MUFU), FP32 FMA and
 * FP64 FMA as thread-instructions per SM per SM clock (median over the SMs; one 1024-thread
 * CTA per SM with eight independent chains per thread, timed by clock64 between CTA
 * barriers, so the rates do not depend on the clock).  rates: HOST array of 6 doubles in that
 * order.  iters: rounds per thread (about 4096 gives a stable figure in well under a second).
 * ws: DEVICE scratch of gp_diag_unit_rates_workspace() bytes.  Synchronises `stream`. */
size_t gp_diag_unit_rates_workspace(void);
int gp_diag_unit_rates(int iters, double *rates, void *ws, size_t ws_bytes, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Kernel matrix-vector products (Sec. 2 H_theta; Eq. standard_system,        */
/* Eq. pathwise_system; every solver's "linear operator H(.)", Alg. 1-3)     */
/* ------------------------------------------------------------------------ */

/* Y[c] = K(X1, X2) V[c] (+ sigma^2 V[c] when add_noise), c < nrhs.
 *   X1 : n1 x d device rows (output points), X2 : n2 x d device columns.
 *   V  : nrhs vectors of length n2 (stride ldv >= n2), Y : nrhs x n1 (ldy >= n1).
 *   add_noise = 1 requires X1 == X2 and n1 == n2 and gives H V.
 *   n1 = 0 or n2 = 0 or nrhs = 0 is a valid no-op (Y is zeroed when n2 = 0).
 * prec: GP_PREC_FP32, GP_PREC_TC16 or GP_PREC_TC16X3 (gp_prec_t).
 * Y must not overlap V or X.  Error: GP_ERR_INVALID_ARG on bad sizes/pointers. */
int gp_kernel_mvm(int kind, const double *theta, int d,
                  const float *X1, int64_t n1, const float *X2, int64_t n2,
                  const float *V, int64_t ldv, int nrhs, float *Y, int64_t ldy,
                  int add_noise, int prec, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_kernel_mvm_workspace(int64_t n1, int64_t n2, int d, int nrhs, int prec);

/* Autotuner of the tensor-core product's schedule (the paper has no counterpart).
 * Times H V = (K(X, X) + sigma^2 I) V for the persistent schedule (one CTA per SM over
 * equal runs of (row tile, column tile) pairs) and a ladder of column-split counts (1 .. 128
 * splits of each 128-row tile's column range); `reps` timed runs each after one warm-up,
 * CUDA events on `stream`; records the fastest for the product's shape (rows, columns and
 * padded right-hand sides in tiles) in a process-wide table.  Every later tensor-core
 * product of that shape, including the solvers' operators, uses the recorded schedule when
 * its workspace holds the partial sums (else the built-in cost model's choice).  Y receives
 * H V.  best_split, best_ms: HOST outputs; best_split = -1 is the persistent schedule, k >= 1
 * k column splits.  1 <= nrhs <= 128.  Synchronises `stream`, so
 * it must not be called inside a stream capture.  Because the split fixes the order of the
 * column sums, results after tuning may differ from untuned ones by rounding.
 * gp_autotune_reset() forgets every recorded choice. */
int gp_autotune_mvm(int kind, const double *theta, int d, const float *X, int64_t n,
                    const float *V, int nrhs, float *Y, int reps, int *best_split, double *best_ms,
                    void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_autotune_mvm_workspace(int64_t n, int d, int nrhs);
void gp_autotune_reset(void);

/* Autotuner of the tensor-core gradient's work split (the paper has no counterpart).  Times
 * the fused estimator of gp_mll_grad_pathwise (Z = NULL: U = W = Vsol, the symmetric sweep
 * over the upper triangle of tiles, candidates = tile pairs per CTA item) or of
 * gp_mll_grad_standard (Z = the s probes: the full sweep, candidates = column splits per
 * 128-row tile), `reps` timed runs each after a warm-up, and records the fastest for the
 * shape (distance and vector contraction widths, row tiles, symmetric or not); later
 * gradients of that shape use it.  best_param, best_ms: HOST outputs.  Vsol: (s+1) x n, Z:
 * s x n, device.  ws: gp_autotune_grad_workspace(n, d, s) bytes.  Synchronises `stream`;
 * not for use inside a stream capture.  GP_ERR_UNSUPPORTED when the tensor-core gradient
 * does not cover (d, s) (d > 32 or s + 1 > 256). */
int gp_autotune_grad(int kind, const double *theta, int d, const float *X, int64_t n,
                     const float *Vsol, int s, const float *Z, int reps, int64_t *best_param,
                     double *best_ms, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_autotune_grad_workspace(int64_t n, int d, int s);

/* The autotuner's table on disk.  gp_autotune_save writes every recorded choice (products and
 * gradients) to a text file tagged with the current device's name, compute capability and SM
 * count; gp_autotune_load adds a file's entries to the table, refusing a file written on
 * another kind of device (GP_ERR_INVALID_ARG, message in gp_last_error()).  When the
 * environment variable GP_AUTOTUNE_CACHE names a file, the library reads it at its first
 * tuned lookup and writes the table back to it after every tuning call.  gp_autotune_count()
 * is the number of recorded choices. */
int gp_autotune_save(const char *path);
int gp_autotune_load(const char *path);
int64_t gp_autotune_count(void);

/* FP64 form of gp_kernel_mvm (plain CUDA-core FP64 tiles). */
int gp_kernel_mvm_f64(int kind, const double *theta, int d,
                      const double *X1, int64_t n1, const double *X2, int64_t n2,
                      const double *V, int64_t ldv, int nrhs, double *Y, int64_t ldy,
                      int add_noise, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_kernel_mvm_f64_workspace(int64_t n1, int64_t n2, int d, int nrhs);

/* ------------------------------------------------------------------------ */
/* Linear system solvers (App. B, Alg. 1-3) on H [v_y, v_1..v_s] = B          */
/* ------------------------------------------------------------------------ */

/* Batched conjugate gradients, Alg. 1 with P = identity.
 *   B        : nrhs right-hand sides (device, stride n), unchanged.
 *   V_inout  : warm start on entry (zeros for a cold start), solution on exit
 *              (device, stride n).  Each column is solved on the normalised
 *              system b / (||b|| + 1e-12) and rescaled on exit (App. B).
 *   max_iters: iteration budget T (one CG iteration = one epoch).
 *   tol      : relative residual tolerance tau; stop_rule a gp_stop_t.
 * A column whose gamma = r^T r falls to <= 1e-30 is frozen.  The iterations carry
 * Alg. 1's recursive residual; when the loop stops on it, the true residual
 * b~ - H v is recomputed once (one product; each difference rounded about once, the
 * norms accumulated in FP64) and the
 * tolerance is judged on it: a solve whose true residual misses tau restarts from
 * it (d = r) within its budget, and info's res_y / res_z are always true-residual
 * norms.  That true residual is taken with an FP32-class product: the split
 * tensor-core product (GP_PREC_TC16X3) for GP_PREC_TC16, the FP64 product of the
 * FP32 inputs for GP_PREC_FP32, the FP64 product for the FP64 form (the initial
 * residual of a warm start uses the form's own product).  A restart that does not lower the true residual by
 * 10% ends the solve (not converged): the form's arithmetic has reached what it
 * can attain on the system.  Returns GP_OK with info filled (synchronises
 * stream), GP_ERR_BREAKDOWN if a residual becomes non-finite. */
int gp_solve_cg(int kind, const double *theta, int d, const float *X, int64_t n,
                const float *B, int nrhs, float *V_inout, int64_t max_iters, double tol,
                int stop_rule, int prec, gp_solve_info_t *info,
                void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_solve_cg_workspace(int64_t n, int d, int nrhs, int prec);

int gp_solve_cg_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                    const double *B, int nrhs, double *V_inout, int64_t max_iters, double tol,
                    int stop_rule, gp_solve_info_t *info, void *ws, size_t ws_bytes,
                    cudaStream_t stream);
size_t gp_solve_cg_f64_workspace(int64_t n, int d, int nrhs);

/* Alg. 1 with the preconditioner of App. B "Conjugate Gradients": P = L^T L + sigma^2 I
 * from a rank-`rank` pivoted Cholesky factor of K (greedy pivots on the largest remaining
 * diagonal, ties to the lowest index; the paper uses rank 100), applied through the
 * Woodbury identity with a k x k Cholesky factor in FP64.  The loop is the listing's:
 * p = P^-1 r, gamma = r^T p, d = p + beta d; split norms and the stop rule use ||r|| as in
 * gp_solve_cg.  rank = 0 is gp_solve_cg; 0 <= rank <= 128 (clamped to n).  The factor is
 * built once per call (2 rank + 3 small launches) and its arithmetic, like the solver's
 * vectors, is FP32 (FP64 in the _f64 form) with FP64 sums across tiles. */
int gp_solve_pcg(int kind, const double *theta, int d, const float *X, int64_t n,
                 const float *B, int nrhs, float *V_inout, int64_t max_iters, double tol,
                 int stop_rule, int prec, int rank, gp_solve_info_t *info,
                 void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_solve_pcg_workspace(int64_t n, int d, int nrhs, int prec, int rank);
int gp_solve_pcg_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                     const double *B, int nrhs, double *V_inout, int64_t max_iters, double tol,
                     int stop_rule, int rank, gp_solve_info_t *info,
                     void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_solve_pcg_f64_workspace(int64_t n, int d, int nrhs, int rank);

/* Alternating projections, Alg. 2.  Blocks are contiguous row ranges
 * [i*block_size, min((i+1)*block_size, n)); each iteration selects the block
 * with the largest ||sum_c r_c[i]|| (ties: lowest index), adds
 * H[i,i]^-1 r[i] to v[i] and subtracts H[:, i] H[i,i]^-1 r[i] from r.  The
 * inverse of every diagonal block is computed once per call from its Cholesky
 * factor (cached for the whole solve).  max_iters counts block iterations
 * (epochs x n / block_size).  1 <= block_size <= 1024.  When the loop stops on the
 * residual the panels maintain, the true residual is recomputed (one full product
 * of the FP32 class, as in gp_solve_cg; not counted in max_iters) and judged as in
 * gp_solve_cg. */
int gp_solve_ap(int kind, const double *theta, int d, const float *X, int64_t n,
                const float *B, int nrhs, float *V_inout, int64_t block_size, int64_t max_iters,
                double tol, int stop_rule, int prec, gp_solve_info_t *info,
                void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_solve_ap_workspace(int64_t n, int d, int nrhs, int64_t block_size, int prec);

int gp_solve_ap_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                    const double *B, int nrhs, double *V_inout, int64_t block_size,
                    int64_t max_iters, double tol, int stop_rule, gp_solve_info_t *info,
                    void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_solve_ap_f64_workspace(int64_t n, int d, int nrhs, int64_t block_size);

/* Stochastic gradient descent with momentum, Alg. 3 (no Polyak averaging).
 *   batch_idx : DEVICE int32 array of max_iters * batch row indices; iteration t
 *               uses batch_idx[t*batch .. t*batch + batch - 1] (distinct rows
 *               within one iteration; every index in [0, n)).
 *   lr, momentum : gamma and rho of Alg. 3.  The momentum starts at zero.
 * The residual estimate r starts at the normalised b and r[i] <- g[i] on the
 * sampled rows.  GP_ERR_DIVERGED if the estimate exceeds 1e6 x its start. */
int gp_solve_sgd(int kind, const double *theta, int d, const float *X, int64_t n,
                 const float *B, int nrhs, float *V_inout, int64_t batch,
                 const int32_t *batch_idx, double lr, double momentum, int64_t max_iters,
                 double tol, int stop_rule, int prec, gp_solve_info_t *info,
                 void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_solve_sgd_workspace(int64_t n, int d, int nrhs, int64_t batch, int prec);

int gp_solve_sgd_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                     const double *B, int nrhs, double *V_inout, int64_t batch,
                     const int32_t *batch_idx, double lr, double momentum, int64_t max_iters,
                     double tol, int stop_rule, gp_solve_info_t *info,
                     void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_solve_sgd_f64_workspace(int64_t n, int d, int nrhs, int64_t batch);

/* ------------------------------------------------------------------------ */
/* Random Fourier features (Sec. 2 "Pathwise Conditioning"; App. B "Kernel     */
/* Function and Random Features")                                            */
/* ------------------------------------------------------------------------ */

/* F[j][i] = f_j(x_i) = s_f sqrt(2/m) sum_{l < m/2} ( W[j][l] cos(w_l . x_i)
 *                                               + W[j][m/2 + l] sin(w_l . x_i) )
 * with frequencies w_l = omega_hat_l / l (RBF) or omega_hat_l / l * sqrt(3 / u_l)
 * (Matern-3/2; u_l ~ chi^2_3, the Student-t spectral density).  The random
 * parameters are inputs, fixed across calls so that the prior sample stays the
 * same function while theta changes (App. B).
 *   omega_hat : (m/2) x d device, chi2 : m/2 device (may be NULL for RBF),
 *   W : s x m device (row j = sample j), F : s x n device (stride ldf >= n).
 * m must be even and >= 2. */
int gp_rff_prior_sample(int kind, const double *theta, int d, const float *X, int64_t n,
                        int m, const float *omega_hat, const float *chi2, const float *W,
                        int s, float *F, int64_t ldf, cudaStream_t stream);
/* Same, in a precision form with a caller workspace (gp_rff_prior_sample_workspace bytes):
 * GP_PREC_FP32 is the CUDA-core form above; GP_PREC_TC16 takes F^T = Phi W^T on the tensor
 * cores, with the features Phi (cos / sin of w_l . x, range-reduced by 2 pi, on the MUFU) and
 * the weights each split into fp16 hi + lo parts and the product summed as hi.hi + hi.lo +
 * lo.hi in FP32 (error ~1e-6 relative, the FP32 form's order), for d <= 32 and s <= 128
 * (larger problems run the CUDA-core form).  Errors: as gp_rff_prior_sample, plus
 * GP_ERR_WORKSPACE and GP_ERR_UNSUPPORTED (GP_PREC_TC16 without tcgen05). */
int gp_rff_prior_sample_ws(int kind, const double *theta, int d, const float *X, int64_t n,
                           int m, const float *omega_hat, const float *chi2, const float *W,
                           int s, float *F, int64_t ldf, int prec, void *ws, size_t ws_bytes,
                           cudaStream_t stream);
size_t gp_rff_prior_sample_workspace(int d, int m, int s, int prec);
int gp_rff_prior_sample_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                            int m, const double *omega_hat, const double *chi2, const double *W,
                            int s, double *F, int64_t ldf, cudaStream_t stream);

/* Pathwise probe right-hand sides (App. B): B = [y, xi_1 .. xi_s] with
 * xi_j = F_j + sigma * w_j (epsilon = sigma w, w fixed).  y : n, F, w : s x n,
 * B : (s+1) x n, all device, stride n. */
int gp_pathwise_rhs(const double *theta, int d, const float *y, const float *F, const float *w,
                    int64_t n, int s, float *B, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Marginal-likelihood gradient estimators (Eq. mll_grad, Eq. trace,           */
/* Eq. pathwise_estimator), fused over kernel tiles                          */
/* ------------------------------------------------------------------------ */

/* Standard (Hutchinson) estimator:
 *   grad_k = 1/2 v_y^T dH_k v_y - 1/(2s) sum_j v_j^T dH_k z_j
 *   Vsol : (s+1) x n = [v_y, v_1..v_s] (solutions), Z : s x n probes.
 * grad : DEVICE array of d+2 doubles, d L / d theta in theta's order (ascent
 * direction of the log marginal likelihood). */
int gp_mll_grad_standard(int kind, const double *theta, int d, const float *X, int64_t n,
                         const float *Vsol, const float *Z, int s, double *grad, int prec,
                         void *ws, size_t ws_bytes, cudaStream_t stream);
/* Pathwise estimator:
 *   grad_k = 1/2 v_y^T dH_k v_y - 1/(2s) sum_j zhat_j^T dH_k zhat_j,
 *   Vsol = [v_y, zhat_1..zhat_s] solving H Vsol = [y, xi_1..xi_s]. */
int gp_mll_grad_pathwise(int kind, const double *theta, int d, const float *X, int64_t n,
                         const float *Vsol, int s, double *grad, int prec,
                         void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_mll_grad_workspace(int64_t n, int d, int s, int prec);

int gp_mll_grad_standard_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                             const double *Vsol, const double *Z, int s, double *grad,
                             void *ws, size_t ws_bytes, cudaStream_t stream);
int gp_mll_grad_pathwise_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                             const double *Vsol, int s, double *grad,
                             void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_mll_grad_f64_workspace(int64_t n, int d, int s);

/* Reverse-mode derivatives of the bilinear form
 *   f(theta, X, U, W) = sum_c lam_c u_c^T H(theta, X) w_c,
 *   lam_0 = lam0, lam_c = lam_rest for c >= 1, H = K + sigma^2 I (Sec. 2).
 * Its theta-gradient is the estimator reduction of Eq. mll_grad (standard:
 * U = [v_y, v_1..v_s], W = [v_y, z_1..z_s]; pathwise: U = W = [v_y, zhat_1..]
 * with lam0 = 1/2, lam_rest = -1/(2s)), and with lam0 = lam_rest = 1 and
 * U = G (an upstream gradient), W = V it is the backward pass of Y = H V with
 * respect to theta and X (the V-gradient is H G, i.e. gp_kernel_mvm).
 *   U, W : R vectors of length n (device, strides ldu, ldw >= n).  U == W with
 *          ldu == ldw is recognised as the symmetric form.
 *   value  : DEVICE double, f itself, or NULL.
 *   dtheta : DEVICE array of d+2 doubles, df/dtheta in theta's order, or NULL.
 *   dX     : DEVICE n x d row-major (same layout as X), df/dX, or NULL.
 *            dk(x, x')/dx = -psi(r) (x - x') / l^2 with psi = k (RBF) or
 *            3 s_f^2 exp(-sqrt3 r) (Matern-3/2); kernel tiles are recomputed.
 * prec applies to value/dtheta as in gp_mll_grad_*; dX always uses CUDA-core
 * tiles in the element type (FP32 here, FP64 in the _f64 form) with FP64
 * accumulation across tiles.  NULL outputs are skipped; all NULL is a no-op.
 * Errors: GP_ERR_INVALID_ARG (sizes, pointers, theta, non-finite lam),
 * GP_ERR_UNSUPPORTED when d and R exceed the point-gradient tile (shared
 * memory), GP_ERR_WORKSPACE. */
int gp_bilinear_grad(int kind, const double *theta, int d, const float *X, int64_t n,
                     const float *U, int64_t ldu, const float *W, int64_t ldw, int R,
                     double lam0, double lam_rest, double *value, double *dtheta, float *dX,
                     int prec, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_bilinear_grad_workspace(int64_t n, int d, int R, int prec);
int gp_bilinear_grad_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                         const double *U, int64_t ldu, const double *W, int64_t ldw, int R,
                         double lam0, double lam_rest, double *value, double *dtheta, double *dX,
                         void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_bilinear_grad_f64_workspace(int64_t n, int d, int R);

/* Pathwise estimator that allocates nothing and takes no workspace (the paper has
 * no counterpart: this is a deployment variant of gp_mll_grad_pathwise).
 * For callers that cannot allocate device memory where they call it: code that
 * runs while a stream is captured into a CUDA graph, host callbacks enqueued on a
 * stream, hosts with a fixed device-memory budget.  Its scratch is one static
 * device array of GP_NOALLOC_SCRATCH_BYTES per GPU (held from library load to
 * process exit).  With prec = GP_PREC_FP32 the scratch holds only block partial
 * sums, enough for n up to about 3.9 million points at d = 16 (2 million at
 * d = 32); with GP_PREC_TC16 it also holds the fp16 tensor-core operands (about
 * 0.9 KB per point at d = 16, s = 64) and the work-split partials, enough for n
 * up to about 8500 points.
 * gp_mll_grad_workspace(n, d, s, prec) is the amount a call needs.  Requests
 * that need more return GP_ERR_INVALID_ARG with the
 * required size in gp_last_error().  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) and also does the library's other
 * one-time set-up for that device (the shared-memory limits of the kernels it
 * launches, the address of the device status word), so make that first call
 * before any stream capture.  All calls on a device share the array: calls whose work
 * overlaps on the GPU (unordered streams) race and must not be issued.  Results
 * equal gp_mll_grad_pathwise's for the same arguments. */
#define GP_NOALLOC_SCRATCH_BYTES (8u << 20)
int gp_mll_grad_pathwise_noalloc(int kind, const double *theta, int d, const float *X, int64_t n,
                                 const float *Vsol, int s, double *grad, int prec, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Posterior samples by pathwise conditioning (Eq. pathwise_conditioning,     */
/* Sec. 3 "Amortising Linear Solves")                                        */
/* ------------------------------------------------------------------------ */

/* out[j](x*) = Fstar[j](x*) + k(x*, X) (v_y - zhat_j),  j < s.
 *   Xstar : nstar x d, X : n x d, Vsol : (s+1) x n (stride n),
 *   Fstar : s x nstar prior samples at Xstar (gp_rff_prior_sample with the same
 *   random parameters), out : s x nstar.  All device. */
int gp_posterior_samples(int kind, const double *theta, int d, const float *Xstar, int64_t nstar,
                         const float *X, int64_t n, const float *Vsol, int s, const float *Fstar,
                         float *out, int prec, void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_posterior_samples_workspace(int64_t nstar, int64_t n, int d, int s, int prec);
/* Predictions from the pathwise solutions (Sec. 3 "Amortising Linear Solves for
 * Optimisation and Prediction"; App. B reports test RMSE and test log-likelihood):
 *   mean_i = k(x*_i, X) v_y,
 *   var_i  = (1/s) sum_j (f_j(x*_i) - k(x*_i, X) zhat_j)^2 + sigma^2
 * (the spread of the s pathwise posterior samples around the exact mean, plus the noise:
 * the predictive variance of y*).  Vsol = [v_y, zhat_1..zhat_s] ((s+1) x n), Fstar: s x nstar
 * prior samples at Xstar (gp_rff_prior_sample with the probes' features).  mean, var:
 * DEVICE nstar floats.  With ystar (DEVICE nstar floats, or NULL) and metrics (DEVICE 2
 * doubles, or NULL): metrics[0] = RMSE, metrics[1] = mean_i log N(ystar_i; mean_i, var_i).
 * Sums in FP64.  Errors as gp_posterior_samples. */
int gp_predict(int kind, const double *theta, int d, const float *Xstar, int64_t nstar,
               const float *X, int64_t n, const float *Vsol, int s, const float *Fstar,
               const float *ystar, float *mean, float *var, double *metrics, int prec,
               void *ws, size_t ws_bytes, cudaStream_t stream);
size_t gp_predict_workspace(int64_t nstar, int64_t n, int d, int s, int prec);

/* ------------------------------------------------------------------------ */
/* Solver diagnostic: initial RKHS distance (Sec. 3, "Initial Distance to the  */
/* Linear System Solution", Eq. RKHS_distance)                               */
/* ------------------------------------------------------------------------ */

/* dist[c] = (Uinit[c] - U[c])^T H (Uinit[c] - U[c]), c < R, H = K(X, X) + sigma^2 I:
 * the squared RKHS distance between a solver's initialisation and a solution.  With
 * Uinit = NULL (the zero initialisation) it is U[c]^T H U[c] = b^T H^-1 b when U[c] solves
 * H u = b; its expectation is tr(H^-1) for the standard estimator's probes (Eq.
 * standard_dist) and n for the pathwise targets (Eq. pathwise_dist).
 *   X : n x d, U and Uinit : R x n (stride n), DEVICE; dist : DEVICE R doubles.
 * One product H E in the requested form (prec), then FP64 dot products summed in a fixed
 * order (deterministic).  Errors: GP_ERR_INVALID_ARG (sizes, null X/U/dist, theta, prec),
 * GP_ERR_WORKSPACE, GP_ERR_UNSUPPORTED (GP_PREC_TC16 without tcgen05). */
int gp_rkhs_sqdist(int kind, const double *theta, int d, const float *X, int64_t n, const float *Uinit,
                   const float *U, int R, double *dist, int prec, void *ws, size_t ws_bytes,
                   cudaStream_t stream);
size_t gp_rkhs_sqdist_workspace(int64_t n, int d, int R, int prec);
int gp_rkhs_sqdist_f64(int kind, const double *theta, int d, const double *X, int64_t n,
                       const double *Uinit, const double *U, int R, double *dist, void *ws,
                       size_t ws_bytes, cudaStream_t stream);
size_t gp_rkhs_sqdist_f64_workspace(int64_t n, int d, int R);

/* ------------------------------------------------------------------------ */
/* Outer loop (Sec. 2.1 "Outer-Loop Optimiser"; App. B "Iterative Optimiser") */
/* ------------------------------------------------------------------------ */

/* One Adam ASCENT step on the softplus parameters nu (theta = log(1 + e^nu)).
 * HOST arrays of P = d+2 doubles: nu, m, v (updated in place), grad_theta (the
 * estimator output copied to the host), theta_out (softplus(nu) after the step).
 * t >= 1 is the step count for bias correction. */
int gp_adam_softplus_step(int P, double *nu, double *m, double *v, int64_t t,
                          const double *grad_theta, double lr, double beta1, double beta2,
                          double eps, double *theta_out);

/* ------------------------------------------------------------------------ */
/* Batches of independent GPs of uneven size (many problems of Sec. 2 solved  */
/* and optimised together; the paper treats one problem at a time)           */
/* ------------------------------------------------------------------------ */

/* A batch plan: G members, member g with n[g] >= 1 points of dimension
 * 1 <= d[g] <= 32, all with the same kernel kind and s probes (R = s+1 vectors
 * per member, R <= 128).  The plan is a HOST object (gp_batch_create allocates
 * it with new; gp_batch_destroy frees it); it owns no device memory.
 *
 * Packed layouts (all DEVICE memory owned by the caller; offsets from
 * gp_batch_member_offsets):
 *   X      : member g's n_g x d_g row-major points at X + x_off[g]
 *            (x_off[g] = sum_{h<g} n_h d_h; total x_len floats).
 *   vectors: member g's block of R vectors at V + vec_off[g], vector c at
 *            V + vec_off[g] + c*n_g (vec_off[g] = R sum_{h<g} n_h; total vec_len).
 *            Right-hand sides B = [y, z_1..z_s] and solutions use this layout.
 *   theta  : member g's d_g+2 doubles [l_1..l_d, s_f, sigma] at theta + theta_off[g]
 *            (DEVICE, so that a step can update it without the host).
 *
 * gp_batch_bind() carves the caller's workspace (gp_batch_workspace() bytes,
 * 256-byte aligned) and copies the plan's tables into it; it synchronises
 * `stream` and must be called once, before any stream capture.  The calls below
 * it never synchronise, allocate or copy from the host: a sequence of them can be
 * captured into a CUDA graph and replayed.  Calls on one plan must not run
 * concurrently (they share the workspace).  Device-side failures (a non-positive
 * theta, a timed-out wait) set a flag read by gp_batch_status(), which synchronises.
 * Arithmetic: tcgen05 fp16 tiles as GP_PREC_TC16 for the products, FP32 vectors,
 * FP64 solver scalars, CUDA-core FP32 tiles for the gradient. */
typedef struct gp_batch gp_batch_t;
int gp_batch_create(int kind, int G, const int64_t *n, const int *d, int s, gp_batch_t **out);
void gp_batch_destroy(gp_batch_t *b);
size_t gp_batch_workspace(const gp_batch_t *b);
int gp_batch_layout(const gp_batch_t *b, int64_t *x_len, int64_t *vec_len, int64_t *theta_len);
/* HOST arrays of G entries each (any may be NULL). */
int gp_batch_member_offsets(const gp_batch_t *b, int64_t *x_off, int64_t *vec_off, int64_t *theta_off);
int gp_batch_bind(gp_batch_t *b, void *ws, size_t ws_bytes, cudaStream_t stream);
int gp_batch_status(const gp_batch_t *b, cudaStream_t stream);

/* Tensor-core operands of every member for the current theta (Sec. 2 H_theta);
 * needed before gp_batch_mvm / gp_batch_solve_cg after theta or X changes. */
int gp_batch_prepare(gp_batch_t *b, const double *theta, const float *X, cudaStream_t stream);
/* Y_g = H_g V_g (add_noise = 1) or K_g V_g for every member (R vectors each). */
int gp_batch_mvm(gp_batch_t *b, const float *V, float *Y, int add_noise, cudaStream_t stream);
/* Alg. 1 on every member (normalised systems, split norms, loop condition
 * GP_STOP_BOTH or GP_STOP_EITHER as gp_solve_cg), V_inout the warm start and
 * the solution.  Exactly `iters` iterations are enqueued; a member whose loop
 * condition fails is skipped from then on.  Every 10 iterations and after the
 * last one, the true residual of each member that stopped on its recursive
 * residual is recomputed (one grouped product over those members); a member whose
 * true residual misses the tolerance restarts from it.  These checks use the split
 * tensor-core product when s + 1 <= 80 (the plain one above; the initial residual
 * always the plain one), and the reported norms are true-residual norms.  info: DEVICE array of G reports (or
 * NULL), written at the end. */
int gp_batch_solve_cg(gp_batch_t *b, const float *B, float *V_inout, int64_t iters, double tol,
                      int stop_rule, gp_solve_info_t *info, cudaStream_t stream);
/* Eq. mll_grad per member into grad (DEVICE, packed like theta): standard
 * estimator (Eq. trace) with probes B[1..s] (pathwise = 0), or the pathwise
 * estimator (Eq. pathwise_estimator, B unused).  Needs gp_batch_prepare's
 * parameters for the same theta. */
int gp_batch_mll_grad(gp_batch_t *b, const double *theta, const float *X, const float *Vsol,
                      const float *B, int pathwise, double *grad, cudaStream_t stream);
/* Adam ascent on softplus parameters, as gp_adam_softplus_step, for all members
 * on the device: nu, m, v, grad, theta packed like theta; *t (DEVICE) counts the
 * completed steps and is incremented.  gp_batch_adam_init sets nu = softplus^-1(theta),
 * m = v = 0, *t = 0. */
int gp_batch_adam_init(gp_batch_t *b, const double *theta, double *nu, double *m, double *v,
                       long long *t, cudaStream_t stream);
int gp_batch_adam_step(gp_batch_t *b, double *nu, double *m, double *v, long long *t,
                       const double *grad, double lr, double beta1, double beta2, double eps,
                       double *theta, cudaStream_t stream);
/* One marginal-likelihood step for every member: prepare(theta), warm-started
 * CG with `iters` iterations and tolerance tol (GP_STOP_BOTH) on B = [y, z],
 * the standard estimator, and an Adam step (beta1 0.9, beta2 0.999, eps 1e-8)
 * that updates theta, nu, m, v and *t in place. */
int gp_batch_step(gp_batch_t *b, const float *X, double *theta, const float *B, float *V_inout,
                  int64_t iters, double tol, double *grad, double *nu, double *m, double *v,
                  long long *t, double lr, gp_solve_info_t *info, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GP_GB300_H */
