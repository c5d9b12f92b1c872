// Internal: operator dispatch, solvers, random features (declarations).
#pragma once

#include "gp_internal.cuh"

namespace gp {

// H V / K V dispatch over precision (CUDA-core FP32/FP64 or tcgen05 fp16).
template <typename T>
size_t mvm_workspace(int64_t n1, int64_t n2, int d, int R, int prec);
template <typename T>
int apply_mvm(const KP<T> &kp, const T *X1, int64_t n1, const T *X2, int64_t n2, const T *V, int64_t ldv,
              int R, T *Y, int64_t ldy, int add_noise, int prec, void *ws, size_t ws_bytes, cudaStream_t st);

template <typename T>
size_t grad_workspace(int64_t n, int d, int R, int prec);
template <typename T>
int apply_grad(const GradArgs<T> &a, int prec, void *ws, size_t ws_bytes, cudaStream_t st);

// Point gradient of sum_c lam_c u_c^T H w_c (backward.cu); sym = 1 when U and W
// are the same block.  value = the form itself from its theta-gradient g.
template <typename T>
size_t bilinear_dx_workspace(int64_t n, int d);
template <typename T>
int bilinear_dx(const GradArgs<T> &a, int sym, T *dX, void *ws, size_t ws_bytes, cudaStream_t st);
template <typename T>
int bilinear_value(const KP<T> &kp, const double *g, double *value, cudaStream_t st);

template <typename T>
int rff_prior(const KP<T> &kp, const T *X, int64_t n, int m, const T *omega_hat, const T *chi2, const T *W,
              int s, T *F, int64_t ldf, cudaStream_t st);
// Same, with a precision form (GP_PREC_TC16: tensor cores within tc_rff_fits, else CUDA cores)
// and a caller workspace.
size_t rff_workspace(int d, int m, int s, int prec);
int rff_prior_ws(const KP<float> &kp, const float *X, int64_t n, int m, const float *omega_hat, const float *chi2,
                 const float *W, int s, float *F, int64_t ldf, int prec, void *ws, size_t ws_bytes, cudaStream_t st);
int pathwise_rhs(float sigma, const float *y, const float *F, const float *w, int64_t n, int s, float *B,
                 cudaStream_t st);

size_t posterior_workspace(int64_t nstar, int64_t n, int d, int s, int prec);
int posterior_samples(const KP<float> &kp, const float *Xstar, int64_t nstar, const float *X, int64_t n,
                      const float *Vsol, int s, const float *Fstar, float *out, int prec, void *ws,
                      size_t ws_bytes, cudaStream_t st);

size_t predict_workspace(int64_t nstar, int64_t n, int d, int s, int prec);
int predict(const KP<float> &kp, const float *Xstar, int64_t nstar, const float *X, int64_t n, const float *Vsol,
            int s, const float *Fstar, const float *ystar, float *mean, float *var, double *metrics, int prec,
            void *ws, size_t ws_bytes, cudaStream_t st);

// RKHS squared distance e_c^T H e_c, e_c = U[c] - U0[c] (U0 may be null), into dist (R doubles).
template <typename T>
size_t rkhs_workspace(int64_t n, int d, int R, int prec);
template <typename T>
int rkhs_sqdist(const KP<T> &kp, const T *X, int64_t n, const T *U0, const T *U, int R, double *dist, int prec,
                void *ws, size_t ws_bytes, cudaStream_t st);

// Pivoted Cholesky preconditioner (precond.cu): P = L^T L + sigma^2 I, applied by Woodbury.
template <typename T>
struct Precond {
    int k;
    int64_t n;
    int R;
    T *L;            // k x n factor rows
    double *G;       // k x k Cholesky factor of sigma^2 I + L L^T (lower triangle)
    double *part;    // per-tile partial sums of L r
    double *w;       // k x R
    double inv_sigma2;
};
template <typename T>
size_t precond_workspace(int64_t n, int R, int k);
template <typename T>
int precond_build(const KP<T> &kp, const T *X, int64_t n, int R, int k, void *ws, size_t ws_bytes, Precond<T> *out,
                  cudaStream_t st);
template <typename T>
int precond_apply(const Precond<T> &P, const T *r, T *p, const int *done, cudaStream_t st);

// The true residual r = b~ - H v of a normalised iterate with the FP64 product of FP32 inputs
// (the check of the FP32 form's solvers), partial sums of ||r||^2 into partN (P x R).
size_t f64_residual_workspace(int64_t n, int d, int R);
int f64_residual(const KP<float> &kp, const float *X, int64_t n, const float *B, const float *V, int R,
                 const double *scale, float *r, double *partN, int P, void *ws, size_t ws_bytes, cudaStream_t st);

// Solvers (App. B, Alg. 1-3).
template <typename T>
size_t cg_workspace(int64_t n, int d, int R, int prec, int pc_rank = 0);
template <typename T>
int cg_solve(const KP<T> &kp, const T *X, int64_t n, const T *B, int R, T *V, int64_t max_iters, double tol,
             int stop_rule, int prec, gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t st,
             int pc_rank = 0);

template <typename T>
size_t ap_workspace(int64_t n, int d, int R, int64_t bs, int prec);
template <typename T>
int ap_solve(const KP<T> &kp, const T *X, int64_t n, const T *B, int R, T *V, int64_t bs, int64_t max_iters,
             double tol, int stop_rule, int prec, gp_solve_info_t *info, void *ws, size_t ws_bytes,
             cudaStream_t st);

template <typename T>
size_t sgd_workspace(int64_t n, int d, int R, int64_t batch, int prec);
template <typename T>
int sgd_solve(const KP<T> &kp, const T *X, int64_t n, const T *B, int R, T *V, int64_t batch,
              const int32_t *idx, double lr, double rho, int64_t max_iters, double tol, int stop_rule,
              int prec, gp_solve_info_t *info, void *ws, size_t ws_bytes, cudaStream_t st);

// Device-resident solver state, read back once per poll.
struct SolverState {
    int done;
    int status;
    int converged;
    int certified;  // CG: res_y / res_z (and converged) come from a recomputed true residual
    long long iter;
    double res_y;
    double res_z;
    double res0;  // SGD: initial residual estimate (divergence guard)
};

}  // namespace gp
