/*
 * gp_oracle.c -- plain FP64 CPU oracle for iterative-GP marginal-likelihood
 * optimisation (Lin, Padhy, Mlodozeniec, Antoran, Hernandez-Lobato, NeurIPS 2024,
 * "Improving Linear System Solvers for Hyperparameter Optimisation in Iterative
 * Gaussian Processes").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle: it is compiled into
 * liboracle_gp.so and may be loaded only by tests/, by __graft_entry__.smoke() and
 * by bench.py's cpu_baseline / reference leg.  The CUDA library never links it
 * and shares no code, header or constant with it.
 *
 * Everything is double precision, written to be read against the paper: no
 * blocking, no fusion, no reordering beyond what a definition states.  OpenMP
 * only splits independent outer loops (rows) across threads.
 *
 * Conventions (independent of the GPU library, chosen for readability):
 *   X      : n x d, row-major (point i at X + i*d)
 *   theta  : d+2 values [l_1..l_d, s_f, sigma]   (natural, positive)
 *   blocks of vectors (right-hand sides, solutions): R x n, row-major, i.e.
 *            vector c occupies V + c*n.  Vector 0 is the y system.
 *   kind   : 0 = RBF-ARD, 1 = Matern-3/2 ARD
 *
 * Readings of the paper taken here (where it is silent, ambiguous or garbled):
 *   - Matern-3/2 with "a scalar signal scale" (Sec. 2, App. B) is
 *     k = s_f^2 (1 + sqrt(3) r) exp(-sqrt(3) r), r^2 = sum_k (x_k-x'_k)^2 / l_k^2,
 *     s_f an amplitude, gradients taken with respect to s_f.
 *   - RBF (not in the paper; used by synthetic workloads): k = s_f^2 exp(-r^2/2).
 *   - The solver loop (Alg. 1-3) continues while t < budget and the relative
 *     residual norms are not BOTH below tau (the text of App. B says both must
 *     reach tau; the listing's conjunction would stop at the first).  stop_rule=1
 *     selects the listing's literal rule instead.
 *   - A CG column whose gamma falls to <= 1e-30 (or whose d^T H d <= 0) is frozen
 *     (alpha = beta = 0); Alg. 1 is silent on 0/0.
 *   - Relative-residual normalisation (App. B "Linear System Solver"):
 *     solve with b~ = b / (||b|| + eps), eps = 1e-12, return (||b|| + eps) u~.
 *   - AP block score is the literal ||r_y[i] + sum_j r_j[i]|| of Alg. 2; ties go to
 *     the lowest block index; block i holds rows [i*b, min((i+1)*b, n)).
 *   - SGD (Alg. 3): r starts at b~ and r[i] <- g[i] on sampled rows; the batch
 *     indices are an input (iteration t uses idx[t*b .. t*b+b-1]).
 *   - RFF (App. B "Kernel Function and Random Features"): m features = m/2
 *     frequencies, each with a cos and a sin feature; f(x) = s_f sqrt(2/m)
 *     sum_l [w_{j,l} cos(w_l.x) + w_{j,m/2+l} sin(w_l.x)], frequency
 *     w_l = omega_hat_l / l (RBF) or omega_hat_l / l * sqrt(3/u_l), u_l ~ chi^2_3
 *     (Matern-3/2 spectral density = Student-t with 3 degrees of freedom).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GPO_RBF 0
#define GPO_MATERN32 1

/* ------------------------------------------------------------------------- */
/* Kernel function (Sec. 2; App. B "Kernel Function and Random Features")      */
/* ------------------------------------------------------------------------- */

/* Scaled squared distance r^2 = sum_k (x_k - x'_k)^2 / l_k^2. */
static double sqdist(int d, const double *ell, const double *x, const double *xp)
{
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = (x[k] - xp[k]) / ell[k];
        r2 += t * t;
    }
    return r2;
}

/* k(x, x'; vartheta) with vartheta = (l_1..l_d, s_f). */
double gpo_kernel(int kind, int d, const double *theta, const double *x, const double *xp)
{
    double sf = theta[d];
    double r2 = sqdist(d, theta, x, xp);
    if (kind == GPO_RBF)
        return sf * sf * exp(-0.5 * r2);
    double r = sqrt(r2);
    return sf * sf * (1.0 + sqrt(3.0) * r) * exp(-sqrt(3.0) * r);
}

/*
 * Partial derivative of k(x, x') with respect to theta_p, p in [0, d+1]:
 *   p <  d : d k / d l_p   (chain rule through r)
 *   p == d : d k / d s_f = 2 k / s_f
 *   p == d+1 (sigma): 0 for the kernel; the noise part of H is handled by
 *            gpo_dH_entry.
 * RBF:      dk/dl_p = k * (x_p - x'_p)^2 / l_p^3
 * Matern32: dk/dr = -3 s_f^2 r exp(-sqrt3 r), dr/dl_p = -(x_p-x'_p)^2 / (r l_p^3)
 *           => dk/dl_p = 3 s_f^2 exp(-sqrt3 r) (x_p-x'_p)^2 / l_p^3
 */
double gpo_dkernel(int kind, int d, const double *theta, const double *x, const double *xp, int p)
{
    double sf = theta[d];
    if (p == d + 1)
        return 0.0;
    if (p == d)
        return 2.0 * gpo_kernel(kind, d, theta, x, xp) / sf;
    double diff = x[p] - xp[p];
    double ell = theta[p];
    double w = diff * diff / (ell * ell * ell);
    double r2 = sqdist(d, theta, x, xp);
    if (kind == GPO_RBF)
        return sf * sf * exp(-0.5 * r2) * w;
    return 3.0 * sf * sf * exp(-sqrt(3.0) * sqrt(r2)) * w;
}

/* Entry (i, j) of dH/dtheta_p, H = K + sigma^2 I (Sec. 2, Eq. mll_grad; App. A.1). */
static double gpo_dH_entry(int kind, int d, const double *theta, const double *X, int64_t i, int64_t j, int p)
{
    if (p == d + 1)
        return (i == j) ? 2.0 * theta[d + 1] : 0.0;
    return gpo_dkernel(kind, d, theta, X + i * d, X + j * d, p);
}

/* Dense K(X1, X2): n1 x n2 row-major. */
void gpo_kernel_matrix(int kind, int d, const double *theta, const double *X1, int64_t n1,
                       const double *X2, int64_t n2, double *K)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n1; ++i)
        for (int64_t j = 0; j < n2; ++j)
            K[i * n2 + j] = gpo_kernel(kind, d, theta, X1 + i * d, X2 + j * d);
}

/* Dense H = K(X, X) + sigma^2 I: n x n row-major. */
void gpo_H_matrix(int kind, int d, const double *theta, const double *X, int64_t n, double *H)
{
    double s2 = theta[d + 1] * theta[d + 1];
    gpo_kernel_matrix(kind, d, theta, X, n, X, n, H);
    for (int64_t i = 0; i < n; ++i)
        H[i * n + i] += s2;
}

/* Dense dH/dtheta_p: n x n row-major. */
void gpo_dH_matrix(int kind, int d, const double *theta, const double *X, int64_t n, int p, double *dH)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            dH[i * n + j] = gpo_dH_entry(kind, d, theta, X, i, j, p);
}

/*
 * Matrix-free product (the operator every solver uses, Alg. 1-3 "Linear operator
 * H(.)"):  Y[c] = K(X1, X2) V[c]  (+ sigma^2 V[c] when add_noise, which requires
 * X1 == X2, i.e. n1 == n2 and the same points).  V: R x n2, Y: R x n1.
 * Only rows listed in `rows` (nrows of them) are produced when rows != NULL;
 * then Y is R x nrows.  This is how the oracle evaluates sampled rows at sizes
 * where the full product would take too long.
 */
void gpo_kernel_mvm(int kind, int d, const double *theta, const double *X1, int64_t n1,
                    const double *X2, int64_t n2, const double *V, int R, int add_noise,
                    const int64_t *rows, int64_t nrows, double *Y)
{
    int64_t nout = rows ? nrows : n1;
    double s2 = theta[d + 1] * theta[d + 1];
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)R);
#pragma omp for schedule(dynamic, 16)
        for (int64_t o = 0; o < nout; ++o) {
            int64_t i = rows ? rows[o] : o;
            for (int c = 0; c < R; ++c)
                acc[c] = 0.0;
            for (int64_t j = 0; j < n2; ++j) {
                double kij = gpo_kernel(kind, d, theta, X1 + i * d, X2 + j * d);
                for (int c = 0; c < R; ++c)
                    acc[c] += kij * V[(int64_t)c * n2 + j];
            }
            for (int c = 0; c < R; ++c) {
                double y = acc[c];
                if (add_noise)
                    y += s2 * V[(int64_t)c * n2 + i];
                Y[(int64_t)c * nout + o] = y;
            }
        }
        free(acc);
    }
}

/* ------------------------------------------------------------------------- */
/* Dense linear algebra: Cholesky (for the exact MLL of Eq. mll and Alg. 2's   */
/* chol_solve)                                                                 */
/* ------------------------------------------------------------------------- */

/* In-place Cholesky A = L L^T (lower triangle overwritten with L, upper zeroed).
 * Returns 0 on success, k+1 if the k-th pivot is not positive. */
int gpo_cholesky(int64_t n, double *A)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; ++k)
            s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0))
            return (int)(j + 1);
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
#pragma omp parallel for schedule(static) if (n > 256)
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; ++k)
                t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            A[i * n + j] = 0.0;
    return 0;
}

/* Solve L L^T x = b for R right-hand sides stored R x n (in place). */
void gpo_chol_solve(int64_t n, const double *L, double *B, int R)
{
    for (int c = 0; c < R; ++c) {
        double *b = B + (int64_t)c * n;
        for (int64_t i = 0; i < n; ++i) { /* forward: L z = b */
            double t = b[i];
            for (int64_t k = 0; k < i; ++k)
                t -= L[i * n + k] * b[k];
            b[i] = t / L[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) { /* backward: L^T x = z */
            double t = b[i];
            for (int64_t k = i + 1; k < n; ++k)
                t -= L[k * n + i] * b[k];
            b[i] = t / L[i * n + i];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Exact log marginal likelihood and gradient (Sec. 2, Eq. mll, Eq. mll_grad)  */
/* ------------------------------------------------------------------------- */

/* L(theta) = -1/2 y^T H^-1 y - 1/2 log det H - n/2 log 2 pi.  Returns NAN if H
 * is not positive definite. */
double gpo_mll(int kind, int d, const double *theta, const double *X, int64_t n, const double *y)
{
    double *H = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *a = (double *)malloc(sizeof(double) * (size_t)n);
    gpo_H_matrix(kind, d, theta, X, n, H);
    if (gpo_cholesky(n, H) != 0) {
        free(H);
        free(a);
        return NAN;
    }
    memcpy(a, y, sizeof(double) * (size_t)n);
    gpo_chol_solve(n, H, a, 1);
    double quad = 0.0, logdet = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        quad += y[i] * a[i];
        logdet += 2.0 * log(H[i * n + i]);
    }
    free(H);
    free(a);
    return -0.5 * quad - 0.5 * logdet - 0.5 * (double)n * log(2.0 * M_PI);
}

/*
 * Exact gradient (Eq. mll_grad):
 *   g_p = 1/2 alpha^T (dH/dtheta_p) alpha - 1/2 tr(H^-1 dH/dtheta_p),  alpha = H^-1 y.
 * H^-1 is formed explicitly from the Cholesky factor; the trace is
 * sum_ij (H^-1)_ij (dH_p)_ji and dH_p is symmetric.  grad has d+2 entries.
 * Returns 0, or the failing Cholesky pivot.
 */
int gpo_mll_grad_exact(int kind, int d, const double *theta, const double *X, int64_t n,
                       const double *y, double *grad)
{
    double *L = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *Hinv = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *alpha = (double *)malloc(sizeof(double) * (size_t)n);
    gpo_H_matrix(kind, d, theta, X, n, L);
    int info = gpo_cholesky(n, L);
    if (info != 0) {
        free(L);
        free(Hinv);
        free(alpha);
        return info;
    }
    memcpy(alpha, y, sizeof(double) * (size_t)n);
    gpo_chol_solve(n, L, alpha, 1);
    memset(Hinv, 0, sizeof(double) * (size_t)(n * n));
    for (int64_t i = 0; i < n; ++i)
        Hinv[i * n + i] = 1.0;
    gpo_chol_solve(n, L, Hinv, (int)n); /* columns of the identity, stored as rows */
    for (int p = 0; p < d + 2; ++p) {
        double quad = 0.0, tr = 0.0;
#pragma omp parallel for reduction(+ : quad, tr) schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                double dh = gpo_dH_entry(kind, d, theta, X, i, j, p);
                quad += alpha[i] * dh * alpha[j];
                tr += Hinv[i * n + j] * dh;
            }
        grad[p] = 0.5 * quad - 0.5 * tr;
    }
    free(L);
    free(Hinv);
    free(alpha);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradient estimators (Eq. trace, Eq. pathwise_estimator) as bilinear forms   */
/* ------------------------------------------------------------------------- */

/*
 * grad_p = sum_c lambda_c * U[c]^T (dH/dtheta_p) W[c]   for p in [0, d+1].
 * U, W: R x n.  Matrix-free: every dH entry is evaluated on the fly.
 *   standard estimator (Eq. mll_grad + Eq. trace): U = [v_y, v_1..v_s],
 *      W = [v_y, z_1..z_s], lambda = [1/2, -1/(2s), ..., -1/(2s)]
 *   pathwise estimator (Eq. pathwise_estimator): U = W = [v_y, zhat_1..zhat_s],
 *      same lambda.
 */
void gpo_grad_bilinear(int kind, int d, const double *theta, const double *X, int64_t n,
                       const double *U, const double *W, const double *lambda, int R, double *grad)
{
    int P = d + 2;
    for (int p = 0; p < P; ++p)
        grad[p] = 0.0;
#pragma omp parallel
    {
        double *loc = (double *)calloc((size_t)P, sizeof(double));
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                /* M_ij = sum_c lambda_c U[c][i] W[c][j] */
                double m = 0.0;
                for (int c = 0; c < R; ++c)
                    m += lambda[c] * U[(int64_t)c * n + i] * W[(int64_t)c * n + j];
                for (int p = 0; p < P; ++p)
                    loc[p] += m * gpo_dH_entry(kind, d, theta, X, i, j, p);
            }
        }
#pragma omp critical
        for (int p = 0; p < P; ++p)
            grad[p] += loc[p];
        free(loc);
    }
}

/*
 * Value of the same bilinear form, f = sum_c lambda_c U[c]^T H W[c] with
 * H = K + sigma^2 I (Sec. 2), matrix-free.
 */
double gpo_bilinear_value(int kind, int d, const double *theta, const double *X, int64_t n,
                          const double *U, const double *W, const double *lambda, int R)
{
    double s2 = theta[d + 1] * theta[d + 1];
    double total = 0.0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : total)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double h = gpo_kernel(kind, d, theta, X + i * d, X + j * d) + (i == j ? s2 : 0.0);
            double m = 0.0;
            for (int c = 0; c < R; ++c)
                m += lambda[c] * U[(int64_t)c * n + i] * W[(int64_t)c * n + j];
            total += m * h;
        }
    }
    return total;
}

/*
 * RKHS squared distance between a solver initialisation and a solution (Sec. 3,
 * "Initial Distance to the Linear System Solution", Eq. RKHS_distance), one value
 * per column c:  dist[c] = (Uinit[c] - U[c])^T H (Uinit[c] - U[c]).
 * Uinit == NULL means the zero initialisation, so dist[c] = U[c]^T H U[c].
 */
void gpo_rkhs_sqdist(int kind, int d, const double *theta, const double *X, int64_t n,
                     const double *Uinit, const double *U, int R, double *dist)
{
    double s2 = theta[d + 1] * theta[d + 1];
    double *e = (double *)malloc(sizeof(double) * (size_t)n);
    for (int c = 0; c < R; ++c) {
        for (int64_t i = 0; i < n; ++i)
            e[i] = (Uinit ? Uinit[(int64_t)c * n + i] : 0.0) - U[(int64_t)c * n + i];
        double total = 0.0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : total)
        for (int64_t i = 0; i < n; ++i) {
            double row = 0.0;
            for (int64_t j = 0; j < n; ++j)
                row += (gpo_kernel(kind, d, theta, X + i * d, X + j * d) + (i == j ? s2 : 0.0)) * e[j];
            total += e[i] * row;
        }
        dist[c] = total;
    }
    free(e);
}

/*
 * Gradient of k(x, x') with respect to its first argument, g (d values).
 * By the chain rule through r (r^2 = sum_p (x_p - x'_p)^2 / l_p^2):
 *   RBF:      dk/dx_p = -k (x_p - x'_p) / l_p^2
 *   Matern32: dk/dr = -3 s_f^2 r exp(-sqrt3 r), dr/dx_p = (x_p - x'_p) / (r l_p^2)
 *             => dk/dx_p = -3 s_f^2 exp(-sqrt3 r) (x_p - x'_p) / l_p^2
 * (finite at r = 0, where it is 0).
 */
void gpo_dkernel_dx(int kind, int d, const double *theta, const double *x, const double *xp, double *g)
{
    double sf = theta[d];
    double r2 = sqdist(d, theta, x, xp);
    double rad;
    if (kind == GPO_RBF)
        rad = sf * sf * exp(-0.5 * r2);
    else
        rad = 3.0 * sf * sf * exp(-sqrt(3.0) * sqrt(r2));
    for (int p = 0; p < d; ++p)
        g[p] = -rad * (x[p] - xp[p]) / (theta[p] * theta[p]);
}

/*
 * Gradient of f(X) = sum_c lambda_c U[c]^T H(theta, X) W[c] with respect to the
 * points, dX (n x d).  With M_ab = sum_c lambda_c U[c][a] W[c][b],
 *   df/dx_a = sum_b M_ab d k(x_a, x_b)/d x_a + sum_b M_ba d k(x_b, x_a)/d x_a,
 * and for a stationary kernel d k(x_b, x_a)/d x_a = -d k(x_b, x_a)/d x_b
 * (k depends on x_b - x_a only).  sigma^2 I does not depend on X.
 */
void gpo_grad_bilinear_X(int kind, int d, const double *theta, const double *X, int64_t n,
                         const double *U, const double *W, const double *lambda, int R, double *dX)
{
#pragma omp parallel
    {
        double *g = (double *)malloc(sizeof(double) * (size_t)d);
#pragma omp for schedule(dynamic, 8)
        for (int64_t a = 0; a < n; ++a) {
            for (int p = 0; p < d; ++p)
                dX[a * d + p] = 0.0;
            for (int64_t b = 0; b < n; ++b) {
                double mab = 0.0, mba = 0.0;
                for (int c = 0; c < R; ++c) {
                    mab += lambda[c] * U[(int64_t)c * n + a] * W[(int64_t)c * n + b];
                    mba += lambda[c] * U[(int64_t)c * n + b] * W[(int64_t)c * n + a];
                }
                /* first argument: k(x_a, x_b) */
                gpo_dkernel_dx(kind, d, theta, X + a * d, X + b * d, g);
                for (int p = 0; p < d; ++p)
                    dX[a * d + p] += mab * g[p];
                /* second argument: k(x_b, x_a) */
                gpo_dkernel_dx(kind, d, theta, X + b * d, X + a * d, g);
                for (int p = 0; p < d; ++p)
                    dX[a * d + p] -= mba * g[p];
            }
        }
        free(g);
    }
}

void gpo_grad_standard(int kind, int d, const double *theta, const double *X, int64_t n,
                       const double *Vsol, const double *Z, int s, double *grad)
{
    /* U = [v_y, v_1..v_s] (the solutions), W = [v_y, z_1..z_s] (y-solution, probes) */
    int R = s + 1;
    double *W = (double *)malloc(sizeof(double) * (size_t)(R * n));
    double *lam = (double *)malloc(sizeof(double) * (size_t)R);
    memcpy(W, Vsol, sizeof(double) * (size_t)n);
    memcpy(W + n, Z, sizeof(double) * (size_t)(s * n));
    lam[0] = 0.5;
    for (int c = 1; c < R; ++c)
        lam[c] = -0.5 / (double)s;
    gpo_grad_bilinear(kind, d, theta, X, n, Vsol, W, lam, R, grad);
    free(W);
    free(lam);
}

void gpo_grad_pathwise(int kind, int d, const double *theta, const double *X, int64_t n,
                       const double *Vsol, int s, double *grad)
{
    int R = s + 1;
    double *lam = (double *)malloc(sizeof(double) * (size_t)R);
    lam[0] = 0.5;
    for (int c = 1; c < R; ++c)
        lam[c] = -0.5 / (double)s;
    gpo_grad_bilinear(kind, d, theta, X, n, Vsol, Vsol, lam, R, grad);
    free(lam);
}

/* ------------------------------------------------------------------------- */
/* Solvers (App. B, Alg. 1-3), each on the normalised systems of App. B        */
/* ------------------------------------------------------------------------- */

static double vnorm(const double *v, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += v[i] * v[i];
    return sqrt(s);
}

/* Split relative residual norms (App. B): ||r_y|| and ||r_z|| = mean_j ||r_j||. */
static void split_norms(const double *r, int64_t n, int R, double *ry, double *rz)
{
    *ry = vnorm(r, n);
    double acc = 0.0;
    for (int c = 1; c < R; ++c)
        acc += vnorm(r + (int64_t)c * n, n);
    *rz = (R > 1) ? acc / (double)(R - 1) : 0.0;
}

/* Loop condition of Alg. 1-3.  stop_rule 0: continue until both norms <= tau
 * (App. B text); stop_rule 1: the listing's conjunction (stop when either is). */
static int keep_going(int64_t t, int64_t tmax, double ry, double rz, double tol, int stop_rule)
{
    if (t >= tmax)
        return 0;
    if (stop_rule == 1)
        return ry > tol && rz > tol;
    return ry > tol || rz > tol;
}

typedef struct {
    int64_t iters;
    int converged;
    double res_y;
    double res_z;
} gpo_info_t;

#define GPO_EPS 1e-12

/* Normalise b and the warm start by (||b_c|| + eps) (App. B). */
static void normalise(const double *B, double *V, int64_t n, int R, double *bt, double *scale)
{
    for (int c = 0; c < R; ++c) {
        scale[c] = vnorm(B + (int64_t)c * n, n) + GPO_EPS;
        for (int64_t i = 0; i < n; ++i) {
            bt[(int64_t)c * n + i] = B[(int64_t)c * n + i] / scale[c];
            V[(int64_t)c * n + i] /= scale[c];
        }
    }
}

static void denormalise(double *V, int64_t n, int R, const double *scale)
{
    for (int c = 0; c < R; ++c)
        for (int64_t i = 0; i < n; ++i)
            V[(int64_t)c * n + i] *= scale[c];
}

/* y = H x for a dense row-major H (n x n), R vectors. */
static void dense_apply(const double *H, int64_t n, const double *X, double *Y, int R)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int c = 0; c < R; ++c)
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j)
                s += H[i * n + j] * X[(int64_t)c * n + j];
            Y[(int64_t)c * n + i] = s;
        }
}

/*
 * Alg. 1, conjugate gradients with P = identity, on H V = B (B: R x n).
 * V holds the warm start on entry (zeros for a cold start) and the solution on
 * exit.  H is built densely (the oracle runs at sizes where that is cheap).
 */
int gpo_solve_cg(int kind, int d, const double *theta, const double *X, int64_t n,
                 const double *B, int R, double *V, int64_t max_iters, double tol, int stop_rule,
                 gpo_info_t *info)
{
    size_t nn = (size_t)n, nr = (size_t)R * nn;
    double *H = malloc(sizeof(double) * nn * nn);
    double *bt = malloc(sizeof(double) * nr), *r = malloc(sizeof(double) * nr);
    double *dd = malloc(sizeof(double) * nr), *Hd = malloc(sizeof(double) * nr);
    double *scale = malloc(sizeof(double) * (size_t)R), *gamma = malloc(sizeof(double) * (size_t)R);
    gpo_H_matrix(kind, d, theta, X, n, H);
    normalise(B, V, n, R, bt, scale);
    dense_apply(H, n, V, Hd, R); /* r = b - H v */
    for (size_t e = 0; e < nr; ++e) {
        r[e] = bt[e] - Hd[e];
        dd[e] = r[e]; /* p = P(r) = r; d = p */
    }
    for (int c = 0; c < R; ++c) {
        double g = 0.0;
        for (int64_t i = 0; i < n; ++i)
            g += r[(int64_t)c * n + i] * r[(int64_t)c * n + i];
        gamma[c] = g;
    }
    int64_t t = 0;
    double ry, rz;
    split_norms(r, n, R, &ry, &rz);
    while (keep_going(t, max_iters, ry, rz, tol, stop_rule)) {
        dense_apply(H, n, dd, Hd, R);
        for (int c = 0; c < R; ++c) {
            double *vc = V + (int64_t)c * n, *rc = r + (int64_t)c * n;
            double *dc = dd + (int64_t)c * n, *hc = Hd + (int64_t)c * n;
            double dHd = 0.0;
            for (int64_t i = 0; i < n; ++i)
                dHd += dc[i] * hc[i];
            double alpha = (gamma[c] > 1e-30 && dHd > 0.0) ? gamma[c] / dHd : 0.0;
            for (int64_t i = 0; i < n; ++i) {
                vc[i] += alpha * dc[i];
                rc[i] -= alpha * hc[i];
            }
            double gnew = 0.0;
            for (int64_t i = 0; i < n; ++i)
                gnew += rc[i] * rc[i];
            double beta = (alpha != 0.0) ? gnew / gamma[c] : 0.0;
            if (alpha != 0.0)
                gamma[c] = gnew;
            for (int64_t i = 0; i < n; ++i)
                dc[i] = rc[i] + beta * dc[i];
        }
        t += 1;
        split_norms(r, n, R, &ry, &rz);
    }
    denormalise(V, n, R, scale);
    info->iters = t;
    info->res_y = ry;
    info->res_z = rz;
    info->converged = !(ry > tol || rz > tol) || (stop_rule == 1 && (ry <= tol || rz <= tol));
    free(H); free(bt); free(r); free(dd); free(Hd); free(scale); free(gamma);
    return 0;
}

/*
 * Rank-k pivoted Cholesky factor of K (App. B "Conjugate Gradients": rank-100 pivoted
 * Cholesky preconditioner, following Wang et al. 2019 / Gardner et al. 2018; the greedy
 * algorithm of Harbrecht, Peters and Schneider 2012).  Starting from the diagonal of K, step m
 * picks the not yet chosen point p with the largest remaining diagonal (ties: lowest index),
 * sets row m of L to (k(x_j, x_p) - sum_{l<m} L[l][j] L[l][p]) / sqrt(diag_p) for every j and
 * subtracts its square from the remaining diagonal.  L is k x n (row m = m-th factor column),
 * K ~ L^T L.  Returns the rank reached (< k if the remaining diagonal vanishes); pivots in piv.
 */
int gpo_pivoted_cholesky(int kind, int d, const double *theta, const double *X, int64_t n, int k,
                         double *L, int64_t *piv)
{
    double *dg = malloc(sizeof(double) * (size_t)n);
    char *used = calloc((size_t)n, 1);
    for (int64_t j = 0; j < n; ++j)
        dg[j] = gpo_kernel(kind, d, theta, X + j * d, X + j * d);
    int m = 0;
    for (; m < k; ++m) {
        int64_t p = -1;
        for (int64_t j = 0; j < n; ++j)
            if (!used[j] && (p < 0 || dg[j] > dg[p]))
                p = j;
        if (p < 0 || !(dg[p] > 0.0))
            break;
        used[p] = 1;
        piv[m] = p;
        double lpp = sqrt(dg[p]);
        for (int64_t j = 0; j < n; ++j) {
            double v = gpo_kernel(kind, d, theta, X + j * d, X + p * d);
            for (int l = 0; l < m; ++l)
                v -= L[(int64_t)l * n + j] * L[(int64_t)l * n + p];
            L[(int64_t)m * n + j] = v / lpp;
        }
        for (int64_t j = 0; j < n; ++j)
            dg[j] -= L[(int64_t)m * n + j] * L[(int64_t)m * n + j];
    }
    free(dg);
    free(used);
    return m;
}

/*
 * Alg. 1 with a preconditioner P (App. B "Conjugate Gradients"): P = L^T L + sigma^2 I from the
 * rank-k pivoted Cholesky factor above (k = 0: P = I, plain CG).  The loop follows the listing:
 * p = P^-1 r, d = p, gamma = r^T p; alpha = gamma / d^T H d; v += alpha d; r -= alpha H d;
 * p = P^-1 r; beta = r^T p / gamma; gamma = r^T p; d = p + beta d.  P^-1 is applied through a
 * dense Cholesky factor of P.  Normalisation, split norms (of r), stop rule and the frozen-column
 * rule as gpo_solve_cg.
 */
int gpo_solve_pcg(int kind, int d, const double *theta, const double *X, int64_t n,
                  const double *B, int R, double *V, int k, int64_t max_iters, double tol, int stop_rule,
                  gpo_info_t *info)
{
    size_t nn = (size_t)n, nr = (size_t)R * nn;
    double *H = malloc(sizeof(double) * nn * nn), *P = malloc(sizeof(double) * nn * nn);
    double *bt = malloc(sizeof(double) * nr), *r = malloc(sizeof(double) * nr), *pz = malloc(sizeof(double) * nr);
    double *dd = malloc(sizeof(double) * nr), *Hd = malloc(sizeof(double) * nr);
    double *scale = malloc(sizeof(double) * (size_t)R), *gamma = malloc(sizeof(double) * (size_t)R);
    double *L = malloc(sizeof(double) * (size_t)(k > 0 ? k : 1) * nn);
    int64_t *piv = malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    gpo_H_matrix(kind, d, theta, X, n, H);
    int rank = k > 0 ? gpo_pivoted_cholesky(kind, d, theta, X, n, k, L, piv) : 0;
    double s2 = theta[d + 1] * theta[d + 1];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double v = (i == j) ? s2 : 0.0;
            for (int l = 0; l < rank; ++l)
                v += L[(int64_t)l * n + i] * L[(int64_t)l * n + j];
            P[i * n + j] = v;
        }
    if (gpo_cholesky(n, P) != 0) {
        free(H); free(P); free(bt); free(r); free(pz); free(dd); free(Hd); free(scale); free(gamma); free(L);
        free(piv);
        return -1;
    }
    normalise(B, V, n, R, bt, scale);
    dense_apply(H, n, V, Hd, R);
    for (size_t e = 0; e < nr; ++e)
        r[e] = bt[e] - Hd[e];
    memcpy(pz, r, sizeof(double) * nr);
    gpo_chol_solve(n, P, pz, R); /* p = P^-1 r */
    memcpy(dd, pz, sizeof(double) * nr);
    for (int c = 0; c < R; ++c) {
        double g = 0.0;
        for (int64_t i = 0; i < n; ++i)
            g += r[(int64_t)c * n + i] * pz[(int64_t)c * n + i];
        gamma[c] = g;
    }
    int64_t t = 0;
    double ry, rz;
    split_norms(r, n, R, &ry, &rz);
    while (keep_going(t, max_iters, ry, rz, tol, stop_rule)) {
        dense_apply(H, n, dd, Hd, R);
        double *alpha = malloc(sizeof(double) * (size_t)R);
        for (int c = 0; c < R; ++c) {
            double *vc = V + (int64_t)c * n, *rc = r + (int64_t)c * n;
            double *dc = dd + (int64_t)c * n, *hc = Hd + (int64_t)c * n;
            double dHd = 0.0;
            for (int64_t i = 0; i < n; ++i)
                dHd += dc[i] * hc[i];
            alpha[c] = (gamma[c] > 1e-30 && dHd > 0.0) ? gamma[c] / dHd : 0.0;
            for (int64_t i = 0; i < n; ++i) {
                vc[i] += alpha[c] * dc[i];
                rc[i] -= alpha[c] * hc[i];
            }
        }
        memcpy(pz, r, sizeof(double) * nr);
        gpo_chol_solve(n, P, pz, R);
        for (int c = 0; c < R; ++c) {
            double *rc = r + (int64_t)c * n, *pc = pz + (int64_t)c * n, *dc = dd + (int64_t)c * n;
            double gnew = 0.0;
            for (int64_t i = 0; i < n; ++i)
                gnew += rc[i] * pc[i];
            double beta = (alpha[c] != 0.0) ? gnew / gamma[c] : 0.0;
            if (alpha[c] != 0.0)
                gamma[c] = gnew;
            for (int64_t i = 0; i < n; ++i)
                dc[i] = pc[i] + beta * dc[i];
        }
        free(alpha);
        t += 1;
        split_norms(r, n, R, &ry, &rz);
    }
    denormalise(V, n, R, scale);
    info->iters = t;
    info->res_y = ry;
    info->res_z = rz;
    info->converged = !(ry > tol || rz > tol) || (stop_rule == 1 && (ry <= tol || rz <= tol));
    free(H); free(P); free(bt); free(r); free(pz); free(dd); free(Hd); free(scale); free(gamma); free(L); free(piv);
    return 0;
}

/*
 * Alg. 2, alternating projections with block size bs.  Each iteration picks the
 * block with the largest ||sum_c r_c[i]||, solves its diagonal block exactly by
 * the cached Cholesky factor, updates v on that block and r everywhere.
 * Returns 0, or a negative value if a diagonal block is not positive definite.
 */
int gpo_solve_ap(int kind, int d, const double *theta, const double *X, int64_t n,
                 const double *B, int R, double *V, int64_t block_size, int64_t max_iters,
                 double tol, int stop_rule, gpo_info_t *info)
{
    size_t nn = (size_t)n, nr = (size_t)R * nn;
    int64_t nb = (n + block_size - 1) / block_size;
    double *H = malloc(sizeof(double) * nn * nn);
    double *bt = malloc(sizeof(double) * nr), *r = malloc(sizeof(double) * nr);
    double *Hv = malloc(sizeof(double) * nr), *scale = malloc(sizeof(double) * (size_t)R);
    double **chol = calloc((size_t)nb, sizeof(double *));
    double *delta = malloc(sizeof(double) * (size_t)R * (size_t)block_size);
    gpo_H_matrix(kind, d, theta, X, n, H);
    /* cache the Cholesky factor of every diagonal block H[i, i] */
    for (int64_t blk = 0; blk < nb; ++blk) {
        int64_t lo = blk * block_size, m = (lo + block_size <= n) ? block_size : n - lo;
        chol[blk] = malloc(sizeof(double) * (size_t)(m * m));
        for (int64_t a = 0; a < m; ++a)
            for (int64_t b = 0; b < m; ++b)
                chol[blk][a * m + b] = H[(lo + a) * n + (lo + b)];
        if (gpo_cholesky(m, chol[blk]) != 0) {
            for (int64_t q = 0; q <= blk; ++q)
                free(chol[q]);
            free(chol); free(H); free(bt); free(r); free(Hv); free(scale); free(delta);
            return -1;
        }
    }
    normalise(B, V, n, R, bt, scale);
    dense_apply(H, n, V, Hv, R);
    for (size_t e = 0; e < nr; ++e)
        r[e] = bt[e] - Hv[e];
    int64_t t = 0;
    double ry, rz;
    split_norms(r, n, R, &ry, &rz);
    while (keep_going(t, max_iters, ry, rz, tol, stop_rule)) {
        /* block selection: argmax_i || r_y[i] + sum_j r_j[i] || */
        int64_t best = 0;
        double best_score = -1.0;
        for (int64_t blk = 0; blk < nb; ++blk) {
            int64_t lo = blk * block_size, hi = (lo + block_size <= n) ? lo + block_size : n;
            double sc = 0.0;
            for (int64_t i = lo; i < hi; ++i) {
                double sum = 0.0;
                for (int c = 0; c < R; ++c)
                    sum += r[(int64_t)c * n + i];
                sc += sum * sum;
            }
            sc = sqrt(sc);
            if (sc > best_score) {
                best_score = sc;
                best = blk;
            }
        }
        int64_t lo = best * block_size, m = (lo + block_size <= n) ? block_size : n - lo;
        /* delta = chol_solve(H[i,i], r[i]) */
        for (int c = 0; c < R; ++c)
            for (int64_t a = 0; a < m; ++a)
                delta[(int64_t)c * m + a] = r[(int64_t)c * n + lo + a];
        gpo_chol_solve(m, chol[best], delta, R);
        /* v[i] += delta ; r -= H[:, i] delta */
        for (int c = 0; c < R; ++c) {
            for (int64_t a = 0; a < m; ++a)
                V[(int64_t)c * n + lo + a] += delta[(int64_t)c * m + a];
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n; ++i) {
                double s = 0.0;
                for (int64_t a = 0; a < m; ++a)
                    s += H[i * n + lo + a] * delta[(int64_t)c * m + a];
                r[(int64_t)c * n + i] -= s;
            }
        }
        t += 1;
        split_norms(r, n, R, &ry, &rz);
    }
    denormalise(V, n, R, scale);
    info->iters = t;
    info->res_y = ry;
    info->res_z = rz;
    info->converged = !(ry > tol || rz > tol) || (stop_rule == 1 && (ry <= tol || rz <= tol));
    for (int64_t q = 0; q < nb; ++q)
        free(chol[q]);
    free(chol); free(H); free(bt); free(r); free(Hv); free(scale); free(delta);
    return 0;
}

/*
 * Alg. 3, stochastic gradient descent with momentum (no Polyak averaging).
 *   g = 0; g[i] = H[i, :] v - b[i];  m = rho m - (lr / b) g;  v = v + m;  r[i] = g[i]
 * idx holds max_iters * batch row indices; iteration t uses idx[t*batch ...].
 * The loop condition uses the residual heuristic r (App. B "Stochastic Gradient
 * Descent").  The momentum starts at zero, as in the listing.
 */
int gpo_solve_sgd(int kind, int d, const double *theta, const double *X, int64_t n,
                  const double *B, int R, double *V, int64_t batch, const int64_t *idx,
                  double lr, double rho, int64_t max_iters, double tol, int stop_rule,
                  gpo_info_t *info)
{
    size_t nn = (size_t)n, nr = (size_t)R * nn;
    double *bt = malloc(sizeof(double) * nr), *r = malloc(sizeof(double) * nr);
    double *m = calloc(nr, sizeof(double)), *g = calloc(nr, sizeof(double));
    double *scale = malloc(sizeof(double) * (size_t)R);
    double s2 = theta[d + 1] * theta[d + 1];
    normalise(B, V, n, R, bt, scale);
    memcpy(r, bt, sizeof(double) * nr); /* r <- b */
    int64_t t = 0;
    double ry, rz;
    split_norms(r, n, R, &ry, &rz);
    while (keep_going(t, max_iters, ry, rz, tol, stop_rule)) {
        const int64_t *bi = idx + t * batch;
        memset(g, 0, sizeof(double) * nr);
        for (int64_t q = 0; q < batch; ++q) { /* g[i] = H[i, :] v - b[i] */
            int64_t i = bi[q];
            for (int c = 0; c < R; ++c) {
                double s = 0.0;
                for (int64_t j = 0; j < n; ++j)
                    s += gpo_kernel(kind, d, theta, X + i * d, X + j * d) * V[(int64_t)c * n + j];
                s += s2 * V[(int64_t)c * n + i];
                g[(int64_t)c * n + i] = s - bt[(int64_t)c * n + i];
            }
        }
        for (size_t e = 0; e < nr; ++e) {
            m[e] = rho * m[e] - (lr / (double)batch) * g[e];
            V[e] += m[e];
        }
        for (int64_t q = 0; q < batch; ++q) {
            int64_t i = bi[q];
            for (int c = 0; c < R; ++c)
                r[(int64_t)c * n + i] = g[(int64_t)c * n + i];
        }
        t += 1;
        split_norms(r, n, R, &ry, &rz);
    }
    denormalise(V, n, R, scale);
    info->iters = t;
    info->res_y = ry;
    info->res_z = rz;
    info->converged = !(ry > tol || rz > tol) || (stop_rule == 1 && (ry <= tol || rz <= tol));
    free(bt); free(r); free(m); free(g); free(scale);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Random Fourier features and pathwise conditioning                           */
/* (Sec. 2 "Pathwise Conditioning", Sec. 3 "Amortising Linear Solves", App. B)  */
/* ------------------------------------------------------------------------- */

/*
 * F[j][i] = f_j(x_i) = s_f sqrt(2/m) sum_{l < m/2} [ W[j][l] cos(w_l . x_i)
 *                                                 + W[j][m/2 + l] sin(w_l . x_i) ]
 * omega_hat: (m/2) x d standard normal; chi2: m/2 chi^2_3 draws (Matern only);
 * W: s x m standard normal; F: s x n.
 */
void gpo_rff_prior(int kind, int d, const double *theta, const double *X, int64_t n, int m,
                   const double *omega_hat, const double *chi2, const double *W, int s, double *F)
{
    int h = m / 2;
    double sf = theta[d];
    double *omega = malloc(sizeof(double) * (size_t)h * (size_t)d);
    for (int l = 0; l < h; ++l) {
        double t = (kind == GPO_MATERN32) ? sqrt(3.0 / chi2[l]) : 1.0;
        for (int k = 0; k < d; ++k)
            omega[l * d + k] = omega_hat[l * d + k] / theta[k] * t;
    }
    double amp = sf * sqrt(2.0 / (double)m);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < s; ++j)
            F[(int64_t)j * n + i] = 0.0;
        for (int l = 0; l < h; ++l) {
            double arg = 0.0;
            for (int k = 0; k < d; ++k)
                arg += omega[l * d + k] * X[i * d + k];
            double cs = cos(arg), sn = sin(arg);
            for (int j = 0; j < s; ++j)
                F[(int64_t)j * n + i] += amp * (W[(int64_t)j * m + l] * cs + W[(int64_t)j * m + h + l] * sn);
        }
    }
    free(omega);
}

/*
 * Pathwise-conditioned posterior samples (Eq. pathwise_conditioning, Sec. 3):
 *   out[j](x*) = f_j(x*) + k(x*, X) (v_y - zhat_j),   j = 1..s
 * Fstar: s x nstar prior samples at X*, Vsol: (s+1) x n = [v_y, zhat_1..zhat_s],
 * out: s x nstar.
 */
void gpo_posterior_samples(int kind, int d, const double *theta, const double *Xstar, int64_t nstar,
                           const double *X, int64_t n, const double *Vsol, int s,
                           const double *Fstar, double *out)
{
    double *Wd = malloc(sizeof(double) * (size_t)s * (size_t)n);
    for (int j = 0; j < s; ++j)
        for (int64_t i = 0; i < n; ++i)
            Wd[(int64_t)j * n + i] = Vsol[i] - Vsol[(int64_t)(j + 1) * n + i];
    gpo_kernel_mvm(kind, d, theta, Xstar, nstar, X, n, Wd, s, 0, NULL, 0, out);
    for (int64_t e = 0; e < (int64_t)s * nstar; ++e)
        out[e] += Fstar[e];
    free(Wd);
}

/* ------------------------------------------------------------------------- */
/* Outer loop (Sec. 2.1 "Outer-Loop Optimiser"; App. B "Iterative Optimiser")   */
/* ------------------------------------------------------------------------- */

/*
 * Predictions from the pathwise solutions (Sec. 3 "Amortising Linear Solves for Optimisation
 * and Prediction"; App. B reports test RMSE and test log-likelihood).  At the test points x*:
 *   mean_i = k(x*_i, X) v_y                                  (the posterior mean)
 *   var_i  = (1/s) sum_j ((f|y)_j(x*_i) - mean_i)^2 + sigma^2, where
 *            (f|y)_j(x*) - mean(x*) = f_j(x*) - k(x*, X) zhat_j  (pathwise conditioning)
 * i.e. the predictive variance of y* from the s posterior samples around the exact mean plus
 * the noise.  With test targets ystar (may be NULL): metrics[0] = RMSE =
 * sqrt(mean_i (ystar_i - mean_i)^2), metrics[1] = mean_i log N(ystar_i; mean_i, var_i).
 * The paper does not print these formulas; this is the reading used throughout.
 * Vsol: (s+1) x n = [v_y, zhat_1..zhat_s]; Fstar: s x nstar prior samples at x*.
 */
void gpo_predict(int kind, int d, const double *theta, const double *Xstar, int64_t nstar,
                 const double *X, int64_t n, const double *Vsol, int s, const double *Fstar,
                 const double *ystar, double *mean, double *var, double *metrics)
{
    int R = s + 1;
    double *M = (double *)malloc(sizeof(double) * (size_t)R * (size_t)nstar);
    gpo_kernel_mvm(kind, d, theta, Xstar, nstar, X, n, Vsol, R, 0, NULL, 0, M);
    double s2 = theta[d + 1] * theta[d + 1];
    double se = 0.0, ll = 0.0;
    for (int64_t i = 0; i < nstar; ++i) {
        mean[i] = M[i];
        double acc = 0.0;
        for (int j = 0; j < s; ++j) {
            double dev = Fstar[(int64_t)j * nstar + i] - M[(int64_t)(j + 1) * nstar + i];
            acc += dev * dev;
        }
        var[i] = acc / (double)s + s2;
        if (ystar) {
            double e = ystar[i] - mean[i];
            se += e * e;
            ll += -0.5 * log(2.0 * M_PI * var[i]) - 0.5 * e * e / var[i];
        }
    }
    if (metrics && ystar && nstar > 0) {
        metrics[0] = sqrt(se / (double)nstar);
        metrics[1] = ll / (double)nstar;
    }
    free(M);
}

/*
 * One Adam ascent step on nu with theta = softplus(nu) = log(1 + e^nu):
 *   g_nu = g_theta * sigmoid(nu)
 *   m = b1 m + (1-b1) g_nu ;  v = b2 v + (1-b2) g_nu^2
 *   nu += lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)      (t >= 1)
 * theta_out = softplus(nu) after the step.
 */
void gpo_adam_softplus(int P, double *nu, double *m, double *v, int64_t t, const double *grad_theta,
                       double lr, double b1, double b2, double eps, double *theta_out)
{
    for (int p = 0; p < P; ++p) {
        double sig = 1.0 / (1.0 + exp(-nu[p]));
        double g = grad_theta[p] * sig;
        m[p] = b1 * m[p] + (1.0 - b1) * g;
        v[p] = b2 * v[p] + (1.0 - b2) * g * g;
        double mh = m[p] / (1.0 - pow(b1, (double)t));
        double vh = v[p] / (1.0 - pow(b2, (double)t));
        nu[p] += lr * mh / (sqrt(vh) + eps);
        theta_out[p] = (nu[p] > 30.0) ? nu[p] : log1p(exp(nu[p]));
    }
}
