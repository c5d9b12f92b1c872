"""Pins for the oracle's gradient estimators (Eq. trace, Eq. pathwise_estimator)
and its random-feature prior / pathwise-conditioning samples (Sec. 2, Sec. 3,
App. B).  Deterministic pins use probe sets for which the estimators are exact;
statistical pins use the exact variances of App. A.1 to set z-score bounds."""
import numpy as np
import pytest

import oracle


def _setup(kind, n=24, d=3, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.6, 1.4, size=d), [1.1, 0.5]])
    y = rng.standard_normal(n)
    return rng, X, th, y


def _sqrtm_inv(H):
    lam, Q = np.linalg.eigh(H)
    return (Q / np.sqrt(lam)) @ Q.T


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_standard_estimator_exact_with_basis_probes(kind):
    """With s = n probes z_j = sqrt(n) e_j, (1/s) sum z_j^T H^-1 dH z_j = tr(H^-1 dH)."""
    rng, X, th, y = _setup(kind)
    n = X.shape[0]
    H = oracle.H_matrix(kind, th, X)
    Z = np.sqrt(n) * np.eye(n)
    V = np.linalg.solve(H, np.vstack([y, Z]).T).T
    g = oracle.grad_standard(kind, th, X, V, Z)
    np.testing.assert_allclose(g, oracle.mll_grad_exact(kind, th, X, y), rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_pathwise_estimator_exact_with_whitened_basis_probes(kind):
    """With zhat_j = H^-1/2 sqrt(n) e_j (second moment H^-1), the pathwise estimator
    equals tr(H^-1/2 dH H^-1/2) = tr(H^-1 dH)."""
    rng, X, th, y = _setup(kind, seed=1)
    n = X.shape[0]
    H = oracle.H_matrix(kind, th, X)
    Zhat = (np.sqrt(n) * _sqrtm_inv(H)).T
    V = np.vstack([np.linalg.solve(H, y), Zhat])
    g = oracle.grad_pathwise(kind, th, X, V)
    np.testing.assert_allclose(g, oracle.mll_grad_exact(kind, th, X, y), rtol=1e-9, atol=1e-11)


def test_bilinear_form_matches_dense_derivative_matrices():
    rng, X, th, y = _setup(oracle.MATERN32, n=15, seed=2)
    d = X.shape[1]
    U = rng.standard_normal((3, 15))
    W = rng.standard_normal((3, 15))
    lam = np.array([0.5, -0.25, 2.0])
    g = oracle.grad_bilinear(oracle.MATERN32, th, X, U, W, lam)
    for p in range(d + 2):
        # dense dH from central differences of H (independent of the derivative formulas)
        h = 1e-6 * th[p]
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        dH = (oracle.H_matrix(oracle.MATERN32, tp, X) - oracle.H_matrix(oracle.MATERN32, tm, X)) / (2 * h)
        ref = sum(lam[c] * U[c] @ dH @ W[c] for c in range(3))
        assert g[p] == pytest.approx(ref, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("estimator", ["standard", "pathwise"])
def test_estimators_unbiased_within_exact_variance_bound(estimator):
    """Mean over N single-probe estimates of the trace term lies within 4 standard
    errors of tr(H^-1 dH); the standard errors come from App. A.1's variances."""
    kind = oracle.MATERN32
    rng, X, th, y = _setup(kind, n=12, d=2, seed=3)
    n, d = X.shape
    H = oracle.H_matrix(kind, th, X)
    Hinv = np.linalg.inv(H)
    L = np.linalg.cholesky(H)
    N = 3000
    ests = np.empty((N, d + 2))
    for t in range(N):
        if estimator == "standard":
            z = rng.standard_normal(n)
            v = Hinv @ z
            ests[t] = oracle.grad_bilinear(kind, th, X, v[None], z[None], np.ones(1))
        else:
            xi = L @ rng.standard_normal(n)  # exact prior + noise draw, xi ~ N(0, H)
            zh = Hinv @ xi
            ests[t] = oracle.grad_bilinear(kind, th, X, zh[None], zh[None], np.ones(1))
    for p in range(d + 2):
        dH = oracle.dH_matrix(kind, th, X, p)
        A = Hinv @ dH
        tr = np.trace(A)
        if estimator == "standard":
            var = np.trace(A @ A) + np.trace(A @ A.T)
        else:
            var = 2.0 * np.trace(dH @ Hinv @ dH @ Hinv)
        se = np.sqrt(var / N)
        assert abs(ests[:, p].mean() - tr) < 4.0 * se + 1e-12
        # the sample variance agrees with the exact variance (chi-square spread, loose)
        assert ests[:, p].var() == pytest.approx(var, rel=0.2)


def test_noise_component_variances_are_equal():
    """App. A.1: for dH/dsigma = 2 sigma I both estimators have the same variance."""
    rng, X, th, y = _setup(oracle.RBF, n=10, d=2, seed=4)
    H = oracle.H_matrix(oracle.RBF, th, X)
    Hinv = np.linalg.inv(H)
    dH = oracle.dH_matrix(oracle.RBF, th, X, X.shape[1] + 1)
    np.testing.assert_allclose(dH, 2 * th[-1] * np.eye(10), rtol=1e-15)
    A = Hinv @ dH
    v_std = np.trace(A @ A) + np.trace(A @ A.T)
    v_path = 2 * np.trace(dH @ Hinv @ dH @ Hinv)
    assert v_std == pytest.approx(v_path, rel=1e-12)


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_rff_feature_inner_product_approximates_kernel(kind):
    """With unit weight vectors the s = m samples are the individual features, so
    sum_j f_j(x) f_j(x') is the random-feature kernel estimate, which converges to
    k(x, x') (Bochner; Student-t frequencies for Matern-3/2) at rate 1/sqrt(m/2)."""
    rng = np.random.default_rng(5)
    d = 3
    th = np.array([0.7, 1.3, 1.0, 1.4, 0.2])
    X = rng.standard_normal((6, d)) * 0.8
    m = 10000
    omega_hat = rng.standard_normal((m // 2, d))
    chi2 = rng.chisquare(3.0, size=m // 2)
    F = oracle.rff_prior(kind, th, X, omega_hat, chi2, np.eye(m))
    K_rff = F.T @ F
    K = oracle.kernel_matrix(kind, th, X, X)
    np.testing.assert_allclose(np.diag(K_rff), th[d] ** 2, rtol=1e-12)  # cos^2 + sin^2 = 1
    assert np.abs(K_rff - K).max() < 5.0 * th[d] ** 2 / np.sqrt(m / 2)


def test_rff_matern_and_rbf_are_distinguishable():
    """Guard against a wrong frequency law: at |x - x'| = 0.5 l the two kernels differ
    by about 0.1, far more than the Monte Carlo error of the feature estimate."""
    rng = np.random.default_rng(6)
    th = np.array([1.0, 1.0, 0.1])
    X = np.array([[0.0], [0.5]])
    m = 8000
    omega_hat = rng.standard_normal((m // 2, 1))
    chi2 = rng.chisquare(3.0, size=m // 2)
    for kind in (oracle.RBF, oracle.MATERN32):
        F = oracle.rff_prior(kind, th, X, omega_hat, chi2, np.eye(m))
        k01 = (F.T @ F)[0, 1]
        assert k01 == pytest.approx(oracle.kernel(kind, th, X[0], X[1]), abs=0.045)
    assert abs(oracle.kernel(oracle.RBF, th, X[0], X[1]) - oracle.kernel(oracle.MATERN32, th, X[0], X[1])) > 0.09


def test_posterior_samples_mean_and_covariance():
    """Pathwise conditioning (Eq. pathwise_conditioning, Sec. 3): with exact solves,
    sample mean -> k(x*, X) H^-1 y and sample covariance -> Eq. gp_posterior."""
    rng = np.random.default_rng(7)
    kind = oracle.RBF
    d, n, ns, s, m = 2, 20, 5, 3000, 8000
    th = np.array([0.8, 1.1, 1.0, 0.3])
    X = rng.uniform(-1, 1, size=(n, d))
    Xs = rng.uniform(-1, 1, size=(ns, d))
    y = rng.standard_normal(n)
    omega_hat = rng.standard_normal((m // 2, d))
    W = rng.standard_normal((s, m))
    Xall = np.vstack([X, Xs])
    Fall = oracle.rff_prior(kind, th, Xall, omega_hat, None, W)
    F, Fs = Fall[:, :n], Fall[:, n:]
    xi = F + th[-1] * rng.standard_normal((s, n))
    H = oracle.H_matrix(kind, th, X)
    Vsol = np.linalg.solve(H, np.vstack([y, xi]).T).T
    out = oracle.posterior_samples(kind, th, Xs, X, Vsol, Fs)
    Ksx = oracle.kernel_matrix(kind, th, Xs, X)
    mu = Ksx @ np.linalg.solve(H, y)
    # the random-feature prior has covariance Phi Phi^T (not exactly K), so compare
    # against the posterior implied by that prior on the same frequencies
    Phi = oracle.rff_prior(kind, th, Xall, omega_hat, None, np.eye(m))
    C = Phi.T @ Phi
    Cs, Csx = C[n:, n:], C[n:, :n]
    cov_ref = Cs - Csx @ np.linalg.solve(H, Ksx.T) - Ksx @ np.linalg.solve(H, Csx.T) \
        + Ksx @ np.linalg.solve(H, (C[:n, :n] + th[-1] ** 2 * np.eye(n)) @ np.linalg.solve(H, Ksx.T))
    sd = np.sqrt(np.diag(cov_ref))
    assert np.all(np.abs(out.mean(axis=0) - mu) < 5 * sd / np.sqrt(s) + 1e-9)
    cov = np.cov(out.T)
    assert np.abs(cov - cov_ref).max() < 6 * np.sqrt(2.0 / s) * sd.max() ** 2
    # and that random-feature posterior is close to the exact one of Eq. gp_posterior
    K_post = oracle.kernel_matrix(kind, th, Xs, Xs) - Ksx @ np.linalg.solve(H, Ksx.T)
    assert np.abs(cov_ref - K_post).max() < 0.05


def test_predictions_from_pathwise_solutions():
    """Predictions (Sec. 3, amortised through pathwise conditioning): the mean is the exact
    posterior mean k(x*, X) H^-1 y; the predictive variance from s samples converges to the
    exact posterior variance of the random-feature prior plus sigma^2; RMSE and test
    log-likelihood equal numpy / scipy evaluations of their definitions on that mean and
    variance."""
    from scipy.stats import norm

    rng = np.random.default_rng(8)
    kind = oracle.MATERN32
    d, n, ns, s, m = 2, 25, 6, 4000, 4000
    th = np.array([0.9, 1.2, 1.1, 0.3])
    X = rng.uniform(-1, 1, size=(n, d))
    Xs = rng.uniform(-1, 1, size=(ns, d))
    y = rng.standard_normal(n)
    ys = rng.standard_normal(ns)
    omega_hat = rng.standard_normal((m // 2, d))
    chi2 = rng.chisquare(3.0, size=m // 2)
    W = rng.standard_normal((s, m))
    Xall = np.vstack([X, Xs])
    Fall = oracle.rff_prior(kind, th, Xall, omega_hat, chi2, W)
    F, Fs = Fall[:, :n], Fall[:, n:]
    xi = F + th[-1] * rng.standard_normal((s, n))
    H = oracle.H_matrix(kind, th, X)
    Vsol = np.linalg.solve(H, np.vstack([y, xi]).T).T
    mean, var, (rmse, llh) = oracle.predict(kind, th, Xs, X, Vsol, Fs, ys)
    Ksx = oracle.kernel_matrix(kind, th, Xs, X)
    np.testing.assert_allclose(mean, Ksx @ np.linalg.solve(H, y), rtol=1e-9, atol=1e-12)
    # exact posterior variance under the random-feature prior covariance C = Phi Phi^T
    Phi = oracle.rff_prior(kind, th, Xall, omega_hat, chi2, np.eye(m))
    C = Phi.T @ Phi
    Cs, Csx = C[n:, n:], C[n:, :n]
    A = np.linalg.solve(H, Ksx.T)
    cov = Cs - Csx @ A - A.T @ Csx.T + A.T @ (C[:n, :n] + th[-1] ** 2 * np.eye(n)) @ A
    v_ref = np.diag(cov) + th[-1] ** 2
    # sample variance of s draws: relative standard error sqrt(2/s)
    assert np.all(np.abs(var / v_ref - 1) < 5 * np.sqrt(2.0 / s))
    np.testing.assert_allclose(rmse, np.sqrt(np.mean((ys - mean) ** 2)), rtol=1e-12)
    np.testing.assert_allclose(llh, np.mean(norm.logpdf(ys, loc=mean, scale=np.sqrt(var))), rtol=1e-12)
