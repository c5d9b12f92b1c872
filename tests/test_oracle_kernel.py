"""Pins for the oracle's kernel function, H, its derivatives, the exact MLL and
its gradient (Sec. 2, Eq. mll, Eq. mll_grad).  Every check compares against
something other than the oracle's own formula: library kernels (scikit-learn),
library densities (scipy), finite differences, eigenvalues and closed forms."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_18457_gb300 import workloads

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _theta(d, rng, sf=1.3, sigma=0.4):
    return np.concatenate([rng.uniform(0.4, 1.6, size=d), [sf, sigma]])


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_kernel_at_zero_distance_is_signal_variance(kind):
    rng = np.random.default_rng(0)
    th = _theta(5, rng, sf=1.7)
    x = rng.standard_normal(5)
    assert oracle.kernel(kind, th, x, x) == pytest.approx(1.7 ** 2, rel=1e-15)


@pytest.mark.parametrize("kind,nu", [(oracle.RBF, None), (oracle.MATERN32, 1.5)])
def test_kernel_matches_scikit_learn(kind, nu):
    sk = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(1)
    d = 4
    th = _theta(d, rng, sf=1.3)
    X1 = rng.standard_normal((7, d))
    X2 = rng.standard_normal((5, d))
    base = sk.RBF(length_scale=th[:d]) if kind == oracle.RBF else sk.Matern(length_scale=th[:d], nu=nu)
    K_ref = (sk.ConstantKernel(th[d] ** 2) * base)(X1, X2)
    K = oracle.kernel_matrix(kind, th, X1, X2)
    np.testing.assert_allclose(K, K_ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_H_symmetric_positive_definite_with_noise_floor(kind):
    rng = np.random.default_rng(2)
    th = _theta(3, rng, sigma=0.3)
    X = rng.uniform(0, 1, size=(40, 3))
    H = oracle.H_matrix(kind, th, X)
    np.testing.assert_array_equal(H, H.T)
    np.testing.assert_allclose(np.diag(H), th[3] ** 2 + th[4] ** 2, rtol=1e-15)
    lam = np.linalg.eigvalsh(H)
    assert lam.min() >= th[4] ** 2 * (1 - 1e-9)
    L = oracle.cholesky(H)
    np.testing.assert_allclose(L, np.linalg.cholesky(H), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_dH_matches_central_finite_differences(kind):
    rng = np.random.default_rng(3)
    d = 3
    th = _theta(d, rng)
    X = rng.standard_normal((12, d))
    for p in range(d + 2):
        h = 1e-6 * th[p]
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (oracle.H_matrix(kind, tp, X) - oracle.H_matrix(kind, tm, X)) / (2 * h)
        an = oracle.dH_matrix(kind, th, X, p)
        np.testing.assert_allclose(an, fd, rtol=2e-7, atol=2e-9)


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_mll_matches_scipy_gaussian_logpdf(kind):
    st = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(4)
    th = _theta(2, rng)
    X = rng.standard_normal((30, 2))
    y = rng.standard_normal(30)
    H = oracle.H_matrix(kind, th, X)
    ref = st.multivariate_normal(mean=np.zeros(30), cov=H).logpdf(y)
    assert oracle.mll(kind, th, X, y) == pytest.approx(ref, rel=1e-12)


def test_mll_single_point_closed_form():
    th = np.array([0.7, 1.2, 0.5])
    y = np.array([0.9])
    h = 1.2 ** 2 + 0.5 ** 2
    ref = -y[0] ** 2 / (2 * h) - 0.5 * math.log(h) - 0.5 * math.log(2 * math.pi)
    for kind in (oracle.RBF, oracle.MATERN32):
        assert oracle.mll(kind, th, np.array([[0.3]]), y) == pytest.approx(ref, rel=1e-14)
        g = oracle.mll_grad_exact(kind, th, np.array([[0.3]]), y)
        # d L / d sigma = (y^2/h^2 - 1/h) sigma ; d L / d s_f = (y^2/h^2 - 1/h) s_f ; d L / d l = 0
        assert g[2] == pytest.approx((y[0] ** 2 / h ** 2 - 1 / h) * 0.5, rel=1e-13)
        assert g[1] == pytest.approx((y[0] ** 2 / h ** 2 - 1 / h) * 1.2, rel=1e-13)
        assert g[0] == 0.0


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_exact_gradient_matches_finite_differences_of_mll(kind):
    rng = np.random.default_rng(5)
    d = 3
    th = _theta(d, rng)
    X = rng.standard_normal((48, d))
    y = rng.standard_normal(48)
    g = oracle.mll_grad_exact(kind, th, X, y)
    for p in range(d + 2):
        h = 1e-5 * th[p]
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (oracle.mll(kind, tp, X, y) - oracle.mll(kind, tm, X, y)) / (2 * h)
        assert g[p] == pytest.approx(fd, rel=1e-7, abs=1e-8)


def test_noise_gradient_closed_form():
    """dH/dsigma = 2 sigma I (App. A.1) gives g_sigma = sigma (||H^-1 y||^2 - tr H^-1)."""
    rng = np.random.default_rng(6)
    th = _theta(2, rng, sigma=0.6)
    X = rng.standard_normal((25, 2))
    y = rng.standard_normal(25)
    H = oracle.H_matrix(oracle.MATERN32, th, X)
    a = np.linalg.solve(H, y)
    ref = th[3] * (a @ a - np.trace(np.linalg.inv(H)))
    assert oracle.mll_grad_exact(oracle.MATERN32, th, X, y)[3] == pytest.approx(ref, rel=1e-11)


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_matrix_free_mvm_equals_dense_product(kind):
    rng = np.random.default_rng(7)
    d = 4
    th = _theta(d, rng)
    X = rng.standard_normal((50, d))
    Xs = rng.standard_normal((17, d))
    V = rng.standard_normal((3, 50))
    H = oracle.H_matrix(kind, th, X)
    np.testing.assert_allclose(oracle.kernel_mvm(kind, th, X, X, V, add_noise=True), V @ H.T,
                               rtol=1e-12, atol=1e-12)
    Kc = oracle.kernel_matrix(kind, th, Xs, X)
    np.testing.assert_allclose(oracle.kernel_mvm(kind, th, Xs, X, V), V @ Kc.T, rtol=1e-12, atol=1e-12)
    rows = np.array([3, 0, 49, 7])
    np.testing.assert_allclose(oracle.kernel_mvm(kind, th, X, X, V, add_noise=True, rows=rows),
                               (V @ H.T)[:, rows], rtol=1e-12, atol=1e-12)


def test_chol_solve_matches_numpy_solve():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((20, 20))
    A = A @ A.T + 20 * np.eye(20)
    B = rng.standard_normal((3, 20))
    L = oracle.cholesky(A)
    np.testing.assert_allclose(oracle.chol_solve(L, B), np.linalg.solve(A, B.T).T, rtol=1e-11)


def test_workload_generators_are_seeded_and_shaped():
    p = workloads.small(n=64, s=4)
    q = workloads.small(n=64, s=4)
    np.testing.assert_array_equal(p.X, q.X)
    assert p.X.shape == (64, 8) and p.Z.shape == (4, 64) and p.theta.shape == (10,)
    idx = workloads.sgd_batches(100, 10, 5)
    assert idx.shape == (5, 10) and all(len(set(r)) == 10 for r in idx)
