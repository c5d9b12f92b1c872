"""Pins for the oracle's solver diagnostics: the RKHS squared distance between a solver
initialisation and the solution (Sec. 3, "Initial Distance to the Linear System Solution",
Eq. RKHS_distance) and its expectations for the two estimators' systems (Eq. standard_dist:
tr(H^-1) for Gaussian probes z; Eq. pathwise_dist: n for targets xi ~ N(0, H)).

The Monte Carlo pins use the exact laws of the quadratic forms: with z ~ N(0, I),
z^T H^-1 z has mean tr(H^-1) and variance 2 tr(H^-2); with xi = L eps (L L^T = H),
xi^T H^-1 xi = eps^T eps ~ chi^2_n (mean n, variance 2n)."""
import numpy as np
import pytest

import oracle


def _setup(kind, n=40, d=3, seed=0, sigma=0.3):
    rng = np.random.default_rng([41, seed])
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.6, 1.4, size=d), [1.1, sigma]])
    return rng, X, th


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_distance_matches_dense_quadratic_form_from_sklearn_kernel(kind):
    sk = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng, X, th = _setup(kind)
    n, d = X.shape
    ls, sf, sig = th[:d], th[d], th[d + 1]
    base = sk.RBF(length_scale=ls) if kind == oracle.RBF else sk.Matern(length_scale=ls, nu=1.5)
    H = sf * sf * base(X) + sig * sig * np.eye(n)
    U = rng.standard_normal((3, n))
    U0 = rng.standard_normal((3, n))
    got = oracle.rkhs_sqdist(kind, th, X, U, U0)
    E = U0 - U
    want = np.einsum("ci,ij,cj->c", E, H, E)
    np.testing.assert_allclose(got, want, rtol=1e-12)
    # zero initialisation: ||u||_H^2 = b^T H^-1 b for u = H^-1 b (Eq. RKHS_distance)
    B = rng.standard_normal((2, n))
    Usol = np.linalg.solve(H, B.T).T
    np.testing.assert_allclose(oracle.rkhs_sqdist(kind, th, X, Usol),
                               np.einsum("ci,ci->c", B, Usol), rtol=1e-9)


def test_distance_is_a_squared_norm():
    rng, X, th = _setup(oracle.MATERN32, seed=1)
    n = X.shape[0]
    U = rng.standard_normal((2, n))
    U0 = rng.standard_normal((2, n))
    d1 = oracle.rkhs_sqdist(oracle.MATERN32, th, X, U, U0)
    assert np.all(d1 > 0)
    np.testing.assert_allclose(oracle.rkhs_sqdist(oracle.MATERN32, th, X, U0, U), d1, rtol=1e-12)
    np.testing.assert_allclose(oracle.rkhs_sqdist(oracle.MATERN32, th, X, U, U), 0.0, atol=1e-12)
    np.testing.assert_allclose(oracle.rkhs_sqdist(oracle.MATERN32, th, X, 2.0 * U), 4.0 * oracle.rkhs_sqdist(
        oracle.MATERN32, th, X, U), rtol=1e-12)
    # lower bound by the smallest eigenvalue of H, which is at least sigma^2
    e = U0 - U
    assert np.all(d1 >= th[-1] ** 2 * np.sum(e * e, axis=1) * (1 - 1e-12))


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_standard_systems_expected_distance_is_trace_of_inverse(kind):
    """Eq. standard_dist: E ||H^-1 z||_H^2 = tr(H^-1), z ~ N(0, I), z-score < 4."""
    rng, X, th = _setup(kind, seed=2, sigma=0.2)
    n = X.shape[0]
    H = oracle.H_matrix(kind, th, X)
    Hinv = np.linalg.inv(H)
    tr = oracle.trace_H_inv(kind, th, X)
    np.testing.assert_allclose(tr, np.trace(Hinv), rtol=1e-10)
    s = 400
    Z = rng.standard_normal((s, n))
    U = np.linalg.solve(H, Z.T).T
    dist = oracle.rkhs_sqdist(kind, th, X, U)
    sd = np.sqrt(2.0 * np.trace(Hinv @ Hinv) / s)
    assert abs(dist.mean() - tr) < 4.0 * sd, (dist.mean(), tr, sd)
    # and the trace lies between the top eigenvalue of H^-1 and n times it
    top = 1.0 / np.linalg.eigvalsh(H)[0]
    assert top <= tr <= n * top


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_pathwise_systems_expected_distance_is_n(kind):
    """Eq. pathwise_dist: E ||H^-1 xi||_H^2 = n for xi ~ N(0, H) (here exact draws L eps),
    whatever the noise level; for these draws the distance is eps^T eps exactly."""
    for sigma in (0.05, 0.5):
        rng, X, th = _setup(kind, seed=3, sigma=sigma)
        n = X.shape[0]
        H = oracle.H_matrix(kind, th, X)
        L = np.linalg.cholesky(H)
        s = 400
        eps = rng.standard_normal((s, n))
        Xi = (L @ eps.T).T
        U = np.linalg.solve(H, Xi.T).T
        dist = oracle.rkhs_sqdist(kind, th, X, U)
        np.testing.assert_allclose(dist, np.sum(eps * eps, axis=1), rtol=1e-7)
        assert abs(dist.mean() - n) < 4.0 * np.sqrt(2.0 * n / s)


def test_standard_distance_grows_with_noise_precision_pathwise_does_not():
    """Sec. 3: as sigma falls (noise precision rises), tr(H^-1) grows like 1/sigma^2 while the
    pathwise expectation stays n."""
    _, X, th = _setup(oracle.RBF, seed=4)
    n = X.shape[0]
    trs = []
    for sigma in (1.0, 0.3, 0.1, 0.03):
        t = th.copy()
        t[-1] = sigma
        trs.append(oracle.trace_H_inv(oracle.RBF, t, X))
    assert all(a < b for a, b in zip(trs, trs[1:]))
    assert trs[-1] > 10 * n > trs[0]
