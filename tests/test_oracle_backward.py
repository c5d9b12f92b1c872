"""Pins for the oracle's reverse-mode derivatives of the bilinear form
f(theta, X, U, W) = sum_c lambda_c U[c]^T H(theta, X) W[c] (Sec. 2 H = K + sigma^2 I;
Eq. mll_grad, Eq. trace and Eq. pathwise_estimator are instances of its theta-gradient).

The X-gradient is pinned by central finite differences of the matrix-free value, by the
translation invariance of a stationary kernel and by the per-dimension scaling identity
that ties it to the (separately pinned) length-scale gradient."""
import numpy as np
import pytest

import oracle

KINDS = [oracle.RBF, oracle.MATERN32]


def _case(kind, n=10, d=3, R=3, seed=0, sym=False):
    rng = np.random.default_rng(seed + 10 * kind)
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.6, 1.5, size=d), [1.2, 0.4]])
    U = rng.standard_normal((R, n))
    W = U.copy() if sym else rng.standard_normal((R, n))
    lam = rng.uniform(-1.0, 1.0, size=R)
    return X, th, U, W, lam


@pytest.mark.parametrize("kind", KINDS)
def test_dkernel_dx_matches_finite_differences(kind):
    rng = np.random.default_rng(3 + kind)
    d = 4
    th = np.concatenate([rng.uniform(0.5, 1.5, size=d), [0.9, 0.3]])
    x = rng.standard_normal(d)
    xp = rng.standard_normal(d)
    g = oracle.dkernel_dx(kind, th, x, xp)
    h = 1e-6
    for p in range(d):
        e = np.zeros(d)
        e[p] = h
        fd = (oracle.kernel(kind, th, x + e, xp) - oracle.kernel(kind, th, x - e, xp)) / (2 * h)
        assert abs(g[p] - fd) <= 1e-8 * max(1.0, abs(fd))
    # r = 0: the gradient vanishes (both kernels are smooth maxima there)
    np.testing.assert_array_equal(oracle.dkernel_dx(kind, th, x, x), np.zeros(d))


@pytest.mark.parametrize("kind", KINDS)
def test_bilinear_value_homogeneity(kind):
    """K scales with s_f^2 and the noise term with sigma^2, so
    f = (s_f/2) df/ds_f + (sigma/2) df/dsigma (Euler's identity for the two
    degree-2 homogeneous parts), tying the value to the pinned theta-gradient."""
    X, th, U, W, lam = _case(kind)
    d = X.shape[1]
    f = oracle.bilinear_value(kind, th, X, U, W, lam)
    g = oracle.grad_bilinear(kind, th, X, U, W, lam)
    np.testing.assert_allclose(f, 0.5 * th[d] * g[d] + 0.5 * th[d + 1] * g[d + 1], rtol=1e-12)
    H = oracle.H_matrix(kind, th, X)
    np.testing.assert_allclose(f, float(np.einsum("c,ci,ij,cj->", lam, U, H, W)), rtol=1e-12)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("sym", [False, True])
def test_grad_X_matches_finite_differences(kind, sym):
    X, th, U, W, lam = _case(kind, sym=sym)
    n, d = X.shape
    dX = oracle.grad_bilinear_X(kind, th, X, U, W, lam)
    h = 1e-6
    scale = np.abs(dX).max()
    for a in range(n):
        for p in range(d):
            Xp = X.copy()
            Xm = X.copy()
            Xp[a, p] += h
            Xm[a, p] -= h
            fd = (oracle.bilinear_value(kind, th, Xp, U, W, lam)
                  - oracle.bilinear_value(kind, th, Xm, U, W, lam)) / (2 * h)
            assert abs(dX[a, p] - fd) <= 1e-7 * scale, (a, p, dX[a, p], fd)


@pytest.mark.parametrize("kind", KINDS)
def test_grad_X_translation_invariance(kind):
    """f(X + t) = f(X) for a common shift t, so the X-gradient sums to zero over points."""
    X, th, U, W, lam = _case(kind, n=16, d=5, R=4, seed=5)
    dX = oracle.grad_bilinear_X(kind, th, X, U, W, lam)
    assert np.abs(dX.sum(axis=0)).max() <= 1e-12 * np.abs(dX).sum()


@pytest.mark.parametrize("kind", KINDS)
def test_grad_X_scaling_identity(kind):
    """f depends on (x_k, l_k) only through x_k / l_k, so scaling dimension k of every
    point and l_k by the same factor leaves f unchanged:
    sum_a x_ak df/dx_ak + l_k df/dl_k = 0 for every k."""
    X, th, U, W, lam = _case(kind, n=14, d=4, R=3, seed=7)
    d = X.shape[1]
    dX = oracle.grad_bilinear_X(kind, th, X, U, W, lam)
    g = oracle.grad_bilinear(kind, th, X, U, W, lam)
    lhs = (X * dX).sum(axis=0) + th[:d] * g[:d]
    assert np.abs(lhs).max() <= 1e-12 * (np.abs(X * dX).sum() + np.abs(th[:d] * g[:d]).sum())
