"""GPU parity of the reverse-mode derivatives: gp_bilinear_grad (value, theta- and
X-gradients of sum_c lam_c u_c^T H w_c) against the FP64 oracle, and the
torch.autograd.Function wrappers against central finite differences and the oracle.

Tolerances (relative to the largest entry of the reference):
  FP64 form : 1e-10          FP32 form : 1e-4
  TC16 form : value/theta 1e-3 (fp16 tiles), X-gradient 1e-4 (always CUDA-core FP32)
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_18457_gb300 import workloads

pytestmark = pytest.mark.gpu

import paper_2405_18457_gb300 as gp  # noqa: E402  (a missing package fails the run)


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    gp.library()
    return torch.device("cuda:0")


def t(a, dev, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


def relmax(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


FORMS = [("f64", None, 1e-10, 1e-10), ("f32", 1, 1e-4, 1e-4), ("tc16", 2, 1e-3, 1e-4)]


def _case(kind, n, d, R, seed, sym):
    rng = np.random.default_rng([11, n, d, R, seed, kind])
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.7, 1.6, size=d), [1.1, 0.3]])
    U = rng.standard_normal((R, n))
    W = U if sym else rng.standard_normal((R, n))
    return X, th, U, W


@pytest.mark.parametrize("form,prec,tol,tolx", FORMS)
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("sym", [False, True])
@pytest.mark.parametrize("n,d,R", [(300, 5, 4), (1, 3, 2), (130, 33, 3)])
def test_bilinear_grad_matches_oracle(dev, form, prec, tol, tolx, kind, sym, n, d, R):
    X, th, U, W = _case(kind, n, d, R, 0, sym)
    lam0, lam_rest = 0.7, -0.3
    lam = np.array([lam0] + [lam_rest] * (R - 1))
    dt = torch.float64 if form == "f64" else torch.float32
    Xt, Ut = t(X, dev, dt), t(U, dev, dt)
    Wt = Ut if sym else t(W, dev, dt)
    if form != "f64":
        Xr = Xt.double().cpu().numpy()
        Ur = Ut.double().cpu().numpy()
        Wr = Wt.double().cpu().numpy()
    else:
        Xr, Ur, Wr = X, U, W
    v, g, gx = gp.gp_bilinear_grad(kind, th, Xt, Ut, Wt, lam0, lam_rest, prec=prec or 1)
    f_ref = oracle.bilinear_value(kind, th, Xr, Ur, Wr, lam)
    g_ref = oracle.grad_bilinear(kind, th, Xr, Ur, Wr, lam)
    x_ref = oracle.grad_bilinear_X(kind, th, Xr, Ur, Wr, lam)
    # K >= 0 for both kernels, so the form on |lam|, |U|, |W| bounds the summed magnitudes
    scale_f = oracle.bilinear_value(kind, th, Xr, np.abs(Ur), np.abs(Wr), np.abs(lam))
    assert abs(v.item() - f_ref) <= tol * scale_f
    assert relmax(g.cpu().numpy(), g_ref) <= tol
    if n > 1:
        assert relmax(gx.cpu().numpy(), x_ref) <= tolx
    else:
        assert np.abs(gx.cpu().numpy()).max() == 0.0


def test_bilinear_grad_optional_outputs_and_errors(dev):
    X, th, U, W = _case(0, 200, 4, 3, 1, False)
    Xt, Ut, Wt = t(X, dev), t(U, dev), t(W, dev)
    v, g, gx = gp.gp_bilinear_grad(0, th, Xt, Ut, Wt, value=False, dtheta=False, dX=True, prec=1)
    assert v is None and g is None and gx.shape == (200, 4)
    v2, g2, gx2 = gp.gp_bilinear_grad(0, th, Xt, Ut, Wt, prec=1)
    assert torch.equal(gx, gx2)  # deterministic: fixed summation order
    with pytest.raises(gp.GPError):
        gp.gp_bilinear_grad(0, th, Xt, Ut, Wt, lam0=float("nan"), prec=1)
    bad = th.copy()
    bad[0] = -1.0
    with pytest.raises(gp.GPError):
        gp.gp_bilinear_grad(0, bad, Xt, Ut, Wt, prec=1)


@pytest.mark.parametrize("kind", [0, 1])
def test_kernel_matvec_gradcheck_fp64(dev, kind):
    """torch.autograd.gradcheck: central finite differences of the FP64 forward against
    the hand-written backward, for X, theta and V."""
    rng = np.random.default_rng(5 + kind)
    n, d, R = 37, 3, 2
    X = torch.tensor(rng.standard_normal((n, d)), dtype=torch.float64, device=dev, requires_grad=True)
    V = torch.tensor(rng.standard_normal((R, n)), dtype=torch.float64, device=dev, requires_grad=True)
    th = torch.tensor(np.concatenate([rng.uniform(0.8, 1.5, d), [1.2, 0.4]]), dtype=torch.float64,
                      requires_grad=True)
    fn = lambda X_, th_, V_: gp.kernel_matvec(X_, th_, V_, kind=kind)  # noqa: E731
    assert torch.autograd.gradcheck(fn, (X, th, V), eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("form,prec,tol,tolx", FORMS)
@pytest.mark.parametrize("kind", [0, 1])
def test_kernel_matvec_backward_matches_oracle(dev, form, prec, tol, tolx, kind):
    """f = sum_c lam_c u_c^T (H V)_c differentiated by torch through kernel_matvec:
    dV = H (lam u), dtheta and dX = the oracle's bilinear-form gradients."""
    X, th, U, W = _case(kind, 257, 6, 3, 2, False)
    lam = np.array([0.5, -0.25, 1.5])
    dt = torch.float64 if form == "f64" else torch.float32
    Xt = t(X, dev, dt).requires_grad_(True)
    Vt = t(W, dev, dt).requires_grad_(True)
    tht = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    Ut = t(U, dev, dt)
    Y = gp.kernel_matvec(Xt, tht, Vt, kind=kind, prec=prec or 1)
    lam_t = torch.tensor(lam, dtype=dt, device=dev)
    f = (lam_t[:, None] * Ut * Y).sum()
    f.backward()
    Xr = Xt.detach().double().cpu().numpy()
    Ur = Ut.double().cpu().numpy()
    Wr = Vt.detach().double().cpu().numpy()
    assert relmax(tht.grad.numpy(), oracle.grad_bilinear(kind, th, Xr, Ur, Wr, lam)) <= tol
    assert relmax(Xt.grad.double().cpu().numpy(), oracle.grad_bilinear_X(kind, th, Xr, Ur, Wr, lam)) <= tolx
    dV_ref = oracle.kernel_mvm(kind, th, Xr, Xr, lam[:, None] * Ur, add_noise=True)
    assert relmax(Vt.grad.double().cpu().numpy(), dV_ref) <= (tol if form != "tc16" else 1e-3)


def _sgd_subset(n=4096):
    p = workloads.sgd(n=n)
    rng = np.random.default_rng([12, n])
    Vsol = rng.standard_normal((p.s + 1, n))
    return p, Vsol


def test_pathwise_surrogate_autograd_equals_estimator_4096(dev):
    """The pathwise surrogate 1/2 v_y^T H v_y - 1/(2s) sum zhat^T H zhat differentiated by
    autograd gives exactly gp_mll_grad_pathwise's estimate (same kernels), on a 4096-point
    subset of the large SGD workload (mixture of Gaussians, d = 11, Matern-3/2, s = 64)."""
    p, Vsol = _sgd_subset()
    s = p.s
    for prec in (1, 2):
        Xt = t(p.X, dev)
        Vt = t(Vsol, dev)
        tht = torch.tensor(p.theta, dtype=torch.float64, requires_grad=True)
        f = gp.bilinear_form(Xt, tht, Vt, Vt, 0.5, -0.5 / s, kind=p.kind, prec=prec)
        f.backward()
        g_est = gp.gp_mll_grad_pathwise(p.kind, p.theta, Xt, Vt, prec=prec).cpu().numpy()
        np.testing.assert_allclose(tht.grad.numpy(), g_est, rtol=1e-12, atol=0)


def test_pathwise_surrogate_finite_differences_4096(dev):
    """Central finite differences of the FP64 surrogate value (GPU forward) against the
    autograd theta- and X-gradients, and both against the oracle, on the 4096-point subset."""
    p, Vsol = _sgd_subset()
    s, n, d = p.s, p.n, p.d
    lam0, lamr = 0.5, -0.5 / s
    Xt = t(p.X, dev, torch.float64).requires_grad_(True)
    Vt = t(Vsol, dev, torch.float64)
    tht = torch.tensor(p.theta, dtype=torch.float64, requires_grad=True)
    f = gp.bilinear_form(Xt, tht, Vt, Vt, lam0, lamr, kind=p.kind)
    f.backward()
    gth = tht.grad.numpy()
    gX = Xt.grad.cpu().numpy()

    def val(th, X):
        v, _, _ = gp.gp_bilinear_grad(p.kind, th, X, Vt, Vt, lam0, lamr, dtheta=False, dX=False)
        return v.item()

    X0 = Xt.detach()
    for k in range(d + 2):
        h = 1e-5 * p.theta[k]
        tp = p.theta.copy()
        tm = p.theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (val(tp, X0) - val(tm, X0)) / (2 * h)
        assert abs(fd - gth[k]) <= 1e-6 * np.abs(gth).max(), (k, fd, gth[k])
    # X: moving point i changes only row and column i of K, so the central difference of
    # f equals 2 sum_c lam_c v_ci [k(x_i + h e_k, X) - k(x_i - h e_k, X)] v~_c with
    # v~_c = v_c with entry i zeroed (the diagonal k(x_i, x_i) = s_f^2 is constant).
    # Each one-row product runs on the GPU in FP64, free of the n^2 roundoff of f.
    lam = np.array([lam0] + [lamr] * s)
    rng = np.random.default_rng(3)
    for _ in range(8):
        i, k = int(rng.integers(n)), int(rng.integers(d))
        h = 1e-5
        Vz = Vt.clone()
        Vz[:, i] = 0.0
        xp = X0[i:i + 1].clone()
        xm = X0[i:i + 1].clone()
        xp[0, k] += h
        xm[0, k] -= h
        kp_ = gp.gp_kernel_mvm(p.kind, p.theta, xp, Vz, X2=X0).cpu().numpy()[:, 0]
        km_ = gp.gp_kernel_mvm(p.kind, p.theta, xm, Vz, X2=X0).cpu().numpy()[:, 0]
        fd = 2.0 * np.sum(lam * Vsol[:, i] * (kp_ - km_)) / (2 * h)
        assert abs(fd - gX[i, k]) <= 1e-6 * max(1.0, np.abs(gX[i]).max()), (i, k, fd, gX[i, k])
    # and both gradients against the oracle on the same inputs
    assert relmax(gth, oracle.grad_bilinear(p.kind, p.theta, p.X, Vsol, Vsol, lam)) <= 1e-10
    assert relmax(gX, oracle.grad_bilinear_X(p.kind, p.theta, p.X, Vsol, Vsol, lam)) <= 1e-10
