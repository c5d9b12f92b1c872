"""FP64 CPU oracle for the iterative-GP hot path (test infrastructure only).

This package is the parity oracle.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s cpu_baseline / ``--impl reference`` leg may import it.  The
product library (``paper_2405_18457_gb300``) never imports, links or executes
anything here, and this package imports nothing from the product.

The arithmetic lives in ``gp_oracle.c`` (plain C99, double precision, OpenMP
over independent rows); this module only marshals numpy arrays through ctypes.
Layout conventions: X is n x d row-major; blocks of vectors are R x n
(vector c contiguous); theta = [l_1..l_d, s_f, sigma]; kind 0 = RBF,
1 = Matern-3/2.  Every function cites the passage of the paper it follows in
``gp_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_gp.so")
_lock = threading.Lock()
_lib = None

RBF = 0
MATERN32 = 1

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("converged", ctypes.c_int),
                ("res_y", ctypes.c_double), ("res_z", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile gp_oracle.c into liboracle_gp.so with gcc (no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=gnu99", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            sig = {
                "gpo_kernel": (_d, [_i, _i, _pd, _pd, _pd]),
                "gpo_dkernel": (_d, [_i, _i, _pd, _pd, _pd, _i]),
                "gpo_kernel_matrix": (None, [_i, _i, _pd, _pd, _i64, _pd, _i64, _pd]),
                "gpo_H_matrix": (None, [_i, _i, _pd, _pd, _i64, _pd]),
                "gpo_dH_matrix": (None, [_i, _i, _pd, _pd, _i64, _i, _pd]),
                "gpo_kernel_mvm": (None, [_i, _i, _pd, _pd, _i64, _pd, _i64, _pd, _i, _i, _pi64, _i64, _pd]),
                "gpo_cholesky": (_i, [_i64, _pd]),
                "gpo_chol_solve": (None, [_i64, _pd, _pd, _i]),
                "gpo_mll": (_d, [_i, _i, _pd, _pd, _i64, _pd]),
                "gpo_mll_grad_exact": (_i, [_i, _i, _pd, _pd, _i64, _pd, _pd]),
                "gpo_grad_bilinear": (None, [_i, _i, _pd, _pd, _i64, _pd, _pd, _pd, _i, _pd]),
                "gpo_bilinear_value": (_d, [_i, _i, _pd, _pd, _i64, _pd, _pd, _pd, _i]),
                "gpo_rkhs_sqdist": (None, [_i, _i, _pd, _pd, _i64, _pd, _pd, _i, _pd]),
                "gpo_dkernel_dx": (None, [_i, _i, _pd, _pd, _pd, _pd]),
                "gpo_grad_bilinear_X": (None, [_i, _i, _pd, _pd, _i64, _pd, _pd, _pd, _i, _pd]),
                "gpo_grad_standard": (None, [_i, _i, _pd, _pd, _i64, _pd, _pd, _i, _pd]),
                "gpo_grad_pathwise": (None, [_i, _i, _pd, _pd, _i64, _pd, _i, _pd]),
                "gpo_solve_cg": (_i, [_i, _i, _pd, _pd, _i64, _pd, _i, _pd, _i64, _d, _i,
                                      ctypes.POINTER(_Info)]),
                "gpo_pivoted_cholesky": (_i, [_i, _i, _pd, _pd, _i64, _i, _pd, _pi64]),
                "gpo_solve_pcg": (_i, [_i, _i, _pd, _pd, _i64, _pd, _i, _pd, _i, _i64, _d, _i,
                                       ctypes.POINTER(_Info)]),
                "gpo_solve_ap": (_i, [_i, _i, _pd, _pd, _i64, _pd, _i, _pd, _i64, _i64, _d, _i,
                                      ctypes.POINTER(_Info)]),
                "gpo_solve_sgd": (_i, [_i, _i, _pd, _pd, _i64, _pd, _i, _pd, _i64, _pi64, _d, _d,
                                       _i64, _d, _i, ctypes.POINTER(_Info)]),
                "gpo_rff_prior": (None, [_i, _i, _pd, _pd, _i64, _i, _pd, _pd, _pd, _i, _pd]),
                "gpo_posterior_samples": (None, [_i, _i, _pd, _pd, _i64, _pd, _i64, _pd, _i, _pd, _pd]),
                "gpo_predict": (None, [_i, _i, _pd, _pd, _i64, _pd, _i64, _pd, _i, _pd, _pd, _pd, _pd, _pd]),
                "gpo_adam_softplus": (None, [_i, _pd, _pd, _pd, _i64, _pd, _d, _d, _d, _d, _pd]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _a(x, dtype=np.float64):
    """C-contiguous copy/view with the requested dtype."""
    return np.ascontiguousarray(x, dtype=dtype)


def _p(x):
    return x.ctypes.data_as(_pd)


def _p64(x):
    return x.ctypes.data_as(_pi64)


def _dims(X, theta):
    X = _a(X)
    if X.ndim == 1:
        X = X[:, None]
    theta = _a(theta)
    d = X.shape[1]
    assert theta.shape == (d + 2,), "theta must hold [l_1..l_d, s_f, sigma]"
    return X, theta, d


def kernel(kind, theta, x, xp):
    """k(x, x') for one pair of points."""
    theta = _a(theta)
    x = _a(x).ravel()
    xp = _a(xp).ravel()
    return _load().gpo_kernel(kind, x.size, _p(theta), _p(x), _p(xp))


def dkernel(kind, theta, x, xp, p):
    theta = _a(theta)
    x = _a(x).ravel()
    xp = _a(xp).ravel()
    return _load().gpo_dkernel(kind, x.size, _p(theta), _p(x), _p(xp), int(p))


def kernel_matrix(kind, theta, X1, X2):
    X1, theta, d = _dims(X1, theta)
    X2 = _a(X2).reshape(-1, d)
    K = np.empty((X1.shape[0], X2.shape[0]))
    _load().gpo_kernel_matrix(kind, d, _p(theta), _p(X1), X1.shape[0], _p(X2), X2.shape[0], _p(K))
    return K


def H_matrix(kind, theta, X):
    X, theta, d = _dims(X, theta)
    n = X.shape[0]
    H = np.empty((n, n))
    _load().gpo_H_matrix(kind, d, _p(theta), _p(X), n, _p(H))
    return H


def dH_matrix(kind, theta, X, p):
    X, theta, d = _dims(X, theta)
    n = X.shape[0]
    dH = np.empty((n, n))
    _load().gpo_dH_matrix(kind, d, _p(theta), _p(X), n, int(p), _p(dH))
    return dH


def kernel_mvm(kind, theta, X1, X2, V, add_noise=False, rows=None):
    """Matrix-free K(X1, X2) V (+ sigma^2 V).  V: R x n2.  Returns R x n1
    (or R x len(rows) when rows is given)."""
    X1, theta, d = _dims(X1, theta)
    X2 = _a(X2).reshape(-1, d)
    V = _a(V)
    if V.ndim == 1:
        V = V[None, :]
    R, n2 = V.shape
    assert n2 == X2.shape[0]
    if add_noise:
        assert X1.shape == X2.shape and np.array_equal(X1, X2)
    if rows is not None:
        rows = _a(rows, np.int64)
        nout = rows.size
        rp = _p64(rows)
    else:
        nout = X1.shape[0]
        rp = None
    Y = np.empty((R, nout))
    _load().gpo_kernel_mvm(kind, d, _p(theta), _p(X1), X1.shape[0], _p(X2), X2.shape[0], _p(V), R,
                           1 if add_noise else 0, rp, nout, _p(Y))
    return Y


def cholesky(A):
    """Lower Cholesky factor (raises on a non-positive pivot)."""
    L = _a(A).copy()
    n = L.shape[0]
    info = _load().gpo_cholesky(n, _p(L))
    if info != 0:
        raise np.linalg.LinAlgError("matrix not positive definite at pivot %d" % info)
    return L


def chol_solve(L, B):
    L = _a(L)
    X = _a(B).copy()
    one = X.ndim == 1
    if one:
        X = X[None, :]
    _load().gpo_chol_solve(L.shape[0], _p(L), _p(X), X.shape[0])
    return X[0] if one else X


def mll(kind, theta, X, y):
    X, theta, d = _dims(X, theta)
    y = _a(y)
    return _load().gpo_mll(kind, d, _p(theta), _p(X), X.shape[0], _p(y))


def mll_grad_exact(kind, theta, X, y):
    X, theta, d = _dims(X, theta)
    y = _a(y)
    g = np.empty(d + 2)
    info = _load().gpo_mll_grad_exact(kind, d, _p(theta), _p(X), X.shape[0], _p(y), _p(g))
    if info != 0:
        raise np.linalg.LinAlgError("H not positive definite")
    return g


def grad_bilinear(kind, theta, X, U, W, lam):
    X, theta, d = _dims(X, theta)
    U = _a(U)
    W = _a(W)
    lam = _a(lam)
    g = np.empty(d + 2)
    _load().gpo_grad_bilinear(kind, d, _p(theta), _p(X), X.shape[0], _p(U), _p(W), _p(lam),
                              U.shape[0], _p(g))
    return g


def bilinear_value(kind, theta, X, U, W, lam):
    """sum_c lam_c U[c]^T H W[c] (Sec. 2 H = K + sigma^2 I)."""
    X, theta, d = _dims(X, theta)
    U = _a(U)
    W = _a(W)
    lam = _a(lam)
    return float(_load().gpo_bilinear_value(kind, d, _p(theta), _p(X), X.shape[0], _p(U), _p(W), _p(lam),
                                            U.shape[0]))


def rkhs_sqdist(kind, theta, X, U, Uinit=None):
    """Per column, ||Uinit[c] - U[c]||_H^2 = (Uinit[c] - U[c])^T H (Uinit[c] - U[c]) (Sec. 3,
    Eq. RKHS_distance); Uinit None is the zero initialisation."""
    X, theta, d = _dims(X, theta)
    U = np.ascontiguousarray(_a(U).reshape(-1, X.shape[0]))
    R = U.shape[0]
    U0 = None if Uinit is None else np.ascontiguousarray(_a(Uinit).reshape(R, X.shape[0]))
    out = np.empty(R)
    _load().gpo_rkhs_sqdist(kind, d, _p(theta), _p(X), X.shape[0], None if U0 is None else _p(U0), _p(U), R,
                            _p(out))
    return out


def trace_H_inv(kind, theta, X):
    """tr(H^-1), the expected initial RKHS distance of the standard estimator's systems
    (Sec. 3, Eq. standard_dist), from the dense H and its Cholesky factor (numpy)."""
    H = H_matrix(kind, theta, X)
    L = np.linalg.cholesky(H)
    Linv = np.linalg.solve(L, np.eye(H.shape[0]))
    return float(np.sum(Linv * Linv))


def dkernel_dx(kind, theta, x, xp):
    """Gradient of k(x, x') with respect to x."""
    theta = _a(theta)
    x = _a(x)
    xp = _a(xp)
    g = np.empty(x.shape[0])
    _load().gpo_dkernel_dx(kind, x.shape[0], _p(theta), _p(x), _p(xp), _p(g))
    return g


def grad_bilinear_X(kind, theta, X, U, W, lam):
    """d/dX of sum_c lam_c U[c]^T H(theta, X) W[c], n x d."""
    X, theta, d = _dims(X, theta)
    U = _a(U)
    W = _a(W)
    lam = _a(lam)
    dX = np.empty_like(X)
    _load().gpo_grad_bilinear_X(kind, d, _p(theta), _p(X), X.shape[0], _p(U), _p(W), _p(lam),
                                U.shape[0], _p(dX))
    return dX


def grad_standard(kind, theta, X, Vsol, Z):
    X, theta, d = _dims(X, theta)
    Vsol = _a(Vsol)
    Z = _a(Z)
    s = Z.shape[0]
    assert Vsol.shape[0] == s + 1
    g = np.empty(d + 2)
    _load().gpo_grad_standard(kind, d, _p(theta), _p(X), X.shape[0], _p(Vsol), _p(Z), s, _p(g))
    return g


def grad_pathwise(kind, theta, X, Vsol):
    X, theta, d = _dims(X, theta)
    Vsol = _a(Vsol)
    s = Vsol.shape[0] - 1
    g = np.empty(d + 2)
    _load().gpo_grad_pathwise(kind, d, _p(theta), _p(X), X.shape[0], _p(Vsol), s, _p(g))
    return g


def _info(inf):
    return {"iters": int(inf.iters), "converged": bool(inf.converged),
            "res_y": float(inf.res_y), "res_z": float(inf.res_z)}


def solve_cg(kind, theta, X, B, V0=None, max_iters=1000, tol=1e-2, stop_rule=0):
    X, theta, d = _dims(X, theta)
    B = _a(B)
    V = np.zeros_like(B) if V0 is None else _a(V0).copy()
    inf = _Info()
    _load().gpo_solve_cg(kind, d, _p(theta), _p(X), X.shape[0], _p(B), B.shape[0], _p(V),
                         int(max_iters), float(tol), int(stop_rule), ctypes.byref(inf))
    return V, _info(inf)


def pivoted_cholesky(kind, theta, X, k):
    """Rank-k pivoted Cholesky factor L (rank x n, K ~ L^T L) and its pivots."""
    X, theta, d = _dims(X, theta)
    n = X.shape[0]
    L = np.zeros((k, n))
    piv = np.zeros(k, dtype=np.int64)
    rank = _load().gpo_pivoted_cholesky(kind, d, _p(theta), _p(X), n, k, _p(L),
                                        piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return L[:rank], piv[:rank]


def solve_pcg(kind, theta, X, B, rank, V0=None, max_iters=1000, tol=1e-2, stop_rule=0):
    """Alg. 1 with the rank-`rank` pivoted Cholesky preconditioner (rank 0: plain CG)."""
    X, theta, d = _dims(X, theta)
    B = _a(B)
    V = np.zeros_like(B) if V0 is None else _a(V0).copy()
    inf = _Info()
    st = _load().gpo_solve_pcg(kind, d, _p(theta), _p(X), X.shape[0], _p(B), B.shape[0], _p(V), int(rank),
                               int(max_iters), float(tol), int(stop_rule), ctypes.byref(inf))
    if st != 0:
        raise np.linalg.LinAlgError("preconditioner not positive definite")
    return V, _info(inf)


def solve_ap(kind, theta, X, B, V0=None, block_size=1000, max_iters=1000, tol=1e-2, stop_rule=0):
    X, theta, d = _dims(X, theta)
    B = _a(B)
    V = np.zeros_like(B) if V0 is None else _a(V0).copy()
    inf = _Info()
    rc = _load().gpo_solve_ap(kind, d, _p(theta), _p(X), X.shape[0], _p(B), B.shape[0], _p(V),
                              int(block_size), int(max_iters), float(tol), int(stop_rule),
                              ctypes.byref(inf))
    if rc != 0:
        raise np.linalg.LinAlgError("diagonal block not positive definite")
    return V, _info(inf)


def solve_sgd(kind, theta, X, B, idx, batch, lr, momentum=0.9, V0=None, max_iters=1000,
              tol=1e-2, stop_rule=0):
    X, theta, d = _dims(X, theta)
    B = _a(B)
    idx = _a(idx, np.int64).ravel()
    assert idx.size >= int(max_iters) * int(batch)
    V = np.zeros_like(B) if V0 is None else _a(V0).copy()
    inf = _Info()
    _load().gpo_solve_sgd(kind, d, _p(theta), _p(X), X.shape[0], _p(B), B.shape[0], _p(V),
                          int(batch), _p64(idx), float(lr), float(momentum), int(max_iters),
                          float(tol), int(stop_rule), ctypes.byref(inf))
    return V, _info(inf)


def rff_prior(kind, theta, X, omega_hat, chi2, W):
    """Prior function samples at X by random Fourier features; W: s x m."""
    X, theta, d = _dims(X, theta)
    omega_hat = _a(omega_hat)
    W = _a(W)
    s, m = W.shape
    assert omega_hat.shape == (m // 2, d)
    c2 = _a(chi2) if chi2 is not None else np.ones(m // 2)
    F = np.empty((s, X.shape[0]))
    _load().gpo_rff_prior(kind, d, _p(theta), _p(X), X.shape[0], m, _p(omega_hat), _p(c2), _p(W),
                          s, _p(F))
    return F


def posterior_samples(kind, theta, Xstar, X, Vsol, Fstar):
    X, theta, d = _dims(X, theta)
    Xstar = _a(Xstar).reshape(-1, d)
    Vsol = _a(Vsol)
    Fstar = _a(Fstar)
    s = Vsol.shape[0] - 1
    out = np.empty((s, Xstar.shape[0]))
    _load().gpo_posterior_samples(kind, d, _p(theta), _p(Xstar), Xstar.shape[0], _p(X), X.shape[0],
                                  _p(Vsol), s, _p(Fstar), _p(out))
    return out


def predict(kind, theta, Xstar, X, Vsol, Fstar, ystar=None):
    """Predictive mean and variance at Xstar from the pathwise solutions, and (RMSE, mean test
    log-likelihood) when ystar is given."""
    X, theta, d = _dims(X, theta)
    Xstar = _a(Xstar).reshape(-1, d)
    Vsol = _a(Vsol)
    Fstar = _a(Fstar)
    s = Vsol.shape[0] - 1
    ns = Xstar.shape[0]
    mean = np.empty(ns)
    var = np.empty(ns)
    metrics = np.full(2, np.nan)
    ys = None if ystar is None else _a(ystar)
    _load().gpo_predict(kind, d, _p(theta), _p(Xstar), ns, _p(X), X.shape[0], _p(Vsol), s, _p(Fstar),
                        None if ys is None else _p(ys), _p(mean), _p(var), _p(metrics))
    return mean, var, (None if ys is None else (float(metrics[0]), float(metrics[1])))


def adam_softplus(nu, m, v, t, grad_theta, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam ascent step in softplus coordinates; updates nu, m, v in place and
    returns theta = softplus(nu)."""
    P = nu.size
    g = _a(grad_theta)
    theta = np.empty(P)
    _load().gpo_adam_softplus(P, _p(nu), _p(m), _p(v), int(t), _p(g), float(lr), float(b1),
                              float(b2), float(eps), _p(theta))
    return theta
