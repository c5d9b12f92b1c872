"""torch.autograd.Function wrappers over the C ABI (argument marshalling only).

* ``kernel_matvec(X, theta, V)`` is Y = H(theta, X) V with H = K + sigma^2 I
  (Sec. 2).  Its backward, for an upstream gradient G, is
  dV = H G (H is symmetric), and (dtheta, dX) = the theta- and X-gradients of
  sum_c G_c^T H V_c, computed by ``gp_bilinear_grad`` with kernel tiles
  recomputed on the GPU (nothing of K is stored by the forward pass).
* ``bilinear_form(X, theta, U, W, lam0, lam_rest)`` is
  f = sum_c lam_c U_c^T H W_c.  With U = W = [v_y, zhat_1..zhat_s] held fixed,
  lam0 = 1/2 and lam_rest = -1/(2s), its theta-gradient is the pathwise
  estimator of Eq. pathwise_estimator (with W = [v_y, z_1..z_s] the standard one
  of Eq. trace): differentiating this scalar in torch reproduces
  ``gp_mll_grad_pathwise`` / ``gp_mll_grad_standard``.  U and W are treated as
  constants (the estimators hold the solutions fixed).

theta may be a sequence or a tensor of d+2 values [l_1..l_d, s_f, sigma]; when
it is a tensor that requires grad its gradient is returned on its own device and
dtype.  float64 inputs use the plain FP64 form; float32 inputs use ``prec``
(GP_PREC_TC16 by default) for the forward product and the theta-gradient, and
CUDA-core FP32 tiles for the X-gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as _b


def _host_theta(theta):
    if isinstance(theta, torch.Tensor):
        return theta.detach().to("cpu", torch.float64).numpy().copy()
    return np.asarray(theta, dtype=np.float64).copy()


class _KernelMatVec(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, theta, V, kind, prec):
        th = _host_theta(theta)
        Y = _b.gp_kernel_mvm(kind, th, X, V, add_noise=True, prec=prec)
        ctx.save_for_backward(X, V)
        ctx.th = th
        ctx.kind = kind
        ctx.prec = prec
        ctx.theta_like = theta if isinstance(theta, torch.Tensor) else None
        return Y

    @staticmethod
    def backward(ctx, G):
        X, V = ctx.saved_tensors
        G = G.contiguous()
        need_x, need_th, need_v = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
        dV = _b.gp_kernel_mvm(ctx.kind, ctx.th, X, G, add_noise=True, prec=ctx.prec) if need_v else None
        dX = dth = None
        if need_x or need_th:
            _, g, gx = _b.gp_bilinear_grad(ctx.kind, ctx.th, X, G, V, 1.0, 1.0, value=False, dtheta=need_th,
                                           dX=need_x, prec=ctx.prec)
            dX = gx
            if need_th:
                ref = ctx.theta_like
                dth = g.to(ref.device, ref.dtype)
        return dX, dth, dV, None, None


def kernel_matvec(X, theta, V, kind=_b.GP_RBF, prec=_b.GP_PREC_TC16):
    """Y = (K(X, X; theta) + sigma^2 I) V, differentiable in X, theta and V.
    X (n, d), V (R, n) or (n,) on the GPU."""
    vec = V.dim() == 1
    Y = _KernelMatVec.apply(X, theta, V.unsqueeze(0) if vec else V, kind, prec)
    return Y.squeeze(0) if vec else Y


class _BilinearForm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, theta, U, W, lam0, lam_rest, kind, prec):
        th = _host_theta(theta)
        v, _, _ = _b.gp_bilinear_grad(kind, th, X, U, W, lam0, lam_rest, value=True, dtheta=False, dX=False,
                                      prec=prec)
        ctx.save_for_backward(X, U, W)
        ctx.args = (th, float(lam0), float(lam_rest), kind, prec)
        ctx.theta_like = theta if isinstance(theta, torch.Tensor) else None
        return v.reshape(())

    @staticmethod
    def backward(ctx, g):
        X, U, W = ctx.saved_tensors
        th, lam0, lam_rest, kind, prec = ctx.args
        need_x, need_th = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if ctx.needs_input_grad[2] or ctx.needs_input_grad[3]:
            raise RuntimeError("bilinear_form treats U and W as constants; detach them")
        dX = dth = None
        if need_x or need_th:
            # the upstream scalar scales the weights lam_c
            gs = float(g)
            _, gt, gx = _b.gp_bilinear_grad(kind, th, X, U, W, lam0 * gs, lam_rest * gs, value=False,
                                            dtheta=need_th, dX=need_x, prec=prec)
            dX = gx
            if need_th:
                ref = ctx.theta_like
                dth = gt.to(ref.device, ref.dtype)
        return dX, dth, None, None, None, None, None, None


def bilinear_form(X, theta, U, W, lam0=1.0, lam_rest=1.0, kind=_b.GP_RBF, prec=_b.GP_PREC_TC16):
    """f = sum_c lam_c U_c^T H(theta, X) W_c (a 0-dim float64 tensor), differentiable in X and theta.
    Pass the same tensor as U and W for the symmetric (pathwise) form."""
    return _BilinearForm.apply(X, theta, U, W, lam0, lam_rest, kind, prec)
