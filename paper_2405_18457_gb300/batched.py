"""Batches of independent GPs of uneven size over the gp_batch_* C ABI
(argument marshalling and packing only; every step runs in the library's kernels).

A batch packs its members one after another:
  points       X      : member g's (n_g, d_g) rows, flattened, concatenated
  vector blocks B, V  : member g's (R, n_g) block (R = s + 1), flattened, concatenated
  hyperparameters     : member g's d_g + 2 values [l_1..l_d, s_f, sigma], concatenated
``pack_*`` / ``unpack_*`` convert between lists of per-member arrays and the packed
device tensors.  After construction no method synchronises the device except
``status()`` and ``info()``, so a sequence of calls (e.g. ``step``) can be captured
with ``torch.cuda.graph`` and replayed.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _binding as _b

_INFO_DTYPE = np.dtype([("iters", "<i8"), ("converged", "<i4"), ("status", "<i4"), ("res_y", "<f8"),
                        ("res_z", "<f8")])


class GPBatch:
    """Plan + bound workspace for G members (kind, n[g], d[g], s probes each)."""

    def __init__(self, kind, n, d, s, device="cuda"):
        lib = _b.library()
        self.kind = int(kind)
        self.n = np.ascontiguousarray(np.asarray(n, dtype=np.int64))
        self.d = np.ascontiguousarray(np.asarray(d, dtype=np.int32))
        if self.n.shape != self.d.shape or self.n.ndim != 1:
            raise ValueError("n and d must be 1-D sequences of equal length")
        self.G = int(self.n.size)
        self.s = int(s)
        self.R = self.s + 1
        h = ctypes.c_void_p()
        _b._check(lib.gp_batch_create(self.kind, self.G, self.n.ctypes.data_as(ctypes.c_void_p),
                                      self.d.ctypes.data_as(ctypes.c_void_p), self.s, ctypes.byref(h)))
        self._h = h
        self._lib = lib
        xl, vl, tl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _b._check(lib.gp_batch_layout(h, ctypes.byref(xl), ctypes.byref(vl), ctypes.byref(tl)))
        self.x_len, self.vec_len, self.theta_len = int(xl.value), int(vl.value), int(tl.value)
        self.x_off = np.zeros(self.G, dtype=np.int64)
        self.vec_off = np.zeros(self.G, dtype=np.int64)
        self.theta_off = np.zeros(self.G, dtype=np.int64)
        _b._check(lib.gp_batch_member_offsets(h, self.x_off.ctypes.data_as(ctypes.c_void_p),
                                              self.vec_off.ctypes.data_as(ctypes.c_void_p),
                                              self.theta_off.ctypes.data_as(ctypes.c_void_p)))
        self.device = torch.device(device)
        nbytes = int(lib.gp_batch_workspace(h))
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        _b._check(lib.gp_batch_bind(h, _b._ptr(self.ws), nbytes, _b._stream()))
        self._info = torch.zeros(self.G * _INFO_DTYPE.itemsize, dtype=torch.uint8, device=self.device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.gp_batch_destroy(h)
            self._h = None

    # ------------------------------------------------------------------ packing
    def pack_points(self, Xs):
        return torch.cat([torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32).reshape(-1)
                          for x in Xs]).to(self.device)

    def pack_vectors(self, blocks):
        out = torch.cat([torch.as_tensor(np.ascontiguousarray(b), dtype=torch.float32).reshape(-1)
                         for b in blocks]).to(self.device)
        if out.numel() != self.vec_len:
            raise ValueError("vector blocks must be (R, n_g) per member")
        return out

    def unpack_vectors(self, V):
        return [V[int(o):int(o) + self.R * int(n)].reshape(self.R, int(n)) for o, n in zip(self.vec_off, self.n)]

    def pack_theta(self, thetas):
        return torch.cat([torch.as_tensor(np.asarray(t, dtype=np.float64)) for t in thetas]).to(self.device)

    def unpack_theta(self, theta):
        return [theta[int(o):int(o) + int(d) + 2] for o, d in zip(self.theta_off, self.d)]

    # ------------------------------------------------------------------ operations
    def _chk(self, t, dtype, numel, name):
        if t.dtype != dtype or not t.is_cuda or not t.is_contiguous() or t.numel() != numel:
            raise ValueError("%s must be a contiguous CUDA %s tensor of %d elements" % (name, dtype, numel))
        return _b._ptr(t)

    def prepare(self, theta, X):
        _b._check(self._lib.gp_batch_prepare(self._h, self._chk(theta, torch.float64, self.theta_len, "theta"),
                                             self._chk(X, torch.float32, self.x_len, "X"), _b._stream()))

    def mvm(self, V, add_noise=True, out=None):
        Y = torch.empty_like(V) if out is None else out
        _b._check(self._lib.gp_batch_mvm(self._h, self._chk(V, torch.float32, self.vec_len, "V"),
                                         self._chk(Y, torch.float32, self.vec_len, "Y"), int(bool(add_noise)),
                                         _b._stream()))
        return Y

    def solve_cg(self, B, V, iters, tol, stop_rule=_b.GP_STOP_BOTH):
        """Alg. 1 on every member; V is the warm start and is overwritten."""
        _b._check(self._lib.gp_batch_solve_cg(self._h, self._chk(B, torch.float32, self.vec_len, "B"),
                                              self._chk(V, torch.float32, self.vec_len, "V"), int(iters),
                                              float(tol), int(stop_rule), _b._ptr(self._info), _b._stream()))
        return V

    def info(self):
        """Per-member solver reports of the last solve (synchronises)."""
        raw = self._info.cpu().numpy().view(_INFO_DTYPE)
        return [dict(iters=int(r["iters"]), converged=bool(r["converged"]), status=int(r["status"]),
                     res_y=float(r["res_y"]), res_z=float(r["res_z"])) for r in raw]

    def mll_grad(self, theta, X, Vsol, B=None, pathwise=False, out=None):
        g = torch.empty(self.theta_len, dtype=torch.float64, device=self.device) if out is None else out
        _b._check(self._lib.gp_batch_mll_grad(
            self._h, self._chk(theta, torch.float64, self.theta_len, "theta"),
            self._chk(X, torch.float32, self.x_len, "X"), self._chk(Vsol, torch.float32, self.vec_len, "Vsol"),
            None if pathwise else self._chk(B, torch.float32, self.vec_len, "B"), int(bool(pathwise)),
            self._chk(g, torch.float64, self.theta_len, "grad"), _b._stream()))
        return g

    def adam_init(self, theta):
        """Adam state for softplus parameters: nu = softplus^-1(theta), m = v = 0, t = 0 (device)."""
        st = {k: torch.empty(self.theta_len, dtype=torch.float64, device=self.device) for k in ("nu", "m", "v")}
        st["t"] = torch.zeros(1, dtype=torch.int64, device=self.device)
        _b._check(self._lib.gp_batch_adam_init(self._h, _b._ptr(theta), _b._ptr(st["nu"]), _b._ptr(st["m"]),
                                               _b._ptr(st["v"]), _b._ptr(st["t"]), _b._stream()))
        return st

    def adam_step(self, state, grad, theta, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _b._check(self._lib.gp_batch_adam_step(self._h, _b._ptr(state["nu"]), _b._ptr(state["m"]),
                                               _b._ptr(state["v"]), _b._ptr(state["t"]), _b._ptr(grad), float(lr),
                                               float(beta1), float(beta2), float(eps), _b._ptr(theta),
                                               _b._stream()))

    def step(self, X, theta, B, V, iters, tol, state, lr, grad):
        """One marginal-likelihood step for every member (prepare, warm-started CG, standard
        estimator, Adam); theta, V, grad and the Adam state are updated in place."""
        _b._check(self._lib.gp_batch_step(
            self._h, self._chk(X, torch.float32, self.x_len, "X"),
            self._chk(theta, torch.float64, self.theta_len, "theta"), self._chk(B, torch.float32, self.vec_len, "B"),
            self._chk(V, torch.float32, self.vec_len, "V"), int(iters), float(tol),
            self._chk(grad, torch.float64, self.theta_len, "grad"), _b._ptr(state["nu"]), _b._ptr(state["m"]),
            _b._ptr(state["v"]), _b._ptr(state["t"]), float(lr), _b._ptr(self._info), _b._stream()))

    def status(self):
        """Raises GPError if a device-side check failed since the bind (synchronises)."""
        _b._check(self._lib.gp_batch_status(self._h, _b._stream()))
