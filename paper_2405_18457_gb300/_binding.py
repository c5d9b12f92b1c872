"""ctypes binding of libgp_gb300.so (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

GP_RBF = 0
GP_MATERN32 = 1
GP_PREC_FP32 = 1
GP_PREC_TC16 = 2
GP_PREC_TC16X3 = 3
GP_STOP_BOTH = 0
GP_STOP_EITHER = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBNAME = "libgp_gb300.so"
_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_d = ctypes.c_double
_sz = ctypes.c_size_t
_pd = ctypes.POINTER(ctypes.c_double)


class GPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("gp status %d: %s" % (status, msg))
        self.status = status


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("converged", ctypes.c_int), ("status", ctypes.c_int),
                ("res_y", ctypes.c_double), ("res_z", ctypes.c_double)]


@dataclass
class SolveInfo:
    iters: int
    converged: bool
    status: int
    res_y: float
    res_z: float


def library_path() -> str:
    return os.path.join(_HERE, _LIBNAME)


_SIGS = {
    "gp_last_error": (ctypes.c_char_p, []),
    "gp_version": (_i, []),
    "gp_kernel_mvm": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i64, _vp, _i64, _i, _vp, _i64, _i, _i, _vp, _sz, _vp]),
    "gp_kernel_mvm_workspace": (_sz, [_i64, _i64, _i, _i, _i]),
    "gp_kernel_mvm_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i64, _vp, _i64, _i, _vp, _i64, _i, _vp, _sz, _vp]),
    "gp_kernel_mvm_f64_workspace": (_sz, [_i64, _i64, _i, _i]),
    "gp_solve_cg": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i64, _d, _i, _i, ctypes.POINTER(_Info), _vp, _sz, _vp]),
    "gp_solve_cg_workspace": (_sz, [_i64, _i, _i, _i]),
    "gp_solve_cg_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i64, _d, _i, ctypes.POINTER(_Info), _vp, _sz, _vp]),
    "gp_solve_cg_f64_workspace": (_sz, [_i64, _i, _i]),
    "gp_solve_pcg": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i64, _d, _i, _i, _i, ctypes.POINTER(_Info), _vp,
                          _sz, _vp]),
    "gp_solve_pcg_workspace": (_sz, [_i64, _i, _i, _i, _i]),
    "gp_solve_pcg_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i64, _d, _i, _i, ctypes.POINTER(_Info), _vp,
                              _sz, _vp]),
    "gp_solve_pcg_f64_workspace": (_sz, [_i64, _i, _i, _i]),
    "gp_solve_ap": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i64, _i64, _d, _i, _i, ctypes.POINTER(_Info), _vp, _sz,
                         _vp]),
    "gp_solve_ap_workspace": (_sz, [_i64, _i, _i, _i64, _i]),
    "gp_solve_ap_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i64, _i64, _d, _i, ctypes.POINTER(_Info), _vp, _sz,
                             _vp]),
    "gp_solve_ap_f64_workspace": (_sz, [_i64, _i, _i, _i64]),
    "gp_solve_sgd": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i64, _vp, _d, _d, _i64, _d, _i, _i,
                          ctypes.POINTER(_Info), _vp, _sz, _vp]),
    "gp_solve_sgd_workspace": (_sz, [_i64, _i, _i, _i64, _i]),
    "gp_solve_sgd_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i64, _vp, _d, _d, _i64, _d, _i,
                              ctypes.POINTER(_Info), _vp, _sz, _vp]),
    "gp_solve_sgd_f64_workspace": (_sz, [_i64, _i, _i, _i64]),
    "gp_bilinear_grad": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i64, _vp, _i64, _i, _d, _d, _vp, _vp, _vp, _i, _vp, _sz,
                              _vp]),
    "gp_bilinear_grad_workspace": (_sz, [_i64, _i, _i, _i]),
    "gp_bilinear_grad_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i64, _vp, _i64, _i, _d, _d, _vp, _vp, _vp, _vp, _sz,
                                  _vp]),
    "gp_bilinear_grad_f64_workspace": (_sz, [_i64, _i, _i]),
    "gp_batch_create": (_i, [_i, _i, _vp, _vp, _i, ctypes.POINTER(_vp)]),
    "gp_batch_destroy": (None, [_vp]),
    "gp_batch_workspace": (_sz, [_vp]),
    "gp_batch_layout": (_i, [_vp, _vp, _vp, _vp]),
    "gp_batch_member_offsets": (_i, [_vp, _vp, _vp, _vp]),
    "gp_batch_bind": (_i, [_vp, _vp, _sz, _vp]),
    "gp_batch_status": (_i, [_vp, _vp]),
    "gp_batch_prepare": (_i, [_vp, _vp, _vp, _vp]),
    "gp_batch_mvm": (_i, [_vp, _vp, _vp, _i, _vp]),
    "gp_batch_solve_cg": (_i, [_vp, _vp, _vp, _i64, _d, _i, _vp, _vp]),
    "gp_batch_mll_grad": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp, _vp]),
    "gp_batch_adam_init": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gp_batch_adam_step": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _d, _d, _d, _d, _vp, _vp]),
    "gp_batch_step": (_i, [_vp, _vp, _vp, _vp, _vp, _i64, _d, _vp, _vp, _vp, _vp, _vp, _d, _vp, _vp]),
    "gp_autotune_mvm": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i, ctypes.POINTER(_i), _pd, _vp, _sz, _vp]),
    "gp_autotune_mvm_workspace": (_sz, [_i64, _i, _i]),
    "gp_autotune_reset": (None, []),
    "gp_autotune_grad": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i, ctypes.POINTER(_i64), _pd, _vp, _sz, _vp]),
    "gp_autotune_grad_workspace": (_sz, [_i64, _i, _i]),
    "gp_autotune_save": (_i, [ctypes.c_char_p]),
    "gp_autotune_load": (_i, [ctypes.c_char_p]),
    "gp_autotune_count": (_i64, []),
    "gp_predict": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i64, _vp, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _sz, _vp]),
    "gp_predict_workspace": (_sz, [_i64, _i64, _i, _i, _i]),
    "gp_rkhs_sqdist": (_i, [_i, _pd, _i, _vp, _i64, _vp, _vp, _i, _vp, _i, _vp, _sz, _vp]),
    "gp_rkhs_sqdist_workspace": (_sz, [_i64, _i, _i, _i]),
    "gp_rkhs_sqdist_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _vp, _i, _vp, _vp, _sz, _vp]),
    "gp_rkhs_sqdist_f64_workspace": (_sz, [_i64, _i, _i]),
    "gp_rff_prior_sample": (_i, [_i, _pd, _i, _vp, _i64, _i, _vp, _vp, _vp, _i, _vp, _i64, _vp]),
    "gp_rff_prior_sample_f64": (_i, [_i, _pd, _i, _vp, _i64, _i, _vp, _vp, _vp, _i, _vp, _i64, _vp]),
    "gp_device_check": (_i, [_vp]),
    "gp_diag_timeout_probe": (_i, [ctypes.c_longlong, _vp]),
    "gp_diag_unit_rates_workspace": (_sz, []),
    "gp_diag_unit_rates": (_i, [_i, _pd, _vp, _sz, _vp]),
    "gp_rff_prior_sample_ws": (_i, [_i, _pd, _i, _vp, _i64, _i, _vp, _vp, _vp, _i, _vp, _i64, _i, _vp, _sz, _vp]),
    "gp_rff_prior_sample_workspace": (_sz, [_i, _i, _i, _i]),
    "gp_pathwise_rhs": (_i, [_pd, _i, _vp, _vp, _vp, _i64, _i, _vp, _vp]),
    "gp_mll_grad_standard": (_i, [_i, _pd, _i, _vp, _i64, _vp, _vp, _i, _vp, _i, _vp, _sz, _vp]),
    "gp_mll_grad_pathwise": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _i, _vp, _sz, _vp]),
    "gp_mll_grad_workspace": (_sz, [_i64, _i, _i, _i]),
    "gp_mll_grad_standard_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _vp, _i, _vp, _vp, _sz, _vp]),
    "gp_mll_grad_pathwise_f64": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i, _vp, _vp, _sz, _vp]),
    "gp_mll_grad_f64_workspace": (_sz, [_i64, _i, _i]),
    "gp_posterior_samples": (_i, [_i, _pd, _i, _vp, _i64, _vp, _i64, _vp, _i, _vp, _vp, _i, _vp, _sz, _vp]),
    "gp_posterior_samples_workspace": (_sz, [_i64, _i64, _i, _i, _i]),
    "gp_adam_softplus_step": (_i, [_i, _pd, _pd, _pd, _i64, _pd, _d, _d, _d, _d, _pd]),
    "gp_diag_reset": (None, [_i]),
    "gp_diag_launches": (ctypes.c_longlong, []),
    "gp_diag_product_time": (_i, [_pd, ctypes.POINTER(ctypes.c_longlong)]),
    "gp_diag_kernel_time": (_i, [_i, _pd, ctypes.POINTER(ctypes.c_longlong)]),
}


def gp_diag_kernel_time(which: int):
    """(total milliseconds, launches) since the reset of the product kernels (0) or
    the tensor-core gradient kernel (1)."""
    ms = ctypes.c_double()
    cnt = ctypes.c_longlong()
    _check(library().gp_diag_kernel_time(int(which), ctypes.byref(ms), ctypes.byref(cnt)))
    return float(ms.value), int(cnt.value)


def gp_diag_reset(time_products: bool = False) -> None:
    """Zero the library's launch counter; optionally time every product kernel."""
    library().gp_diag_reset(1 if time_products else 0)


def gp_diag_launches() -> int:
    return int(library().gp_diag_launches())


def gp_device_check():
    """Raise GPError(GP_ERR_TIMEOUT) if a bounded device wait gave up since the last check."""
    _check(library().gp_device_check(_stream()))


UNIT_RATE_NAMES = ("ex2", "rsqrt", "sin", "cos", "ffma", "dfma")


def gp_diag_unit_rates(iters=4096, device=None):
    """Measured thread-instructions per SM per clock of ex2, rsqrt, sin, cos (MUFU), FP32 FMA and
    FP64 FMA on the current device (gp_diag_unit_rates), as a dict."""
    lib = library()
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    ws, wsb = _ws(lib.gp_diag_unit_rates_workspace(), dev)
    out = (ctypes.c_double * 6)()
    _check(lib.gp_diag_unit_rates(int(iters), out, _ptr(ws), wsb, _stream()))
    return {k: float(v) for k, v in zip(UNIT_RATE_NAMES, out)}


def gp_diag_timeout_probe(wait_cycles):
    """Launch one bounded wait that nothing completes (exercises the time-out status)."""
    _check(library().gp_diag_timeout_probe(int(wait_cycles), _stream()))


def gp_diag_product_time():
    """(total milliseconds, launches) of the timed product kernels since the reset."""
    ms = ctypes.c_double()
    cnt = ctypes.c_longlong()
    _check(library().gp_diag_product_time(ctypes.byref(ms), ctypes.byref(cnt)))
    return float(ms.value), int(cnt.value)


def library():
    """Loads libgp_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise ImportError("%s is missing: run __graft_entry__.build() (nvcc, sm_103a) first" % path)
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != 0:
        msg = library().gp_last_error().decode(errors="replace")
        raise GPError(status, msg)


def _theta(theta, d):
    arr = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).ravel())
    if arr.size != d + 2:
        raise ValueError("theta must hold d+2 = %d values" % (d + 2))
    return arr, arr.ctypes.data_as(_pd)


def _dev(t: torch.Tensor, dtype, name: str, ndim=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor (no CPU fallback)" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if ndim is not None and t.dim() != ndim:
        raise ValueError("%s must have %d dims" % (name, ndim))
    return t


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _stream():
    return _vp(torch.cuda.current_stream().cuda_stream)


def _ws(nbytes: int, device):
    if nbytes == 0:
        return None, 0
    buf = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
    assert buf.data_ptr() % 256 == 0
    return buf, int(nbytes)


def _f64(X: torch.Tensor) -> bool:
    return X.dtype == torch.float64


def gp_kernel_mvm(kind, theta, X1, V, X2=None, add_noise=False, prec=GP_PREC_TC16, out=None):
    """Y = K(X1, X2) V (+ sigma^2 V).  X1 (n1, d), X2 (n2, d), V (R, n2) -> Y (R, n1).
    float64 inputs use the plain FP64 form (prec ignored)."""
    lib = library()
    dt = X1.dtype
    _dev(X1, dt, "X1", 2)
    X2 = X1 if X2 is None else _dev(X2, dt, "X2", 2)
    _dev(V, dt, "V", 2)
    n1, d = X1.shape
    n2 = X2.shape[0]
    R = V.shape[0]
    if V.shape[1] != n2:
        raise ValueError("V must be (R, n2)")
    th, thp = _theta(theta, d)
    Y = torch.empty((R, n1), dtype=dt, device=X1.device) if out is None else _dev(out, dt, "out", 2)
    if _f64(X1):
        wsb = lib.gp_kernel_mvm_f64_workspace(n1, n2, d, R)
        ws, wsb = _ws(wsb, X1.device)
        _check(lib.gp_kernel_mvm_f64(kind, thp, d, _ptr(X1), n1, _ptr(X2), n2, _ptr(V), n2, R, _ptr(Y), n1,
                                     int(bool(add_noise)), _ptr(ws), wsb, _stream()))
    else:
        wsb = lib.gp_kernel_mvm_workspace(n1, n2, d, R, prec)
        ws, wsb = _ws(wsb, X1.device)
        _check(lib.gp_kernel_mvm(kind, thp, d, _ptr(X1), n1, _ptr(X2), n2, _ptr(V), n2, R, _ptr(Y), n1,
                                 int(bool(add_noise)), prec, _ptr(ws), wsb, _stream()))
    return Y


def gp_autotune_mvm(kind, theta, X, V, reps=3):
    """Times the tensor-core product H V for a ladder of column-split counts and records the
    fastest for its shape (used by later products of that shape).  Returns (splits, ms)."""
    lib = library()
    _dev(X, torch.float32, "X", 2)
    _dev(V, torch.float32, "V", 2)
    n, d = X.shape
    R = V.shape[0]
    th, thp = _theta(theta, d)
    Y = torch.empty_like(V)
    ws, wsb = _ws(lib.gp_autotune_mvm_workspace(n, d, R), X.device)
    best = ctypes.c_int()
    ms = ctypes.c_double()
    _check(lib.gp_autotune_mvm(kind, thp, d, _ptr(X), n, _ptr(V), R, _ptr(Y), int(reps), ctypes.byref(best),
                               ctypes.byref(ms), _ptr(ws), wsb, _stream()))
    return int(best.value), float(ms.value)


def gp_autotune_reset():
    library().gp_autotune_reset()


def gp_autotune_grad(kind, theta, X, Vsol, Z=None, reps=3):
    """Times the tensor-core gradient's work splits for this shape (pathwise estimator when Z is
    None, else the standard estimator with probes Z) and records the fastest; returns
    (best work-split parameter, its time in ms)."""
    lib = library()
    _dev(X, torch.float32, "X", 2)
    n, d = X.shape
    _dev(Vsol, torch.float32, "Vsol", 2)
    s = Vsol.shape[0] - 1
    if Z is not None:
        _dev(Z, torch.float32, "Z", 2)
    th, thp = _theta(theta, d)
    ws, wsb = _ws(lib.gp_autotune_grad_workspace(n, d, s), X.device)
    best = ctypes.c_int64(0)
    ms = ctypes.c_double(0.0)
    _check(lib.gp_autotune_grad(kind, thp, d, _ptr(X), n, _ptr(Vsol), s, _ptr(Z), int(reps), ctypes.byref(best),
                                ctypes.byref(ms), _ptr(ws), wsb, _stream()))
    return int(best.value), float(ms.value)


def gp_autotune_save(path):
    """Writes the autotuner's recorded choices to `path` (tagged with this device)."""
    _check(library().gp_autotune_save(str(path).encode()))


def gp_autotune_load(path):
    """Adds the choices recorded in `path` (written on this kind of device) to the table."""
    _check(library().gp_autotune_load(str(path).encode()))


def gp_autotune_count():
    return int(library().gp_autotune_count())


def _info(inf: _Info) -> SolveInfo:
    return SolveInfo(int(inf.iters), bool(inf.converged), int(inf.status), float(inf.res_y), float(inf.res_z))


def _solver_prep(X, B, V0):
    dt = X.dtype
    _dev(X, dt, "X", 2)
    _dev(B, dt, "B", 2)
    n, d = X.shape
    R = B.shape[0]
    if B.shape[1] != n:
        raise ValueError("B must be (R, n)")
    V = torch.zeros_like(B) if V0 is None else _dev(V0, dt, "V0", 2)
    if V.shape != B.shape:
        raise ValueError("V0 must match B")
    return dt, n, d, R, V


def gp_solve_cg(kind, theta, X, B, V0=None, max_iters=1000, tol=1e-2, stop_rule=GP_STOP_BOTH, prec=GP_PREC_TC16,
                precond_rank=0):
    """Alg. 1 (CG).  V0 (R, n) is the warm start and is overwritten with the solution.
    precond_rank > 0: the rank-k pivoted Cholesky preconditioner of App. B (gp_solve_pcg)."""
    lib = library()
    dt, n, d, R, V = _solver_prep(X, B, V0)
    th, thp = _theta(theta, d)
    inf = _Info()
    if precond_rank > 0:
        k = int(precond_rank)
        if _f64(X):
            ws, wsb = _ws(lib.gp_solve_pcg_f64_workspace(n, d, R, k), X.device)
            _check(lib.gp_solve_pcg_f64(kind, thp, d, _ptr(X), n, _ptr(B), R, _ptr(V), int(max_iters), float(tol),
                                        stop_rule, k, ctypes.byref(inf), _ptr(ws), wsb, _stream()))
        else:
            ws, wsb = _ws(lib.gp_solve_pcg_workspace(n, d, R, prec, k), X.device)
            _check(lib.gp_solve_pcg(kind, thp, d, _ptr(X), n, _ptr(B), R, _ptr(V), int(max_iters), float(tol),
                                    stop_rule, prec, k, ctypes.byref(inf), _ptr(ws), wsb, _stream()))
        return V, _info(inf)
    if _f64(X):
        ws, wsb = _ws(lib.gp_solve_cg_f64_workspace(n, d, R), X.device)
        _check(lib.gp_solve_cg_f64(kind, thp, d, _ptr(X), n, _ptr(B), R, _ptr(V), int(max_iters), float(tol),
                                   stop_rule, ctypes.byref(inf), _ptr(ws), wsb, _stream()))
    else:
        ws, wsb = _ws(lib.gp_solve_cg_workspace(n, d, R, prec), X.device)
        _check(lib.gp_solve_cg(kind, thp, d, _ptr(X), n, _ptr(B), R, _ptr(V), int(max_iters), float(tol),
                               stop_rule, prec, ctypes.byref(inf), _ptr(ws), wsb, _stream()))
    return V, _info(inf)


def gp_solve_ap(kind, theta, X, B, V0=None, block_size=1024, max_iters=1000, tol=1e-2, stop_rule=GP_STOP_BOTH,
                prec=GP_PREC_TC16):
    """Alg. 2 (alternating projections); max_iters counts block iterations."""
    lib = library()
    dt, n, d, R, V = _solver_prep(X, B, V0)
    th, thp = _theta(theta, d)
    inf = _Info()
    if _f64(X):
        ws, wsb = _ws(lib.gp_solve_ap_f64_workspace(n, d, R, block_size), X.device)
        _check(lib.gp_solve_ap_f64(kind, thp, d, _ptr(X), n, _ptr(B), R, _ptr(V), int(block_size), int(max_iters),
                                   float(tol), stop_rule, ctypes.byref(inf), _ptr(ws), wsb, _stream()))
    else:
        ws, wsb = _ws(lib.gp_solve_ap_workspace(n, d, R, block_size, prec), X.device)
        _check(lib.gp_solve_ap(kind, thp, d, _ptr(X), n, _ptr(B), R, _ptr(V), int(block_size), int(max_iters),
                               float(tol), stop_rule, prec, ctypes.byref(inf), _ptr(ws), wsb, _stream()))
    return V, _info(inf)


def gp_solve_sgd(kind, theta, X, B, batch_idx, lr, momentum=0.9, V0=None, max_iters=None, tol=1e-2,
                 stop_rule=GP_STOP_BOTH, prec=GP_PREC_TC16):
    """Alg. 3 (SGD).  batch_idx: int32 CUDA tensor (iters, batch) of row indices."""
    lib = library()
    dt, n, d, R, V = _solver_prep(X, B, V0)
    _dev(batch_idx, torch.int32, "batch_idx", 2)
    iters, batch = batch_idx.shape
    max_iters = iters if max_iters is None else int(max_iters)
    if max_iters > iters:
        raise ValueError("batch_idx holds %d iterations, %d requested" % (iters, max_iters))
    th, thp = _theta(theta, d)
    inf = _Info()
    if _f64(X):
        ws, wsb = _ws(lib.gp_solve_sgd_f64_workspace(n, d, R, batch), X.device)
        _check(lib.gp_solve_sgd_f64(kind, thp, d, _ptr(X), n, _ptr(B), R, _ptr(V), batch, _ptr(batch_idx),
                                    float(lr), float(momentum), max_iters, float(tol), stop_rule,
                                    ctypes.byref(inf), _ptr(ws), wsb, _stream()))
    else:
        ws, wsb = _ws(lib.gp_solve_sgd_workspace(n, d, R, batch, prec), X.device)
        _check(lib.gp_solve_sgd(kind, thp, d, _ptr(X), n, _ptr(B), R, _ptr(V), batch, _ptr(batch_idx), float(lr),
                                float(momentum), max_iters, float(tol), stop_rule, prec, ctypes.byref(inf),
                                _ptr(ws), wsb, _stream()))
    return V, _info(inf)


def gp_rff_prior_sample(kind, theta, X, omega_hat, chi2, W, out=None, prec=GP_PREC_TC16):
    """Prior samples F (s, n) at X from fixed random-feature parameters.  float32: prec selects
    the tensor-core form (GP_PREC_TC16) or the CUDA-core form (GP_PREC_FP32)."""
    lib = library()
    dt = X.dtype
    _dev(X, dt, "X", 2)
    _dev(omega_hat, dt, "omega_hat", 2)
    _dev(W, dt, "W", 2)
    if chi2 is not None:
        _dev(chi2, dt, "chi2", 1)
    n, d = X.shape
    s, m = W.shape
    if omega_hat.shape != (m // 2, d):
        raise ValueError("omega_hat must be (m/2, d)")
    th, thp = _theta(theta, d)
    F = torch.empty((s, n), dtype=dt, device=X.device) if out is None else out
    if _f64(X):
        _check(lib.gp_rff_prior_sample_f64(kind, thp, d, _ptr(X), n, m, _ptr(omega_hat), _ptr(chi2), _ptr(W), s,
                                           _ptr(F), F.stride(0), _stream()))
    else:
        ws, wsb = _ws(lib.gp_rff_prior_sample_workspace(d, m, s, prec), X.device)
        _check(lib.gp_rff_prior_sample_ws(kind, thp, d, _ptr(X), n, m, _ptr(omega_hat), _ptr(chi2), _ptr(W), s,
                                          _ptr(F), F.stride(0), prec, _ptr(ws), wsb, _stream()))
    return F


def gp_pathwise_rhs(theta, d, y, F, w):
    """B = [y, F_j + sigma w_j] (float32)."""
    lib = library()
    _dev(y, torch.float32, "y", 1)
    _dev(F, torch.float32, "F", 2)
    _dev(w, torch.float32, "w", 2)
    n = y.shape[0]
    s = F.shape[0]
    th, thp = _theta(theta, d)
    B = torch.empty((s + 1, n), dtype=torch.float32, device=y.device)
    _check(lib.gp_pathwise_rhs(thp, d, _ptr(y), _ptr(F), _ptr(w), n, s, _ptr(B), _stream()))
    return B


def gp_mll_grad_standard(kind, theta, X, Vsol, Z, prec=GP_PREC_TC16):
    """Standard estimator of d L / d theta (CUDA float64 tensor of d+2)."""
    lib = library()
    dt = X.dtype
    _dev(X, dt, "X", 2)
    _dev(Vsol, dt, "Vsol", 2)
    _dev(Z, dt, "Z", 2)
    n, d = X.shape
    s = Z.shape[0]
    th, thp = _theta(theta, d)
    g = torch.empty(d + 2, dtype=torch.float64, device=X.device)
    if _f64(X):
        ws, wsb = _ws(lib.gp_mll_grad_f64_workspace(n, d, s), X.device)
        _check(lib.gp_mll_grad_standard_f64(kind, thp, d, _ptr(X), n, _ptr(Vsol), _ptr(Z), s, _ptr(g), _ptr(ws),
                                            wsb, _stream()))
    else:
        ws, wsb = _ws(lib.gp_mll_grad_workspace(n, d, s, prec), X.device)
        _check(lib.gp_mll_grad_standard(kind, thp, d, _ptr(X), n, _ptr(Vsol), _ptr(Z), s, _ptr(g), prec, _ptr(ws),
                                        wsb, _stream()))
    return g


def gp_mll_grad_pathwise(kind, theta, X, Vsol, prec=GP_PREC_TC16):
    """Pathwise estimator of d L / d theta (CUDA float64 tensor of d+2)."""
    lib = library()
    dt = X.dtype
    _dev(X, dt, "X", 2)
    _dev(Vsol, dt, "Vsol", 2)
    n, d = X.shape
    s = Vsol.shape[0] - 1
    th, thp = _theta(theta, d)
    g = torch.empty(d + 2, dtype=torch.float64, device=X.device)
    if _f64(X):
        ws, wsb = _ws(lib.gp_mll_grad_f64_workspace(n, d, s), X.device)
        _check(lib.gp_mll_grad_pathwise_f64(kind, thp, d, _ptr(X), n, _ptr(Vsol), s, _ptr(g), _ptr(ws), wsb,
                                            _stream()))
    else:
        ws, wsb = _ws(lib.gp_mll_grad_workspace(n, d, s, prec), X.device)
        _check(lib.gp_mll_grad_pathwise(kind, thp, d, _ptr(X), n, _ptr(Vsol), s, _ptr(g), prec, _ptr(ws), wsb,
                                        _stream()))
    return g


def gp_bilinear_grad(kind, theta, X, U, W, lam0=1.0, lam_rest=1.0, value=True, dtheta=True, dX=True,
                     prec=GP_PREC_TC16):
    """Derivatives of f = sum_c lam_c U[c]^T H W[c] (lam_0 = lam0, lam_c = lam_rest for c >= 1).
    Returns (value, dtheta, dX): a CUDA float64 tensor of shape (1,), a CUDA float64 tensor of
    d+2 and an (n, d) tensor in X's dtype; outputs not requested are None.  Passing the same
    tensor as U and W selects the symmetric form."""
    lib = library()
    dt = X.dtype
    _dev(X, dt, "X", 2)
    _dev(U, dt, "U", 2)
    _dev(W, dt, "W", 2)
    n, d = X.shape
    R = U.shape[0]
    if U.shape != (R, n) or W.shape != (R, n):
        raise ValueError("U and W must be (R, n)")
    th, thp = _theta(theta, d)
    dev = X.device
    v = torch.empty(1, dtype=torch.float64, device=dev) if value else None
    g = torch.empty(d + 2, dtype=torch.float64, device=dev) if dtheta else None
    gx = torch.empty((n, d), dtype=dt, device=dev) if dX else None
    if _f64(X):
        ws, wsb = _ws(lib.gp_bilinear_grad_f64_workspace(n, d, R), dev)
        _check(lib.gp_bilinear_grad_f64(kind, thp, d, _ptr(X), n, _ptr(U), n, _ptr(W), n, R, float(lam0),
                                        float(lam_rest), _ptr(v), _ptr(g), _ptr(gx), _ptr(ws), wsb, _stream()))
    else:
        ws, wsb = _ws(lib.gp_bilinear_grad_workspace(n, d, R, prec), dev)
        _check(lib.gp_bilinear_grad(kind, thp, d, _ptr(X), n, _ptr(U), n, _ptr(W), n, R, float(lam0),
                                    float(lam_rest), _ptr(v), _ptr(g), _ptr(gx), prec, _ptr(ws), wsb, _stream()))
    return v, g, gx


def gp_posterior_samples(kind, theta, Xstar, X, Vsol, Fstar, prec=GP_PREC_TC16):
    """Pathwise-conditioned posterior samples (s, nstar) at Xstar."""
    lib = library()
    _dev(Xstar, torch.float32, "Xstar", 2)
    _dev(X, torch.float32, "X", 2)
    _dev(Vsol, torch.float32, "Vsol", 2)
    _dev(Fstar, torch.float32, "Fstar", 2)
    nstar, d = Xstar.shape
    n = X.shape[0]
    s = Vsol.shape[0] - 1
    th, thp = _theta(theta, d)
    out = torch.empty((s, nstar), dtype=torch.float32, device=X.device)
    ws, wsb = _ws(lib.gp_posterior_samples_workspace(nstar, n, d, s, prec), X.device)
    _check(lib.gp_posterior_samples(kind, thp, d, _ptr(Xstar), nstar, _ptr(X), n, _ptr(Vsol), s, _ptr(Fstar),
                                    _ptr(out), prec, _ptr(ws), wsb, _stream()))
    return out


def gp_predict(kind, theta, Xstar, X, Vsol, Fstar, ystar=None, prec=GP_PREC_TC16):
    """Predictive mean and variance (nstar each) from the pathwise solutions; with ystar also
    a CUDA float64 tensor (RMSE, mean test log-likelihood)."""
    lib = library()
    for t_, nm in ((Xstar, "Xstar"), (X, "X"), (Vsol, "Vsol"), (Fstar, "Fstar")):
        _dev(t_, torch.float32, nm, 2)
    if ystar is not None:
        _dev(ystar, torch.float32, "ystar", 1)
    nstar, d = Xstar.shape
    n = X.shape[0]
    s = Vsol.shape[0] - 1
    th, thp = _theta(theta, d)
    mean = torch.empty(nstar, dtype=torch.float32, device=X.device)
    var = torch.empty(nstar, dtype=torch.float32, device=X.device)
    metrics = torch.empty(2, dtype=torch.float64, device=X.device) if ystar is not None else None
    ws, wsb = _ws(lib.gp_predict_workspace(nstar, n, d, s, prec), X.device)
    _check(lib.gp_predict(kind, thp, d, _ptr(Xstar), nstar, _ptr(X), n, _ptr(Vsol), s, _ptr(Fstar), _ptr(ystar),
                          _ptr(mean), _ptr(var), _ptr(metrics), prec, _ptr(ws), wsb, _stream()))
    return mean, var, metrics


def gp_rkhs_sqdist(kind, theta, X, U, Uinit=None, prec=GP_PREC_TC16):
    """Per column, the squared RKHS distance (Uinit[c] - U[c])^T H (Uinit[c] - U[c]) (Sec. 3,
    Eq. RKHS_distance); Uinit None is the zero initialisation.  CUDA float64 tensor of R."""
    lib = library()
    dt = X.dtype
    _dev(X, dt, "X", 2)
    _dev(U, dt, "U", 2)
    n, d = X.shape
    R = U.shape[0]
    if U.shape[1] != n:
        raise ValueError("U must be (R, n)")
    if Uinit is not None:
        _dev(Uinit, dt, "Uinit", 2)
        if Uinit.shape != U.shape:
            raise ValueError("Uinit must have U's shape")
    th, thp = _theta(theta, d)
    dist = torch.empty(R, dtype=torch.float64, device=X.device)
    if _f64(X):
        ws, wsb = _ws(lib.gp_rkhs_sqdist_f64_workspace(n, d, R), X.device)
        _check(lib.gp_rkhs_sqdist_f64(kind, thp, d, _ptr(X), n, _ptr(Uinit), _ptr(U), R, _ptr(dist), _ptr(ws), wsb,
                                      _stream()))
    else:
        ws, wsb = _ws(lib.gp_rkhs_sqdist_workspace(n, d, R, prec), X.device)
        _check(lib.gp_rkhs_sqdist(kind, thp, d, _ptr(X), n, _ptr(Uinit), _ptr(U), R, _ptr(dist), prec, _ptr(ws),
                                  wsb, _stream()))
    return dist


def gp_adam_softplus_step(nu, m, v, t, grad_theta, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam ascent step on softplus parameters (host float64 numpy arrays, updated in place);
    returns theta = softplus(nu)."""
    lib = library()
    for a in (nu, m, v):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise TypeError("nu, m, v must be contiguous float64 numpy arrays")
    g = np.ascontiguousarray(np.asarray(grad_theta, dtype=np.float64))
    P = nu.size
    theta = np.empty(P)
    pd = lambda a: a.ctypes.data_as(_pd)  # noqa: E731
    _check(lib.gp_adam_softplus_step(P, pd(nu), pd(m), pd(v), int(t), pd(g), float(lr), float(beta1), float(beta2),
                                     float(eps), pd(theta)))
    return theta
