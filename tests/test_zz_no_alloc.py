"""gp_mll_grad_pathwise_noalloc: the allocation-free pathwise estimator.

Some callers cannot allocate device memory where they call the library (inside a
stream capture, in a stream host callback, under a fixed memory budget).  This
entry point keeps its scratch in a static device array instead of a workspace.
The test calls it through the C ABI twice in a row (the second call reuses the
array left as the first call left it) and compares each result with the
regular, workspace-taking gp_mll_grad_pathwise on the same inputs, within the
gradient tolerance the parity tests use, and with the FP64 oracle.  It also
checks that a request larger than the static array is refused with a clear
message.  This file sorts last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2405_18457_gb300 import _binding as b
from paper_2405_18457_gb300 import workloads

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, kind, theta, X, V, s, grad, prec):
    pd = ctypes.POINTER(ctypes.c_double)
    fn = lib.gp_mll_grad_pathwise_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, pd, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    th = np.ascontiguousarray(theta, dtype=np.float64)
    return fn(kind, th.ctypes.data_as(pd), X.shape[1], ctypes.c_void_p(X.data_ptr()), X.shape[0],
              ctypes.c_void_p(V.data_ptr()), s, ctypes.c_void_p(grad.data_ptr()), prec,
              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec", [b.GP_PREC_FP32, b.GP_PREC_TC16])
def test_noalloc_gradient_matches_workspace_entry_point_twice(prec):
    assert torch.cuda.is_available()
    lib = b.library()
    dev = torch.device("cuda:0")
    p = workloads.pathwise(n=1500, d=7, s=12, m=64, seed=11)
    X = torch.tensor(p.X, dtype=torch.float32, device=dev)
    for call in range(2):
        V = torch.tensor(workloads.vectors(p.s + 1, p.n, seed=20 + call), dtype=torch.float32, device=dev)
        ref = b.gp_mll_grad_pathwise(p.kind, p.theta, X, V, prec=prec).cpu().numpy()
        g = torch.full((p.d + 2,), float("nan"), dtype=torch.float64, device=dev)
        st = _call_noalloc(lib, p.kind, p.theta, X, V, p.s, g, prec)
        assert st == 0, lib.gp_last_error()
        got = g.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
        # and the estimator itself (FP64 oracle on the same FP32 inputs), per component
        Vh = V.double().cpu().numpy()
        Xh = p.X.astype(np.float32).astype(np.float64)
        exact = oracle.grad_pathwise(p.kind, p.theta, Xh, Vh)
        lam = np.concatenate([[0.5], np.full(p.s, -0.5 / p.s)])
        scale = oracle.grad_bilinear(p.kind, p.theta, Xh, np.abs(Vh), np.abs(Vh), np.abs(lam))
        tol = 1e-4 if prec == b.GP_PREC_FP32 else 1e-3
        assert np.all(np.abs(got - exact) <= tol * (np.abs(exact) + scale))


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    """A real request that needs more than the array: the tensor-core form at n = 20000, d = 16,
    s = 64 needs about 18 MB of fp16 operands; the buffers passed are of that real size."""
    lib = b.library()
    dev = torch.device("cuda:0")
    n, d, s = 20000, 16, 64
    need = lib.gp_mll_grad_workspace(n, d, s, b.GP_PREC_TC16)
    assert need > (8 << 20)
    X = torch.zeros((n, d), dtype=torch.float32, device=dev)
    V = torch.zeros((s + 1, n), dtype=torch.float32, device=dev)
    g = torch.zeros(d + 2, dtype=torch.float64, device=dev)
    st = _call_noalloc(lib, 1, np.ones(d + 2), X, V, s, g, b.GP_PREC_TC16)
    assert st == -1
    assert b"static scratch" in lib.gp_last_error()
