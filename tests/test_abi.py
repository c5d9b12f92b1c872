"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a,
loads, exports every entry point include/gp.h declares, rejects invalid
arguments before touching the device, and runs its host-only Adam step like
the oracle."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2405_18457_gb300 import build

    build.build()
    from paper_2405_18457_gb300 import _binding

    return _binding.library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["gp_kernel_mvm", "gp_solve_cg", "gp_solve_ap", "gp_solve_sgd", "gp_rff_prior_sample",
                     "gp_mll_grad_standard", "gp_mll_grad_pathwise", "gp_posterior_samples",
                     "gp_adam_softplus_step", "gp_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_arguments_are_rejected_on_the_host(lib):
    from paper_2405_18457_gb300 import _binding as b

    pd = ctypes.POINTER(ctypes.c_double)
    bad = np.array([1.0, -1.0, 1.0, 0.1])  # negative length scale
    st = lib.gp_kernel_mvm(0, bad.ctypes.data_as(pd), 2, ctypes.c_void_p(16), 4, ctypes.c_void_p(16), 4,
                           ctypes.c_void_p(16), 4, 1, ctypes.c_void_p(16), 4, 0, b.GP_PREC_FP32, None, 0, None)
    assert st == -1 and b"theta[1]" in lib.gp_last_error()
    good = np.array([1.0, 1.0, 1.0, 0.1])
    st = lib.gp_kernel_mvm(0, good.ctypes.data_as(pd), 2, ctypes.c_void_p(16), 4, ctypes.c_void_p(16), 4,
                           ctypes.c_void_p(16), 2, 1, ctypes.c_void_p(16), 4, 0, b.GP_PREC_FP32, None, 0, None)
    assert st == -1 and b"ldv" in lib.gp_last_error()
    st = lib.gp_kernel_mvm(7, good.ctypes.data_as(pd), 2, ctypes.c_void_p(16), 4, ctypes.c_void_p(16), 4,
                           ctypes.c_void_p(16), 4, 1, ctypes.c_void_p(16), 4, 0, b.GP_PREC_FP32, None, 0, None)
    assert st == -1 and b"kind" in lib.gp_last_error()
    info = b._Info()
    st = lib.gp_solve_ap(0, good.ctypes.data_as(pd), 2, ctypes.c_void_p(16), 8, ctypes.c_void_p(16), 1,
                         ctypes.c_void_p(16), 4096, 10, 0.01, 0, b.GP_PREC_FP32, ctypes.byref(info), None, 0, None)
    assert st == -1 and b"block_size" in lib.gp_last_error()
    # a zero-sized product is a valid no-op that touches nothing
    assert lib.gp_kernel_mvm(0, good.ctypes.data_as(pd), 2, None, 0, None, 0, None, 0, 3, None, 0, 0,
                             b.GP_PREC_FP32, None, 0, None) == 0


def test_workspace_queries_are_consistent(lib):
    a = lib.gp_solve_cg_workspace(1000, 8, 9, 1)
    b = lib.gp_solve_cg_workspace(2000, 8, 9, 1)
    assert 0 < a < b and a % 256 == 0
    assert lib.gp_solve_ap_workspace(1000, 8, 9, 100, 1) > 10 * 100 * 100 * 4


def test_adam_step_matches_oracle(lib):
    from paper_2405_18457_gb300 import _binding as b

    rng = np.random.default_rng(0)
    nu1, m1, v1 = rng.standard_normal(6), np.zeros(6), np.zeros(6)
    nu2, m2, v2 = nu1.copy(), m1.copy(), v1.copy()
    for t in range(1, 6):
        g = rng.standard_normal(6)
        th1 = b.gp_adam_softplus_step(nu1, m1, v1, t, g, lr=0.05)
        th2 = oracle.adam_softplus(nu2, m2, v2, t, g, lr=0.05)
        np.testing.assert_allclose(th1, th2, rtol=1e-14)
        np.testing.assert_allclose(nu1, nu2, rtol=1e-14)


def test_batch_plan_layout_on_the_host(lib):
    """The batch plan is a host object: packed offsets and workspace size need no device."""
    vp = ctypes.c_void_p
    n = np.array([5, 300, 1000], dtype=np.int64)
    d = np.array([4, 32, 16], dtype=np.int32)
    s = 2
    h = vp()
    assert lib.gp_batch_create(0, 3, n.ctypes.data_as(vp), d.ctypes.data_as(vp), s, ctypes.byref(h)) == 0
    try:
        xl, vl, tl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        assert lib.gp_batch_layout(h, ctypes.byref(xl), ctypes.byref(vl), ctypes.byref(tl)) == 0
        assert xl.value == int((n * d).sum())
        assert vl.value == (s + 1) * int(n.sum())
        assert tl.value == int((d + 2).sum())
        xo, vo, to = (np.zeros(3, dtype=np.int64) for _ in range(3))
        assert lib.gp_batch_member_offsets(h, xo.ctypes.data_as(vp), vo.ctypes.data_as(vp),
                                           to.ctypes.data_as(vp)) == 0
        np.testing.assert_array_equal(xo, [0, 20, 20 + 300 * 32])
        np.testing.assert_array_equal(vo, [0, 15, 15 + 900])
        np.testing.assert_array_equal(to, [0, 6, 40])
        ws = lib.gp_batch_workspace(h)
        assert ws > 0 and ws % 256 == 0
        # device work before gp_batch_bind is refused on the host
        assert lib.gp_batch_prepare(h, vp(16), vp(16), None) == -1
        assert b"bind" in lib.gp_last_error()
    finally:
        lib.gp_batch_destroy(h)


@pytest.mark.parametrize("kind,nn,dd,s,msg", [(0, [10, 0], [4, 4], 2, b"n ="), (0, [10], [33], 2, b"d ="),
                                              (0, [10], [4], 0, b"s must"), (5, [10], [4], 2, b"kind")])
def test_batch_plan_rejects_bad_shapes(lib, kind, nn, dd, s, msg):
    vp = ctypes.c_void_p
    n = np.array(nn, dtype=np.int64)
    d = np.array(dd, dtype=np.int32)
    h = vp()
    assert lib.gp_batch_create(kind, len(nn), n.ctypes.data_as(vp), d.ctypes.data_as(vp), s,
                               ctypes.byref(h)) == -1
    assert msg in lib.gp_last_error() and not h.value
