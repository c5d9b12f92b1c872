"""Parity of the RKHS-distance diagnostic (Sec. 3, Eq. RKHS_distance) with the FP64 oracle:
FP64 form 1e-10, FP32 form 1e-5, tensor-core form 1e-3 (relative, per column), with and
without an initialisation, on a ragged size spanning several 128-row tiles; and at the
pathwise workload's full size (n = 32768, d = 16, Matern-3/2, 65 columns) on two sampled
columns, which the oracle computes exactly."""
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


@pytest.mark.parametrize("kind", [gp.GP_RBF, gp.GP_MATERN32])
@pytest.mark.parametrize("form", ["f64", "fp32", "tc16"])
@pytest.mark.parametrize("with_init", [False, True])
def test_rkhs_sqdist_parity(dev, kind, form, with_init):
    rng = np.random.default_rng([51, kind])
    n, d, R = 777, 6, 5
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.7, 1.5, size=d), [1.2, 0.25]])
    U = rng.standard_normal((R, n))
    U0 = U + 0.1 * rng.standard_normal((R, n)) if with_init else None
    dt = torch.float64 if form == "f64" else torch.float32
    Xr = X.astype(np.float32).astype(np.float64) if form != "f64" else X
    Ur = U.astype(np.float32).astype(np.float64) if form != "f64" else U
    U0r = None if U0 is None else (U0.astype(np.float32).astype(np.float64) if form != "f64" else U0)
    ref = oracle.rkhs_sqdist(kind, th, Xr, Ur, U0r)
    t = lambda a: torch.tensor(a, dtype=dt, device=dev)  # noqa: E731
    prec = gp.GP_PREC_TC16 if form == "tc16" else gp.GP_PREC_FP32
    got = gp.gp_rkhs_sqdist(kind, th, t(X), t(U), None if U0 is None else t(U0), prec=prec).cpu().numpy()
    tol = {"f64": 1e-10, "fp32": 1e-5, "tc16": 1e-3}[form]
    np.testing.assert_allclose(got, ref, rtol=tol)


def test_rkhs_sqdist_edge_cases(dev):
    X = torch.randn(130, 3, device=dev)
    th = [1.0, 1.0, 1.0, 1.0, 0.5]
    U = torch.randn(2, 130, device=dev)
    # zero distance from a point to itself; R = 0 returns an empty result
    np.testing.assert_allclose(gp.gp_rkhs_sqdist(gp.GP_RBF, th, X, U, U.clone(), prec=gp.GP_PREC_FP32).cpu(),
                               0.0, atol=1e-12)
    assert gp.gp_rkhs_sqdist(gp.GP_RBF, th, X, U[:0]).numel() == 0
    # n = 1: (u0 - u)^2 (s_f^2 + sigma^2)
    X1 = torch.zeros(1, 3, device=dev)
    u = torch.tensor([[2.0]], device=dev)
    got = gp.gp_rkhs_sqdist(gp.GP_MATERN32, th, X1, u, prec=gp.GP_PREC_FP32).item()
    assert abs(got - 4.0 * (1.0 + 0.25)) < 1e-6
    with pytest.raises(ValueError):
        gp.gp_rkhs_sqdist(gp.GP_RBF, th, X, U, U[:1])


def test_rkhs_sqdist_full_size_sampled_columns(dev):
    p = workloads.pathwise()
    n, R = p.n, p.s + 1
    X32 = p.X.astype(np.float32)
    U = workloads.vectors(R, n, seed=52).astype(np.float32)
    U0 = workloads.vectors(R, n, seed=53).astype(np.float32)
    got = gp.gp_rkhs_sqdist(p.kind, p.theta, torch.tensor(X32, device=dev), torch.tensor(U, device=dev),
                            torch.tensor(U0, device=dev), prec=gp.GP_PREC_TC16).cpu().numpy()
    cols = [0, 37]
    ref = oracle.rkhs_sqdist(p.kind, p.theta, X32.astype(np.float64), U[cols].astype(np.float64),
                             U0[cols].astype(np.float64))
    np.testing.assert_allclose(got[cols], ref, rtol=1e-3)
