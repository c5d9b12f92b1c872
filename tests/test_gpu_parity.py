"""GPU-vs-oracle parity of every C-ABI entry point (CUDA-core FP64 and FP32
forms, and the tcgen05 fp16 form where it is built).  Inputs come from the
seeded generators; expected values come from the FP64 CPU oracle only.

Tolerances (relative Frobenius unless stated):
  FP64 path  : 1e-10 (same arithmetic, different summation order)
  FP32 path  : MVM 1e-5, solutions/gradients 1e-4
  TC16 path  : MVM 1e-3, gradient 1e-3 (fp16 operands, FP32 accumulation)
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
    gp.library()  # fail loudly if the CUDA library is missing
    return torch.device("cuda:0")


def t(a, dev, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)


from parity_util import close, rel  # noqa: E402


PRECS = [("f64", None, 1e-10), ("f32", gp.GP_PREC_FP32, 1e-5), ("tc16", gp.GP_PREC_TC16, 1e-3),
         ("tc16x3", gp.GP_PREC_TC16X3, 1e-5)]


def run_mvm(prec_name, prec, kind, th, X1, X2, V, add_noise, dev):
    dt = torch.float64 if prec_name == "f64" else torch.float32
    X1t = t(X1, dev, dt)
    X2t = X1t if X2 is None else t(X2, dev, dt)
    Y = gp.gp_kernel_mvm(kind, th, X1t, t(V, dev, dt), X2=X2t, add_noise=add_noise,
                         prec=prec if prec is not None else gp.GP_PREC_FP32)
    torch.cuda.synchronize()
    return Y.double().cpu().numpy()


# --------------------------------------------------------------------------- MVM
@pytest.mark.parametrize("prec_name,prec,tol", PRECS)
@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
@pytest.mark.parametrize("n,d,R", [(333, 5, 9), (257, 16, 65), (130, 26, 70), (1, 3, 1), (64, 1, 17),
                                   (200, 4, 150)])
def test_hv_matches_oracle(dev, prec_name, prec, tol, kind, n, d, R):
    rng = np.random.default_rng(n * 100 + d)
    X = rng.uniform(-1, 1, size=(n, d))
    th = np.concatenate([rng.uniform(0.5, 1.5, size=d), [1.2, 0.3]])
    V = rng.standard_normal((R, n))
    Y = run_mvm(prec_name, prec, kind, th, X, None, V, True, dev)
    ref = oracle.kernel_mvm(kind, th, X, X, V, add_noise=True)
    assert close(Y, ref, tol)


@pytest.mark.parametrize("prec_name,prec,tol", PRECS)
def test_cross_kernel_product_matches_oracle(dev, prec_name, prec, tol):
    rng = np.random.default_rng(11)
    X1 = rng.standard_normal((301, 7))
    X2 = rng.standard_normal((517, 7))
    th = np.concatenate([rng.uniform(0.8, 2.0, size=7), [0.9, 0.2]])
    V = rng.standard_normal((12, 517))
    Y = run_mvm(prec_name, prec, oracle.MATERN32, th, X1, X2, V, False, dev)
    assert close(Y, oracle.kernel_mvm(oracle.MATERN32, th, X1, X2, V), tol)


@pytest.mark.parametrize("prec_name,prec,tol", PRECS)
def test_small_problem_workload_matches_oracle(dev, prec_name, prec, tol):
    """The small workload (n=2048, d=8, RBF, s=8 probes): full product."""
    p = workloads.small()
    B = np.vstack([p.y, p.Z])
    Y = run_mvm(prec_name, prec, p.kind, p.theta, p.X, None, B, True, dev)
    assert close(Y, oracle.kernel_mvm(p.kind, p.theta, p.X, p.X, B, add_noise=True), tol)


@pytest.mark.parametrize("prec_name,prec,tol", PRECS[1:])
def test_full_size_pathwise_workload_sampled_rows(dev, prec_name, prec, tol):
    """The pathwise workload at its full size (n=32768, d=16, R=65, Matern-3/2):
    the GPU product is compared with the oracle on 48 sampled rows."""
    p = workloads.pathwise()
    V = workloads.vectors(65, p.n, seed=1)
    Y = run_mvm(prec_name, prec, p.kind, p.theta, p.X.astype(np.float32), None, V.astype(np.float32), True, dev)
    rows = np.random.default_rng(2).choice(p.n, size=48, replace=False)
    Xr = p.X.astype(np.float32).astype(np.float64)
    ref = oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.astype(np.float32).astype(np.float64), add_noise=True,
                            rows=rows)
    assert close(Y[:, rows], ref, tol)


def test_empty_column_set_gives_zeros(dev):
    X1 = t(np.ones((5, 2)), dev)
    X2 = torch.zeros((0, 2), device=dev)
    V = torch.zeros((3, 0), device=dev)
    Y = gp.gp_kernel_mvm(0, [1.0, 1.0, 1.0, 0.1], X1, V, X2=X2, prec=gp.GP_PREC_FP32)
    assert torch.count_nonzero(Y).item() == 0


# --------------------------------------------------------------------------- gradients
@pytest.mark.parametrize("prec_name,prec,tol", [("f64", None, 1e-10), ("f32", gp.GP_PREC_FP32, 1e-4),
                                                ("tc16", gp.GP_PREC_TC16, 1e-3)])
@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
@pytest.mark.parametrize("estimator", ["standard", "pathwise"])
def test_gradient_estimators_match_oracle(dev, prec_name, prec, tol, kind, estimator):
    rng = np.random.default_rng(5)
    n, d, s = 203, 6, 8
    X = rng.uniform(-1, 1, size=(n, d))
    th = np.concatenate([rng.uniform(0.5, 1.5, size=d), [1.1, 0.4]])
    Vsol = rng.standard_normal((s + 1, n))
    Z = rng.standard_normal((s, n))
    dt = torch.float64 if prec_name == "f64" else torch.float32
    Xr = X.astype(np.float32).astype(np.float64) if dt == torch.float32 else X
    Vr = Vsol.astype(np.float32).astype(np.float64) if dt == torch.float32 else Vsol
    Zr = Z.astype(np.float32).astype(np.float64) if dt == torch.float32 else Z
    pr = prec if prec is not None else gp.GP_PREC_FP32
    lam = np.concatenate([[0.5], np.full(s, -0.5 / s)])
    if estimator == "standard":
        g = gp.gp_mll_grad_standard(kind, th, t(X, dev, dt), t(Vsol, dev, dt), t(Z, dev, dt), prec=pr)
        ref = oracle.grad_standard(kind, th, Xr, Vr, Zr)
        W = np.vstack([Vr[:1], Zr])
    else:
        g = gp.gp_mll_grad_pathwise(kind, th, t(X, dev, dt), t(Vsol, dev, dt), prec=pr)
        ref = oracle.grad_pathwise(kind, th, Xr, Vr)
        W = Vr
    scale = oracle.grad_bilinear(kind, th, Xr, np.abs(Vr), np.abs(W), np.abs(lam))
    _per_component_ok(g.cpu().numpy(), ref, scale, tol)


def _grad_case(kind, n, d, s, seed, full_pathwise=False):
    """Inputs of a gradient check in FP32 (as the GPU sees them) and the estimator's terms."""
    if full_pathwise:
        p = workloads.pathwise()
        X = p.X.astype(np.float32)
        th = p.theta
    else:
        rng = np.random.default_rng([seed, n, d, s])
        X = rng.standard_normal((n, d)).astype(np.float32)
        th = np.concatenate([rng.uniform(0.7, 1.6, size=d) * np.sqrt(d / 8.0), [1.1, 0.3]])
    Vsol = (workloads.vectors(s + 1, X.shape[0], seed=seed) * 0.8).astype(np.float32)
    Z = workloads.vectors(s, X.shape[0], seed=seed + 1).astype(np.float32)
    return X, th, Vsol, Z


def _per_component_ok(g, ref, scale, rtol):
    """|g_k - ref_k| <= rtol |ref_k| + rtol S_k, with S_k = sum_c |lambda_c| |u_c|^T |dH/dtheta_k| |w_c|
    (the estimator evaluated on absolute values: every dH/dtheta_k is elementwise non-negative),
    so each length-scale component is checked against its own size, not the largest one."""
    err = np.abs(g - ref)
    bound = rtol * np.abs(ref) + rtol * scale
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).tolist()


@pytest.mark.parametrize("estimator", ["pathwise", "standard"])
@pytest.mark.parametrize("kind,n,d,s", [
    (oracle.MATERN32, 4099, 16, 63),    # R = 64: one 64-wide U/W atom, four GEMM-M steps
    (oracle.MATERN32, 4099, 16, 64),    # R = 65: the benched shape; second atom, five steps
    (oracle.MATERN32, 4099, 16, 79),    # R = 80
    (oracle.RBF, 4099, 16, 127),        # R = 128: two full atoms
    (oracle.RBF, 2500, 26, 64),         # d = 26: two 64-wide atoms of the distance contraction
    (oracle.MATERN32, 2049, 32, 64),    # d = 32: the widest tensor-core gradient
])
def test_tc16_gradient_matches_oracle_per_component(dev, estimator, kind, n, d, s):
    """The tensor-core gradient kernel at the right-hand-side counts and dimensions the solvers
    and the benchmark use (Eq. mll_grad with Eq. trace / Eq. pathwise_estimator), against the
    oracle, component by component (ragged n: the last 128-row and 64-column tiles are partial)."""
    X, th, Vsol, Z = _grad_case(kind, n, d, s, seed=40 + s)
    Xr, Vr, Zr = (a.astype(np.float64) for a in (X, Vsol, Z))
    lam = np.concatenate([[0.5], np.full(s, -0.5 / s)])
    if estimator == "pathwise":
        g = gp.gp_mll_grad_pathwise(kind, th, t(X, dev), t(Vsol, dev), prec=gp.GP_PREC_TC16).cpu().numpy()
        ref = oracle.grad_pathwise(kind, th, Xr, Vr)
        W = Vr
    else:
        g = gp.gp_mll_grad_standard(kind, th, t(X, dev), t(Vsol, dev), t(Z, dev),
                                    prec=gp.GP_PREC_TC16).cpu().numpy()
        ref = oracle.grad_standard(kind, th, Xr, Vr, Zr)
        W = np.vstack([Vr[:1], Zr])
    scale = oracle.grad_bilinear(kind, th, Xr, np.abs(Vr), np.abs(W), np.abs(lam))
    _per_component_ok(g, ref, scale, 1e-3)


@pytest.mark.parametrize("estimator", ["pathwise", "standard"])
def test_tc16_gradient_full_pathwise_workload_per_component(dev, estimator):
    """The benchmark's gradient call at full size: n = 32768, d = 16, Matern-3/2, s = 64 (R = 65),
    against the FP64 oracle over all n^2 pairs, component by component."""
    X, th, Vsol, Z = _grad_case(oracle.MATERN32, 0, 16, 64, seed=77, full_pathwise=True)
    Xr, Vr, Zr = (a.astype(np.float64) for a in (X, Vsol, Z))
    s = 64
    lam = np.concatenate([[0.5], np.full(s, -0.5 / s)])
    if estimator == "pathwise":
        g = gp.gp_mll_grad_pathwise(oracle.MATERN32, th, t(X, dev), t(Vsol, dev), prec=gp.GP_PREC_TC16)
        ref = oracle.grad_pathwise(oracle.MATERN32, th, Xr, Vr)
        W = Vr
    else:
        g = gp.gp_mll_grad_standard(oracle.MATERN32, th, t(X, dev), t(Vsol, dev), t(Z, dev),
                                    prec=gp.GP_PREC_TC16)
        ref = oracle.grad_standard(oracle.MATERN32, th, Xr, Vr, Zr)
        W = np.vstack([Vr[:1], Zr])
    scale = oracle.grad_bilinear(oracle.MATERN32, th, Xr, np.abs(Vr), np.abs(W), np.abs(lam))
    _per_component_ok(g.cpu().numpy(), ref, scale, 1e-3)


# --------------------------------------------------------------------------- solvers
@pytest.mark.parametrize("prec_name,prec,tol,iters", [("f64", None, 1e-9, 6), ("f32", gp.GP_PREC_FP32, 1e-4, 6),
                                                      ("tc16", gp.GP_PREC_TC16, 3e-3, 2)])
def test_cg_iterates_match_oracle(dev, prec_name, prec, tol, iters):
    """Fixed iterations from a warm start: iterate-by-iterate parity with Alg. 1.
    CG amplifies product rounding from one iteration to the next, so the fp16
    tensor-core form is compared after 2 iterations."""
    rng = np.random.default_rng(7)
    n, d, R = 300, 4, 5
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.7, 1.3, size=d), [1.0, 0.5]])
    B = rng.standard_normal((R, n))
    V0 = 0.1 * rng.standard_normal((R, n))
    dt = torch.float64 if prec_name == "f64" else torch.float32
    V, info = gp.gp_solve_cg(oracle.MATERN32, th, t(X, dev, dt), t(B, dev, dt), V0=t(V0, dev, dt),
                             max_iters=iters, tol=0.0, prec=prec if prec is not None else gp.GP_PREC_FP32)
    Vr, ir = oracle.solve_cg(oracle.MATERN32, th, X, B, V0=V0, max_iters=iters, tol=0.0)
    assert info.iters == ir["iters"] == iters
    assert rel(V.double().cpu().numpy(), Vr) < tol
    assert info.res_y == pytest.approx(ir["res_y"], rel=100 * tol)


@pytest.mark.parametrize("prec_name,prec", [("f64", None), ("f32", gp.GP_PREC_FP32)])
@pytest.mark.parametrize("stop_rule", [0, 1])
def test_cg_reaches_tolerance_with_true_residual(dev, prec_name, prec, stop_rule):
    """The small workload's shape (RBF, l=0.5, sigma=0.1: condition number ~1e3-1e4):
    the reported convergence holds for the true residual recomputed in FP64."""
    p = workloads.small(n=700, s=8, seed=1)
    B = np.vstack([p.y, p.Z])
    dt = torch.float64 if prec_name == "f64" else torch.float32
    tol = 1e-6 if prec_name == "f64" else 1e-4
    V, info = gp.gp_solve_cg(p.kind, p.theta, t(p.X, dev, dt), t(B, dev, dt), max_iters=500, tol=tol,
                             stop_rule=stop_rule, prec=prec if prec is not None else gp.GP_PREC_FP32)
    assert info.converged
    Vh = V.double().cpu().numpy()
    Xr = p.X if dt == torch.float64 else p.X.astype(np.float32).astype(np.float64)
    Br = B if dt == torch.float64 else B.astype(np.float32).astype(np.float64)
    r = Br - oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, Vh, add_noise=True)
    rn = np.linalg.norm(r, axis=1) / np.linalg.norm(Br, axis=1)
    if stop_rule == 0:
        assert rn[0] <= tol and rn[1:].mean() <= tol
    else:
        assert min(rn[0], rn[1:].mean()) <= tol
    # the reported norms are those of the recomputed true residual
    slack = (1e-2 if prec_name == "f32" else 1e-6) * tol  # FP32-rounded hyperparameters in the check
    assert info.res_y == pytest.approx(rn[0], rel=1e-3, abs=slack)
    assert info.res_z == pytest.approx(rn[1:].mean(), rel=1e-3, abs=slack)


@pytest.mark.parametrize("warm", [False, True])
def test_tc16_cg_at_the_paper_tolerance_true_residual(dev, warm):
    """fp16 tensor-core products at tau = 0.01 on the pathwise workload's shape (Matern-3/2,
    X ~ N(0, I), sigma = 0.3): the true FP64 residual of the returned solution meets tau, and a
    warm start from the previous solution after a small theta change needs fewer iterations."""
    p = workloads.pathwise(n=3000, d=8, s=16, m=256, seed=3)
    X32 = p.X.astype(np.float32)
    Xr = X32.astype(np.float64)
    B = np.vstack([p.y_noise, p.Z]).astype(np.float32)
    Br = B.astype(np.float64)
    th = p.theta.copy()
    V, info = gp.gp_solve_cg(p.kind, th, t(X32, dev), t(B, dev), max_iters=500, tol=1e-2, prec=gp.GP_PREC_TC16)
    assert info.converged
    if warm:
        th2 = th * 1.02
        V2, info2 = gp.gp_solve_cg(p.kind, th2, t(X32, dev), t(B, dev), V0=V.clone(), max_iters=500, tol=1e-2,
                                   prec=gp.GP_PREC_TC16)
        cold, info_c = gp.gp_solve_cg(p.kind, th2, t(X32, dev), t(B, dev), max_iters=500, tol=1e-2,
                                      prec=gp.GP_PREC_TC16)
        assert info2.converged and info2.iters < info_c.iters
        V, th, info = V2, th2, info2
    r = Br - oracle.kernel_mvm(p.kind, th, Xr, Xr, V.double().cpu().numpy(), add_noise=True)
    rn = np.linalg.norm(r, axis=1) / np.linalg.norm(Br, axis=1)
    assert rn[0] <= 1e-2 and rn[1:].mean() <= 1e-2
    # reported norms: the true residual, taken with the split (FP32-class) tensor-core product
    assert abs(info.res_y - rn[0]) <= 1e-4 and abs(info.res_z - rn[1:].mean()) <= 1e-4


@pytest.mark.parametrize("R", [1, 4, 9])
@pytest.mark.parametrize("prec_name,prec,tol", [("f64", None, 1e-9), ("f32", gp.GP_PREC_FP32, 1e-4)])
@pytest.mark.parametrize("n,bs", [(250, 64), (97, 32), (130, 130)])
def test_ap_iterates_match_oracle(dev, prec_name, prec, tol, n, bs, R):
    """Alg. 2 iterate by iterate; R = 1 and 9 leave column groups of the score pass empty or
    uneven."""
    rng = np.random.default_rng(n)
    d = 3
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.7, 1.3, size=d), [1.0, 0.4]])
    B = rng.standard_normal((R, n))
    dt = torch.float64 if prec_name == "f64" else torch.float32
    iters = 7
    V, info = gp.gp_solve_ap(oracle.RBF, th, t(X, dev, dt), t(B, dev, dt), block_size=bs, max_iters=iters, tol=0.0,
                             prec=prec if prec is not None else gp.GP_PREC_FP32)
    Vr, ir = oracle.solve_ap(oracle.RBF, th, X, B, block_size=bs, max_iters=iters, tol=0.0)
    assert info.iters == ir["iters"]
    assert rel(V.double().cpu().numpy(), Vr) < tol
    # the reported norms are the returned iterate's true residual (recomputed when the loop stops)
    Xr = X if dt == torch.float64 else X.astype(np.float32).astype(np.float64)
    Br = B if dt == torch.float64 else B.astype(np.float32).astype(np.float64)
    res = Br - oracle.kernel_mvm(oracle.RBF, th, Xr, Xr, V.double().cpu().numpy(), add_noise=True)
    rn = np.linalg.norm(res, axis=1) / np.linalg.norm(Br, axis=1)
    # (the FP32 form's check runs in FP64 on the FP32-rounded hyperparameters); with the target
    # column alone (R = 1) there are no probe systems and res_z is reported as 0
    res_z = rn[1:].mean() if R > 1 else 0.0
    assert info.res_y == pytest.approx(rn[0], rel=1e-3, abs=(1e-2 if prec_name == "f32" else 1e-3) * tol)
    assert info.res_z == pytest.approx(res_z, rel=1e-3, abs=(1e-2 if prec_name == "f32" else 1e-3) * tol)


def test_ap_converges_to_dense_solution(dev):
    rng = np.random.default_rng(3)
    n, d, R = 200, 3, 3
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.7, 1.3, size=d), [1.0, 0.5]])
    B = rng.standard_normal((R, n))
    V, info = gp.gp_solve_ap(oracle.MATERN32, th, t(X, dev, torch.float64), t(B, dev, torch.float64),
                             block_size=50, max_iters=5000, tol=1e-10)
    assert info.converged
    H = oracle.H_matrix(oracle.MATERN32, th, X)
    assert rel(V.cpu().numpy(), np.linalg.solve(H, B.T).T) < 1e-8


@pytest.mark.parametrize("R", [4, 9])
@pytest.mark.parametrize("n,bs", [(250, 64), (300, 128), (130, 130)])
def test_tc16_ap_iterates_match_oracle(dev, n, bs, R):
    """Tensor-core column panel (device-resident block offset; the block update writes the
    panel's fp16 operand and the score pass applies the residual update): a few iterations of
    Alg. 2 against the oracle; the fp16 panel error is below 1e-3 per iteration."""
    rng = np.random.default_rng(n + 1)
    d = 5
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.7, 1.3, size=d), [1.0, 0.4]])
    B = rng.standard_normal((R, n))
    X32 = X.astype(np.float32)
    iters = 3
    V, info = gp.gp_solve_ap(oracle.RBF, th, t(X32, dev), t(B, dev), block_size=bs, max_iters=iters, tol=0.0,
                             prec=gp.GP_PREC_TC16)
    Vr, ir = oracle.solve_ap(oracle.RBF, th, X32.astype(np.float64), B.astype(np.float32).astype(np.float64),
                             block_size=bs, max_iters=iters, tol=0.0)
    assert info.iters == ir["iters"] == iters
    assert rel(V.double().cpu().numpy(), Vr) < 5e-3


def test_tc16_ap_reaches_tolerance_true_residual(dev):
    """Alg. 2 with the tensor-core panel to tau = 0.01 on the pathwise workload's shape; the true
    FP64 residual of the returned solution meets tau."""
    p = workloads.pathwise(n=2000, d=8, s=8, m=256, seed=5)
    X32 = p.X.astype(np.float32)
    B = np.vstack([p.y_noise, p.Z]).astype(np.float32)
    V, info = gp.gp_solve_ap(p.kind, p.theta, t(X32, dev), t(B, dev), block_size=256, max_iters=4000, tol=1e-2,
                             prec=gp.GP_PREC_TC16)
    assert info.converged
    Xr, Br = X32.astype(np.float64), B.astype(np.float64)
    r = Br - oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.double().cpu().numpy(), add_noise=True)
    rn = np.linalg.norm(r, axis=1) / np.linalg.norm(Br, axis=1)
    assert rn[0] <= 1e-2 and rn[1:].mean() <= 1e-2
    assert abs(info.res_y - rn[0]) <= 1e-4 and abs(info.res_z - rn[1:].mean()) <= 1e-4


@pytest.mark.parametrize("n", [3000, 3001])
def test_tc16_sgd_iterates_match_oracle(dev, n):
    """Tensor-core row panel (batch rows against all points, many column splits): a few
    iterations of Alg. 3 against the oracle (n = 3001: the step's scalar path, rows not a
    multiple of the 16-byte vector)."""
    rng = np.random.default_rng(19)
    d, R, batch, iters = 4, 4, 64, 4
    X = rng.standard_normal((n, d)).astype(np.float32)
    th = np.concatenate([rng.uniform(0.7, 1.3, size=d), [1.0, 0.6]])
    B = rng.standard_normal((R, n)).astype(np.float32)
    idx = workloads.sgd_batches(n, batch, iters, seed=6)
    V, info = gp.gp_solve_sgd(oracle.MATERN32, th, t(X, dev), t(B, dev), torch.tensor(idx, dtype=torch.int32, device=dev),
                              lr=2.0, momentum=0.9, tol=0.0, prec=gp.GP_PREC_TC16)
    Vr, ir = oracle.solve_sgd(oracle.MATERN32, th, X.astype(np.float64), B.astype(np.float64), idx, batch=batch,
                              lr=2.0, momentum=0.9, max_iters=iters, tol=0.0)
    assert info.iters == ir["iters"] == iters
    assert rel(V.double().cpu().numpy(), Vr) < 5e-3


@pytest.mark.parametrize("n", [180, 181])
@pytest.mark.parametrize("prec_name,prec,tol", [("f64", None, 1e-9), ("f32", gp.GP_PREC_FP32, 1e-4)])
def test_sgd_iterates_match_oracle(dev, prec_name, prec, tol, n):
    rng = np.random.default_rng(9)
    d, R, batch, iters = 3, 4, 16, 25
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.7, 1.3, size=d), [1.0, 0.6]])
    B = rng.standard_normal((R, n))
    idx = workloads.sgd_batches(n, batch, iters, seed=4)
    dt = torch.float64 if prec_name == "f64" else torch.float32
    V, info = gp.gp_solve_sgd(oracle.MATERN32, th, t(X, dev, dt), t(B, dev, dt),
                              torch.tensor(idx, dtype=torch.int32, device=dev), lr=2.0, momentum=0.9, tol=0.0,
                              prec=prec if prec is not None else gp.GP_PREC_FP32)
    Vr, ir = oracle.solve_sgd(oracle.MATERN32, th, X, B, idx, batch=batch, lr=2.0, momentum=0.9, max_iters=iters,
                              tol=0.0)
    assert info.iters == ir["iters"] == iters
    assert rel(V.double().cpu().numpy(), Vr) < tol
    assert info.res_y == pytest.approx(ir["res_y"], rel=100 * tol)
    assert info.res_z == pytest.approx(ir["res_z"], rel=100 * tol)


def test_sgd_reports_divergence(dev):
    rng = np.random.default_rng(1)
    n = 64
    X = rng.standard_normal((n, 2))
    th = [1.0, 1.0, 1.0, 0.5]
    B = rng.standard_normal((2, n))
    idx = torch.tensor(workloads.sgd_batches(n, 16, 200), dtype=torch.int32, device=dev)
    with pytest.raises(gp.GPError) as e:
        gp.gp_solve_sgd(0, th, t(X, dev), t(B, dev), idx, lr=1e4, momentum=0.9, tol=0.0, prec=gp.GP_PREC_FP32)
    assert e.value.status == -4


# --------------------------------------------------------------------------- random features, posterior
@pytest.mark.parametrize("dtype,prec,tol", [(torch.float64, gp.GP_PREC_FP32, 1e-11),
                                            (torch.float32, gp.GP_PREC_FP32, 2e-5),
                                            (torch.float32, gp.GP_PREC_TC16, 2e-5)])
@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_rff_prior_sample_matches_oracle(dev, dtype, prec, tol, kind):
    """Ragged n, s not a multiple of 16, m/2 not a multiple of the 32-frequency chunk."""
    p = workloads.pathwise(n=517, d=9, s=33, m=130, seed=2)
    F = gp.gp_rff_prior_sample(kind, p.theta, t(p.X, dev, dtype), t(p.omega_hat, dev, dtype),
                               t(p.chi2, dev, dtype), t(p.W_probe, dev, dtype), prec=prec)
    cast = (lambda a: a) if dtype == torch.float64 else (lambda a: a.astype(np.float32).astype(np.float64))
    ref = oracle.rff_prior(kind, p.theta, cast(p.X), cast(p.omega_hat), cast(p.chi2), cast(p.W_probe))
    assert close(F.double().cpu().numpy(), ref, tol)


@pytest.mark.parametrize("n,d,s,m", [(300, 32, 128, 64), (260, 4, 129, 96), (128, 1, 1, 2)])
def test_rff_tensor_core_limits(dev, n, d, s, m):
    """The largest tensor-core shape (d = 32, s = 128), the CUDA-core fallback past it
    (s = 129) and the smallest case (one point row tile, one sample, one frequency)."""
    p = workloads.pathwise(n=n, d=d, s=s, m=m, seed=4)
    F = gp.gp_rff_prior_sample(p.kind, p.theta, t(p.X, dev), t(p.omega_hat, dev), t(p.chi2, dev),
                               t(p.W_probe, dev), prec=gp.GP_PREC_TC16)
    f = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    ref = oracle.rff_prior(p.kind, p.theta, f(p.X), f(p.omega_hat), f(p.chi2), f(p.W_probe))
    assert close(F.double().cpu().numpy(), ref, 2e-5)


def test_rff_full_size_sampled_points(dev):
    """The pathwise workload's prior samples (n = 32768, d = 16, m = 2048, s = 64, Matern-3/2)
    in both forms, checked on sampled points (a point's features do not depend on the others)."""
    p = workloads.pathwise()
    f = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    rows = np.random.default_rng(31).choice(p.n, size=200, replace=False)
    ref = oracle.rff_prior(p.kind, p.theta, f(p.X)[rows], f(p.omega_hat), f(p.chi2), f(p.W_probe))
    for prec in (gp.GP_PREC_TC16, gp.GP_PREC_FP32):
        F = gp.gp_rff_prior_sample(p.kind, p.theta, t(p.X, dev), t(p.omega_hat, dev), t(p.chi2, dev),
                                   t(p.W_probe, dev), prec=prec)
        assert close(F.double().cpu().numpy()[:, rows], ref, 2e-5)


def test_pathwise_rhs_and_posterior_samples_match_oracle(dev):
    p = workloads.pathwise(n=400, d=4, s=10, m=64, seed=5)
    f = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
    F = oracle.rff_prior(p.kind, p.theta, f(p.X), f(p.omega_hat), f(p.chi2), f(p.W_probe))
    y = f(p.y_noise)
    B = gp.gp_pathwise_rhs(p.theta, p.d, t(y, dev), t(F, dev), t(p.Z, dev))
    Bref = np.vstack([y, f(F) + p.theta[-1] * f(p.Z)])
    assert rel(B.double().cpu().numpy(), Bref) < 1e-6
    rng = np.random.default_rng(0)
    Xs = rng.standard_normal((150, 4))
    Vsol = rng.standard_normal((11, 400))
    Fs = rng.standard_normal((10, 150))
    out = gp.gp_posterior_samples(p.kind, p.theta, t(Xs, dev), t(p.X, dev), t(Vsol, dev), t(Fs, dev),
                                  prec=gp.GP_PREC_FP32)
    ref = oracle.posterior_samples(p.kind, p.theta, f(Xs), f(p.X), f(Vsol), f(Fs))
    assert close(out.double().cpu().numpy(), ref, 1e-5)


def test_autotuned_split_is_used_and_keeps_parity(dev):
    """The autotuner times candidate column splits for one shape and records the fastest;
    products of that shape (standalone and inside CG) still match the oracle."""
    p = workloads.pathwise(n=2500, d=6, s=8, m=64, seed=7)
    X32 = p.X.astype(np.float32)
    V = workloads.vectors(9, 2500, seed=3).astype(np.float32)
    try:
        best, ms = gp.gp_autotune_mvm(p.kind, p.theta, t(X32, dev), t(V, dev), reps=2)
        assert (best >= 1 or best == -1) and ms > 0.0
        Y = gp.gp_kernel_mvm(p.kind, p.theta, t(X32, dev), t(V, dev), add_noise=True, prec=gp.GP_PREC_TC16)
        Xr = X32.astype(np.float64)
        ref = oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.astype(np.float64), add_noise=True)
        assert close(Y.cpu().numpy(), ref, 1e-3)
        B = np.vstack([p.y_noise, p.Z]).astype(np.float32)
        Vs, info = gp.gp_solve_cg(p.kind, p.theta, t(X32, dev), t(B, dev), max_iters=300, tol=1e-2,
                                  prec=gp.GP_PREC_TC16)
        assert info.converged
    finally:
        gp.gp_autotune_reset()


@pytest.mark.parametrize("n,R", [(20000, 9), (40000, 65)])
def test_persistent_schedule_rows_straddling_ctas(dev, n, R):
    """At these sizes the product runs one CTA per SM over equal runs of tile pairs, so most
    128-row tiles are shared by two or more CTAs and summed by the reduction; rows of shared
    and unshared tiles (first, last, ragged) match the oracle, and so does CG with it."""
    p = workloads.pathwise(n=n, d=8, s=R - 1, m=64, seed=17)
    X32 = p.X.astype(np.float32)
    V = workloads.vectors(R, n, seed=18).astype(np.float32)
    Y = gp.gp_kernel_mvm(p.kind, p.theta, t(X32, dev), t(V, dev), add_noise=True,
                         prec=gp.GP_PREC_TC16).cpu().numpy()
    rt = -(-n // 128)
    rows = np.concatenate([np.arange(0, 128, 9), np.arange(128 * (rt // 2), 128 * (rt // 2) + 128, 11),
                           np.arange(128 * (rt - 1), n, 5),
                           np.random.default_rng(19).choice(n, size=48, replace=False)])
    Xr = X32.astype(np.float64)
    ref = oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.astype(np.float64), add_noise=True, rows=rows)
    assert close(Y[:, rows], ref, 1e-3)
    # deterministic: the same call twice gives the same bits
    Y2 = gp.gp_kernel_mvm(p.kind, p.theta, t(X32, dev), t(V, dev), add_noise=True,
                          prec=gp.GP_PREC_TC16).cpu().numpy()
    assert np.array_equal(Y, Y2)
    if n == 20000:
        # CG on the same schedule: its products also return d^T H d per CTA for the step size
        B = workloads.vectors(R, n, seed=20).astype(np.float32)
        V0 = (0.1 * workloads.vectors(R, n, seed=21)).astype(np.float32)
        Vg, info = gp.gp_solve_cg(p.kind, p.theta, t(X32, dev), t(B, dev), V0=t(V0, dev), max_iters=2, tol=0.0,
                                  prec=gp.GP_PREC_TC16)
        Vr, ir = oracle.solve_cg(p.kind, p.theta, Xr, B.astype(np.float64), V0=V0.astype(np.float64), max_iters=2,
                                 tol=0.0)
        assert info.iters == ir["iters"] == 2
        assert close(Vg.double().cpu().numpy(), Vr, 3e-3)


@pytest.mark.parametrize("n,R", [(2048, 9), (1500, 65)])
def test_persistent_schedule_many_ctas_per_row_tile(dev, tmp_path, n, R):
    """The persistent schedule forced through the tuning table on a small problem: 152 CTAs take
    the 256 tile pairs of n = 2048, or 144 CTAs one tile pair each at n = 1500, so a 128-row
    tile is shared by up to 12 CTAs, whose partial sums the last-arriving warps add in CTA
    order.  The product's rows (twice, bit for bit) and two CG iterations, whose step sizes
    use the products' d^T H d partials, match the oracle."""
    p = workloads.pathwise(n=n, d=8, s=R - 1, m=64, seed=21)
    X32 = p.X.astype(np.float32)
    V = workloads.vectors(R, n, seed=22).astype(np.float32)
    tiles = -(-n // 128)
    r_pad = 16 * (-(-R // 16))
    gp.gp_autotune_reset()
    try:
        # this device's cache header (an empty table), then the product's entry: persistent (-1)
        f = tmp_path / "force_persistent.txt"
        gp.gp_autotune_save(f)
        f.write_text(f.read_text() + "0 %d %d %d 0 -1\n" % (r_pad, tiles, tiles))
        gp.gp_autotune_load(f)
        assert gp.gp_autotune_count() == 1
        Xr = X32.astype(np.float64)
        Y = gp.gp_kernel_mvm(p.kind, p.theta, t(X32, dev), t(V, dev), add_noise=True,
                             prec=gp.GP_PREC_TC16).cpu().numpy()
        ref = oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.astype(np.float64), add_noise=True)
        assert close(Y, ref, 1e-3)
        Y2 = gp.gp_kernel_mvm(p.kind, p.theta, t(X32, dev), t(V, dev), add_noise=True,
                              prec=gp.GP_PREC_TC16).cpu().numpy()
        assert np.array_equal(Y, Y2)
        B = workloads.vectors(R, n, seed=23).astype(np.float32)
        V0 = (0.1 * workloads.vectors(R, n, seed=24)).astype(np.float32)
        Vg, info = gp.gp_solve_cg(p.kind, p.theta, t(X32, dev), t(B, dev), V0=t(V0, dev), max_iters=2, tol=0.0,
                                  prec=gp.GP_PREC_TC16)
        Vr, ir = oracle.solve_cg(p.kind, p.theta, Xr, B.astype(np.float64), V0=V0.astype(np.float64), max_iters=2,
                                 tol=0.0)
        assert info.iters == ir["iters"] == 2
        assert close(Vg.double().cpu().numpy(), Vr, 3e-3)
    finally:
        gp.gp_autotune_reset()


@pytest.mark.parametrize("prec_name,prec,tol", [("f32", gp.GP_PREC_FP32, 1e-5), ("tc16", gp.GP_PREC_TC16, 2e-3)])
def test_predictions_match_oracle(dev, prec_name, prec, tol):
    """Predictive mean/variance and test RMSE/log-likelihood from the pathwise solutions."""
    p = workloads.pathwise(n=1500, d=6, s=12, m=256, seed=9)
    rng = np.random.default_rng(10)
    Xs = rng.standard_normal((700, 6)).astype(np.float32)
    X32 = p.X.astype(np.float32)
    Vsol = (0.3 * rng.standard_normal((13, 1500))).astype(np.float32)
    Fs = rng.standard_normal((12, 700)).astype(np.float32)
    ys = rng.standard_normal(700).astype(np.float32)
    mean, var, met = gp.gp_predict(p.kind, p.theta, t(Xs, dev), t(X32, dev), t(Vsol, dev), t(Fs, dev), t(ys, dev),
                                   prec=prec)
    m_ref, v_ref, (rmse, llh) = oracle.predict(p.kind, p.theta, Xs.astype(np.float64), X32.astype(np.float64),
                                               Vsol.astype(np.float64), Fs.astype(np.float64), ys.astype(np.float64))
    assert close(mean.cpu().numpy(), m_ref, tol)
    assert close(var.cpu().numpy(), v_ref, tol)
    met = met.cpu().numpy()
    assert abs(met[0] - rmse) <= tol * rmse and abs(met[1] - llh) <= 10 * tol * abs(llh)


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_pcg_iterates_match_oracle_fp64(dev, kind):
    """Preconditioned CG (App. B: pivoted Cholesky, here rank 20) iterate by iterate in FP64."""
    rng = np.random.default_rng(50 + kind)
    n, d, R = 230, 3, 4
    X = rng.uniform(0, 1, size=(n, d))
    th = np.concatenate([rng.uniform(0.4, 0.7, size=d), [1.0, 0.1]])
    B = rng.standard_normal((R, n))
    V, info = gp.gp_solve_cg(kind, th, t(X, dev, torch.float64), t(B, dev, torch.float64), max_iters=6, tol=0.0,
                             precond_rank=20)
    Vr, ir = oracle.solve_pcg(kind, th, X, B, 20, max_iters=6, tol=0.0)
    assert info.iters == ir["iters"] == 6
    assert rel(V.cpu().numpy(), Vr) < 1e-9


def test_pcg_full_rank_converges_in_one_iteration(dev):
    rng = np.random.default_rng(52)
    n, R = 90, 3
    X = rng.standard_normal((n, 2))
    th = np.array([0.8, 1.2, 1.0, 0.4])
    B = rng.standard_normal((R, n))
    V, info = gp.gp_solve_cg(oracle.RBF, th, t(X, dev, torch.float64), t(B, dev, torch.float64), max_iters=5,
                             tol=1e-8, precond_rank=128)
    assert info.converged and info.iters == 1
    H = oracle.H_matrix(oracle.RBF, th, X)
    assert rel(V.cpu().numpy(), np.linalg.solve(H, B.T).T) < 1e-7


def test_pcg_reaches_tolerance_in_fewer_iterations_fp32(dev):
    """The small workload's shape (RBF, l = 0.5, sigma = 0.1, ill-conditioned): with the rank-100
    preconditioner CG meets the tolerance (true FP64 residual) in fewer iterations."""
    tol = 1e-4
    p = workloads.small(n=1500, s=4, seed=2)
    X32 = p.X.astype(np.float32)
    B = np.vstack([p.y, p.Z]).astype(np.float32)
    V0, info0 = gp.gp_solve_cg(p.kind, p.theta, t(X32, dev), t(B, dev), max_iters=3000, tol=tol,
                               prec=gp.GP_PREC_FP32)
    V, info = gp.gp_solve_cg(p.kind, p.theta, t(X32, dev), t(B, dev), max_iters=3000, tol=tol,
                             prec=gp.GP_PREC_FP32, precond_rank=100)
    assert info.converged and info0.converged and info.iters < info0.iters
    Xr, Br = X32.astype(np.float64), B.astype(np.float64)
    r = Br - oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.double().cpu().numpy(), add_noise=True)
    rn = np.linalg.norm(r, axis=1) / np.linalg.norm(Br, axis=1)
    assert rn[0] <= tol and rn[1:].mean() <= tol


def test_tc16_pcg_at_the_paper_tolerance_true_residual(dev):
    """Tensor-core products with the rank-100 preconditioner at tau = 0.01 on the pathwise
    workload's shape (sigma = 0.3; an fp16 product cannot certify tau on the ill-conditioned small
    workload, see the plain-CG tests): converged and the true FP64 residual meets tau.  In this
    high-dimensional shape the kernel spectrum is flat, so a rank-100 factor barely changes the
    iteration count (the FP32 test above shows the reduction on the small workload)."""
    p = workloads.pathwise(n=3000, d=8, s=16, m=256, seed=3)
    X32 = p.X.astype(np.float32)
    B = np.vstack([p.y_noise, p.Z]).astype(np.float32)
    V, info = gp.gp_solve_cg(p.kind, p.theta, t(X32, dev), t(B, dev), max_iters=500, tol=1e-2,
                             prec=gp.GP_PREC_TC16, precond_rank=100)
    assert info.converged
    Xr, Br = X32.astype(np.float64), B.astype(np.float64)
    r = Br - oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.double().cpu().numpy(), add_noise=True)
    rn = np.linalg.norm(r, axis=1) / np.linalg.norm(Br, axis=1)
    assert rn[0] <= 1e-2 and rn[1:].mean() <= 1e-2
