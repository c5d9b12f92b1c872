"""Pins for the oracle's solvers (App. B, Alg. 1 CG, Alg. 2 AP, Alg. 3 SGD) and the
outer-loop Adam step (Sec. 2.1, App. B "Iterative Optimiser").  Solutions are
checked against numpy's dense solve; structural facts (CG terminates in at most
n steps, one AP iteration with b = n is exact, the first SGD step has a closed
form) catch index and sign mistakes; Adam is checked against torch.optim.Adam."""
import numpy as np
import pytest

import oracle


def _problem(kind=oracle.MATERN32, n=30, d=3, R=4, seed=0, sigma=0.5):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.7, 1.3, size=d), [1.0, sigma]])
    B = rng.standard_normal((R, n))
    return rng, X, th, B


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_cg_matches_dense_solve(kind):
    rng, X, th, B = _problem(kind)
    H = oracle.H_matrix(kind, th, X)
    V, info = oracle.solve_cg(kind, th, X, B, max_iters=200, tol=1e-12)
    assert info["converged"]
    np.testing.assert_allclose(V, np.linalg.solve(H, B.T).T, rtol=1e-9, atol=1e-10)
    assert info["res_y"] <= 1e-12 and info["res_z"] <= 1e-12


def test_cg_terminates_within_n_iterations():
    rng, X, th, B = _problem(n=16, sigma=0.8)
    V, info = oracle.solve_cg(oracle.RBF, th, X, B, max_iters=1000, tol=1e-10)
    assert info["converged"] and info["iters"] <= 16 + 2  # n steps in exact arithmetic, FP64 slack


def test_cg_warm_start_at_solution_needs_no_iteration_and_scales_linearly():
    rng, X, th, B = _problem()
    H = oracle.H_matrix(oracle.MATERN32, th, X)
    Vx = np.linalg.solve(H, B.T).T
    V, info = oracle.solve_cg(oracle.MATERN32, th, X, B, V0=Vx, tol=1e-8)
    assert info["iters"] == 0
    V1, _ = oracle.solve_cg(oracle.MATERN32, th, X, B, max_iters=5, tol=0.0)
    V2, _ = oracle.solve_cg(oracle.MATERN32, th, X, 2.0 * B, max_iters=5, tol=0.0)
    np.testing.assert_allclose(V2, 2.0 * V1, rtol=1e-10)


def test_cg_stop_rules():
    """Default: iterate until both split norms reach tau (App. B); rule 1: the
    listing's literal conjunction stops as soon as one does."""
    rng, X, th, B = _problem(n=40, R=6, seed=3)
    B[0] *= 1e-3  # make the y system converge at a different rate
    V0, i0 = oracle.solve_cg(oracle.RBF, th, X, B, max_iters=500, tol=1e-6, stop_rule=0)
    V1, i1 = oracle.solve_cg(oracle.RBF, th, X, B, max_iters=500, tol=1e-6, stop_rule=1)
    assert i0["res_y"] <= 1e-6 and i0["res_z"] <= 1e-6
    assert min(i1["res_y"], i1["res_z"]) <= 1e-6
    assert i1["iters"] <= i0["iters"]


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_ap_matches_dense_solve(kind):
    rng, X, th, B = _problem(kind, n=37)
    H = oracle.H_matrix(kind, th, X)
    V, info = oracle.solve_ap(kind, th, X, B, block_size=8, max_iters=5000, tol=1e-11)
    assert info["converged"]
    np.testing.assert_allclose(V, np.linalg.solve(H, B.T).T, rtol=1e-8, atol=1e-9)


def test_ap_with_one_block_is_exact_in_one_iteration():
    rng, X, th, B = _problem(n=25)
    H = oracle.H_matrix(oracle.MATERN32, th, X)
    V, info = oracle.solve_ap(oracle.MATERN32, th, X, B, block_size=25, max_iters=10, tol=1e-10)
    assert info["iters"] == 1
    np.testing.assert_allclose(V, np.linalg.solve(H, B.T).T, rtol=1e-10, atol=1e-12)


def test_ap_first_iteration_zeroes_the_largest_block_residual():
    """One AP iteration solves the selected diagonal block exactly, so the residual
    on that block vanishes; the block must be argmax ||r_y[i] + sum_j r_j[i]||."""
    rng, X, th, B = _problem(n=40, R=3, seed=5)
    H = oracle.H_matrix(oracle.RBF, th, X)
    V, _ = oracle.solve_ap(oracle.RBF, th, X, B, block_size=10, max_iters=1, tol=0.0)
    r = B - V @ H.T
    scores = [np.linalg.norm(B[:, i * 10:(i + 1) * 10].sum(axis=0)) for i in range(4)]
    best = int(np.argmax(scores))
    assert np.abs(r[:, best * 10:(best + 1) * 10]).max() < 1e-10 * np.abs(B).max()
    others = [i for i in range(4) if i != best]
    assert all(np.abs(r[:, i * 10:(i + 1) * 10]).max() > 1e-6 for i in others)


def test_ap_ragged_last_block():
    rng, X, th, B = _problem(n=23, R=2, seed=6)
    H = oracle.H_matrix(oracle.MATERN32, th, X)
    V, info = oracle.solve_ap(oracle.MATERN32, th, X, B, block_size=5, max_iters=4000, tol=1e-11)
    np.testing.assert_allclose(V, np.linalg.solve(H, B.T).T, rtol=1e-8, atol=1e-9)


def test_sgd_first_step_closed_form():
    """From v = 0 with m = 0: g[i] = -b~[i] on the batch, so v1 = (lr/b) b~ on the
    batch rows and 0 elsewhere; the returned solution is rescaled by ||b|| + eps."""
    rng, X, th, B = _problem(n=20, R=2)
    idx = np.array([[3, 7, 11, 0]])
    V, info = oracle.solve_sgd(oracle.MATERN32, th, X, B, idx, batch=4, lr=0.5, momentum=0.9,
                               max_iters=1, tol=0.0)
    ref = np.zeros_like(B)
    ref[:, idx[0]] = (0.5 / 4) * B[:, idx[0]]
    np.testing.assert_allclose(V, ref, rtol=1e-12, atol=1e-15)
    assert info["iters"] == 1


def test_sgd_residual_heuristic_tracks_true_residual_on_sampled_rows():
    rng, X, th, B = _problem(n=20, R=2, seed=8)
    H = oracle.H_matrix(oracle.RBF, th, X)
    idx = np.array([[1, 2, 3, 4], [5, 6, 7, 8]])
    V1, _ = oracle.solve_sgd(oracle.RBF, th, X, B, idx, batch=4, lr=0.3, max_iters=1, tol=0.0)
    V2, info = oracle.solve_sgd(oracle.RBF, th, X, B, idx, batch=4, lr=0.3, max_iters=2, tol=0.0)
    bn = np.linalg.norm(B, axis=1, keepdims=True) + 1e-12
    # after step 2, r on rows 5..8 equals -(b~ - H v~1) there; rows 9.. keep b~
    r_true_at_v1 = (B - V1 @ H.T) / bn
    r = (B / bn).copy()
    r[:, idx[0]] = -(B / bn - 0.0)[:, idx[0]]
    r[:, idx[1]] = -r_true_at_v1[:, idx[1]]
    ry = np.linalg.norm(r[0])
    assert info["res_y"] == pytest.approx(ry, rel=1e-10)


def test_sgd_converges_to_the_solution():
    rng, X, th, B = _problem(n=24, R=2, seed=9, sigma=1.0)
    H = oracle.H_matrix(oracle.RBF, th, X)
    iters, batch = 4000, 6
    idx = np.stack([rng.choice(24, size=batch, replace=False) for _ in range(iters)])
    V, info = oracle.solve_sgd(oracle.RBF, th, X, B, idx, batch=batch, lr=0.5, momentum=0.9,
                               max_iters=iters, tol=0.0)
    np.testing.assert_allclose(V, np.linalg.solve(H, B.T).T, rtol=1e-6, atol=1e-7)


def test_adam_softplus_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    P = 5
    nu = rng.standard_normal(P)
    m = np.zeros(P)
    v = np.zeros(P)
    t_nu = torch.tensor(nu.copy(), requires_grad=True)
    opt = torch.optim.Adam([t_nu], lr=0.1, maximize=True)
    for t in range(1, 12):
        g_theta = rng.standard_normal(P)
        sig = 1.0 / (1.0 + np.exp(-t_nu.detach().numpy()))
        t_nu.grad = torch.tensor(g_theta * sig)
        opt.step()
        theta = oracle.adam_softplus(nu, m, v, t, g_theta, lr=0.1)
        np.testing.assert_allclose(nu, t_nu.detach().numpy(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(theta, np.log1p(np.exp(nu)), rtol=1e-14)


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_warm_start_first_order_identity(kind):
    """App. A.2 "Taylor Approximation View of Warm Start": for theta' = theta + eps * delta with the same right-hand side,
    v(theta') = v(theta) - H(theta)^-1 (H(theta') - H(theta)) v(theta) + O(eps^2), so the previous
    solution is an O(eps) warm start and the first-order correction leaves an O(eps^2) error."""
    rng = np.random.default_rng(31 + kind)
    n, d = 40, 3
    X = rng.standard_normal((n, d))
    th = np.concatenate([rng.uniform(0.8, 1.4, size=d), [1.1, 0.5]])
    delta = rng.uniform(-1.0, 1.0, size=d + 2) * th
    y = rng.standard_normal(n)
    H0 = oracle.H_matrix(kind, th, X)
    v0 = np.linalg.solve(H0, y)
    errs, dists = [], []
    for eps in (1e-2, 5e-3, 2.5e-3):
        H1 = oracle.H_matrix(kind, th + eps * delta, X)
        v1 = np.linalg.solve(H1, y)
        taylor = v0 - np.linalg.solve(H0, (H1 - H0) @ v0)
        errs.append(np.linalg.norm(v1 - taylor))
        dists.append(np.linalg.norm(v1 - v0))
    # first-order distance, second-order remainder
    assert 1.8 < dists[0] / dists[1] < 2.2 and 1.8 < dists[1] / dists[2] < 2.2
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


@pytest.mark.parametrize("kind", [oracle.RBF, oracle.MATERN32])
def test_pivoted_cholesky_full_rank_reproduces_K(kind):
    rng = np.random.default_rng(40 + kind)
    n, d = 30, 2
    X = rng.standard_normal((n, d))
    th = np.array([0.9, 1.3, 1.1, 0.2])
    L, piv = oracle.pivoted_cholesky(kind, th, X, n)
    K = oracle.kernel_matrix(kind, th, X, X)
    assert L.shape[0] >= n - 2  # numerically full rank (the remaining diagonal may vanish a step early)
    np.testing.assert_allclose(L.T @ L, K, atol=1e-9)
    assert piv[0] == 0 and len(set(piv.tolist())) == len(piv)  # equal diagonals: ties to index 0
    # each pivot column is interpolated exactly from the first step that picks it on
    for m, p in enumerate(piv):
        np.testing.assert_allclose(L[: m + 1].T @ L[: m + 1, p], K[:, p], atol=1e-9)


def test_pivoted_cholesky_trace_error_decreases():
    rng = np.random.default_rng(41)
    n = 80
    X = rng.uniform(-1, 1, size=(n, 2))
    th = np.array([0.5, 0.5, 1.0, 0.1])
    K = oracle.kernel_matrix(oracle.RBF, th, X, X)
    errs = []
    for k in (2, 5, 10, 20):
        L, _ = oracle.pivoted_cholesky(oracle.RBF, th, X, k)
        E = K - L.T @ L
        assert np.min(np.linalg.eigvalsh(E)) > -1e-10  # the remainder is PSD
        errs.append(np.trace(E))
    assert all(a > b for a, b in zip(errs, errs[1:]))


def test_pcg_rank_zero_is_plain_cg():
    rng = np.random.default_rng(42)
    n, R = 60, 3
    X = rng.standard_normal((n, 3))
    th = np.array([1.0, 0.8, 1.2, 1.0, 0.3])
    B = rng.standard_normal((R, n))
    Va, ia = oracle.solve_cg(oracle.MATERN32, th, X, B, max_iters=6, tol=0.0)
    Vb, ib = oracle.solve_pcg(oracle.MATERN32, th, X, B, 0, max_iters=6, tol=0.0)
    np.testing.assert_allclose(Vb, Va, rtol=1e-12, atol=1e-14)
    assert ia["iters"] == ib["iters"] == 6


def test_pcg_with_the_exact_preconditioner_needs_one_iteration():
    """Full rank: P = K + sigma^2 I = H, so the first step lands on the solution."""
    rng = np.random.default_rng(43)
    n, R = 40, 2
    X = rng.standard_normal((n, 2))
    th = np.array([0.7, 1.1, 1.0, 0.5])
    B = rng.standard_normal((R, n))
    V, info = oracle.solve_pcg(oracle.RBF, th, X, B, n, max_iters=5, tol=1e-9)
    assert info["iters"] == 1 and info["converged"]
    H = oracle.H_matrix(oracle.RBF, th, X)
    np.testing.assert_allclose(V, np.linalg.solve(H, B.T).T, rtol=1e-7, atol=1e-9)


def test_pcg_matches_dense_solve_and_needs_fewer_iterations():
    p_rng = np.random.default_rng(44)
    n, R = 300, 3
    X = p_rng.uniform(0, 1, size=(n, 4))
    th = np.array([0.5, 0.5, 0.5, 0.5, 1.0, 0.1])  # the small workload's hyperparameters
    B = p_rng.standard_normal((R, n))
    V, info = oracle.solve_pcg(oracle.RBF, th, X, B, 20, max_iters=2000, tol=1e-8)
    _, info_cg = oracle.solve_cg(oracle.RBF, th, X, B, max_iters=2000, tol=1e-8)
    H = oracle.H_matrix(oracle.RBF, th, X)
    np.testing.assert_allclose(V, np.linalg.solve(H, B.T).T, rtol=1e-5, atol=1e-6)
    assert info["converged"] and info["iters"] < info_cg["iters"]
