"""GPU parity of batches of independent GPs (gp_batch_* C ABI): every member's product,
CG iterates and convergence, gradient estimators and Adam step against the FP64 oracle,
and a CUDA-graph replay of the whole marginal-likelihood step against eager execution.

Members follow the batched workload's recipe (RBF, X ~ U[0,1]^d, l = 0.5, s_f = 1) at
sizes that span one to several 128-row tiles with ragged tails and every contraction
class (d = 3, 4, 8, 16, 32).  Tolerances as for the single-problem tensor-core form:
products 1e-3, CG iterates after 2 iterations 3e-3, gradients (CUDA-core FP32) 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_18457_gb300 import workloads

pytestmark = pytest.mark.gpu

import paper_2405_18457_gb300 as gp  # noqa: E402  (a missing package fails the run)

SHAPES = [(1, 3), (100, 4), (300, 8), (700, 16), (257, 32)]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    gp.library()
    return torch.device("cuda:0")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def members(shapes, s, sigma=None, seed=0):
    out = []
    for g, (n, d) in enumerate(shapes):
        p = workloads.batched_member(n, d, s=s, m=64, seed=seed, index=g)
        th = p.theta.copy()
        if sigma is not None:
            th[-1] = sigma
        out.append((p.X.astype(np.float32), th, p))
    return out


def make_batch(kind, shapes, s, dev, sigma=None, seed=0):
    ms = members(shapes, s, sigma, seed)
    b = gp.GPBatch(kind, [n for n, _ in shapes], [d for _, d in shapes], s, device=dev)
    X = b.pack_points([m[0] for m in ms])
    th = b.pack_theta([m[1] for m in ms])
    return b, ms, X, th


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("add_noise", [True, False])
def test_batch_product_matches_oracle(dev, kind, add_noise):
    s = 2
    b, ms, X, th = make_batch(kind, SHAPES, s, dev)
    rng = np.random.default_rng(1)
    Vs = [rng.standard_normal((s + 1, n)).astype(np.float32) for n, _ in SHAPES]
    V = b.pack_vectors(Vs)
    b.prepare(th, X)
    Y = b.mvm(V, add_noise=add_noise)
    b.status()
    for (Xg, thg, _), Vg, Yg in zip(ms, Vs, b.unpack_vectors(Y)):
        Xr = Xg.astype(np.float64)
        ref = oracle.kernel_mvm(kind, thg, Xr, Xr, Vg.astype(np.float64), add_noise=add_noise)
        assert rel(Yg.cpu().numpy(), ref) < 1e-3


def test_batch_pack_unpack_round_trip(dev):
    b, ms, X, th = make_batch(0, SHAPES, 3, dev)
    rng = np.random.default_rng(2)
    Vs = [rng.standard_normal((4, n)).astype(np.float32) for n, _ in SHAPES]
    for a, c in zip(Vs, b.unpack_vectors(b.pack_vectors(Vs))):
        np.testing.assert_array_equal(a, c.cpu().numpy())
    for (_, thg, _), t in zip(ms, b.unpack_theta(th)):
        np.testing.assert_array_equal(thg, t.cpu().numpy())


def test_batch_cg_iterates_match_oracle(dev):
    """Two iterations of Alg. 1 from a warm start, every member against the oracle."""
    s = 3
    b, ms, X, th = make_batch(0, SHAPES, s, dev, sigma=0.3)
    rng = np.random.default_rng(3)
    Bs = [rng.standard_normal((s + 1, n)).astype(np.float32) for n, _ in SHAPES]
    V0s = [(0.1 * rng.standard_normal((s + 1, n))).astype(np.float32) for n, _ in SHAPES]
    B = b.pack_vectors(Bs)
    V = b.pack_vectors(V0s)
    b.prepare(th, X)
    b.solve_cg(B, V, iters=2, tol=0.0)
    info = b.info()
    b.status()
    for g, ((Xg, thg, _), Bg, V0g, Vg) in enumerate(zip(ms, Bs, V0s, b.unpack_vectors(V))):
        Vr, ir = oracle.solve_cg(0, thg, Xg.astype(np.float64), Bg.astype(np.float64),
                                 V0=V0g.astype(np.float64), max_iters=2, tol=0.0)
        assert info[g]["iters"] == ir["iters"] == 2
        assert rel(Vg.cpu().numpy(), Vr) < 3e-3, g


def test_batch_cg_reaches_tolerance_with_true_residual(dev):
    s = 4
    shapes = SHAPES[1:]
    b, ms, X, th = make_batch(0, shapes, s, dev, sigma=0.3)
    Bs = [np.vstack([m[2].y_noise, m[2].Z]).astype(np.float32) for m in ms]
    B = b.pack_vectors(Bs)
    V = torch.zeros_like(B)
    b.prepare(th, X)
    b.solve_cg(B, V, iters=300, tol=1e-2)
    info = b.info()
    b.status()
    for g, ((Xg, thg, _), Bg, Vg) in enumerate(zip(ms, Bs, b.unpack_vectors(V))):
        assert info[g]["converged"], (g, info[g])
        Xr = Xg.astype(np.float64)
        Br = Bg.astype(np.float64)
        r = Br - oracle.kernel_mvm(0, thg, Xr, Xr, Vg.double().cpu().numpy(), add_noise=True)
        rn = np.linalg.norm(r, axis=1) / np.linalg.norm(Br, axis=1)
        assert rn[0] <= 1e-2 and rn[1:].mean() <= 1e-2, (g, rn)
        # reported norms: the member's true residual, taken with the split tensor-core product
        assert abs(info[g]["res_y"] - rn[0]) <= 1e-4 and abs(info[g]["res_z"] - rn[1:].mean()) <= 1e-4, (g, info[g])


def test_batch_cg_members_stop_independently(dev):
    """A member whose right-hand sides are zero meets the loop condition at t = 0 and is
    skipped from then on; the others iterate to their own tolerance."""
    s = 2
    shapes = [(300, 8), (200, 4)]
    b, ms, X, th = make_batch(0, shapes, s, dev, sigma=0.3)
    rng = np.random.default_rng(4)
    Bs = [np.zeros((s + 1, 300), dtype=np.float32), rng.standard_normal((s + 1, 200)).astype(np.float32)]
    B = b.pack_vectors(Bs)
    V = torch.zeros_like(B)
    b.prepare(th, X)
    b.solve_cg(B, V, iters=100, tol=1e-3)
    info = b.info()
    assert info[0]["iters"] == 0 and info[0]["converged"]
    assert info[1]["converged"] and 0 < info[1]["iters"] < 100
    assert torch.count_nonzero(b.unpack_vectors(V)[0]).item() == 0


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("pathwise", [False, True])
def test_batch_gradient_matches_oracle(dev, kind, pathwise):
    s = 3
    b, ms, X, th = make_batch(kind, SHAPES, s, dev)
    rng = np.random.default_rng(5)
    Vs = [rng.standard_normal((s + 1, n)).astype(np.float32) for n, _ in SHAPES]
    Bs = [rng.standard_normal((s + 1, n)).astype(np.float32) for n, _ in SHAPES]
    V = b.pack_vectors(Vs)
    B = b.pack_vectors(Bs)
    b.prepare(th, X)
    g = b.mll_grad(th, X, V, B=None if pathwise else B, pathwise=pathwise)
    for (Xg, thg, _), Vg, Bg, gg in zip(ms, Vs, Bs, b.unpack_theta(g)):
        Xr, Vr = Xg.astype(np.float64), Vg.astype(np.float64)
        if pathwise:
            ref = oracle.grad_pathwise(kind, thg, Xr, Vr)
        else:
            ref = oracle.grad_standard(kind, thg, Xr, Vr, Bg[1:].astype(np.float64))
        assert rel(gg.cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("pathwise", [False, True])
def test_batch_gradient_tensor_core_members_match_oracle(dev, kind, pathwise):
    """Members of 1024 points or more take the fused tensor-core estimator (hyperparameters
    read on the device), the others the CUDA-core one; tolerance of the 16-bit form (1e-3)."""
    s = 3
    shapes = [(1100, 4), (300, 8), (2048, 16), (1500, 32)]
    b, ms, X, th = make_batch(kind, shapes, s, dev)
    rng = np.random.default_rng(15)
    Vs = [rng.standard_normal((s + 1, n)).astype(np.float32) for n, _ in shapes]
    Bs = [rng.standard_normal((s + 1, n)).astype(np.float32) for n, _ in shapes]
    V = b.pack_vectors(Vs)
    B = b.pack_vectors(Bs)
    b.prepare(th, X)
    g = b.mll_grad(th, X, V, B=None if pathwise else B, pathwise=pathwise)
    for (Xg, thg, _), Vg, Bg, gg, (n, _) in zip(ms, Vs, Bs, b.unpack_theta(g), shapes):
        Xr, Vr = Xg.astype(np.float64), Vg.astype(np.float64)
        if pathwise:
            ref = oracle.grad_pathwise(kind, thg, Xr, Vr)
        else:
            ref = oracle.grad_standard(kind, thg, Xr, Vr, Bg[1:].astype(np.float64))
        assert rel(gg.cpu().numpy(), ref) < (1e-3 if n >= 1024 else 1e-4), n


def test_batch_adam_matches_oracle(dev):
    b, ms, X, th = make_batch(0, SHAPES, 2, dev)
    st = b.adam_init(th)
    rng = np.random.default_rng(6)
    host = [(np.log(np.expm1(m[1])), np.zeros(m[1].size), np.zeros(m[1].size)) for m in ms]
    for t in (1, 2):
        grads = [rng.standard_normal(m[1].size) for m in ms]
        g = b.pack_theta(grads)
        b.adam_step(st, g, th, lr=0.05)
        for (nu, m_, v_), gr in zip(host, grads):
            oracle.adam_softplus(nu, m_, v_, t, gr, 0.05)
    assert int(st["t"].item()) == 2
    for (nu, _, _), tg in zip(host, b.unpack_theta(th)):
        np.testing.assert_allclose(tg.cpu().numpy(), np.log1p(np.exp(nu)), rtol=1e-12)


def _step_inputs(b, ms, s):
    Bs = [np.vstack([m[2].y_noise, m[2].Z[:s]]).astype(np.float32) for m in ms]
    return b.pack_vectors(Bs), Bs


def test_batch_step_first_update_matches_oracle(dev):
    """One step: the gradient it used equals the oracle's standard estimator on the solution it
    produced, and theta moved by the oracle's Adam step with that gradient."""
    s = 3
    b, ms, X, th = make_batch(0, SHAPES, s, dev, sigma=0.3)
    th0 = th.clone()
    B, Bs = _step_inputs(b, ms, s)
    V = torch.zeros_like(B)
    st = b.adam_init(th)
    grad = torch.empty_like(th)
    b.step(X, th, B, V, iters=50, tol=1e-2, state=st, lr=0.05, grad=grad)
    b.status()
    for (Xg, thg, _), Bg, Vg, gg, t0, t1 in zip(ms, Bs, b.unpack_vectors(V), b.unpack_theta(grad),
                                                b.unpack_theta(th0), b.unpack_theta(th)):
        ref = oracle.grad_standard(0, thg, Xg.astype(np.float64), Vg.double().cpu().numpy(),
                                   Bg[1:].astype(np.float64))
        assert rel(gg.cpu().numpy(), ref) < 1e-4
        nu = np.log(np.expm1(t0.cpu().numpy()))
        z = np.zeros_like(nu)
        th_ref = oracle.adam_softplus(nu, z.copy(), z.copy(), 1, gg.cpu().numpy(), 0.05)
        np.testing.assert_allclose(t1.cpu().numpy(), th_ref, rtol=1e-12)


def test_batch_step_graph_replay_equals_eager(dev):
    """The whole step (prepare, 20 CG iterations, gradient, Adam) captured once into a CUDA
    graph and replayed twice gives bitwise the same theta and solutions as two eager steps."""
    s = 3
    b, ms, X, th_e = make_batch(0, SHAPES, s, dev, sigma=0.3)
    B, _ = _step_inputs(b, ms, s)
    th_g = th_e.clone()
    V_e = torch.zeros_like(B)
    V_g = torch.zeros_like(B)
    st_e = b.adam_init(th_e)
    st_g = b.adam_init(th_g)
    grad_e = torch.empty_like(th_e)
    grad_g = torch.empty_like(th_g)
    for _ in range(2):
        b.step(X, th_e, B, V_e, iters=20, tol=1e-3, state=st_e, lr=0.05, grad=grad_e)
    torch.cuda.synchronize()
    # warm-up on a side stream (kernel attributes and tensor maps), then capture
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.step(X, th_g, B, V_g, iters=20, tol=1e-3, state=st_g, lr=0.05, grad=grad_g)
    torch.cuda.synchronize()
    # capture does not execute: state is still the initial one
    assert int(st_g["t"].item()) == 0
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    b.status()
    assert int(st_g["t"].item()) == 2
    assert torch.equal(th_e, th_g)
    assert torch.equal(V_e, V_g)
    assert torch.equal(grad_e, grad_g)


def test_batch_invalid_theta_is_reported(dev):
    b, ms, X, th = make_batch(0, SHAPES[:2], 2, dev)
    th[1] = -1.0
    b.prepare(th, X)
    with pytest.raises(gp.GPError):
        b.status()
