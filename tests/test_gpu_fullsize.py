"""Parity at the full sizes of the benchmark workloads, on outputs the FP64 oracle computes one
by one (sampled rows of the product), in the tensor-core launch configurations the solvers use:

  ap        n = 262144, d = 26, RBF, 65 right-hand sides: the square product (CG / AP operator)
            and the alternating-projection column panel shape (all rows against one block)
  sgd       n = 2,000,000, d = 11, Matern-3/2, 65 right-hand sides: the stochastic-gradient row
            panel (512 batch rows against all points, tens of column splits)
  batched   256 RBF members, n ~ LogUniform[512, 65536], d in {4, 8, 16, 32}, 17 vectors each:
            the grouped product of gp_batch_mvm

Tolerance: 1e-3 relative (Frobenius over the sampled rows), the bound for the 16-bit form, and
4e-3 for each sampled row on its own (parity_util.close).
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
    gp.library()
    return torch.device("cuda:0")


from parity_util import close  # noqa: E402


def test_ap_workload_full_size_product_and_panel_sampled_rows(dev):
    p = workloads.ap()
    n, R = p.n, p.s + 1
    X32 = p.X.astype(np.float32)
    Xr = X32.astype(np.float64)
    V = workloads.vectors(R, n, seed=21).astype(np.float32)
    Xt = torch.tensor(X32, device=dev)
    Y = gp.gp_kernel_mvm(p.kind, p.theta, Xt, torch.tensor(V, device=dev), add_noise=True,
                         prec=gp.GP_PREC_TC16).cpu().numpy()
    rows = np.random.default_rng(22).choice(n, size=24, replace=False)
    ref = oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.astype(np.float64), add_noise=True, rows=rows)
    assert close(Y[:, rows], ref, 1e-3)
    # panel shape of Alg. 2: every row against one block of b = 1024 columns
    blk = slice(5 * 1024, 6 * 1024)
    Vb = V[:, blk].copy()
    Yp = gp.gp_kernel_mvm(p.kind, p.theta, Xt, torch.tensor(Vb, device=dev), X2=Xt[blk].contiguous(),
                          prec=gp.GP_PREC_TC16).cpu().numpy()
    refp = oracle.kernel_mvm(p.kind, p.theta, Xr, Xr[blk], Vb.astype(np.float64), rows=rows)
    assert close(Yp[:, rows], refp, 1e-3)


def test_sgd_workload_full_size_row_panel_sampled_rows(dev):
    p = workloads.sgd()
    n, R = p.n, p.s + 1
    X32 = p.X.astype(np.float32)
    batch = workloads.sgd_batches(n, 512, 1, seed=23)[0]
    V = workloads.vectors(R, n, seed=24).astype(np.float32)
    Xt = torch.tensor(X32, device=dev)
    Xb = Xt[torch.tensor(batch, device=dev)].contiguous()
    G = gp.gp_kernel_mvm(p.kind, p.theta, Xb, torch.tensor(V, device=dev), X2=Xt,
                         prec=gp.GP_PREC_TC16).cpu().numpy()
    pick = np.random.default_rng(25).choice(512, size=12, replace=False)
    Xr = X32.astype(np.float64)
    ref = oracle.kernel_mvm(p.kind, p.theta, Xr[batch], Xr, V.astype(np.float64), rows=pick)
    assert close(G[:, pick], ref, 1e-3)


def test_batched_workload_full_size_sampled_rows(dev):
    s = 16
    ns, ds = workloads.batched_sizes()
    mem = [workloads.batched_member(int(n), int(d), s=s, m=64, seed=0, index=g) for g, (n, d) in enumerate(zip(ns, ds))]
    b = gp.GPBatch(gp.GP_RBF, ns, ds, s, device=dev)
    X = b.pack_points([m.X for m in mem])
    th = b.pack_theta([m.theta for m in mem])
    rng = np.random.default_rng(26)
    Vs = [rng.standard_normal((s + 1, int(n))).astype(np.float32) for n in ns]
    V = b.pack_vectors(Vs)
    b.prepare(th, X)
    Y = b.mvm(V, add_noise=True)
    b.status()
    order = np.argsort(ns)
    check = [int(order[0]), int(order[len(order) // 2]), int(order[-1]), int(np.argmax(ds))]
    Ys = b.unpack_vectors(Y)
    for g in check:
        m = mem[g]
        Xr = m.X.astype(np.float32).astype(np.float64)
        rows = np.random.default_rng(27 + g).choice(m.n, size=min(16, m.n), replace=False)
        ref = oracle.kernel_mvm(m.kind, m.theta, Xr, Xr, Vs[g].astype(np.float64), add_noise=True, rows=rows)
        assert close(Ys[g].cpu().numpy()[:, rows], ref, 1e-3), g
