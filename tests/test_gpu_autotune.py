"""The autotuner beyond the product's schedule: the tensor-core gradient's work split (items of
the symmetric sweep for the pathwise estimator, column splits for the standard one) is timed
and recorded; a recorded choice keeps oracle parity; the table survives a round trip through its
cache file (written, reset, read back: same entries, same bits of the gradient), a file tagged
with another device is refused, and a fresh process picks the file up from GP_AUTOTUNE_CACHE."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2405_18457_gb300 import workloads

pytestmark = pytest.mark.gpu

import paper_2405_18457_gb300 as gp  # noqa: E402  (a missing package fails the run)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    gp.library()
    return torch.device("cuda:0")


def _case(dev, n=6000, d=8, s=16):
    p = workloads.pathwise(n=n, d=d, s=s, m=64, seed=21)
    X = p.X.astype(np.float32)
    V = (0.7 * workloads.vectors(s + 1, n, seed=22)).astype(np.float32)
    Z = workloads.vectors(s, n, seed=23).astype(np.float32)
    t = lambda a: torch.tensor(a, device=dev)  # noqa: E731
    return p, X, V, Z, t(X), t(V), t(Z)


def _oracle_ok(p, X, V, Z, g, pathwise):
    Xr, Vr, Zr = (a.astype(np.float64) for a in (X, V, Z))
    s = V.shape[0] - 1
    lam = np.concatenate([[0.5], np.full(s, -0.5 / s)])
    if pathwise:
        ref, W = oracle.grad_pathwise(p.kind, p.theta, Xr, Vr), Vr
    else:
        ref, W = oracle.grad_standard(p.kind, p.theta, Xr, Vr, Zr), np.vstack([Vr[:1], Zr])
    scale = oracle.grad_bilinear(p.kind, p.theta, Xr, np.abs(Vr), np.abs(W), np.abs(lam))
    assert np.all(np.abs(g - ref) <= 1e-3 * (np.abs(ref) + scale))


@pytest.mark.parametrize("pathwise", [True, False])
def test_tuned_gradient_split_keeps_parity(dev, pathwise):
    p, X, V, Z, Xt, Vt, Zt = _case(dev)
    try:
        best, ms = gp.gp_autotune_grad(p.kind, p.theta, Xt, Vt, None if pathwise else Zt, reps=2)
        assert best >= 1 and ms > 0.0
        if pathwise:
            g = gp.gp_mll_grad_pathwise(p.kind, p.theta, Xt, Vt, prec=gp.GP_PREC_TC16)
        else:
            g = gp.gp_mll_grad_standard(p.kind, p.theta, Xt, Vt, Zt, prec=gp.GP_PREC_TC16)
        _oracle_ok(p, X, V, Z, g.cpu().numpy(), pathwise)
    finally:
        gp.gp_autotune_reset()


def test_cache_file_round_trip(dev, tmp_path):
    p, X, V, Z, Xt, Vt, Zt = _case(dev)
    gp.gp_autotune_reset()
    try:
        gp.gp_autotune_grad(p.kind, p.theta, Xt, Vt, None, reps=1)
        gp.gp_autotune_mvm(p.kind, p.theta, Xt, Vt, reps=1)
        g_tuned = gp.gp_mll_grad_pathwise(p.kind, p.theta, Xt, Vt, prec=gp.GP_PREC_TC16).cpu().numpy()
        n0 = gp.gp_autotune_count()
        assert n0 == 2
        f1 = tmp_path / "tune1.txt"
        gp.gp_autotune_save(f1)
        gp.gp_autotune_reset()
        assert gp.gp_autotune_count() == 0
        gp.gp_autotune_load(f1)
        assert gp.gp_autotune_count() == n0
        f2 = tmp_path / "tune2.txt"
        gp.gp_autotune_save(f2)
        assert f1.read_text() == f2.read_text()
        # the reloaded choice: the same work split, so the same reduction order and bits
        g_loaded = gp.gp_mll_grad_pathwise(p.kind, p.theta, Xt, Vt, prec=gp.GP_PREC_TC16).cpu().numpy()
        assert np.array_equal(g_tuned, g_loaded)
        _oracle_ok(p, X, V, Z, g_loaded, True)
        # another device's file is refused and leaves the table as it was
        lines = f1.read_text().splitlines()
        head = lines[0].split()
        head[2] = "Some_Other_GPU_sm90_x132"
        bad = tmp_path / "other.txt"
        bad.write_text("\n".join([" ".join(head)] + lines[1:]) + "\n")
        with pytest.raises(gp.GPError):
            gp.gp_autotune_load(bad)
        assert gp.gp_autotune_count() == n0
    finally:
        gp.gp_autotune_reset()


def test_cache_file_is_read_from_the_environment(dev, tmp_path):
    p, X, V, Z, Xt, Vt, Zt = _case(dev)
    gp.gp_autotune_reset()
    try:
        gp.gp_autotune_grad(p.kind, p.theta, Xt, Vt, None, reps=1)
        f = tmp_path / "tune_env.txt"
        gp.gp_autotune_save(f)
    finally:
        gp.gp_autotune_reset()
    env = dict(os.environ, GP_AUTOTUNE_CACHE=str(f))
    code = ("import torch, paper_2405_18457_gb300 as gp; torch.zeros(1, device='cuda'); "
            "print(gp.gp_autotune_count())")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().splitlines()[-1] == "1"
