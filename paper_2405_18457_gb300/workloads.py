"""Seeded synthetic inputs shaped like the paper's regression workloads.

This module only draws random numbers; it holds none of the method's arithmetic
(no kernel, no solver, no random-feature evaluation).  Both the CUDA path and the
FP64 oracle take their inputs from here, so the two sides see identical data.

The paper measures on UCI regression sets (App. B "Datasets": pol 13500x26 ...
houseelectric 1844352x11), which are not available here.  The synthetic recipes
below stand in for them with the same n/d range; each follows the workload
descriptions used by the benchmarks and tests:

  small     n=2048,  d=8,  X~U[0,1]^d, y = sin(2 pi sum x) + N(0, 0.1^2), RBF,
            l=0.5, s_f=1, sigma=0.1, s=8 Gaussian probes, CG tol 1e-6, cold.
  pathwise  n=32768, d=16, X~N(0,I), y = RFF prior draw (m=2048, Matern-3/2,
            l=1, s_f=1) + N(0, 0.3^2), s=64, CG tol 0.01, warm start.
  ap        n=262144, d=26, X~U[-1,1]^d, y = RFF draw (m=4096, RBF) + N(0, 0.2^2),
            s=64 pathwise probes, AP block 1024, 10 epochs per step.
  sgd       n=2e6, d=11, X ~ mixture of 32 Gaussians (weights 1/32, means N(0,I),
            isotropic std U[0.1,1]), y = RFF draw (m=8192, Matern-3/2) + N(0,0.1^2),
            s=64, SGD batch 512, momentum 0.9, 1000 iterations per step.
  batched   256 independent RBF GPs, n ~ LogUniform[512, 65536], d in {4,8,16,32},
            X~U[0,1]^d, y = RFF draw + N(0, 0.1^2), s=16.

All draws are float64 from numpy's PCG64 generator seeded per workload; callers
cast to the dtype their path computes in.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RBF = 0
MATERN32 = 1


@dataclass
class Problem:
    name: str
    kind: int
    X: np.ndarray            # n x d
    theta: np.ndarray        # [l_1..l_d, s_f, sigma] initial hyperparameters
    s: int                   # number of probe vectors
    m: int                   # number of random Fourier features (total, cos + sin)
    omega_hat: np.ndarray    # (m/2) x d standard normal frequencies
    chi2: np.ndarray         # m/2 chi^2_3 draws (used by Matern-3/2 only)
    W_probe: np.ndarray      # s x m RFF weights for the s prior samples (pathwise probes)
    W_y: np.ndarray          # 1 x m RFF weights for the target function
    Z: np.ndarray            # s x n standard-normal probes (standard estimator) = fixed w
    y_noise: np.ndarray      # n standard-normal noise for the targets
    noise_y: float           # std of the target noise
    y: np.ndarray | None = None  # targets when they need no method arithmetic (small)
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]


def _rff_parts(rng, m, d, s):
    omega_hat = rng.standard_normal((m // 2, d))
    chi2 = rng.chisquare(3.0, size=m // 2)
    W_probe = rng.standard_normal((s, m))
    W_y = rng.standard_normal((1, m))
    return omega_hat, chi2, W_probe, W_y


def small(n: int = 2048, d: int = 8, s: int = 8, seed: int = 0) -> Problem:
    rng = np.random.default_rng([1, seed])
    X = rng.uniform(0.0, 1.0, size=(n, d))
    y_noise = rng.standard_normal(n)
    y = np.sin(2.0 * np.pi * X.sum(axis=1)) + 0.1 * y_noise
    theta = np.concatenate([np.full(d, 0.5), [1.0, 0.1]])
    m = 2048
    omega_hat, chi2, W_probe, W_y = _rff_parts(rng, m, d, s)
    Z = rng.standard_normal((s, n))
    return Problem("small", RBF, X, theta, s, m, omega_hat, chi2, W_probe, W_y, Z, y_noise, 0.1, y,
                   {"tol": 1e-6, "warm": False, "steps": 20, "lr": 0.1})


def pathwise(n: int = 32768, d: int = 16, s: int = 64, m: int = 2048, seed: int = 0) -> Problem:
    rng = np.random.default_rng([2, seed])
    X = rng.standard_normal((n, d))
    y_noise = rng.standard_normal(n)
    theta = np.concatenate([np.full(d, 1.0), [1.0, 0.3]])
    omega_hat, chi2, W_probe, W_y = _rff_parts(rng, m, d, s)
    Z = rng.standard_normal((s, n))
    return Problem("pathwise", MATERN32, X, theta, s, m, omega_hat, chi2, W_probe, W_y, Z, y_noise,
                   0.3, None, {"tol": 1e-2, "warm": True, "steps": 50, "lr": 0.1})


def ap(n: int = 262144, d: int = 26, s: int = 64, m: int = 4096, seed: int = 0) -> Problem:
    rng = np.random.default_rng([3, seed])
    X = rng.uniform(-1.0, 1.0, size=(n, d))
    y_noise = rng.standard_normal(n)
    theta = np.concatenate([np.full(d, 1.0), [1.0, 0.2]])
    omega_hat, chi2, W_probe, W_y = _rff_parts(rng, m, d, s)
    Z = rng.standard_normal((s, n))
    return Problem("ap", RBF, X, theta, s, m, omega_hat, chi2, W_probe, W_y, Z, y_noise, 0.2, None,
                   {"tol": 1e-2, "warm": True, "steps": 100, "block": 1024, "epochs": 10, "lr": 0.03})


def sgd(n: int = 2_000_000, d: int = 11, s: int = 64, m: int = 8192, seed: int = 0) -> Problem:
    rng = np.random.default_rng([4, seed])
    n_comp = 32
    means = rng.standard_normal((n_comp, d))
    stds = rng.uniform(0.1, 1.0, size=n_comp)
    comp = rng.integers(0, n_comp, size=n)
    X = means[comp] + stds[comp, None] * rng.standard_normal((n, d))
    y_noise = rng.standard_normal(n)
    theta = np.concatenate([np.full(d, 1.0), [1.0, 0.1]])
    omega_hat, chi2, W_probe, W_y = _rff_parts(rng, m, d, s)
    Z = rng.standard_normal((s, n))
    return Problem("sgd", MATERN32, X, theta, s, m, omega_hat, chi2, W_probe, W_y, Z, y_noise, 0.1,
                   None, {"tol": 1e-2, "warm": True, "batch": 512, "momentum": 0.9, "iters": 1000,
                          "lr": 0.03})


def batched_sizes(n_gps: int = 256, n_min: int = 512, n_max: int = 65536, seed: int = 0):
    """n_g ~ round(exp(U[ln n_min, ln n_max])), d_g uniform in {4, 8, 16, 32}."""
    rng = np.random.default_rng([5, seed])
    ns = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_gps))).astype(np.int64)
    ds = rng.choice(np.array([4, 8, 16, 32]), size=n_gps)
    return ns, ds


def batched_member(n: int, d: int, s: int = 16, m: int = 1024, seed: int = 0, index: int = 0) -> Problem:
    rng = np.random.default_rng([6, seed, index])
    X = rng.uniform(0.0, 1.0, size=(n, d))
    y_noise = rng.standard_normal(n)
    theta = np.concatenate([np.full(d, 0.5), [1.0, 0.1]])
    omega_hat, chi2, W_probe, W_y = _rff_parts(rng, m, d, s)
    Z = rng.standard_normal((s, n))
    return Problem("batched", RBF, X, theta, s, m, omega_hat, chi2, W_probe, W_y, Z, y_noise, 0.1,
                   None, {"tol": 1e-2, "warm": True, "iters": 50})


def sgd_batches(n: int, batch: int, iters: int, seed: int = 0) -> np.ndarray:
    """Row indices for Alg. 3: iters x batch, distinct within each batch."""
    rng = np.random.default_rng([7, seed])
    out = np.empty((iters, batch), dtype=np.int64)
    for t in range(iters):
        out[t] = rng.choice(n, size=batch, replace=False)
    return out


def vectors(R: int, n: int, seed: int = 0) -> np.ndarray:
    """R x n standard-normal block (right-hand sides / multiplicands)."""
    return np.random.default_rng([8, seed]).standard_normal((R, n))


def points(n: int, d: int, seed: int = 0, low: float = -1.0, high: float = 1.0) -> np.ndarray:
    return np.random.default_rng([9, seed]).uniform(low, high, size=(n, d))
