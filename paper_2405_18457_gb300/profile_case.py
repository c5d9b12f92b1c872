"""Small, self-contained invocations of single hot-path operations, for profilers.

    python -m paper_2405_18457_gb300.profile_case --op mvm --n 16384 --repeat 3

runs `repeat` launches of the chosen operation on the pathwise workload's shape
(d=16, Matern-3/2, 65 right-hand sides) with seeded synthetic inputs, so that a
profiler can capture one kernel on a case that ends in seconds.  Operations:
mvm (gp_kernel_mvm, H V), grad (gp_mll_grad_pathwise), rff (gp_rff_prior_sample),
cg (gp_solve_cg, 10 iterations).
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

import paper_2405_18457_gb300 as gp
from paper_2405_18457_gb300 import workloads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["mvm", "grad", "rff", "cg"], default="mvm")
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--d", type=int, default=16)
    ap.add_argument("--s", type=int, default=64)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--prec", choices=["tc16", "fp32"], default="tc16")
    ap.add_argument("--time", action="store_true", help="print the mean time per call (CUDA events)")
    args = ap.parse_args()
    prec = gp.GP_PREC_TC16 if args.prec == "tc16" else gp.GP_PREC_FP32
    dev = torch.device("cuda:0")
    p = workloads.pathwise(n=args.n, d=args.d, s=args.s, m=2048, seed=0)
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    X = t(p.X)
    V = t(workloads.vectors(p.s + 1, p.n, seed=1))
    om, c2, Wp = t(p.omega_hat), t(p.chi2), t(p.W_probe)

    def call():
        if args.op == "mvm":
            gp.gp_kernel_mvm(p.kind, p.theta, X, V, add_noise=True, prec=prec)
        elif args.op == "grad":
            gp.gp_mll_grad_pathwise(p.kind, p.theta, X, V, prec=prec)
        elif args.op == "rff":
            gp.gp_rff_prior_sample(p.kind, p.theta, X, om, c2, Wp, prec=prec)
        else:
            gp.gp_solve_cg(p.kind, p.theta, X, V, max_iters=10, tol=0.0, prec=prec)

    if args.time:
        call()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.repeat):
            call()
        e1.record()
        torch.cuda.synchronize()
        print("time_ms %s n=%d %.4f" % (args.op, args.n, e0.elapsed_time(e1) / args.repeat))
        return
    for _ in range(args.repeat):
        call()
    torch.cuda.synchronize()
    print("done", args.op, args.n)


if __name__ == "__main__":
    main()
