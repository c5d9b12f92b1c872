"""Benchmark of the iterative-GP hot path on GB300.

One step = one warm-started pathwise marginal-likelihood step on the pathwise
workload (n=32768, d=16, Matern-3/2, s=64 probes -> 65 right-hand sides,
m=2048 random features, CG to relative tolerance 0.01 with the stop rule of
App. B):
    random-feature prior samples -> pathwise right-hand sides -> CG solve
    (warm start from the previous step; the tolerance certified on the true
    residual) -> fused pathwise gradient -> gradient to the host -> Adam ascent
    step in softplus coordinates.
Inputs are synthetic (seeded generators) and resident in HBM for `value`.

value = kernel-matrix pair x RHS work of the step (every H V product of the
solve's iterations and its initial residual, plus the gradient pass counted as
one n^2 x 65 pass; the true-residual check product is not counted) divided by
the step time, in Gpair*RHS/s.  The product kernel's own rate is beside it
(`mvm_kernel`).  The plain FP64 GPU form of the same steps (replayed from the
same optimiser state, same tolerance on the true residual) is timed beside it.

The same line carries sub-records for the other single-GPU workloads: one
warm-started step of the alternating-projection workload (n=262144, 10-epoch
budget), one of the SGD workload (n=2,000,000, 1000 iterations) and a few
steps of the batched workload (256 uneven GPs, p50/p99), each with the
roofline of its dominant kernel and the oracle's rate on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       python bench.py --op mvm|grad|rff|cg|unit-rates [--n N] [--repeat R]   (single
           operations, for profilers)
With torchrun (N > 1) every rank runs an independent replica (weak scaling, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "kernel-MVM Gpair*RHS/s (whole warm-started pathwise MLL step; sec per step vs plain FP64 GPU form)"
UNIT = "Gpair*RHS/s"
L2_BYTES = 129 * 1024 * 1024
# Sec. 5 "The Effects of Early Stopping": solver budgets of 10 to 50 epochs per step
EPOCH_BUDGETS = (10, 20, 30, 40, 50)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def pair_roofline(kind, d, R, pairs, launch_s, rates, peaks, peak_src, sms, clk_mhz, kd, r_pad, kernel):
    """Roofline of one kernel-matrix launch over `pairs` (i, j) pairs: the slower of
      MUFU   : Matern-3/2 needs one rsqrt and one ex2 per pair, RBF one ex2, at the unit rates
               measured on this GPU (gp_diag_unit_rates: per SM per clock) x SMs x max SM clock;
      tensor : the algorithmic contraction, 2 d flops (distance cross term) + 2 R flops (K V)
               per pair, at the measured sustained bf16 dense rate (fp16 runs at the same rate).
    The kernel's own contraction is wider (hi/lo split distance columns padded to KD, right-hand
    sides padded to R_pad); that padding is reported, not counted."""
    per_pair_clk = 1.0 / rates["ex2"] + (1.0 / rates["rsqrt"] if kind == 1 else 0.0)
    mufu = sms * clk_mhz * 1e6 / per_pair_clk  # pairs/s
    tpeak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * 1e12
    tensor = tpeak / (2.0 * d + 2.0 * R)  # pairs/s
    peak = min(mufu, tensor)
    achieved = pairs / launch_s if launch_s else None
    return {"bound": "alu" if mufu <= tensor else "tensor", "unit": "Gpair/s",
            "achieved": achieved / 1e9 if achieved else None, "peak": peak / 1e9,
            "frac": (achieved / peak) if achieved else None, "traffic": None,
            "peak_derivation": "min(MUFU: %d SMs x %.0f MHz / (%s), tensor: %.0f TFLOP/s / (2d + 2R = %d flops))"
                               % (sms, clk_mhz, "1/ex2 + 1/rsqrt" if kind == 1 else "1/ex2", tpeak / 1e12,
                                  2 * d + 2 * R),
            "mufu_gpairs_per_s": mufu / 1e9, "tensor_alg_gpairs_per_s": tensor / 1e9,
            "unit_rates_per_sm_clk": {k: round(v, 2) for k, v in rates.items()},
            "peak_source": "%s (unit rates measured live; bf16 rate from MEASURED_PEAKS.json)" % peak_src,
            "kernel": kernel, "avg_launch_ms": launch_s * 1e3 if launch_s else None, "pairs_per_launch": pairs,
            "padded_contraction_flops_per_pair": 2 * kd + 2 * r_pad,
            "algorithmic_flops_per_pair": 2 * d + 2 * R}


def kd_of(d):
    """Width of the tensor-core distance contraction (hi/lo split columns, padded to 64)."""
    return 64 * -(-(3 * d + 4) // 64)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index

    def start(self):
        if shutil.which("nvidia-smi") is None:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits", "-lms", "50"],
                                     stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        # the sampler is running (first row written) before the timed region starts
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        if len(rows) > 1:
            rows = rows[1:]  # the first row was taken before the region started
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


class Replica:
    """State of one warm-started marginal-likelihood optimisation run."""

    def __init__(self, gp, torch, prob, dev, dtype, prec, max_iters):
        self.gp = gp
        self.torch = torch
        self.p = prob
        self.dev = dev
        self.dtype = dtype
        self.prec = prec
        self.max_iters = max_iters
        t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)  # noqa: E731
        self.host = {k: np.ascontiguousarray(v, dtype=np.float64 if dtype == torch.float64 else np.float32)
                     for k, v in dict(X=prob.X, om=prob.omega_hat, c2=prob.chi2, Wp=prob.W_probe, w=prob.Z).items()}
        self.X = t(prob.X)
        self.om = t(prob.omega_hat)
        self.c2 = t(prob.chi2)
        self.Wp = t(prob.W_probe)
        self.w = t(prob.Z)
        # fixed targets: one prior draw at the initial hyperparameters plus noise
        fy = gp.gp_rff_prior_sample(prob.kind, prob.theta, self.X, self.om, self.c2, t(prob.W_y))[0]
        self.y = (fy + prob.noise_y * t(prob.y_noise)).contiguous()
        self.host["y"] = self.y.cpu().numpy()
        self.theta = prob.theta.copy()
        self.nu = np.log(np.expm1(self.theta))
        self.m = np.zeros_like(self.nu)
        self.v = np.zeros_like(self.nu)
        self.t = 1
        self.V = torch.zeros((prob.s + 1, prob.n), dtype=dtype, device=dev)
        self.last = None
        self.phase_ms = None
        self._events = []

    def snapshot(self):
        """The optimiser's state (hyperparameters, Adam moments, warm start), to replay the
        same steps later."""
        return (self.theta.copy(), self.nu.copy(), self.m.copy(), self.v.copy(), self.t, self.V.clone())

    def restore(self, snap):
        theta, nu, m, v, self.t, V = snap
        self.theta, self.nu, self.m, self.v = theta.copy(), nu.copy(), m.copy(), v.copy()
        self.V.copy_(V)

    def pinned_inputs(self):
        torch = self.torch
        return {k: torch.from_numpy(v).pin_memory() for k, v in self.host.items()}

    def load_inputs(self, pinned):
        """Host-to-device copy of every input of a step (end-to-end timing)."""
        self.X.copy_(pinned["X"], non_blocking=True)
        self.om.copy_(pinned["om"], non_blocking=True)
        self.c2.copy_(pinned["c2"], non_blocking=True)
        self.Wp.copy_(pinned["Wp"], non_blocking=True)
        self.w.copy_(pinned["w"], non_blocking=True)
        self.y.copy_(pinned["y"], non_blocking=True)
        return sum(v.numel() * v.element_size() for v in pinned.values())

    def _mark(self, name):
        if self.phase_ms is not None:
            ev = self.torch.cuda.Event(enable_timing=True)
            ev.record()
            self._events.append((name, ev))

    def step(self):
        gp, p = self.gp, self.p
        th = self.theta
        self._events = []
        self._mark("start")
        if self.dtype == self.torch.float64:
            F = gp.gp_rff_prior_sample(p.kind, th, self.X, self.om, self.c2, self.Wp)
            sig = th[-1]
            B = self.torch.cat([self.y[None], F + sig * self.w], 0)
        else:
            F = gp.gp_rff_prior_sample(p.kind, th, self.X, self.om, self.c2, self.Wp)
            B = gp.gp_pathwise_rhs(th, p.d, self.y, F, self.w)
        self._mark("rff+rhs")
        V, info = gp.gp_solve_cg(p.kind, th, self.X, B, V0=self.V, max_iters=self.max_iters, tol=0.01,
                                 prec=self.prec)
        self._mark("cg")
        g = gp.gp_mll_grad_pathwise(p.kind, th, self.X, V, prec=self.prec)
        self._mark("grad")
        gh = g.cpu().numpy()  # device -> host read of the step's result
        if self.phase_ms is not None:
            for (_, e0), (name, e1) in zip(self._events[:-1], self._events[1:]):
                self.phase_ms[name] = self.phase_ms.get(name, 0.0) + e0.elapsed_time(e1)
        self.last_theta = th
        self.theta = gp.gp_adam_softplus_step(self.nu, self.m, self.v, self.t, gh, lr=0.1)
        self.t += 1
        self.last = info
        return info, gh

    def work(self, info):
        n, R = self.p.n, self.p.s + 1
        return float(info.iters + 2) * n * n * R  # solve products (+1 initial residual) + gradient pass


def recorded_traffic(n, prec_tc16):
    """DRAM bytes per launch of the product kernel from the committed ncu capture
    (profiles/tc_mvm_kernel_traffic.json), or None when the kernel source has changed since
    the counters were taken or the workload differs."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "tc_mvm_kernel_traffic.json")
    if not (prec_tc16 and n == 32768 and os.path.exists(path)):
        return None
    with open(path) as f:
        rec = json.load(f)
    with open(os.path.join(ROOT, rec["source"]), "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    return rec["traffic_bytes_per_launch"] if digest == rec["source_sha256"] else None


def combine_ranks(dist, device, seconds, work):
    """Whole-job figures of the replicas: the slowest rank's time and the summed work
    (weak scaling; no data-path collective, only this reduction of two scalars)."""
    import torch

    if dist is None:
        return seconds, work
    tt = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ww = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(ww)
    return float(tt.item()), float(ww.item())


def flush_l2(torch, buf):
    buf.add_(1.0)


def run_ours(args):
    import torch

    import paper_2405_18457_gb300 as gp
    from paper_2405_18457_gb300 import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    assert torch.cuda.is_available(), "bench.py needs a CUDA device (no CPU fallback)"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gp.library()
    prec = gp.GP_PREC_TC16 if args.prec == "tc16" else gp.GP_PREC_FP32
    n = args.n
    prob = workloads.pathwise(n=n, seed=rank)
    rates = gp.gp_diag_unit_rates(4096)  # MUFU / FMA unit rates of this GPU (roofline peaks)
    rep = Replica(gp, torch, prob, dev, torch.float32, prec, args.max_iters)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    tuned = None
    if prec == gp.GP_PREC_TC16 and not args.no_autotune:
        # schedule of the product chosen by timing (column splits), before any timed work
        Vt = torch.randn((prob.s + 1, n), dtype=torch.float32, device=dev)
        best, best_ms = gp.gp_autotune_mvm(prob.kind, prob.theta, rep.X, Vt, reps=3)
        gbest, gbest_ms = gp.gp_autotune_grad(prob.kind, prob.theta, rep.X, Vt, None, reps=3)
        tuned = {"column_splits": best, "ms": best_ms, "gradient_tile_pairs_per_item": gbest, "gradient_ms": gbest_ms}

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        rep.step()
    # ---- device-resident timed steps
    start_state = rep.snapshot()
    clocks = Clocks(local)
    barrier()
    gp.gp_diag_reset(True)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    work = 0.0
    iters, res = [], []
    for k in range(args.steps):
        flush_l2(torch, flush)
        starts[k].record()
        info, gh = rep.step()
        ends[k].record()
        work += rep.work(info)
        iters.append(info.iters)
        res.append((info.res_y, info.res_z, bool(info.converged)))
    barrier()
    launches = gp.gp_diag_launches()
    gp.gp_diag_reset(False)
    # Dominant-kernel timing: CUDA events around each launch of the product kernel (and the
    # gradient kernel) on the step's own inputs, L2 flushed between launches.  Timed apart
    # from the solver, whose speculatively enqueued iterations past convergence return at once.
    barrier()
    gp.gp_diag_reset(True)
    for _ in range(args.kernel_reps):
        flush_l2(torch, flush)
        gp.gp_kernel_mvm(prob.kind, rep.theta, rep.X, rep.V, add_noise=True, prec=prec)
    for _ in range(max(1, args.kernel_reps // 2)):
        flush_l2(torch, flush)
        gp.gp_mll_grad_pathwise(prob.kind, rep.theta, rep.X, rep.V, prec=prec)
    torch.cuda.synchronize()
    prod_ms, prod_cnt = gp.gp_diag_kernel_time(0)
    grad_ms, grad_cnt = gp.gp_diag_kernel_time(1)
    gp.gp_diag_reset(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(step_ms) / 1e3
    # one extra, separately timed step for the per-phase breakdown (not in `value`)
    rep.phase_ms = {}
    rep.step()
    phases = {k: round(v, 3) for k, v in rep.phase_ms.items()}
    rep.phase_ms = None
    total_s, work = combine_ranks(dist, dev, total_s, work)
    value = work / total_s / 1e9

    # ---- end-to-end: inputs copied from pinned host memory every step, gradient read back.
    # The same steps as the timed ones (the optimiser state is rewound): warm-started CG needs
    # fewer iterations as the optimisation proceeds, so later steps would carry a larger share
    # of the per-step fixed work (random features, gradient pass) and not be comparable.
    pinned = rep.pinned_inputs()
    rep.restore(start_state)
    barrier()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_work = 0.0
    h2d = 0
    e_iters = []
    e_start.record()
    for k in range(args.steps):
        h2d = rep.load_inputs(pinned)
        info, gh = rep.step()
        e_work += rep.work(info)
        e_iters.append(info.iters)
    e_end.record()
    barrier()
    clk = clocks.stop()  # sampled from the first timed step to the last end-to-end step
    if clk:
        clk["region"] = "timed steps, kernel timing and end-to-end steps"
    e_s = e_start.elapsed_time(e_end) / 1e3
    e_s, e_work = combine_ranks(dist, dev, e_s, e_work)

    # ---- plain FP64 GPU form of the same steps: the first `fp64_steps` timed steps replayed
    # from the same optimiser state (hyperparameters, Adam moments, warm start), each solved to
    # the same tolerance on its true residual, device-timed like the mixed form's steps.
    fp64 = None
    if args.fp64_steps > 0:
        F = min(args.fp64_steps, args.steps)
        rep64 = Replica(gp, torch, prob, dev, torch.float64, gp.GP_PREC_FP32, args.max_iters)
        rep64.restore(start_state)
        per64 = []
        for k in range(F):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            flush_l2(torch, flush)
            e0.record()
            info64, _ = rep64.step()
            e1.record()
            torch.cuda.synchronize()
            per64.append({"ms": e0.elapsed_time(e1), "cg_iters": int(info64.iters), "res_y": info64.res_y,
                          "res_z": info64.res_z, "converged": bool(info64.converged)})
        mixed = [{"ms": step_ms[k], "cg_iters": int(iters[k]), "res_y": res[k][0], "res_z": res[k][1],
                  "converged": res[k][2]} for k in range(F)]
        f_s = float(np.mean([r["ms"] for r in per64])) / 1e3
        m_s = float(np.mean([r["ms"] for r in mixed])) / 1e3
        fp64 = {"steps_replayed": F, "sec_per_step": f_s, "mixed_sec_per_step_same_steps": m_s,
                "ms_per_cg_iteration": float(np.sum([r["ms"] for r in per64]) / max(1, sum(r["cg_iters"] for r in per64))),
                "mixed_ms_per_cg_iteration": float(np.sum([r["ms"] for r in mixed]) /
                                                   max(1, sum(r["cg_iters"] for r in mixed))),
                "fp64_steps": per64, "mixed_steps": mixed,
                "residuals": "true residual norms of the returned solutions (FP64 form: exact operator; mixed "
                             "form: its tensor-core operator, certified at tau - 1e-3); both meet tau = 0.01"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    peaks, peak_src = _peaks()
    d, R = prob.d, prob.s + 1
    avg_launch_s = (prod_ms / 1e3) / max(prod_cnt, 1)
    clk_mhz = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    pairs = float(n) * n
    if prec == gp.GP_PREC_TC16:
        roof = pair_roofline(prob.kind, d, R, pairs, avg_launch_s if prod_cnt else None, rates, peaks, peak_src, sms,
                             clk_mhz, kd_of(d), 16 * -(-R // 16), "tc_mvm_kernel (H V)")
        tpeak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        tflops = (2.0 * kd_of(d) + 2.0 * 16 * -(-R // 16)) * pairs / avg_launch_s / 1e12 if prod_cnt else None
        roof["tensor_pipe_tflops_padded"] = tflops
        roof["tensor_pipe_frac_of_measured_bf16_sustained"] = (tflops / tpeak) if tflops else None
    else:
        # FP32 CUDA-core peak at the measured FMA rate: per pair ~3d + 2R + 10 FP32 flops
        flops_pair = 3.0 * d + 2.0 * R + 10.0
        peak = sms * rates["ffma"] * 2 * clk_mhz * 1e6 / 1e12
        achieved = flops_pair * pairs / avg_launch_s / 1e12 if prod_cnt else None
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak": peak, "algorithmic_flops_per_pair": flops_pair,
                "achieved": achieved, "frac": (achieved / peak) if achieved else None, "traffic": None,
                "kernel": "mvm_simt_kernel (H V)", "avg_launch_ms": avg_launch_s * 1e3}
    roof["traffic"] = recorded_traffic(n, prec == gp.GP_PREC_TC16)
    roof["launches_timed"] = prod_cnt
    grad_kernel = None
    if grad_cnt:
        g_avg = grad_ms / 1e3 / grad_cnt
        # the pathwise estimator's summand is symmetric: the kernel sweeps the upper triangle of
        # tiles (n^2 / 2 evaluated pairs, the off-diagonal ones counted twice)
        ev = pairs / 2.0 + 64.0 * n
        groof = pair_roofline(prob.kind, d, R, ev, g_avg, rates, peaks, peak_src, sms, clk_mhz, kd_of(d),
                              16 * -(-R // 16), "tc_grad_kernel (fused pathwise gradient, upper triangle)")
        grad_kernel = {"kernel": "tc_grad_kernel", "avg_launch_ms": g_avg * 1e3, "launches_timed": grad_cnt,
                       "logical_gpairs_per_s": pairs / g_avg / 1e9, "evaluated_pairs_per_launch": ev,
                       "frac_of_roofline_evaluated": groof["frac"], "roofline": groof}
    cpu = cpu_baseline(prob, R, budget_s=args.cpu_seconds)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16-tensor/f32/f64" if prec == gp.GP_PREC_TC16 else "f32",
        "data": "synthetic (seeded; shaped like the paper's UCI regression workloads)",
        "config": {"workload": "pathwise MLL step: n=%d d=%d Matern-3/2 s=%d (R=%d) m=%d RFF, CG tol 0.01 warm start,"
                               " pathwise gradient, Adam lr 0.1" % (n, d, prob.s, R, prob.m),
                   "n": n, "d": d, "rhs": R, "precision": args.prec, "l2": "flushed between timed steps",
                   "parallelism": "replicas" if world > 1 else "single GPU", "autotuned": tuned},
        "sec_per_step": total_s / args.steps,
        "cg_iters_per_step": iters,
        "final_true_residuals": [[round(r[0], 5), round(r[1], 5)] for r in res],
        "phase_ms_one_step": phases,
        "mvm_kernel": {"gpair_rhs_per_s": pairs * R / avg_launch_s / 1e9 if prod_cnt else None,
                       "note": "the product kernel alone (n^2 x R per launch / its mean launch time)"},
        "fp64_form": fp64,
        "speedup_vs_fp64_form": (fp64["sec_per_step"] / fp64["mixed_sec_per_step_same_steps"]) if fp64 else None,
        "e2e": {"value": e_work / e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 8 * (d + 2), "ms_per_step": 1e3 * e_s / args.steps, "cg_iters_per_step": e_iters},
        "gpu_launches": launches,
        "roofline": roof,
        "gradient_kernel": grad_kernel,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    del rep, flush, pinned
    if world == 1 and not args.no_subrecords:
        torch.cuda.empty_cache()
        out["workloads"] = {
            "ap": solver_record(torch, gp, workloads, dev, "ap", rates, peaks, peak_src, sms, clk_mhz,
                                args.sub_cpu_seconds),
            "sgd": solver_record(torch, gp, workloads, dev, "sgd", rates, peaks, peak_src, sms, clk_mhz,
                                 args.sub_cpu_seconds),
            "batched": batched_record(torch, gp, workloads, dev, rates, peaks, peak_src, sms, clk_mhz,
                                      steps=args.batched_steps, warmup=1, kernel_reps=3, n_gps=args.n_gps,
                                      cpu_seconds=args.sub_cpu_seconds, rank=0, local=local),
        }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def run_solver_workload(args):
    """The alternating-projection or SGD workload on its own (python bench.py --workload ap|sgd):
    solver_record's line.  --solver-iters overrides the iteration budget (for profiling)."""
    torch, gp, workloads, dev = _gpu_setup()
    rates = gp.gp_diag_unit_rates(4096)
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = solver_record(torch, gp, workloads, dev, args.workload, rates, peaks, peak_src, sms,
                        peaks.get("sm_max_mhz", 2070.0), args.cpu_seconds, iters_override=args.solver_iters)
    out.update({"n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f16-tensor/f32/f64", "data": "synthetic (seeded)"})
    print(json.dumps(out))


def solver_record(torch, gp, workloads, dev, which, rates, peaks, peak_src, sms, clk_mhz, cpu_seconds,
                  iters_override=0):
    """One warm-started pathwise marginal-likelihood step of the alternating-projection workload
    (which = "ap": n = 262144, d = 26, RBF, AP with 1024-row blocks, a budget of 10 epochs = 2560
    block iterations; Alg. 2, Sec. 5 "The Effects of Early Stopping") or the SGD workload
    (which = "sgd": n = 2,000,000, d = 11, Matern-3/2, SGD with 512-row batches, momentum 0.9,
    1000 iterations; Alg. 3): random features -> pathwise right-hand sides -> solver (tau = 0.01,
    warm start from an untimed first solve) -> pathwise gradient -> Adam.  The step is timed with
    CUDA events, its dominant kernel (the solver's panel product) in a loop of its own."""
    p = workloads.ap() if which == "ap" else workloads.sgd()
    n, d, R = p.n, p.d, p.s + 1
    bs = 1024 if which == "ap" else 512
    iters = 10 * n // bs if which == "ap" else 1000
    if iters_override:
        iters = iters_override
    tf = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    X = tf(p.X)
    om, c2, Wp, w = tf(p.omega_hat), tf(p.chi2), tf(p.W_probe), tf(p.Z)
    y = (gp.gp_rff_prior_sample(p.kind, p.theta, X, om, c2, tf(p.W_y))[0] + p.noise_y * tf(p.y_noise)).contiguous()
    V = torch.zeros((R, n), dtype=torch.float32, device=dev)
    idx = None
    if which == "sgd":
        idx = torch.tensor(workloads.sgd_batches(n, bs, iters, seed=13), dtype=torch.int32, device=dev)
    theta = p.theta.copy()
    nu = np.log(np.expm1(theta))
    m_, v_ = np.zeros_like(nu), np.zeros_like(nu)
    lr_sgd = None

    def rhs(th):
        F = gp.gp_rff_prior_sample(p.kind, th, X, om, c2, Wp)
        return gp.gp_pathwise_rhs(th, d, y, F, w)

    def solve(th, B, lr=None):
        if which == "ap":
            return gp.gp_solve_ap(p.kind, th, X, B, V0=V, block_size=bs, max_iters=iters, tol=0.01,
                                  prec=gp.GP_PREC_TC16)
        return gp.gp_solve_sgd(p.kind, th, X, B, idx, lr=lr, momentum=0.9, V0=V, tol=0.01, prec=gp.GP_PREC_TC16)

    # untimed first step (cold solve, gradient, Adam), which gives the timed step its warm start
    # at new hyperparameters; the SGD step size is the largest of the grid that does not diverge
    # on the first solve (App. B "Stochastic Gradient Descent"; the reading of the paper's rule)
    B = rhs(theta)
    if which == "sgd":
        for lr in (50.0, 20.0, 10.0, 5.0, 2.0, 1.0, 0.5):
            V.zero_()
            try:
                solve(theta, B, lr)
                lr_sgd = lr
                break
            except gp.GPError:
                continue
    else:
        solve(theta, B)
    g = gp.gp_mll_grad_pathwise(p.kind, theta, X, V, prec=gp.GP_PREC_TC16)
    lr_adam = 0.1 if n < 50000 else 0.03  # App. B "Iterative Optimiser": 0.03 above 50k points
    theta = gp.gp_adam_softplus_step(nu, m_, v_, 1, g.cpu().numpy(), lr=lr_adam)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    B = rhs(theta)
    ev[1].record()
    _, info = solve(theta, B, lr_sgd)
    ev[2].record()
    g = gp.gp_mll_grad_pathwise(p.kind, theta, X, V, prec=gp.GP_PREC_TC16)
    gh = g.cpu().numpy()
    ev[3].record()
    theta = gp.gp_adam_softplus_step(nu, m_, v_, 2, gh, lr=lr_adam)
    torch.cuda.synchronize()
    step_s = ev[0].elapsed_time(ev[3]) / 1e3
    solve_s = ev[1].elapsed_time(ev[2]) / 1e3
    grad_s = ev[2].elapsed_time(ev[3]) / 1e3
    it = int(info.iters)
    panel_pairs = float(n) * bs
    # solver work: its panel products, its initial-residual product (AP), the gradient pass
    work = (it * panel_pairs + (float(n) * n if which == "ap" else 0.0) + float(n) * n) * R
    # dominant kernel: the panel product in the solver's shape, events per launch, L2 flushed
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    if which == "ap":
        blk = slice(5 * bs, 6 * bs)
        Xc, Vc, Xr_ = X[blk].contiguous(), V[:, blk].contiguous(), X
    else:
        rows = torch.tensor(workloads.sgd_batches(n, bs, 1, seed=14)[0], dtype=torch.int64, device=dev)
        Xc, Vc, Xr_ = X, V, X[rows].contiguous()
    gp.gp_diag_reset(True)
    for _ in range(5):
        flush_l2(torch, flush)
        gp.gp_kernel_mvm(p.kind, theta, Xr_, Vc, X2=Xc, prec=gp.GP_PREC_TC16)
    torch.cuda.synchronize()
    k_ms, k_cnt = gp.gp_diag_kernel_time(0)
    gp.gp_diag_reset(False)
    launch_s = k_ms / 1e3 / max(k_cnt, 1)
    roof = pair_roofline(p.kind, d, R, panel_pairs, launch_s, rates, peaks, peak_src, sms, clk_mhz, kd_of(d),
                         16 * -(-R // 16), "tc_mvm_kernel (%s panel: %s)" % (
                             which, "all n rows x one 1024-column block" if which == "ap"
                             else "512 batch rows x all n columns"))
    # oracle on the host cores: sampled rows of the same panel product
    import oracle

    Xh = p.X.astype(np.float32).astype(np.float64)
    Vh = Vc.double().cpu().numpy()
    Xrows = Xh if which == "ap" else Xh[workloads.sgd_batches(n, bs, 1, seed=14)[0]]
    Xcols = Xh[5 * bs:6 * bs] if which == "ap" else Xh
    t0 = time.perf_counter()
    oracle.kernel_mvm(p.kind, theta, Xrows, Xcols, Vh, rows=np.arange(2))
    t2 = max(time.perf_counter() - t0, 1e-6)
    k = int(max(2, min(Xrows.shape[0], 2 * cpu_seconds / t2)))
    sample = np.random.default_rng(3).choice(Xrows.shape[0], size=k, replace=False)
    t0 = time.perf_counter()
    oracle.kernel_mvm(p.kind, theta, Xrows, Xcols, Vh, rows=sample)
    dt = time.perf_counter() - t0
    cols = Xcols.shape[0]
    cpu = {"value": k * cols * R / dt / 1e9, "unit": "Gpair*RHS/s",
           "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
           "sample": "%d sampled rows of the %s panel product (%d columns, R=%d), FP64, %.1f s"
                     % (k, which, cols, R, dt)}
    return {"metric": "Gpair*RHS/s of one warm-started pathwise MLL step (%s solver)" % which.upper(),
            "value": work / step_s / 1e9, "unit": "Gpair*RHS/s",
            "config": {"workload": ("alternating projections: n=%d d=%d RBF s=%d b=%d, 10 epochs (%d block iterations), "
                                    "tol 0.01, warm start" % (n, d, p.s, bs, iters)) if which == "ap" else
                                   ("SGD: n=%d d=%d Matern-3/2 mixture of 32 Gaussians s=%d b=%d momentum 0.9 lr %s, "
                                    "%d iterations, tol 0.01, warm start" % (n, d, p.s, bs, lr_sgd, iters)),
                       "n": n, "d": d, "rhs": R},
            "ms_per_step": step_s * 1e3, "solver_ms": solve_s * 1e3, "gradient_and_readback_ms": grad_s * 1e3,
            "solver_iters": it, "converged": bool(info.converged), "res_y": info.res_y, "res_z": info.res_z,
            "residual_kind": "true residual (recomputed)" if which == "ap" else "Alg. 3 residual estimate",
            "roofline": roof, "cpu_baseline": cpu}


SMALL_METRIC = "sec per MLL step, small workload (CG to 1e-6, cold start), plain vs pivoted-Cholesky preconditioned CG"


def run_small(args):
    """The small workload (n = 2048, d = 8, RBF l = 0.5, sigma = 0.1, s = 8 Gaussian probes, CG to
    relative tolerance 1e-6 from a cold start, standard estimator, Adam lr 0.1): seconds per MLL
    step with plain CG and with the rank-100 pivoted Cholesky preconditioner of App. B in the
    FP64 form (a true residual of 1e-6 on this system, condition number about 1e4, is below
    what FP32 vectors attain, and CG certifies its tolerance on the true residual), next to the
    FP32 form of both at 1e-4."""
    import torch

    import paper_2405_18457_gb300 as gp
    from paper_2405_18457_gb300 import workloads

    assert torch.cuda.is_available(), "bench.py needs a CUDA device (no CPU fallback)"
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    gp.library()
    p = workloads.small()
    res = {}
    for name, dtype, rank, tol in (("fp64_plain", torch.float64, 0, 1e-6), ("fp64_pc100", torch.float64, 100, 1e-6),
                                   ("fp32_plain_tol1e-4", torch.float32, 0, 1e-4),
                                   ("fp32_pc100_tol1e-4", torch.float32, 100, 1e-4)):
        Xt = torch.tensor(p.X, dtype=dtype, device=dev)
        B = torch.tensor(np.vstack([p.y, p.Z]), dtype=dtype, device=dev)
        Zt = B[1:].contiguous()
        nu = np.log(np.expm1(p.theta))
        m = np.zeros_like(nu)
        v = np.zeros_like(nu)
        theta = p.theta.copy()
        steps = args.steps
        times, iters, conv = [], [], []
        for t in range(1, args.warmup + steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            V, info = gp.gp_solve_cg(p.kind, theta, Xt, B, max_iters=20000, tol=tol, prec=gp.GP_PREC_FP32,
                                     precond_rank=rank)
            g = gp.gp_mll_grad_standard(p.kind, theta, Xt, V, Zt, prec=gp.GP_PREC_FP32).cpu().numpy()
            theta = gp.gp_adam_softplus_step(nu, m, v, t, g, lr=0.1)
            torch.cuda.synchronize()
            if t > args.warmup:
                times.append(time.perf_counter() - t0)
                iters.append(info.iters)
                conv.append(bool(info.converged))
        res[name] = {"sec_per_step": float(np.mean(times)), "cg_iters": iters, "tol": tol,
                     "converged_steps": int(sum(conv))}
    out = {"metric": SMALL_METRIC, "value": res["fp64_pc100"]["sec_per_step"], "unit": "s per step",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * res["fp64_pc100"]["sec_per_step"], "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic (seeded)",
           "config": {"workload": "small: n=2048 d=8 RBF l=0.5 sigma=0.1 s=8, CG tol 1e-6 cold (FP64 form), standard "
                                  "estimator, Adam lr 0.1"},
           "forms": res,
           "speedup_pc_vs_plain": res["fp64_plain"]["sec_per_step"] / res["fp64_pc100"]["sec_per_step"]}
    print(json.dumps(out))


ABL_METRIC = "solver time to tolerance per MLL step: standard vs pathwise x cold vs warm x CG/AP/SGD"


class SolverGrid:
    """Shared set-up of the solver ablations (Table 1's design, Sec. 5's budgets) on synthetic data:
    Matern-3/2, n = 8192, d = 8, s = 64, sigma = 0.3, targets an RFF prior draw plus noise, the
    tensor-core form, tau = 0.01, AP with 1024-row blocks, SGD with 512-row batches and momentum 0.9
    (step size: the largest of a grid that does not diverge on the first system), Adam lr 0.1."""

    def __init__(self, torch, gp, workloads, dev, n=8192, s=64):
        self.torch, self.gp, self.wl, self.dev = torch, gp, workloads, dev
        self.n, self.s = n, s
        p = self.p = workloads.pathwise(n=n, d=8, s=s, m=1024, seed=11)
        tf = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
        self.X = tf(p.X)
        self.om, self.c2, self.Wp, self.w = tf(p.omega_hat), tf(p.chi2), tf(p.W_probe), tf(p.Z)
        fy = gp.gp_rff_prior_sample(p.kind, p.theta, self.X, self.om, self.c2, tf(p.W_y))[0]
        self.y = (fy + p.noise_y * tf(p.y_noise)).contiguous()
        self.B_std = torch.cat([self.y[None], self.w], 0).contiguous()
        self.prec = gp.GP_PREC_TC16
        self.bs_ap, self.bs_sgd = 1024, 512
        self.rng = np.random.default_rng(12)
        self.lr_sgd = None
        for lr in (50.0, 20.0, 10.0, 5.0, 2.0, 1.0, 0.5):
            try:
                self.solve("sgd", p.theta, self.B_std, None, 40, lr=lr)
                self.lr_sgd = lr
                break
            except gp.GPError:
                continue

    def solve(self, solver, theta, B, V0, epochs, lr=None):
        gp, p, n = self.gp, self.p, self.n
        if solver == "cg":
            return gp.gp_solve_cg(p.kind, theta, self.X, B, V0=V0, max_iters=epochs, tol=0.01, prec=self.prec)
        if solver == "ap":
            return gp.gp_solve_ap(p.kind, theta, self.X, B, V0=V0, block_size=self.bs_ap,
                                  max_iters=epochs * n // self.bs_ap, tol=0.01, prec=self.prec)
        iters = epochs * n // self.bs_sgd
        idx = self.torch.tensor(self.wl.sgd_batches(n, self.bs_sgd, iters, seed=int(self.rng.integers(1 << 30))),
                                dtype=self.torch.int32, device=self.dev)
        return gp.gp_solve_sgd(p.kind, theta, self.X, B, idx, lr=self.lr_sgd if lr is None else lr, momentum=0.9,
                               V0=V0, tol=0.01, prec=self.prec)

    def rhs(self, theta, pathwise):
        gp, p = self.gp, self.p
        if not pathwise:
            return self.B_std
        F = gp.gp_rff_prior_sample(p.kind, theta, self.X, self.om, self.c2, self.Wp)
        return gp.gp_pathwise_rhs(theta, p.d, self.y, F, self.w)

    def true_residuals(self, theta, B, V):
        """Relative residual norms ||b - H v|| / ||b|| of the y system and the mean over the probes'
        systems, from one product (measurement only)."""
        HV = self.gp.gp_kernel_mvm(self.p.kind, theta, self.X, V, add_noise=True, prec=self.prec)
        rel = ((B - HV).norm(dim=1) / B.norm(dim=1)).double().cpu().numpy()
        return float(rel[0]), float(rel[1:].mean())

    def run(self, solver, pathwise, warm, steps, epochs, residuals=False):
        """`steps` marginal-likelihood steps; per step the solver's wall time, iterations, convergence
        flag and (optionally) the true residual norms reached."""
        torch, gp, p = self.torch, self.gp, self.p
        theta = p.theta.copy()
        nu = np.log(np.expm1(theta))
        m_, v_ = np.zeros_like(nu), np.zeros_like(nu)
        V = None
        out = {"sec": [], "iters": [], "converged": [], "res_y": [], "res_z": []}
        for t in range(1, steps + 1):
            B = self.rhs(theta, pathwise)
            V0 = V.clone() if (warm and V is not None) else None
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                V, info = self.solve(solver, theta, B, V0, epochs)
            except gp.GPError:
                V, info = None, None
            torch.cuda.synchronize()
            out["sec"].append(time.perf_counter() - t0)
            if info is None:
                out["iters"].append(-1)
                out["converged"].append(False)
                continue
            out["iters"].append(int(info.iters))
            out["converged"].append(bool(info.converged))
            if residuals:
                ry, rz = self.true_residuals(theta, B, V)
                out["res_y"].append(ry)
                out["res_z"].append(rz)
            if pathwise:
                g = gp.gp_mll_grad_pathwise(p.kind, theta, self.X, V, prec=self.prec)
            else:
                g = gp.gp_mll_grad_standard(p.kind, theta, self.X, V, self.w, prec=self.prec)
            theta = gp.gp_adam_softplus_step(nu, m_, v_, t, g.cpu().numpy(), lr=0.1)
        return out


def _gpu_setup():
    import torch

    import paper_2405_18457_gb300 as gp
    from paper_2405_18457_gb300 import workloads

    assert torch.cuda.is_available(), "bench.py needs a CUDA device (no CPU fallback)"
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    gp.library()
    return torch, gp, workloads, dev


def run_ablation(args):
    """Table 1's design on synthetic data: for each solver (CG, AP, SGD) and each of standard /
    pathwise probes x cold / warm start, `--abl-steps` marginal-likelihood steps solved to
    tau = 0.01 (budgets: 1000 CG iterations, 40 epochs of AP / SGD); reports the solver's time
    and iterations per step and the speed-up over standard-cold (SolverGrid has the workload)."""
    torch, gp, workloads, dev = _gpu_setup()
    grid = SolverGrid(torch, gp, workloads, dev)
    steps = args.abl_steps
    rows = {}
    for solver in ("cg", "ap", "sgd"):
        for pathwise in (False, True):
            for warm in (False, True):
                r = grid.run(solver, pathwise, warm, steps, 1000 if solver == "cg" else 40)
                rows["%s/%s/%s" % (solver, "pathwise" if pathwise else "standard", "warm" if warm else "cold")] = {
                    "solver_sec_per_step": float(np.mean(r["sec"])), "iters": r["iters"],
                    "converged_steps": int(sum(r["converged"]))}
    for solver in ("cg", "ap", "sgd"):
        base = rows["%s/standard/cold" % solver]["solver_sec_per_step"]
        for k, r in rows.items():
            if k.startswith(solver + "/"):
                r["speedup_vs_standard_cold"] = base / r["solver_sec_per_step"]
    out = {"metric": ABL_METRIC, "value": rows["cg/pathwise/warm"]["speedup_vs_standard_cold"],
           "unit": "x speed-up of CG pathwise+warm over standard+cold", "n_gpus": 1, "steps": steps, "warmup": 0,
           "ms_per_step": 1e3 * rows["cg/pathwise/warm"]["solver_sec_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f16-tensor/f32/f64", "data": "synthetic (seeded)",
           "config": {"workload": "ablation: n=%d d=8 Matern-3/2 sigma=0.3 s=%d, tau 0.01, CG <= 1000 iters, AP b=%d "
                                  "and SGD b=%d (lr %s, momentum 0.9) <= 40 epochs, Adam lr 0.1, %d steps"
                                  % (grid.n, grid.s, grid.bs_ap, grid.bs_sgd, grid.lr_sgd, steps)},
           "grid": rows}
    print(json.dumps(out))


DIAG_METRIC = "solver diagnostics: initial RKHS distance, probe-count cost, residual norm under epoch budgets"


def run_diagnostics(args):
    """Sec. 3-5 diagnostics on the GPU path.
    (1) Initial RKHS distance (Eq. RKHS_distance) along a pathwise warm-started optimisation of the
        pathwise workload (n = 32768): per step the mean over the probes' systems of ||u||_H^2 for the
        standard systems (expectation tr(H^-1), Eq. standard_dist), for the pathwise systems (n, Eq.
        pathwise_dist) and ||u_prev - u||_H^2 for the warm start.
    (2) Cost of the probe count (Sec. 3, "How Many Probe Vectors"): seconds per warm pathwise step and
        per solver iteration at s = 16, 32, 64 on the pathwise workload.
    (3) Epoch budgets (Sec. 5, "The Effects of Early Stopping"): true relative residual norms reached
        with 10-50 epochs by CG / AP / SGD, standard-cold against pathwise-warm (SolverGrid's workload)."""
    torch, gp, workloads, dev = _gpu_setup()
    steps = args.abl_steps
    # (1) RKHS distances
    p = workloads.pathwise()
    rep = Replica(gp, torch, p, dev, torch.float32, gp.GP_PREC_TC16, 1000)
    Bstd = torch.cat([rep.y[None], rep.w], 0).contiguous()
    rk = {"std_cold": [], "pathwise_cold": [], "pathwise_warm": [], "n": p.n, "pathwise_iters": []}
    for t in range(steps):
        V_prev = rep.V.clone()
        info, _ = rep.step()  # warm pathwise solve into rep.V, gradient, Adam (advances rep.theta)
        th = rep.last_theta
        rk["pathwise_iters"].append(int(info.iters))
        rk["pathwise_cold"].append(float(gp.gp_rkhs_sqdist(p.kind, th, rep.X, rep.V[1:]).mean()))
        if t > 0:
            rk["pathwise_warm"].append(float(gp.gp_rkhs_sqdist(p.kind, th, rep.X, rep.V[1:], V_prev[1:]).mean()))
        Vs, _ = gp.gp_solve_cg(p.kind, th, rep.X, Bstd, max_iters=1000, tol=0.01, prec=gp.GP_PREC_TC16)
        rk["std_cold"].append(float(gp.gp_rkhs_sqdist(p.kind, th, rep.X, Vs[1:]).mean()))
    # (2) probe count
    probe = {}
    for s in (16, 32, 64):
        ps = workloads.pathwise(s=s)
        r = Replica(gp, torch, ps, dev, torch.float32, gp.GP_PREC_TC16, 1000)
        for _ in range(3):
            r.step()
        secs, its = [], []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info, _ = r.step()
            torch.cuda.synchronize()
            secs.append(time.perf_counter() - t0)
            its.append(int(info.iters))
        probe["s=%d" % s] = {"sec_per_step": float(np.mean(secs)), "cg_iters": its,
                             "sec_per_product": float(np.sum(secs) / (np.sum(its) + 2 * steps))}
    base = probe["s=16"]["sec_per_product"]
    for v in probe.values():
        v["product_cost_vs_s16"] = v["sec_per_product"] / base
    # (3) epoch budgets
    grid = SolverGrid(torch, gp, workloads, dev)
    budget = {}
    for solver in ("cg", "ap", "sgd"):
        for epochs in EPOCH_BUDGETS:
            for pathwise, warm in ((False, False), (True, True)):
                r = grid.run(solver, pathwise, warm, steps, epochs, residuals=True)
                budget["%s/%d/%s" % (solver, epochs, "pathwise-warm" if pathwise else "standard-cold")] = {
                    "res_y_last": r["res_y"][-1] if r["res_y"] else None,
                    "res_z_last": r["res_z"][-1] if r["res_z"] else None,
                    "res_z_mean": float(np.mean(r["res_z"])) if r["res_z"] else None,
                    "iters": r["iters"]}
    out = {"metric": DIAG_METRIC, "value": probe["s=64"]["product_cost_vs_s16"],
           "unit": "x cost per solver product at s=64 vs s=16", "n_gpus": 1, "steps": steps, "warmup": 3,
           "ms_per_step": 1e3 * probe["s=64"]["sec_per_step"], "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f16-tensor/f32/f64", "data": "synthetic (seeded)",
           "config": {"workload": "pathwise n=32768 d=16 Matern-3/2 (RKHS distances, probe counts); "
                                  "n=8192 d=8 Matern-3/2 s=64 (epoch budgets 10-50)"},
           "rkhs_distance": rk, "probe_count": probe, "epoch_budget": budget}
    print(json.dumps(out))


BATCH_METRIC = "batched MLL step time (256 independent uneven RBF GPs, one captured CUDA graph per step)"


def run_batched(args):
    """The batched workload on its own (python bench.py --workload batched): batched_record's line."""
    import torch

    import paper_2405_18457_gb300 as gp
    from paper_2405_18457_gb300 import workloads

    assert torch.cuda.is_available(), "bench.py needs a CUDA device (no CPU fallback)"
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gp.library()
    rates = gp.gp_diag_unit_rates(4096)
    peaks, peak_src = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = batched_record(torch, gp, workloads, dev, rates, peaks, peak_src, sms, peaks.get("sm_max_mhz", 2070.0),
                         steps=args.steps, warmup=args.warmup, kernel_reps=args.kernel_reps, n_gps=args.n_gps,
                         cpu_seconds=args.cpu_seconds, rank=rank, local=local)
    if rank != 0:
        return
    out.update({"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None})
    print(json.dumps(out))


def batched_record(torch, gp, workloads, dev, rates, peaks, peak_src, sms, clk_mhz, steps, warmup, kernel_reps,
                   n_gps, cpu_seconds, rank, local):
    """The batched workload: 256 independent RBF-ARD GPs, n ~ LogUniform[512, 65536],
    d in {4, 8, 16, 32}, X ~ U[0,1]^d, y = RFF prior draw + N(0, 0.1^2), s = 16 standard
    probes (R = 17); per step: operands from theta, warm-started CG with a budget of 50
    iterations (tolerance 0.01 on the true residual, per-member early stop), standard estimator,
    Adam (lr 0.1), all captured once into a CUDA graph and replayed.  Reports p50/p99 step time."""
    s, iters, tol, lr = 16, 50, 0.01, 0.1
    ns, ds = workloads.batched_sizes(n_gps=n_gps, seed=rank)
    mem = [workloads.batched_member(int(n), int(d), s=s, m=1024, seed=rank, index=g)
           for g, (n, d) in enumerate(zip(ns, ds))]
    b = gp.GPBatch(gp.GP_RBF, ns, ds, s, device=dev)
    Bs = []
    for p in mem:
        Xg = torch.tensor(p.X, dtype=torch.float32, device=dev)
        tf = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
        F = gp.gp_rff_prior_sample(p.kind, p.theta, Xg, tf(p.omega_hat), None, tf(p.W_y))
        # y = f(X) + 0.1 w  (the second block of [y', F + sigma w] with sigma = 0.1)
        y = gp.gp_pathwise_rhs(p.theta, p.d, torch.zeros(p.n, device=dev), F, tf(p.y_noise[None]))[1]
        Bs.append(torch.cat([y[None], tf(p.Z)], 0).cpu().numpy())
    X = b.pack_points([p.X for p in mem])
    B = b.pack_vectors(Bs)
    theta = b.pack_theta([p.theta for p in mem])
    V = torch.zeros_like(B)
    grad = torch.empty_like(theta)
    st = b.adam_init(theta)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    # one eager step (attributes, tensor maps), then capture the step once
    b.step(X, theta, B, V, iters, tol, st, lr, grad)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.step(X, theta, B, V, iters, tol, st, lr, grad)
    torch.cuda.synchronize()
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize()
    b.status()
    nsq = np.asarray(ns, dtype=np.float64) ** 2
    R = s + 1
    clocks = Clocks(local)
    clocks.start()
    times, work, its = [], 0.0, []
    for _ in range(steps):
        flush_l2(torch, flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        info = b.info()  # outside the timed region
        it = np.array([r["iters"] for r in info], dtype=np.float64)
        its.append(float(it.mean()))
        work += float(((it + 2.0) * nsq).sum()) * R  # CG products (+1 initial residual) + gradient pass
    clk = clocks.stop()
    b.status()
    total_s = sum(times) / 1e3
    # dominant kernel: the grouped product (one launch per contraction class), events per launch
    gp.gp_diag_reset(True)
    for _ in range(kernel_reps):
        flush_l2(torch, flush)
        b.mvm(V, add_noise=True)
    torch.cuda.synchronize()
    prod_ms, prod_cnt = gp.gp_diag_kernel_time(0)
    gp.gp_diag_reset(False)
    prod_s = prod_ms / 1e3 / kernel_reps  # all classes of one batched product
    pairs = float(nsq.sum())
    # roofline of one batched product (all classes): per pair the algorithmic contraction
    # 2 d_g + 2 R flops (tensor, measured bf16 rate) and one ex2 (MUFU, measured rate), summed
    # over the members; the kernel's padded contraction (KD, R_pad = 32) is reported beside it
    tpeak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * 1e12
    dd = np.asarray(ds, dtype=np.float64)
    t_tensor = float((nsq * (2.0 * dd + 2.0 * R)).sum()) / tpeak
    t_mufu = pairs / (sms * rates["ex2"] * clk_mhz * 1e6)
    bound_s = max(t_tensor, t_mufu)
    kd = np.array([kd_of(int(x)) for x in ds], dtype=np.float64)
    padded = float((nsq * (2.0 * kd + 2.0 * 32)).sum()) / float((nsq * (2.0 * dd + 2.0 * R)).sum())
    achieved = pairs / prod_s / 1e9
    roof = {"bound": "tensor" if t_tensor >= t_mufu else "alu", "unit": "Gpair/s", "achieved": achieved,
            "peak": pairs / bound_s / 1e9, "frac": bound_s / prod_s, "traffic": None,
            "peak_derivation": "max over pipes of sum over members of n^2 x (tensor: (2 d + 2 R) flops / %.0f TFLOP/s; "
                               "MUFU: 1 ex2 / (%d SMs x %.1f ex2/clk x %.0f MHz))"
                               % (tpeak / 1e12, sms, rates["ex2"], clk_mhz),
            "padded_over_algorithmic_tensor_flops": padded,
            "peak_source": "%s (unit rates measured live)" % peak_src, "kernel": "tc_mvm_kernel (grouped H V, all classes)",
            "avg_launch_ms": prod_s * 1e3, "launches_timed": prod_cnt, "pairs_per_launch": pairs}
    # end to end: points and right-hand sides from pinned host memory every step, theta read back
    Xh = X.cpu().pin_memory()
    Bh = B.cpu().pin_memory()
    th_h = torch.empty(theta.numel(), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        X.copy_(Xh, non_blocking=True)
        B.copy_(Bh, non_blocking=True)
        graph.replay()
        th_h.copy_(theta, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e_s = e0.elapsed_time(e1) / 1e3
    cpu = None
    if rank == 0:
        big = int(np.argmax(ns))
        p = mem[big]
        Vh = np.random.default_rng(0).standard_normal((R, p.n))
        rows = np.arange(8)
        t0 = time.perf_counter()
        import oracle

        oracle.kernel_mvm(p.kind, p.theta, p.X, p.X, Vh, add_noise=True, rows=rows)
        t8 = time.perf_counter() - t0
        k = int(max(8, min(p.n, 8 * cpu_seconds / max(t8, 1e-6))))
        rows = np.random.default_rng(1).choice(p.n, size=k, replace=False)
        t0 = time.perf_counter()
        oracle.kernel_mvm(p.kind, p.theta, p.X, p.X, Vh, add_noise=True, rows=rows)
        dt = time.perf_counter() - t0
        cpu = {"value": k * p.n * R / dt / 1e9, "unit": "Gpair*RHS/s",
               "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), "kind": "oracle",
               "sample": "%d sampled rows of H V of the largest member (n=%d, d=%d, R=%d), FP64, %.1f s"
                         % (k, p.n, p.d, R, dt)}
    ts = np.array(times)
    out = {
        "metric": BATCH_METRIC, "value": float(np.percentile(ts, 50)), "unit": "ms per step (p50)",
        "steps": steps, "ms_per_step": float(ts.mean()), "dtype": "f16-tensor/f32/f64",
        "data": "synthetic (seeded)",
        "config": {"workload": "batched: %d RBF GPs, n~LogUniform[512,65536] (sum n=%d), d in {4,8,16,32}, s=%d, "
                               "CG budget %d tol %.2g warm, standard estimator, Adam lr %.2g"
                               % (len(ns), int(np.sum(ns)), s, iters, tol, lr),
                   "l2": "flushed between timed steps", "parallelism": "single GPU"},
        "p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
        "gpair_rhs_per_s": work / total_s / 1e9, "mean_cg_iters_per_member": its,
        "e2e": {"value": 1e3 * e_s / steps, "unit": "ms per step (mean)",
                "h2d_bytes_per_step": int(Xh.numel() * 4 + Bh.numel() * 4), "d2h_bytes_per_step": int(th_h.numel() * 8)},
        "roofline": roof, "cpu_baseline": cpu, "clocks": clk, "fp64_form": None,
    }
    return out


def cpu_baseline(prob, R, budget_s=15.0, rows_per_step=None):
    """The FP64 CPU oracle (as it stands) on a bounded sample of the same product:
    sampled rows of H V over all n columns and R right-hand sides."""
    import oracle

    X = prob.X
    V = np.random.default_rng(0).standard_normal((R, prob.n))
    rows = np.arange(128)
    oracle.kernel_mvm(prob.kind, prob.theta, X, X, V, add_noise=True, rows=rows[:8])  # thread start-up
    t0 = time.perf_counter()
    oracle.kernel_mvm(prob.kind, prob.theta, X, X, V, add_noise=True, rows=rows)
    t128 = time.perf_counter() - t0
    k = rows_per_step or int(max(128, min(prob.n, 128 * budget_s / max(t128, 1e-6))))
    rows = np.random.default_rng(1).choice(prob.n, size=k, replace=False)
    t0 = time.perf_counter()
    oracle.kernel_mvm(prob.kind, prob.theta, X, X, V, add_noise=True, rows=rows)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": k * prob.n * R / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d sampled rows of H V (n=%d, R=%d), FP64, %.1f s" % (k, prob.n, R, dt)}


def run_reference(args):
    """The oracle timed on the host cores, one bounded sample of the product per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2405_18457_gb300 import workloads

    import oracle

    prob = workloads.pathwise(n=args.n, seed=0)
    R = prob.s + 1
    X = prob.X
    V = np.random.default_rng(0).standard_normal((R, prob.n))
    rows_per_step = args.ref_rows
    for _ in range(args.warmup):
        oracle.kernel_mvm(prob.kind, prob.theta, X, X, V, add_noise=True, rows=np.arange(rows_per_step))
    t0 = time.perf_counter()
    for k in range(args.steps):
        rows = np.random.default_rng(k).choice(prob.n, size=rows_per_step, replace=False)
        oracle.kernel_mvm(prob.kind, prob.theta, X, X, V, add_noise=True, rows=rows)
    dt = time.perf_counter() - t0
    value = args.steps * rows_per_step * prob.n * R / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "pathwise workload product H V: %d sampled rows x n=%d x R=%d per step"
                                  % (rows_per_step, prob.n, R), "n": prob.n, "d": prob.d, "rhs": R},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "%d rows per step" % rows_per_step},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_op(args):
    """Single hot-path operations on the pathwise workload's shape (d = 16, Matern-3/2, 65
    right-hand sides, seeded synthetic inputs), `repeat` calls, for profilers (a capture of one
    kernel on a case that ends in seconds): mvm (gp_kernel_mvm, H V), grad (gp_mll_grad_pathwise),
    rff (gp_rff_prior_sample), cg (gp_solve_cg, 10 iterations), unit-rates (gp_diag_unit_rates);
    panel: the alternating-projections column panel's shape (K(X, X_block) V, n = 262144, d = 26,
    RBF, a block of 1024 points, 65 vectors).
    Prints the mean time per call (CUDA events).  --autotune tunes the shape first; with
    GP_AUTOTUNE_CACHE set the choice is saved, and a later run (under a profiler) reads it."""
    import torch

    import paper_2405_18457_gb300 as gp
    from paper_2405_18457_gb300 import workloads

    assert torch.cuda.is_available(), "bench.py needs a CUDA device (no CPU fallback)"
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    gp.library()
    if args.op == "unit-rates":
        rates = gp.gp_diag_unit_rates(4096)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peaks, _ = _peaks()
        clk = peaks.get("sm_max_mhz", 2070.0)
        print(json.dumps({"unit_rates_per_sm_per_clk": rates, "sms": sms, "sm_max_mhz": clk,
                          "mufu_bound_gpairs_per_s": {
                              "matern32 (rsqrt + ex2)": sms * clk * 1e6 / (1 / rates["ex2"] + 1 / rates["rsqrt"]) / 1e9,
                              "rbf (ex2)": sms * clk * 1e6 * rates["ex2"] / 1e9},
                          "ffma_tflops": sms * rates["ffma"] * 2 * clk * 1e6 / 1e12,
                          "dfma_tflops": sms * rates["dfma"] * 2 * clk * 1e6 / 1e12}))
        return
    prec = {"tc16": gp.GP_PREC_TC16, "fp32": gp.GP_PREC_FP32, "tc16x3": gp.GP_PREC_TC16X3}[args.prec]
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    if args.op == "panel":
        # the alternating-projections column panel's shape: all n = 262144 points (d = 26, RBF)
        # against one block of 1024 points, 65 vectors
        p = workloads.ap()
        X = t(p.X)
        Xb = X[:1024].contiguous()
        V = t(workloads.vectors(p.s + 1, 1024, seed=1))
    else:
        p = workloads.pathwise(n=args.n, d=16, s=64, m=2048, seed=0)
        X = t(p.X)
        V = t(workloads.vectors(p.s + 1, p.n, seed=1))
        om, c2, Wp = t(p.omega_hat), t(p.chi2), t(p.W_probe)

    def call():
        if args.op == "panel":
            gp.gp_kernel_mvm(p.kind, p.theta, X, V, X2=Xb, prec=prec)
        elif args.op == "mvm":
            gp.gp_kernel_mvm(p.kind, p.theta, X, V, add_noise=True, prec=prec)
        elif args.op == "grad":
            gp.gp_mll_grad_pathwise(p.kind, p.theta, X, V, prec=prec)
        elif args.op == "rff":
            gp.gp_rff_prior_sample(p.kind, p.theta, X, om, c2, Wp, prec=prec)
        else:
            gp.gp_solve_cg(p.kind, p.theta, X, V, max_iters=10, tol=0.0, prec=prec)

    if args.autotune:
        # record this shape's tuned choices (written to GP_AUTOTUNE_CACHE when set, so that a later
        # process -- a profiler run -- uses them without tuning)
        if args.op in ("mvm", "cg"):
            gp.gp_autotune_mvm(p.kind, p.theta, X, V, reps=3)
        if args.op == "grad":
            gp.gp_autotune_grad(p.kind, p.theta, X, V, None, reps=3)
    call()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.repeat):
        call()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"op": args.op, "n": p.n, "repeat": args.repeat,
                      "ms_per_call": e0.elapsed_time(e1) / args.repeat}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["tc16", "fp32", "tc16x3"], default="tc16",
                    help="tc16x3 (the split tensor-core product) for --op mvm only")
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--max-iters", type=int, default=1000)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--sub-cpu-seconds", type=float, default=3.0)
    ap.add_argument("--batched-steps", type=int, default=3)
    ap.add_argument("--no-subrecords", action="store_true")
    ap.add_argument("--ref-rows", type=int, default=256)
    ap.add_argument("--kernel-reps", type=int, default=10)
    ap.add_argument("--workload", choices=["pathwise", "batched", "small", "ablation", "diagnostics", "ap", "sgd"],
                    default="pathwise")
    ap.add_argument("--solver-iters", type=int, default=0, help="--workload ap|sgd: iteration budget override")
    ap.add_argument("--op", choices=["mvm", "panel", "grad", "rff", "cg", "unit-rates"], default=None)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--autotune", action="store_true", help="--op: tune the operation's shape first")
    ap.add_argument("--abl-steps", type=int, default=10)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--n-gps", type=int, default=256)
    args = ap.parse_args()
    if args.op is not None:
        if args.op != "unit-rates" and args.n == 32768 and "--n" not in sys.argv:
            args.n = 16384
        run_op(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.prec == "tc16x3":
        raise SystemExit("--prec tc16x3 applies to --op mvm only")
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "small":
        run_small(args)
        return
    if args.workload == "ablation":
        run_ablation(args)
        return
    if args.workload == "diagnostics":
        run_diagnostics(args)
        return
    if args.workload in ("ap", "sgd"):
        run_solver_workload(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
