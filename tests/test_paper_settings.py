"""The workloads follow the experimental settings the paper prints (tests/golden/
paper_settings.json, each value with its passage) wherever the paper fixes them."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2405_18457_gb300 import workloads  # noqa: E402

with open(os.path.join(ROOT, "tests", "golden", "paper_settings.json")) as f:
    PAPER = {k: v for k, v in json.load(f).items() if not k.startswith("_")}


def val(key):
    return PAPER[key]["value"]


def test_every_setting_cites_a_passage():
    for key, entry in PAPER.items():
        assert "value" in entry and entry["cite"], key


def test_tolerance_workloads_solve_to_the_papers_tau():
    # the small workload solves to 1e-6 by its own specification (exact-gradient comparisons)
    probs = [workloads.pathwise(n=256, s=8, m=64), workloads.ap(n=256, s=8, m=64),
             workloads.sgd(n=256, s=8, m=64), workloads.batched_member(256, 4, m=64)]
    for p in probs:
        assert p.extra["tol"] == val("tolerance_tau"), p.name


def test_learning_rates_follow_the_dataset_size_rule():
    # n < 50k: 0.1; n > 50k: 0.03 (the default sizes of the workloads)
    assert workloads.pathwise(n=256, s=8, m=64).extra["lr"] == val("adam_lr_small")
    assert workloads.small(n=256).extra["lr"] == val("adam_lr_small")
    assert workloads.ap(n=256, s=8, m=64).extra["lr"] == val("adam_lr_large")
    assert workloads.sgd(n=256, s=8, m=64).extra["lr"] == val("adam_lr_large")


def test_probe_counts_budgets_and_initial_scales():
    import inspect

    for fn in (workloads.pathwise, workloads.ap, workloads.sgd):
        assert inspect.signature(fn).parameters["s"].default == val("probes_main"), fn.__name__
    assert workloads.ap(n=256, s=8, m=64).extra["epochs"] == val("budget_epochs_large")
    assert list(bench.EPOCH_BUDGETS) == val("budget_epochs_sweep")
    p = workloads.pathwise(n=256, d=4, s=8, m=64)
    init = val("init_hyperparameters_small")
    assert np.all(p.theta[:4] == init) and p.theta[4] == init  # length scales and signal scale


def test_random_features_come_in_sin_cos_pairs():
    # m features = m / 2 frequencies, each with a cosine and a sine (2000 features = 1000 pairs)
    assert val("rff_features") == 2 * PAPER["rff_features"]["pairs"]
    for m in (64, 2048):
        p = workloads.pathwise(n=256, d=4, s=8, m=m)
        assert p.omega_hat.shape == (m // 2, 4)
        assert p.W_probe.shape == (8, m) and p.W_y.shape[-1] == m
