"""Host-side logic of bench.py that needs no GPU: the optimiser-state snapshot that lets the
end-to-end loop replay the timed steps, and the clock-record summary."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_snapshot_restore_replays_the_same_state():
    r = bench.Replica.__new__(bench.Replica)
    r.theta = np.array([0.7, 1.3, 0.2])
    r.nu = np.log(np.expm1(r.theta))
    r.m = np.array([0.1, -0.2, 0.3])
    r.v = np.array([0.01, 0.02, 0.03])
    r.t = 4
    r.V = torch.arange(6, dtype=torch.float32).reshape(2, 3)
    snap = r.snapshot()
    want = (r.theta.copy(), r.nu.copy(), r.m.copy(), r.v.copy(), r.t, r.V.clone())
    for _ in range(2):
        # a few optimiser steps change every part of the state in place
        r.theta += 1.0
        r.nu *= 2.0
        r.m[:] = 5.0
        r.v[:] = 6.0
        r.t += 3
        r.V.add_(1.0)
        r.restore(snap)
        assert np.array_equal(r.theta, want[0]) and np.array_equal(r.nu, want[1])
        assert np.array_equal(r.m, want[2]) and np.array_equal(r.v, want[3]) and r.t == want[4]
        assert torch.equal(r.V, want[5])
    # the snapshot is not aliased by the restored state
    r.theta[0] = -1.0
    r.restore(snap)
    assert r.theta[0] == want[0][0]


def test_clock_summary_drops_the_pre_region_row_and_flags_reasons(tmp_path):
    rows = ["0, 1980, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 940.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.Clocks(0)
    c.proc, c.path = Done(), str(path)
    out = c.stop()
    assert out["samples"] == 3  # the first row was taken before the region
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
