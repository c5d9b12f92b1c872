"""The bounded-wait path of the tensor-core kernels, exercised without a GPU fault: a kernel
waits on a barrier that nothing completes, gives up after about a millisecond, and sets the
device status word; the host reads GP_ERR_TIMEOUT once, the word is cleared, and the context
keeps working (a product afterwards still matches the oracle)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_18457_gb300 import workloads

pytestmark = pytest.mark.gpu

import paper_2405_18457_gb300 as gp  # noqa: E402  (a missing package fails the run)


def test_timed_out_wait_is_reported_once_and_context_survives():
    assert torch.cuda.is_available()
    dev = torch.device("cuda:0")
    gp.library()
    gp.gp_device_check()  # clean start
    gp.gp_diag_timeout_probe(2_000_000)  # about 1 ms at 2 GHz
    with pytest.raises(gp.GPError) as e:
        gp.gp_device_check()
    assert e.value.status == -5
    gp.gp_device_check()  # cleared
    p = workloads.pathwise(n=700, d=5, s=4, m=64, seed=9)
    X32 = p.X.astype(np.float32)
    V = workloads.vectors(5, 700, seed=10).astype(np.float32)
    Y = gp.gp_kernel_mvm(p.kind, p.theta, torch.tensor(X32, device=dev), torch.tensor(V, device=dev),
                         add_noise=True, prec=gp.GP_PREC_TC16).cpu().numpy()
    Xr = X32.astype(np.float64)
    ref = oracle.kernel_mvm(p.kind, p.theta, Xr, Xr, V.astype(np.float64), add_noise=True)
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) < 1e-3
    gp.gp_device_check()


def test_probe_rejects_out_of_range_limit():
    with pytest.raises(gp.GPError):
        gp.gp_diag_timeout_probe(-1)
