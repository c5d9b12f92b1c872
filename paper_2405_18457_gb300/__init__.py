"""GB300 (sm_103a) iterative-GP hot path: Python binding of libgp_gb300.so.

Every function here only marshals arguments (torch CUDA tensors -> raw device
pointers, the current CUDA stream, caller-owned workspace) into the C ABI of
``include/gp.h``; all arithmetic runs in the library's CUDA kernels.  There is
no CPU fallback: if the library cannot be loaded or no CUDA device is present
the call raises.

Layouts follow the C ABI: points X are (n, d) float32/float64 row-major, blocks
of vectors are (R, n) with one right-hand side per row, theta is a sequence of
d+2 floats [l_1..l_d, s_f, sigma].
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    GP_MATERN32,
    GP_PREC_FP32,
    GP_PREC_TC16,
    GP_PREC_TC16X3,
    GP_RBF,
    GP_STOP_BOTH,
    GP_STOP_EITHER,
    GPError,
    SolveInfo,
    gp_adam_softplus_step,
    gp_autotune_count,
    gp_autotune_grad,
    gp_autotune_load,
    gp_autotune_mvm,
    gp_autotune_reset,
    gp_autotune_save,
    gp_bilinear_grad,
    gp_diag_kernel_time,
    gp_diag_launches,
    gp_diag_product_time,
    gp_diag_reset,
    gp_kernel_mvm,
    gp_mll_grad_pathwise,
    gp_mll_grad_standard,
    gp_pathwise_rhs,
    gp_posterior_samples,
    gp_predict,
    gp_device_check,
    gp_diag_timeout_probe,
    gp_diag_unit_rates,
    gp_rkhs_sqdist,
    gp_rff_prior_sample,
    gp_solve_ap,
    gp_solve_cg,
    gp_solve_sgd,
    library,
    library_path,
)
from .autograd import bilinear_form, kernel_matvec  # noqa: F401,E402
from .batched import GPBatch  # noqa: F401,E402
