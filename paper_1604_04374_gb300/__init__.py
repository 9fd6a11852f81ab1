"""GB300-native convolution-product expansion (Escande & Weiss, arXiv:1604.04374).

H_m u = sum_k h_k * (w_k . u) (Eq. 1.4) and its adjoint on periodic 1D/2D
grids, computed by the CUDA library libpce.so (hand-written sm_103a kernels)
behind the C ABI of include/pce.h.  This package is the thin Python binding:
``pce`` mirrors the C entry points one to one, ``Plan`` marshals torch CUDA
tensors into them.  There is no CPU fallback: without the built library or a
CUDA device every call raises.
"""
from .pce import (Batch, PceError, Plan, apply_batch, construct_projection_1d, construct_projection_2d, pce_construct_projection_1d, pce_construct_projection_2d, pce_construct_projection_bspline_1d, construct_svd_1d, pce_construct_svd_1d, pce_apply_batch, pce_batch_create, pce_batch_destroy,
                  pce_batch_info, pce_batch_launch, pce_batch_run, pce_plan_autotune, pce_plan_tuning,
                  pce_schedule_lpt, pce_apply, pce_apply_adjoint, pce_apply_noalloc, pce_backward,
                  pce_backward_workspace_bytes, pce_last_error_string,
                  pce_launch_count, pce_plan_create, pce_plan_create_from_spectra,
                  pce_plan_destroy, pce_plan_hhat, pce_plan_info, pce_plan_set_timing,
                  pce_plan_timing, load_library)

__all__ = ["Batch", "apply_batch", "construct_projection_1d", "construct_projection_2d", "pce_construct_projection_1d", "pce_construct_projection_2d", "pce_construct_projection_bspline_1d", "construct_svd_1d", "pce_construct_svd_1d", "pce_apply_batch", "pce_batch_create", "pce_batch_destroy",
           "pce_batch_info", "pce_batch_launch", "pce_batch_run", "pce_plan_autotune", "pce_plan_tuning",
           "pce_schedule_lpt", "PceError", "Plan", "pce_apply", "pce_apply_adjoint", "pce_apply_noalloc", "pce_backward",
           "pce_backward_workspace_bytes", "ConvolutionProduct", "convolution_product", "pce_last_error_string",
           "pce_launch_count", "pce_plan_create", "pce_plan_create_from_spectra",
           "pce_plan_destroy", "pce_plan_hhat", "pce_plan_info", "pce_plan_set_timing",
           "pce_plan_timing", "load_library"]
from .autograd import ConvolutionProduct, convolution_product  # noqa: E402
