"""GB300 (sm_103a) implementation of accelerated filtered back projection: recursive (IIR)
ramp filtering and fast-Hough-transform back projection (arXiv 2007.06289).

The compute path is ``libfbp.so`` (CUDA kernels behind the C ABI of include/fbp.h);
``binding`` exposes its entry points to Python with the same names.  ``build`` compiles
the library in-tree.  ``iir_fit`` fits the recursive-filter coefficients (host prep).
``autograd`` wraps the reconstruction and its adjoint as a differentiable torch operation
(import it explicitly; it needs torch).
"""
from .binding import (FbpError, Plan, fbp_default_coeffs, fbp_direct_reconstruct,  # noqa: F401
                      fbp_fht_backproject, fbp_filter_iir, fbp_last_device_error, fbp_plan,
                      fbp_plan_destroy, fbp_plan_info, fbp_profile_enable,
                      fbp_profile_read, fbp_profile_reset, fbp_reconstruct, fbp_reconstruct_host,
                      fbp_resample_st, fbp_set_workspace, fbp_status_str, fbp_workspace_bytes,
                      fbp_set_chunk, fbp_fht_backproject_adjoint, fbp_resample_st_adjoint,
                      fbp_reconstruct_adjoint, Volume, fbp_volume_create, load_library)
