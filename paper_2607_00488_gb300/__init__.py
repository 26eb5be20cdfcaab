"""srw: spectrum-reweighting likelihood for solar nu-e scattering on GB300.

The computation runs in the in-tree CUDA library ``libsrw.so`` (C ABI in
``include/srw.h``); ``srw`` is its ctypes binding.  Build the library with
``paper_2607_00488_gb300.build.build()``.
"""

from .srw import (  # noqa: F401
    EXPORTS,
    LIB_PATH,
    PRECISIONS,
    SRW_BF16,
    SRW_BF16X3,
    SRW_DEVICE,
    SRW_EDOMAIN,
    SRW_FP16X3,
    SRW_FP32,
    SRW_HOST,
    SRW_SCAN_ERROR_BARS,
    SRW_SCAN_FLAG_CELLS,
    GroupedLikelihood,
    Likelihood,
    SrwError,
    Surrogate,
    lib,
    srw_autotune,
    srw_create,
    srw_destroy,
    srw_get_basis,
    srw_group_autotune,
    srw_group_create,
    srw_group_destroy,
    srw_group_loglik,
    srw_group_profile,
    srw_group_profile_read,
    srw_group_schedule,
    srw_group_set_schedule,
    srw_info,
    srw_last_error,
    srw_loglik,
    srw_loglik_point_noalloc,
    srw_loglik_points,
    srw_profile,
    srw_set_reference,
    srw_profile_read,
    srw_set_data,
    srw_spectrum,
    srw_spectrum_batch,
)
