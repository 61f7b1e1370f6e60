"""GB300-native steered response power maps: conventional FD-SRP, SLRI-SRP and SSPI-SRP
(Dietzen, De Sena, van Waterschoot, "Scalable-Complexity Steered Response Power Based on
Low-Rank and Sparse Interpolation"), with SI-SRP and conv. TD-SRP, and a serving runtime.

The computation lives in ``libsrp.so`` (CUDA for sm_103a, C-ABI in include/libsrp.h);
this package is its Python binding.
"""
from ._abi import (  # noqa: F401
    Plan, Server, SrpError, srp_plan_create, srp_plan_info, srp_plan_lags, srp_map,
    srp_map_host, srp_gcc_samples, srp_plan_sspi_taps, srp_plan_slri_sigma,
    srp_plan_set_profiling, srp_plan_stage_ms, srp_plan_status, srp_slri_apply_static,
    srp_plan_estimate_bytes, srp_server_now, srp_destroy, srp_last_error, srp_debug_fail_allocations,
    srp_plan_save, srp_plan_create_from_file,
    make_desc, lib, SIGNATURES, LIB_PATH,
    SRP_OK, SRP_EINVAL, SRP_ENOMEM, SRP_ECUDA, SRP_ETIMEOUT, SRP_EUNSUPPORTED, SRP_EAGAIN,
    SRP_CONV, SRP_SLRI, SRP_SSPI, SRP_SI, SRP_TD, SRP_LR, SRP_FP32, SRP_BF16, SRP_FP16, SRP_FP16X3,
    SRP_BF16X3, SRP_TF32X3, SRP_TF32, PRECISIONS,
)
