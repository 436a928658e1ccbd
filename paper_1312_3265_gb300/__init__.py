"""GB300 (sm_103a) staggered Wilson / Wilson CGNE library.

Thin Python binding over the C ABI in include/sw_cgne.h: it only marshals
arguments (torch tensors -> device pointers, the current CUDA stream) and
turns error codes into exceptions.  Every step of the computation runs in the
library's CUDA kernels; there is no other implementation behind these names.

Field layouts (complex128, canonical, site index n = x0 + L0*(x1 + L1*(x2 + L2*x3))):
  U (V,4,3,3)   W (V,8,3,3)   staggered vectors (V,3)   Wilson spinors (V,4,3)
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    SWError, SolveInfo, Server, lib, lib_path,
    SW_OK, SW_NOT_CONVERGED, SW_OP_STAGGERED_WILSON, SW_OP_WILSON, SW_OP_WILSON_EVEN_ODD,
    SW_PREC_F64, SW_PREC_F32_RELIABLE, SW_PREC_F16_RELIABLE,
    sw_hypercube_build, sw_dslash_apply, wilson_dslash_apply, dslash_apply_inner, cgne_solve, cgne_solve_batch,
    sw_status_string, sw_last_cuda_error, sw_profile_enable, sw_profile_reset, sw_profile_read,
    sw_kernel_launches, sw_measure_fp64_peak, sw_workspace_reserved, sw_trim_workspace, cgne_solve_noalloc, sw_set_param, sw_get_param,
    sw_autotune, sw_autotune_layout, SW_PARAM_CHUNK, SW_PARAM_RELIABLE_DELTA, SW_PARAM_NS_SW, SW_PARAM_NS_WILSON, SW_PARAM_GRAPHS,
    SW_PARAM_SITE_BLOCKING, SW_PARAM_GROUP_FAST,
    SW_PARAM_RELIABLE_DELTA_F16, SW_PARAM_PERSISTENT, SW_PARAM_WILSON_LEAN, SW_SITE_SHAPES,
)
