"""GB300-native fast CP gradients and CP_ALS (Phan, Tichavsky, Cichocki).

The computation lives in ``libcpgrad.so`` (CUDA, sm_103a) behind the C ABI
of ``include/cpgrad.h``; ``cpgrad`` is its argument-marshalling binding.
"""
from .cpgrad import (  # noqa: F401
    cpg_split_point, cpg_workspace_size, cp_gradient_all, cp_gradient_mode, cp_als_iter, cp_als_batched,
    cpg_device_status, cp_gradient_autotune, gradient_plan, autotune_clear, cp_gradient_full, cp_gradient_step,
    cp_ntf_iter, selftest_timeout, als_candidates, cp_als_autotune, als_plan, set_gradient_plan, set_als_plan,
    colmajor, launch_count, profile_lead, profile_read, Workspace, CpgError, PRECISIONS, LAUNCH_KINDS, lib,
    CPG_OK, CPG_ERR_ARG, CPG_ERR_WORKSPACE, CPG_ERR_UNSUPPORTED, CPG_ERR_TIMEOUT,
)
