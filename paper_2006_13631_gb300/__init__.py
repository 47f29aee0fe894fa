"""GB300 moving-grid hybrid lattice Boltzmann solver (CUDA, sm_103a).

The solver lives in the C-ABI library built from ``csrc/`` (declared in
``include/hlbm.h``); this package only binds it.  Nothing here computes the
method on the CPU: without the compiled library every entry point raises.
"""
from .hlbm import (HLBMError, Solver, Sweep, hlbm_clear_status, hlbm_create, hlbm_destroy, hlbm_fit_static, hlbm_force, hlbm_gamma, hlbm_get_class, hlbm_get_level_fields,
                   hlbm_get_fields, hlbm_get_fv, hlbm_get_patch_f, hlbm_get_refill, hlbm_info, hlbm_inject_fault,
                   hlbm_profile, hlbm_profile_read, hlbm_set_fv_depth, hlbm_set_overlap, hlbm_set_overlap_share, hlbm_load, hlbm_save, hlbm_status, hlbm_step, hlbm_theta_adjoint, hlbm_theta_gradient, theta_function,
                   use_torch_allocator, workload_inputs)
from . import _native

__all__ = ["HLBMError", "Solver", "Sweep", "hlbm_clear_status", "hlbm_create", "hlbm_destroy", "hlbm_fit_static", "hlbm_force", "hlbm_gamma", "hlbm_get_class", "hlbm_get_level_fields",
           "hlbm_get_fields", "hlbm_get_fv", "hlbm_get_patch_f", "hlbm_get_refill", "hlbm_info", "hlbm_inject_fault", "hlbm_profile", "hlbm_set_fv_depth", "hlbm_set_overlap", "hlbm_set_overlap_share",
           "hlbm_profile_read", "hlbm_load", "hlbm_save", "hlbm_status",
           "hlbm_step", "hlbm_theta_adjoint", "hlbm_theta_gradient", "theta_function", "use_torch_allocator", "workload_inputs",
           "_native"]
