"""Lanczos full-frequency GW hot path on GB300 (sm_103a).

The compute path is the C-ABI library ``liblgw.so`` (CUDA kernels); the
Python side (:mod:`.lgw`) only marshals arguments to it.
"""
from .lgw import (Handle, LgwError, Options, Problem, System, load_library,  # noqa: F401
                  lgw_apply_casida, lgw_create, lgw_destroy, lgw_last_error,
                  lgw_lanczos_coeffs, lgw_prepare_system, lgw_release_system, lgw_sigma_c,
                  lgw_sigma_c_backward, lgw_sigma_c_batched, lgw_sigma_from_coeffs,
                  lgw_status_string)
