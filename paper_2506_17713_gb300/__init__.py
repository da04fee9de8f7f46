"""GB300-native Shan-Chen multiphase lattice Boltzmann step (arXiv 2506.17713).

The lattice update runs in hand-written CUDA kernels for sm_103a, behind the C
ABI of ``include/lbm.h`` (``liblbm.so``); ``lbm`` is its ctypes binding.
"""
from .build import build as build_library
from .lbm import (EXPORTS, Batch, Lattice, LbmError, lbm_create, lbm_destroy, lbm_diagnostics,
                  lbm_get_populations, lbm_init_fields, lbm_kernel_launches, lbm_macroscopic,
                  lbm_params, lbm_profile_step, lbm_stream_probe, lbm_set_geometry, lbm_set_populations, lbm_status_str, lbm_step,
                  lbm_sync, lbm_temperature, lbm_velocity_set, lbm_workspace_size, library,
                  params_from_case)

__all__ = ["build_library", "EXPORTS", "Batch", "Lattice", "LbmError", "lbm_create", "lbm_destroy",
           "lbm_diagnostics", "lbm_get_populations", "lbm_init_fields", "lbm_kernel_launches",
           "lbm_macroscopic", "lbm_params", "lbm_profile_step", "lbm_stream_probe", "lbm_set_geometry", "lbm_set_populations",
           "lbm_status_str", "lbm_step", "lbm_sync", "lbm_temperature", "lbm_velocity_set",
           "lbm_workspace_size", "library", "params_from_case"]
