"""GB300-native (sm_103a) pseudo-potential MRT lattice Boltzmann method with
the kappa-scaled pressure-tensor surface-tension adjustment of Hu, Li &
Uddin (arXiv:1412.7228).

The compute path is liblbm.so (include/lbm.h); ``lbm`` is its ctypes binding.
"""
from .lbm import (Batch, Eos, Lattice, LbmError, LBM_EOS_CS, LBM_EOS_PR, LBM_EOS_VDW, LBM_FP32, LBM_FP64,
                  LBM_FLAG_LI_EPS, LBM_FLAG_TEST_FORCE_TIMEOUT, lbm_eos_critical, lbm_eos_maxwell,
                  lbm_eos_pressure, lbm_fp64_math_check, lbm_laplace_fit, lbm_required_bytes,
                  lbm_batch_required_bytes, lbm_run_chunk_plan, lbm_tile_configs, lib)

__all__ = ["Batch", "Eos", "Lattice", "LbmError", "LBM_EOS_CS", "LBM_EOS_PR", "LBM_EOS_VDW", "LBM_FP32",
           "LBM_FP64", "LBM_FLAG_LI_EPS", "LBM_FLAG_TEST_FORCE_TIMEOUT", "lbm_eos_critical", "lbm_eos_maxwell",
           "lbm_eos_pressure", "lbm_fp64_math_check", "lbm_laplace_fit", "lbm_required_bytes",
           "lbm_batch_required_bytes", "lbm_run_chunk_plan", "lbm_tile_configs", "lib"]
