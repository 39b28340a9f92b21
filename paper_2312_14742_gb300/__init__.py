"""GB300-native Tau1 lattice Boltzmann solver (arXiv 2312.14742, hot path).

The solver is the CUDA library liblbm_tau1.so behind the C ABI in
include/lbm_tau1.h; ``paper_2312_14742_gb300.lbm`` is its ctypes binding.
Nothing here computes on the CPU: without the built library the binding
raises.
"""
from .lbm import (Batch, LbmError, Tau1, load, lbm_tau1_abi_version, lbm_tau1_create, lbm_tau1_destroy,  # noqa: F401
                  lbm_tau1_get_fields, lbm_tau1_last_error, lbm_tau1_launch_count, lbm_tau1_reduce,
                  lbm_tau1_set_fields, lbm_tau1_set_geometry, lbm_tau1_step, lbm_tau1_synchronize)

__all__ = ["Batch", "LbmError", "Tau1", "load"]
