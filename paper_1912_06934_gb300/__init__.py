"""GB300 (sm_103a) implementation of the enhanced MsRSB preconditioner
(arXiv 1912.06934): C ABI in include/msrsb.h, CUDA kernels in csrc/, ctypes
binding in msrsb.py. Importing the package does no device work."""
from . import msrsb  # noqa: F401
from .msrsb import (Mat, Handle, MsrsbError, grid, opts, basis_opts, load,  # noqa: F401
                    msrsb_partition_size, msrsb_partition, msrsb_filter, msrsb_build_basis, msrsb_coarse_op,
                    msrsb_setup, msrsb_apply, msrsb_solve, msrsb_get_setup, msrsb_get_info, msrsb_destroy,
                    msrsb_solve_host, msrsb_profile, msrsb_profile_read, msrsb_fma_rate,
                    msrsb_build_basis_noalloc, msrsb_solve_ensemble, msrsb_transpose_values,
                    msrsb_pattern_outer, msrsb_wait_selftest, msrsb_mpfa_assemble, msrsb_mpfa_gradient,
                    msrsb_tune_mode, msrsb_tune_reset, msrsb_tune_table, MSRSB_TUNE_AUTO, MSRSB_TUNE_SMOOTH)
