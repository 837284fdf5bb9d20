"""Tucker-format sketched GMRES (RHOSVD-Tucker sGMRES, MLN-Tucker sGMRES) for B300 (sm_103a).

The solvers run in the CUDA library libtuckersgmres.so (C ABI: include/tuckersgmres.h);
this package is its thin Python binding.  The library is loaded on first use and loading
fails loudly when it has not been built; nothing here computes on the CPU.
"""
from ._lib import EXPORTS, LIB_PATH, load  # noqa: F401
from .api import (DeviceOperator, DeviceTucker, Handle, Options, Report, TuckerError,  # noqa: F401
                  fortran_empty, handle, to_fortran, tk_apply, tk_gaussian, tk_inner, tk_kron_sketch,
                  tk_mln_roundsum, tk_philox, tk_profile, tk_profile_report, tk_residual, tk_roundsum,
                  tk_sketched_ls, tk_sketched_ls_static, tk_solve, tk_sum_norm, tk_adjoint_grads,
                  tk_solve_precond, tk_expsum_laplacian, tk_checkpoint_save, tk_checkpoint_load,
                  tk_set_workspace_limit, tk_fma_peak, tk_solve_expsum,
                  tk_solve_concurrent, tk_selftest_qr_wait)

from . import autograd  # noqa: E402,F401
