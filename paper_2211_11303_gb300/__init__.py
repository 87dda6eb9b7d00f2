"""GB300-native H-LU preconditioned solver for the Nedelec edge-element
discretisation of time-harmonic Maxwell (arXiv 2211.11303, Algorithm 1).

The numerical path lives in libhlu.so (CUDA for sm_103a + a C++ task
scheduler) behind the C ABI of include/hlu.h; ``hlu`` is its thin binding.
"""
from . import hlu  # noqa: F401
from .hlu import (HLU_FP32, HLU_FP64, HluError, Problem, colmajor, gmres_solve,  # noqa: F401
                  hlu_build, hlu_destroy, hlu_export_csr, hlu_export_trees, hlu_factor,
                  hlu_factor_batch, hlu_factor_bytes_estimate, hlu_factor_stats, hlu_n,
                  hlu_rhs_manufactured, hlu_richardson, hlu_set_wait_limit_ms, hlu_solve,
                  hlu_solve_batch, hlu_spmv)
