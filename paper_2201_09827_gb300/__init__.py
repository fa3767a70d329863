"""GB300 (sm_103a) recycled mixed-precision GMRES-IR for dense Ax = b.

The solver (Algorithms 2-4 of Oktay & Carson, arXiv 2201.09827) is the CUDA library
``libgir.so`` behind the C ABI in ``include/gir.h``; ``gir`` is its thin ctypes binding.
"""
from .gir import (  # noqa: F401
    Params, Info, Factorization, GirSolve, GirError, solve, residual, backward_errors, gemv, small_eig, batch_solve, batch_engine, load, lu_panel, lu_update, trace_enable, trace_report, trace_select, launch_count,
    library_path, autotune, tune_report, GIR_FLAG_AUTOTUNE, GIR_FLAG_CW_BERR, GIR_FLAG_SIR, GIR_FLAG_ADAPTIVE_K, GIR_FLAG_BATCH_STREAMS, GIR_FLAG_BATCH_PERSISTENT,
)
