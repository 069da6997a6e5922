"""GB300 (sm_103a) low-rank primal-dual SDP solver (LR-PD-SDP, Alg. 2 of
Souto, Garcia & Veiga) behind the C ABI of ``include/proxsdp_gpu.h``.

The Python layer only marshals arguments to ``libproxsdp_gpu.so``; build the
library with ``python -m paper_1810_05231_gb300.build``.
"""
from ._binding import (  # noqa: F401
    CONVERGED,
    ERR_BAD_STATE,
    ERR_CUDA,
    ERR_INVALID_ARG,
    ERR_OOM,
    ERR_TIMEOUT,
    ERR_UNSUPPORTED,
    MAX_ITER,
    NUMERIC_ERROR,
    OP_AUTO,
    OP_EXPLICIT,
    OP_FACTORED,
    STALLED_AT_MAX_RANK,
    TIME_LIMIT,
    EXPORTED,
    Info,
    ProxSDPError,
    Settings,
    Solver,
    analyze_problem,
    aproj,
    aproj_noalloc,
    block_matvec,
    default_settings,
    lib,
    solve_batch,
    sym_eig,
)
