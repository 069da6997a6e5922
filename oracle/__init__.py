"""FP64 CPU oracle for the paper's PD-SDP (Alg. 1) and LR-PD-SDP (Alg. 2).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or executes this package; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA path.

Everything here is plain, slow and written to be checked against the paper by
eye: dense FP64 matrices, ``numpy.linalg.eigh`` for every eigendecomposition,
one function per formula.  Every function names the section / equation /
algorithm it follows.  The pins that tie it to something other than itself
(closed forms, identities, brute force) live in ``tests/test_oracle_pins.py``.

Parity status: every function is pinned except the per-iteration trajectory
and rank path of ``solve`` (they depend on the window / step-size / rank-rule
readings the paper leaves open); only the fixed points, final objective values
and certificates of ``solve`` are pinned ("parity unpinned" for trajectories).
"""
from .sdp import (  # noqa: F401
    DENSE_ROW,
    ConstraintOperator,
    aproj_psd,
    brute_force_maxcut,
    brute_force_binary_ls,
    certificates,
    dual_prox,
    normalize_rows,
    operator_norm,
    pd_iteration,
    proj_box,
    proj_psd,
    solve,
    svec_unpack,
)
