"""FP64 CPU oracle for rAPDB on convex QCQPs -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference arms may import, call or execute anything in this package.  The
product path (the CUDA library and its Python binding) never touches it, and
this package shares no code with the CUDA path: the only module both sides use
is the seeded workload generator, which holds no solver arithmetic.

Parity status of each function is stated in ``rapdb_oracle``'s header.
"""
from .rapdb_oracle import (  # noqa: F401
    Params, Problem, Result, default_params, rapdb, apdb, kkt_residual,
    smoothed_gap, gap_x_subproblem, start_routine, apdb_iteration,
    yx_trial, xy_trial, BacktrackError, proj_simplex, simplex_cone_distance,
    proj_box_hyperplane, hyperplane_cone_distance, box_cone_residual,
)
from .quant import bf16_round, e4m3_round, e4m3_decode_table, fp8_jacobi_quantize  # noqa: F401
