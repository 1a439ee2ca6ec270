"""GB300-native selective diagonal-block-inversion TRSM (arXiv:1612.01855).

``binding`` exposes the C ABI of ``include/trsm_gb300.h`` under the same
names; ``inputs`` draws the seeded synthetic workloads; ``build`` compiles
the CUDA library in-tree for sm_103a.
"""
from .binding import (Batch, Plan, TrsmError, colmajor, fp32_peak, fp64_peak, launch_count, load_library,  # noqa: F401
                      trsm_host, trsm_host_ptr, trsm_plan, trsm_plan_mixed, trsm_plan_sliced, trsm_solve, trsm_solve_mixed, trsm_solve_schedule,
                      trsm_solve_noalloc,
                      trsm_solve_workspace_size, trsm_solve_ws, trsm_sync_status, trtri_blocks,
                      workspace_reserved_bytes, workspace_trim)

__all__ = ["Batch", "Plan", "TrsmError", "colmajor", "fp32_peak", "fp64_peak", "launch_count", "load_library",
           "trsm_host", "trsm_host_ptr", "trsm_plan", "trsm_plan_mixed", "trsm_plan_sliced", "trsm_solve", "trsm_solve_mixed", "trsm_solve_schedule", "trsm_solve_noalloc", "trsm_solve_workspace_size",
           "trsm_solve_ws", "trsm_sync_status", "trtri_blocks", "workspace_reserved_bytes", "workspace_trim"]
