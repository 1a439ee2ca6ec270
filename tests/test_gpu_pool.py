"""The library's workspace pool: per-call scratch is a stream-ordered
allocation from a pool the library owns, which keeps freed memory mapped
for the next call (the device's default pool unmaps it at every
synchronisation).  A solve leaves its workspace reserved, a second solve of
the same size reuses it without growing the pool, trsm_workspace_trim hands
the idle memory back, and results do not depend on whether the workspace
was fresh or reused."""
import numpy as np
import pytest

import oracle
from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda().t()


def test_workspace_is_kept_reused_and_trimmed(cuda_lib):
    import torch
    import paper_1612_01855_gb300 as g
    n, k, n0 = 1200, 700, 128
    L, B = inputs.well_conditioned(n, k, seed=77)
    Ld, Bd = _dev(L), _dev(B)
    plan = g.trsm_plan(Ld, n0)
    g.workspace_trim(0)
    torch.cuda.synchronize()
    base = g.workspace_reserved_bytes()
    X1 = g.trsm_solve(plan, Bd)
    g.trsm_sync_status(plan)
    after_first = g.workspace_reserved_bytes()
    # the solve's workspace (a copy of B plus counters) stays reserved
    assert after_first - base >= 8 * n * k
    X2 = g.trsm_solve(plan, Bd)
    g.trsm_sync_status(plan)
    assert g.workspace_reserved_bytes() == after_first  # reused, not grown
    assert torch.equal(X1, X2)
    want = oracle.forward_subst(L, B)
    assert float(np.max(np.abs(X1.cpu().numpy() - want)) / np.max(np.abs(want))) < 1e-12
    g.workspace_trim(0)
    torch.cuda.synchronize()
    assert g.workspace_reserved_bytes() <= base
    # a solve after the trim maps its workspace again and gives the same bits
    X3 = g.trsm_solve(plan, Bd)
    g.trsm_sync_status(plan)
    assert torch.equal(X1, X3)
    plan.destroy()
