"""The three schedules of the blocked solve (dependency-driven kernel, the
paper's right-looking loop with look-ahead, Rec-TRSM) against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda().t()


@pytest.mark.parametrize("schedule", ["right-looking", "recursive"])
@pytest.mark.parametrize("n,k,n0", [(512, 512, 64), (1000, 37, 64), (777, 5, 100), (300, 100, 300),
                                    (2048, 96, 128), (64, 3, 16), (130, 70, 32)])
def test_schedule_parity(cuda_lib, schedule, n, k, n0):
    import paper_1612_01855_gb300 as g
    L, B = inputs.well_conditioned(n, k, seed=n + 7 * k)
    p = g.trsm_plan(_dev(L), n0)
    X = g.trsm_solve_schedule(p, _dev(B), schedule=schedule)
    g.trsm_sync_status(p)
    want = oracle.forward_subst(L, B)
    assert np.max(np.abs(X.cpu().numpy() - want)) / np.max(np.abs(want)) < TOL


def test_schedules_agree_and_are_deterministic(cuda_lib):
    import torch
    import paper_1612_01855_gb300 as g
    n, k, n0 = 1536, 64, 128
    L, B = inputs.well_conditioned(n, k, seed=3)
    p = g.trsm_plan(_dev(L), n0)
    Bd = _dev(B)
    xs = {s: g.trsm_solve_schedule(p, Bd, schedule=s) for s in ("dag", "right-looking", "recursive")}
    again = g.trsm_solve_schedule(p, Bd, schedule="right-looking")
    g.trsm_sync_status(p)
    assert torch.equal(again, xs["right-looking"])
    ref = xs["dag"].cpu().numpy()
    for s, x in xs.items():
        assert np.max(np.abs(x.cpu().numpy() - ref)) / np.max(np.abs(ref)) < TOL, s


def test_schedule_autotuner_picks_a_correct_fastest(cuda_lib):
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300 import autotune
    L, B = inputs.well_conditioned(1024, 48, seed=11)
    p = g.trsm_plan(_dev(L), 128)
    Bd = _dev(B)
    best, times = autotune.tune_schedule(p, Bd)
    assert best in times and times[best] == min(times.values())
    X = g.trsm_solve_schedule(p, Bd, schedule=best)
    g.trsm_sync_status(p)
    want = oracle.forward_subst(L, B)
    assert np.max(np.abs(X.cpu().numpy() - want)) / np.max(np.abs(want)) < TOL
