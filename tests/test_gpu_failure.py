"""Failure detection without a GPU fault: a wait that nothing will satisfy
must run out after its limit, record the error, free what it holds and
return, leaving the device usable for the next solve."""
import ctypes
import time

import numpy as np
import pytest

import oracle
from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1])  # dependency counter, mbarrier
def test_unsatisfiable_wait_times_out_and_device_stays_usable(cuda_lib, kind):
    import torch
    import paper_1612_01855_gb300 as g
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    rc = cuda_lib.trsm_wait_selftest(kind, 50_000, s)  # 50 ms limit
    dt = time.perf_counter() - t0
    assert rc == -5  # TRSM_ETIMEOUT
    assert 0.045 <= dt < 2.0
    # the context is intact: a normal solve right after is correct
    L, B = inputs.well_conditioned(300, 7, seed=kind)
    Ld = torch.from_numpy(np.ascontiguousarray(L.T)).cuda().t()
    Bd = torch.from_numpy(np.ascontiguousarray(B.T)).cuda().t()
    p = g.trsm_plan(Ld, 64)
    X = g.trsm_solve(p, Bd)
    g.trsm_sync_status(p)  # raises on a recorded timeout
    want = oracle.forward_subst(L, B)
    assert np.max(np.abs(X.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want))


def test_wait_selftest_argument_errors(cuda_lib):
    assert cuda_lib.trsm_wait_selftest(2, 1000, None) == -1
    assert cuda_lib.trsm_wait_selftest(0, 0, None) == -1
