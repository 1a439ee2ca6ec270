"""trsm_solve_noalloc: the solve for callers that may not allocate device
memory while solving (an application that owns all GPU memory through its
own arena, or a latency-critical loop that cannot pay for an allocation).
It must give the same X as trsm_solve and the oracle, call after call and in
place, from its fixed 64 MiB scratch array, and refuse problems whose
workspace does not fit.

This file is named to be collected last, so that a failure here cannot hide
the results of the other GPU tests in a run that stops at the first failure.
"""
import ctypes

import numpy as np
import pytest

from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 parity tolerance of the other GPU tests


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda().t()


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("n,k,n0", [(1000, 300, 64), (777, 33, 100)])
def test_noalloc_matches_trsm_solve_twice(cuda_lib, n, k, n0):
    """Two calls in a row with different B: each equals trsm_solve and the
    oracle.  (777, 33, 100) leaves a short last block row (77 rows) and a
    narrow last column tile, so ragged tiles go through the shared scratch."""
    import torch
    import oracle
    import paper_1612_01855_gb300 as g
    lib = cuda_lib
    L = inputs.well_conditioned_L(n, seed=21)
    plan = g.trsm_plan(_dev(L), n0)
    need = ctypes.c_size_t()
    assert lib.trsm_solve_workspace_size(plan.handle, k, ctypes.byref(need)) == 0
    assert need.value <= 64 << 20
    for call, seed in enumerate((31, 32)):  # two calls in a row, different B
        Bh = inputs.rhs(n, k, seed)
        B = _dev(Bh)
        X_ref = g.trsm_solve(plan, B)
        X = torch.full((k, n), float("nan"), dtype=torch.float64, device="cuda").t()
        rc = lib.trsm_solve_noalloc(plan.handle, ctypes.c_void_p(B.data_ptr()), k, B.stride(1),
                                    ctypes.c_void_p(X.data_ptr()), X.stride(1), _stream())
        assert rc == 0, lib.trsm_error_string(rc)
        g.trsm_sync_status(plan)
        assert torch.isfinite(X).all().item(), call
        got = X.cpu().numpy()
        assert _rel(got, X_ref.cpu().numpy()) < TOL, call
        assert _rel(got, oracle.forward_subst(L, Bh)) < TOL, call


def test_noalloc_in_place(cuda_lib):
    """X_dev == B_dev (same leading dimension) is allowed: the solve
    overwrites B with X."""
    import torch
    import oracle
    import paper_1612_01855_gb300 as g
    lib = cuda_lib
    n, k, n0 = 777, 33, 100
    L = inputs.well_conditioned_L(n, seed=23)
    plan = g.trsm_plan(_dev(L), n0)
    Bh = inputs.rhs(n, k, 33)
    B = _dev(Bh)
    rc = lib.trsm_solve_noalloc(plan.handle, ctypes.c_void_p(B.data_ptr()), k, B.stride(1),
                                ctypes.c_void_p(B.data_ptr()), B.stride(1), _stream())
    assert rc == 0, lib.trsm_error_string(rc)
    g.trsm_sync_status(plan)
    assert torch.isfinite(B).all().item()
    assert _rel(B.cpu().numpy(), oracle.forward_subst(L, Bh)) < TOL


def test_noalloc_rejects_oversized_workspace(cuda_lib):
    import torch
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300 import binding
    lib = cuda_lib
    n, k = 4096, 4096  # workspace about 128 MiB > 64 MiB
    plan = g.trsm_plan(_dev(inputs.well_conditioned_L(n, seed=22)), 256)
    B = torch.zeros((k, n), dtype=torch.float64, device="cuda").t()
    rc = lib.trsm_solve_noalloc(plan.handle, ctypes.c_void_p(B.data_ptr()), k, n,
                                ctypes.c_void_p(B.data_ptr()), n, _stream())
    assert rc == binding.TRSM_ENOSCRATCH
    assert b"scratch" in lib.trsm_error_string(rc)
    g.trsm_sync_status(plan)
