"""Mixed-precision solve with iterative refinement (tcgen05 bf16/tf32
updates, FP64 inverses, FP64-class residual) against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda().t()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("inner", ["tf32", "bf16"])
@pytest.mark.parametrize("residual,s32", [("sliced", False), ("fp64", False), ("sliced", True)])
@pytest.mark.parametrize("n,k,n0", [(1024, 64, 128), (1000, 37, 64), (300, 5, 300)])
def test_mixed_well_conditioned(cuda_lib, inner, residual, s32, n, k, n0):
    import paper_1612_01855_gb300 as g
    L, B = inputs.well_conditioned(n, k, seed=n + k)
    Ld = _dev(L)
    plan = g.trsm_plan(Ld, n0)
    g.trsm_plan_mixed(plan, Ld, inner)
    X, iters, upd = g.trsm_solve_mixed(plan, _dev(B), residual=residual, max_iter=40, tol=1e-15,
                                       raise_on_noconv=False, s_fp32=s32)
    got = X.cpu().numpy()
    want = oracle.forward_subst(L, B)
    err = _rel(got, want)
    print(f"mixed {inner}/{residual} n={n} k={k} n0={n0}: {iters} iterations, last update {upd:.2e}, rel err {err:.2e}")
    # the refinement's limit is the residual's accuracy: ~2^-40 of |L||X| (sliced), ~n eps (fp64)
    assert err < (5e-12 if residual == "sliced" else 1e-13)
    assert iters <= (12 if inner == "tf32" else 25)


def test_mixed_graded_diagonal_forward_error(cuda_lib):
    """Diagonal graded from 1 to 1e-2: forward error against the
    double-double substitution stays below 1e-10."""
    import paper_1612_01855_gb300 as g
    n, k, n0 = 1024, 16, 128
    L, B = inputs.graded_diagonal(n, k, 2, seed=3)
    Ld = _dev(L)
    plan = g.trsm_plan(Ld, n0)
    g.trsm_plan_mixed(plan, Ld, "tf32")
    X, iters, upd = g.trsm_solve_mixed(plan, _dev(B), residual="sliced", max_iter=40, tol=1e-15,
                                       raise_on_noconv=False)
    hi, lo = oracle.forward_subst_dd(L, B)
    ref = hi + lo
    err = _rel(X.cpu().numpy(), ref)
    fp64 = _rel(oracle.forward_subst(L, B), ref)
    print(f"graded c=2: {iters} iterations, forward error {err:.2e} (FP64 oracle: {fp64:.2e})")
    assert err < 1e-10


def test_mixed_overflowing_solution_is_reported(cuda_lib):
    """Diagonal graded to 1e-4: X outgrows the FP32/bf16 range of the inner
    solve; the refinement must report non-convergence, not return garbage."""
    import paper_1612_01855_gb300 as g
    n, k, n0 = 512, 4, 64
    L, B = inputs.graded_diagonal(n, k, 4, seed=1)
    Ld = _dev(L)
    plan = g.trsm_plan(Ld, n0)
    g.trsm_plan_mixed(plan, Ld, "tf32")
    with pytest.raises(g.TrsmError) as ei:
        g.trsm_solve_mixed(plan, _dev(B), residual="sliced", max_iter=10, tol=1e-14)
    assert ei.value.code == -7


def test_mixed_argument_errors(cuda_lib):
    import paper_1612_01855_gb300 as g
    L, B = inputs.well_conditioned(64, 2, seed=0)
    plan = g.trsm_plan(_dev(L), 32)
    Bd = _dev(B)
    with pytest.raises(g.TrsmError):  # no mixed data in the plan
        g.trsm_solve_mixed(plan, Bd)
    g.trsm_plan_mixed(plan, _dev(L), "bf16")
    with pytest.raises(g.TrsmError):  # in place not allowed
        g.trsm_solve_mixed(plan, Bd, X=Bd)
