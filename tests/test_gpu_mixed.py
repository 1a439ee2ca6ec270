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


def _smode(smode):
    """Keyword arguments of a diagonal-multiply mode: fp64, fp32, or the
    tensor cores with 3 (tc), 2 (tc2) or 1 (tc1) tf32 planes per factor."""
    planes = {"tc": 3, "tc2": 2, "tc1": 1}.get(smode)
    return dict(s_fp32=smode == "fp32", s_tc=planes is not None, s_tc_planes=planes or 3)


def test_mixed_tensor_core_flags_are_exclusive(cuda_lib):
    """Two of the tensor-core diagonal-multiply flags at once, or one with
    TRSM_SOLVE_S_FP32, are rejected."""
    import ctypes
    import torch
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300 import binding as b
    n, k = 256, 8
    L, B = inputs.well_conditioned(n, k, seed=5)
    Ld, Bd = _dev(L), _dev(B)
    plan = g.trsm_plan(Ld, 64)
    g.trsm_plan_mixed(plan, Ld, "tf32")
    X = torch.empty((k, n), dtype=torch.float64, device="cuda").t()
    lib = b.load_library()
    it, upd = ctypes.c_int(), ctypes.c_double()
    for flags in (b.TRSM_SOLVE_S_TC | b.TRSM_SOLVE_S_TC2, b.TRSM_SOLVE_S_TC2 | b.TRSM_SOLVE_S_TC1,
                  b.TRSM_SOLVE_S_FP32 | b.TRSM_SOLVE_S_TC1):
        rc = lib.trsm_solve_mixed(plan.handle, ctypes.c_void_p(Bd.data_ptr()), k, n, ctypes.c_void_p(X.data_ptr()),
                                  n, b.TRSM_RESIDUAL_SLICED | flags, 10, 1e-12, ctypes.byref(it), ctypes.byref(upd),
                                  None)
        assert rc == b.TRSM_EINVAL
    plan.destroy()


@pytest.mark.parametrize("inner", ["tf32", "bf16", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("residual,smode", [("sliced", "fp64"), ("fp64", "fp64"), ("sliced", "fp32"),
                                            ("sliced", "tc"), ("sliced", "tc2"), ("sliced", "tc1"),
                                            ("progressive", "fp32")])
@pytest.mark.parametrize("n,k,n0", [(1024, 64, 128), (1000, 37, 64), (300, 5, 300)])
def test_mixed_well_conditioned(cuda_lib, inner, residual, smode, n, k, n0):
    """smode: the diagonal multiplies in FP64, in FP32, or on the tensor
    cores (split tf32)."""
    import paper_1612_01855_gb300 as g
    L, B = inputs.well_conditioned(n, k, seed=n + k)
    Ld = _dev(L)
    plan = g.trsm_plan(Ld, n0)
    g.trsm_plan_mixed(plan, Ld, inner)
    X, iters, upd = g.trsm_solve_mixed(plan, _dev(B), residual=residual, max_iter=40, tol=1e-15,
                                       raise_on_noconv=False, **_smode(smode))
    got = X.cpu().numpy()
    want = oracle.forward_subst(L, B)
    err = _rel(got, want)
    print(f"mixed {inner}/{residual}/{smode} n={n} k={k} n0={n0}: {iters} iterations, last update {upd:.2e}, "
          f"rel err {err:.2e}")
    # the refinement's limit is the residual's accuracy: ~2^-40 of |L||X| (sliced), ~n eps (fp64)
    assert err < (1e-13 if residual == "fp64" else 5e-12)
    assert iters <= {"tf32": 12, "bf16": 25, "bf16x3": 6, "fp16x3": 6}[inner]


@pytest.mark.parametrize("inner", ["tf32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("smode", ["fp32", "tc", "tc2", "tc1"])
@pytest.mark.parametrize("n,k,n0", [(1500, 70, 600), (2048, 33, 1024), (1100, 130, 512), (700, 21, 250)])
def test_mixed_wide_blocks_fp32_diagonal_multiply(cuda_lib, inner, smode, n, k, n0):
    """Blocks of 512 rows and more take the 64 x 64 register-blocked FP32
    diagonal multiply (ragged last blocks the 32 x 32 tile), or the
    tensor-core one (several row tiles per block, ragged last blocks)."""
    import paper_1612_01855_gb300 as g
    L, B = inputs.well_conditioned(n, k, seed=n + 3 * k)
    Ld = _dev(L)
    plan = g.trsm_plan(Ld, n0)
    g.trsm_plan_mixed(plan, Ld, inner)
    X, iters, upd = g.trsm_solve_mixed(plan, _dev(B), residual="sliced", max_iter=40, tol=1e-15,
                                       raise_on_noconv=False, **_smode(smode))
    err = _rel(X.cpu().numpy(), oracle.forward_subst(L, B))
    print(f"mixed {inner}/{smode} n={n} k={k} n0={n0}: {iters} iterations, rel err {err:.2e}")
    assert err < 5e-12
    assert iters <= 12


@pytest.mark.parametrize("inner", ["tf32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("smode", ["fp64", "fp32", "tc", "tc2", "tc1"])
def test_mixed_power_of_two_scaling_is_exact(cuda_lib, inner, smode):
    """Every scale in the refined solve (chunk exponents of the sliced
    residual, the fp16 panel and D_i scales, the FP32 inner solve) is a power
    of two, so solving with 2^s B gives 2^s X bit for bit while nothing leaves
    the normal range: s = -60 and +60 keep the FP32 residuals normal."""
    import paper_1612_01855_gb300 as g
    n, k, n0 = 600, 7, 128
    L, B = inputs.well_conditioned(n, k, seed=11)
    Ld = _dev(L)
    plan = g.trsm_plan(Ld, n0)
    g.trsm_plan_mixed(plan, Ld, inner)
    runs = {}
    for sc in (0, -60, 60):
        X, iters, upd = g.trsm_solve_mixed(plan, _dev(np.ldexp(B, sc)), residual="sliced", max_iter=40, tol=1e-13,
                                           raise_on_noconv=False, **_smode(smode))
        runs[sc] = (X.cpu().numpy(), iters)
    for sc in (-60, 60):
        assert runs[sc][1] == runs[0][1]
        assert np.array_equal(runs[sc][0], np.ldexp(runs[0][0], sc))


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


def test_mixed_residual_planes_set_the_floor(cuda_lib):
    """Diagonal graded from 1 to 1e-3 (componentwise condition ~1e3): the
    refinement stops at the condition times the residual's accuracy.  Seven
    digit planes (~2^-44) leave it near 1e-10; eight (~2^-49), alone or after
    seven stagnate, reach well below, against the double-double
    substitution."""
    import paper_1612_01855_gb300 as g
    n, k, n0 = 2048, 8, 128
    L, B = inputs.graded_diagonal(n, k, 3, seed=5)
    Ld = _dev(L)
    plan = g.trsm_plan(Ld, n0)
    g.trsm_plan_mixed(plan, Ld, "tf32")
    hi, lo = oracle.forward_subst_dd(L, B)
    ref = hi + lo
    errs = {}
    for res in ("sliced", "sliced8", "adaptive"):
        X, iters, upd = g.trsm_solve_mixed(plan, _dev(B), residual=res, max_iter=40, tol=1e-16,
                                           raise_on_noconv=False)
        errs[res] = (_rel(X.cpu().numpy(), ref), iters, upd)
    print(f"graded c=3 n={n}: {errs}")
    for res in ("sliced8", "adaptive"):
        assert errs[res][0] < 1e-11
        assert errs[res][0] < 0.25 * errs["sliced"][0]
    assert errs["adaptive"][1] > errs["sliced"][1]  # it went on after seven planes stagnated


def test_mixed_split_inner_reaches_the_floor(cuda_lib):
    """Diagonal graded from 1 to 1e-3: the split updates (bf16: about 16
    bits per factor; fp16, scaled into range: about 22) reach the eight-plane
    residual's floor in no more sweeps than tf32 (11 bits)."""
    import paper_1612_01855_gb300 as g
    n, k, n0 = 2048, 8, 128
    L, B = inputs.graded_diagonal(n, k, 3, seed=5)
    Ld = _dev(L)
    hi, lo = oracle.forward_subst_dd(L, B)
    ref = hi + lo
    out = {}
    for inner in ("tf32", "bf16x3", "fp16x3"):
        plan = g.trsm_plan(Ld, n0)
        g.trsm_plan_mixed(plan, Ld, inner)
        X, iters, upd = g.trsm_solve_mixed(plan, _dev(B), residual="sliced8", max_iter=40, tol=1e-12,
                                           raise_on_noconv=False)
        out[inner] = (_rel(X.cpu().numpy(), ref), iters, upd)
    print(f"graded c=3 n={n}, eight planes: {out}")
    for split in ("bf16x3", "fp16x3"):
        assert out[split][0] < 1e-11
        assert out[split][1] <= out["tf32"][1]


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


@pytest.mark.parametrize("c", [2, 4])
@pytest.mark.parametrize("smode,residual", [("fp32", "adaptive"), ("tc", "adaptive"), ("tc2", "adaptive"),
                                            ("fp32", "progressive")])
def test_full_size_precision_config(cuda_lib, c, smode, residual):
    """The precision configuration at its full size and in the bench's launch
    configuration: n = 16384, k = 4096, n0 = 1024, graded diagonal
    geomspace(1, 10^-c) permuted, split-fp16 updates, FP32 diagonal
    multiplies (FP32, or split tf32 on the tensor cores), the adaptive
    residual (seven digit planes, then eight) or the progressive one (five or
    six while the iterate is far from converged, then seven, then eight).  The
    forward error on a seeded sample of columns, against the double-double
    substitution of the same columns (columns of X are independent), stays
    within the 1e-10 target; the backward error of those columns is FP64
    class."""
    import torch
    import paper_1612_01855_gb300 as g
    n, k, n0 = 16384, 4096, 1024
    L, B = inputs.graded_diagonal(n, k, c, seed=0)
    cols = np.sort(np.random.default_rng(17).choice(k, size=6, replace=False))
    hi, lo = oracle.forward_subst_dd(L, B[:, cols])
    ref = hi + lo
    assert np.all(np.isfinite(ref))
    Ld, Bd = _dev(L), _dev(B)
    del L
    plan = g.trsm_plan(Ld, n0)
    g.trsm_plan_mixed(plan, Ld, "fp16x3")
    X, iters, upd = g.trsm_solve_mixed(plan, Bd, residual=residual, max_iter=30, tol=1e-12,
                                       **_smode(smode))
    ci = torch.from_numpy(cols).cuda()
    got = X[:, ci].cpu().numpy()
    fwd = _rel(got, ref)
    Lt = torch.tril(Ld)
    Xs = X[:, ci]
    bwd = (Bd[:, ci] - Lt @ Xs).abs().max().item() / (Lt.abs().sum(dim=1).max().item() * Xs.abs().max().item())
    print(f"precision config c={c} {smode} {residual}: {iters} sweeps, last update {upd:.2e}, forward error {fwd:.2e}, "
          f"backward error {bwd:.2e}")
    assert fwd <= 1e-10
    assert bwd <= 1e-14
    plan.destroy()
