"""The sliced schedule (both matrix multiplies of It-Inv-TRSM as FP64-class
digit-sliced tensor-core products) against the oracle at the FP64
tolerance, at small and full sizes, in place, and bit for bit from call to
call."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the FP64 parity tolerance of the other schedules


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda().t()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("n,k,n0", [(512, 512, 64),     # the oracle-sized configuration
                                    (1000, 37, 64),     # ragged last block (40 rows), one narrow column tile
                                    (777, 81, 128),     # ragged block and column tiles (81 = 80 + 1)
                                    (2048, 300, 256),
                                    (4096, 96, 512),
                                    (3000, 200, 2048),  # the longest block, a ragged second one
                                    (300, 5, 300),      # one block: the full inverse
                                    (2048, 160, 4096),  # n0 > n: one block of order 2048
                                    (64, 1, 64), (1, 1, 1)])
def test_sliced_schedule_parity(cuda_lib, n, k, n0):
    import paper_1612_01855_gb300 as g
    L, B = inputs.well_conditioned(n, k, seed=n + 3 * k)
    p = g.trsm_plan(_dev(L), n0)
    X = g.trsm_solve_schedule(p, _dev(B), schedule="sliced")
    g.trsm_sync_status(p)
    got = X.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert _rel(got, oracle.forward_subst(L, B)) < TOL


def test_sliced_schedule_in_place_and_deterministic(cuda_lib):
    import torch
    import paper_1612_01855_gb300 as g
    n, k, n0 = 1536, 130, 128
    L, B = inputs.well_conditioned(n, k, seed=5)
    p = g.trsm_plan(_dev(L), n0)
    Bd = _dev(B)
    X1 = g.trsm_solve_schedule(p, Bd, schedule="sliced")
    X2 = g.trsm_solve_schedule(p, Bd, schedule="sliced")
    Bi = Bd.clone()
    g.trsm_solve_schedule(p, Bi, X=Bi, schedule="sliced")
    g.trsm_sync_status(p)
    assert torch.equal(X1, X2) and torch.equal(X1, Bi)
    assert _rel(X1.cpu().numpy(), oracle.forward_subst(L, B)) < TOL
    # the plan's device bytes include the digit planes: 16 n^2 + 16 n n0 (and exponents)
    assert p.device_bytes() >= 8 * n * n + 16 * n * n + 16 * n * n0


def test_sliced_schedule_rejects_unsupported_block_orders(cuda_lib):
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300 import binding
    lib = cuda_lib
    L = inputs.well_conditioned_L(1000, seed=9)
    for n0 in (100, 4096 // 2 + 64):  # not a multiple of 64; longer than 2048 with several blocks
        p = g.trsm_plan(_dev(L if n0 == 100 else inputs.well_conditioned_L(5000, seed=9)), n0)
        s = ctypes.c_void_p(0)
        assert lib.trsm_plan_sliced(p.handle, s) == binding.TRSM_EINVAL
        B = _dev(np.ones((p.n, 2)))
        rc = lib.trsm_solve_schedule(p.handle, ctypes.c_void_p(B.data_ptr()), 2, p.n,
                                     ctypes.c_void_p(B.data_ptr()), p.n, 3, s)
        assert rc == binding.TRSM_EINVAL  # no sliced data on the plan


@pytest.mark.parametrize("n,k,n0", [(16384, 256, 256), (8192, 8192, 512), (2048, 131072, 2048)])
def test_sliced_schedule_full_size_sampled_columns(cuda_lib, n, k, n0):
    """The FP64 sweep's three shapes: a seeded sample of columns computed by
    the oracle one by one (columns of X are independent), and the backward
    error of those columns."""
    import torch
    import paper_1612_01855_gb300 as g
    L, B = inputs.well_conditioned(n, k, seed=0)
    cols = np.sort(np.random.default_rng(5).choice(k, size=min(6, k), replace=False))
    want = oracle.forward_subst_columns(L, B, cols)
    Ld = _dev(L)
    p = g.trsm_plan(Ld, n0)
    Bd = _dev(B)
    X = g.trsm_solve_schedule(p, Bd, schedule="sliced")
    g.trsm_sync_status(p)
    ci = torch.from_numpy(cols).cuda()
    got = X[:, ci].cpu().numpy()
    assert _rel(got, want) < TOL
    Xs = torch.from_numpy(got).cuda()
    Lt = torch.tril(Ld)
    r = (Bd[:, ci] - Lt @ Xs).abs().max().item()
    bwd = r / (Lt.abs().sum(dim=1).max().item() * Xs.abs().max().item())
    assert bwd <= 10 * n * np.finfo(np.float64).eps, bwd


@pytest.mark.parametrize("c", [2, 4])
def test_sliced_schedule_precision_config(cuda_lib, c):
    """The precision configuration (n = 16384, k = 4096, graded diagonal
    geomspace(1, 10^-c) permuted) solved directly by the sliced schedule at
    n0 = 1024, with no refinement: the forward error of a seeded sample of
    columns against the double-double substitution meets the 1e-10 target
    of the refined solves."""
    import torch
    import paper_1612_01855_gb300 as g
    n, k, n0 = 16384, 4096, 1024
    L, B = inputs.graded_diagonal(n, k, c, seed=0)
    cols = np.sort(np.random.default_rng(17).choice(k, size=6, replace=False))
    hi, lo = oracle.forward_subst_dd(L, B[:, cols])
    ref = hi + lo
    Ld, Bd = _dev(L), _dev(B)
    del L
    p = g.trsm_plan(Ld, n0)
    X = g.trsm_solve_schedule(p, Bd, schedule="sliced")
    g.trsm_sync_status(p)
    got = X[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    fwd = _rel(got, ref)
    print(f"sliced schedule, precision config c={c}: forward error {fwd:.2e}")
    assert fwd <= 1e-10
