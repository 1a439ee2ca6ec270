"""FP64-class residual R = B - tril(L) X on the BF16 tensor cores (integer
digit slices, exact FP32 group sums) against an exactly rounded reference:
products split exactly (Dekker/Veltkamp TwoProduct) and summed with
math.fsum."""
import ctypes
import math

import numpy as np
import pytest

from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu


def _two_product(a, b):
    """Exact a*b = p + e for float64 arrays (Dekker, with Veltkamp splitting)."""
    p = a * b
    c = 134217729.0  # 2^27 + 1
    def split(x):
        t = c * x
        hi = t - (t - x)
        return hi, x - hi
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_residual(L, X, B):
    n, k = B.shape
    Lt = np.tril(L)
    R = np.empty_like(B)
    for j in range(k):
        x = X[:, j]
        for i in range(n):
            p, e = _two_product(Lt[i, : i + 1], x[: i + 1])
            R[i, j] = math.fsum(np.concatenate(([B[i, j]], -p, -e)))
    return R


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda().t()


@pytest.mark.parametrize("planes", [5, 6, 7, 8])
@pytest.mark.parametrize("n,k,kind", [(1024, 8, "well"), (1500, 5, "well"), (700, 17, "graded2"),
                                      (2100, 3, "well"), (130, 64, "well"), (100, 9, "well"),
                                      (300, 40, "graded2")])
def test_sliced_residual_accuracy(cuda_lib, n, k, kind, planes):
    import torch
    lib = cuda_lib
    if kind == "well":
        L, B = inputs.well_conditioned(n, k, seed=n)
    else:
        L, B = inputs.graded_diagonal(n, k, 2, seed=n)
    rng = np.random.default_rng(n + k)
    X = rng.uniform(-1, 1, size=(n, k)) * 2.0 ** rng.integers(-8, 8, size=(1, k))
    Ld, Xd, Bd = _dev(L), _dev(X), _dev(B)
    Rd = torch.full((k, n), float("nan"), dtype=torch.float64, device="cuda").t()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.trsm_residual_sliced(ctypes.c_void_p(Ld.data_ptr()), n, Ld.stride(1),
                                  ctypes.c_void_p(Xd.data_ptr()), k, Xd.stride(1),
                                  ctypes.c_void_p(Bd.data_ptr()), Bd.stride(1),
                                  ctypes.c_void_p(Rd.data_ptr()), Rd.stride(1), planes,
                                  ctypes.c_void_p(err.data_ptr()), s)
    assert rc == 0
    torch.cuda.synchronize()
    assert err.item() == 0
    R = Rd.cpu().numpy()
    Rref = exact_residual(L, X, B)
    # componentwise measure |B| + |L||X|: the final FP64 rounding of R is
    # relative to |B - L X|, which |L||X| alone does not bound when X is small
    scale = np.abs(B) + np.abs(np.tril(L)) @ np.abs(X)
    rel = np.max(np.abs(R - Rref) / scale)
    assert np.all(np.isfinite(R))
    # P digits of 6 bits: each factor exact to 2^-(6P+1) of its (row, chunk)
    # maximum, dropped digit pairs below 2^-(6P-1) per product; relative to
    # |B| + |L||X| the max error stays near 2^-43 for P = 7 and 2^-48 for
    # P = 8 (two bits more when a small diagonal shrinks |L||X|), so 6 bits
    # less per plane fewer: the bound is 2^-(6P - 2), three bits of margin
    print(f"sliced residual P={planes} n={n} k={k} {kind}: max rel err {rel:.3e} (2^{np.log2(rel):.1f})")
    assert rel < 2.0 ** -(6 * planes - 2 if planes < 8 else 45), rel
