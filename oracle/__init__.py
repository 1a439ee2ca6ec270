"""Plain FP64 CPU oracle for selective diagonal-block-inversion TRSM.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The CUDA product path never imports this package, and this package
imports nothing from the product.

Every function follows a passage of Wicky, Solomonik & Hoefler,
arXiv:1612.01855 (cited per function) or the textbook definition of the
result; the arithmetic lives in ``trsm_oracle.c`` (plain loops, FP64,
``-ffp-contract=off``), this module only marshals numpy arrays.

Matrices are numpy arrays holding the mathematical matrix (row index first);
they are passed to C in column-major (Fortran) order.

Planted mistakes for the pin-strength tests (``set_mutation``):
  1  RecTriInv loses the minus sign of L'21 = -(L22^-1 L21)
  2  RecTriInv multiplies by the transpose of L22^-1
  3  substitution drops the term l = j-1 from x_j's sum
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_c_i64 = ctypes.c_int64
_c_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, dp = _c_i64, _c_dp
        lib.oracle_forward_subst.argtypes = [i64, i64, dp, i64, dp, i64, dp, i64]
        lib.oracle_tri_inv_columns.argtypes = [i64, dp, i64, dp, i64]
        lib.oracle_rec_tri_inv.argtypes = [i64, dp, i64, dp, i64, i64]
        lib.oracle_diagonal_inverter.argtypes = [i64, i64, dp, i64, dp, i64, i64]
        lib.oracle_it_inv_trsm.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64, i64,
                                           ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_rec_trsm.argtypes = [i64, i64, i64, dp, i64, dp, i64, dp, i64]
        lib.oracle_forward_subst_dd.argtypes = [i64, i64, dp, i64, dp, i64, dp, dp, i64]
        lib.oracle_set_mutation.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        for f in ("oracle_forward_subst", "oracle_tri_inv_columns", "oracle_rec_tri_inv",
                  "oracle_diagonal_inverter", "oracle_it_inv_trsm", "oracle_rec_trsm",
                  "oracle_forward_subst_dd"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _f(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return a.ctypes.data_as(_c_dp)


def _ld(a):
    return max(1, a.shape[0])


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} returned {rc}")


def set_mutation(m: int) -> None:
    """Plant one deliberate mistake (see module docstring); 0 restores."""
    _load().oracle_set_mutation(int(m))


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def forward_subst(L, B):
    """X = L^-1 B by forward substitution (the problem statement L X = B of
    Section 1; textbook column sweep, sum in increasing index)."""
    L, B = _f(L), _f(B)
    if B.ndim == 1:
        return forward_subst(L, B[:, None])[:, 0]
    n, k = B.shape
    X = np.empty((n, k), dtype=np.float64, order="F")
    _check(_load().oracle_forward_subst(n, k, _p(L), _ld(L), _p(B), _ld(B), _p(X), _ld(X)),
           "forward_subst")
    return X


def tri_inv_columns(L):
    """L^-1 by definition: column j solves L y = e_j."""
    L = _f(L)
    m = L.shape[0]
    Li = np.empty((m, m), dtype=np.float64, order="F")
    _check(_load().oracle_tri_inv_columns(m, _p(L), _ld(L), _p(Li), _ld(Li)), "tri_inv_columns")
    return Li


def rec_tri_inv(L, base=16):
    """Algorithm RecTriInv (Section 5.1): recursive halving with
    L21^-1 = -(L22^-1 L21) L11^-1; base case by definition when m <= base."""
    L = _f(L)
    m = L.shape[0]
    Li = np.empty((m, m), dtype=np.float64, order="F")
    _check(_load().oracle_rec_tri_inv(m, _p(L), _ld(L), _p(Li), _ld(Li), int(base)), "rec_tri_inv")
    return Li


def diagonal_inverter(L, n0, base=16):
    """Algorithm Diagonal-Inverter (Section 6.1): L~ = L with every n0 x n0
    diagonal block replaced by its RecTriInv inverse (last block may be short)."""
    L = _f(L)
    n = L.shape[0]
    Lt = np.empty((n, n), dtype=np.float64, order="F")
    _check(_load().oracle_diagonal_inverter(n, int(n0), _p(L), _ld(L), _p(Lt), _ld(Lt), int(base)),
           "diagonal_inverter")
    return Lt


def diag_block_inverses(L, n0, base=16):
    """The n/n0 inverted diagonal blocks packed as an array (N, n0, n0); a
    short last block sits in the leading corner of a zero-filled slot."""
    n = np.asarray(L).shape[0]
    Lt = diagonal_inverter(L, n0, base)
    N = (n + n0 - 1) // n0
    out = np.zeros((N, n0, n0))
    for b in range(N):
        s = b * n0
        m = min(n0, n - s)
        out[b, :m, :m] = Lt[s:s + m, s:s + m]
    return out


def it_inv_trsm(L, B, n0, base=16, return_counts=False):
    """Algorithm It-Inv-TRSM (Section 6.2) on one processor, right-looking
    order of the paper.  With return_counts, also the multiply-add counts
    (solve, update)."""
    L, B = _f(L), _f(B)
    n, k = B.shape
    X = np.empty((n, k), dtype=np.float64, order="F")
    counts = (ctypes.c_int64 * 2)()
    _check(_load().oracle_it_inv_trsm(n, k, int(n0), _p(L), _ld(L), _p(B), _ld(B), _p(X), _ld(X),
                                      int(base), counts), "it_inv_trsm")
    if return_counts:
        return X, (int(counts[0]), int(counts[1]))
    return X


def rec_trsm(L, B, n0):
    """Algorithm Rec-TRSM (Section 4), sequential: halve L until n <= n0."""
    L, B = _f(L), _f(B)
    n, k = B.shape
    X = np.empty((n, k), dtype=np.float64, order="F")
    _check(_load().oracle_rec_trsm(n, k, int(n0), _p(L), _ld(L), _p(B), _ld(B), _p(X), _ld(X)),
           "rec_trsm")
    return X


def forward_subst_dd(L, B):
    """Forward substitution in double-double arithmetic (TwoSum / FMA-based
    TwoProd); returns (hi, lo) with X ~= hi + lo to about 2^-104 relative."""
    L, B = _f(L), _f(B)
    n, k = B.shape
    Xh = np.empty((n, k), dtype=np.float64, order="F")
    Xl = np.empty((n, k), dtype=np.float64, order="F")
    _check(_load().oracle_forward_subst_dd(n, k, _p(L), _ld(L), _p(B), _ld(B), _p(Xh), _p(Xl),
                                           _ld(Xh)), "forward_subst_dd")
    return Xh, Xl


def forward_subst_columns(L, B, cols):
    """Columns `cols` of X = L^-1 B only (the columns of X are independent,
    Section 2.3.4), for sampled checks at sizes where the full oracle is slow."""
    B = np.asarray(B)
    return forward_subst(L, B[:, np.asarray(cols)])
