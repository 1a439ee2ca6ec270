"""Seeded synthetic inputs for L X = B (numpy PCG64 streams).

This module holds no arithmetic of the method: it only draws the matrices the
tests, the smoke check and the bench feed to both the CUDA path and the CPU
oracle.  Every matrix is returned in column-major (Fortran) order, the layout
the C ABI expects.

Recipes (the paper runs no experiments, so these are the workloads the
method's cost analysis is stated for, at the sizes of the measured configs):

* ``well_conditioned``: L lower-triangular, diagonal ~ U[2, 3], strictly lower
  entries ~ U[-1, 1] / n (diagonally dominant, condition number O(1));
  B ~ U[-1, 1].  Draw order from one ``Generator(PCG64(seed))``: n*n values
  for the strictly-lower part in column-major order (the upper half of the
  draw is discarded), then n diagonal values, then n*k values of B in
  column-major order.
* ``graded_diagonal``: as above, but the diagonal is geomspace(1, 10^-c, n)
  permuted by the same generator (ill-conditioned for large c).
* ``log_uniform_sizes``: sizes drawn log-uniformly, for batches of uneven
  systems.
"""
import numpy as np

_CHUNK = 1 << 24  # values per draw when filling large matrices


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _fill_uniform_f(rng, shape, lo, hi, scale=1.0):
    """Column-major matrix of U[lo, hi] * scale, drawn in column-major order."""
    n, m = shape
    out = np.empty((n, m), dtype=np.float64, order="F")
    flat = out.reshape(-1, order="F")  # a view: `out` is F-contiguous
    total = n * m
    for s in range(0, total, _CHUNK):
        e = min(total, s + _CHUNK)
        flat[s:e] = rng.uniform(lo, hi, size=e - s)
    if scale != 1.0:
        flat *= scale
    return out


def _lower_offdiag(rng, n):
    L = _fill_uniform_f(rng, (n, n), -1.0, 1.0, 1.0 / max(n, 1))
    # zero the strict upper triangle column by column (in place, no n x n temporaries)
    for j in range(1, n):
        L[:j, j] = 0.0
    return L


def well_conditioned(n, k, seed=0):
    """(L, B) with diag(L) ~ U[2,3], tril(L,-1) ~ U[-1,1]/n, B ~ U[-1,1]."""
    rng = _rng(seed)
    L = _lower_offdiag(rng, n)
    d = rng.uniform(2.0, 3.0, size=n)
    L[np.arange(n), np.arange(n)] = d
    B = _fill_uniform_f(rng, (n, k), -1.0, 1.0)
    return L, B


def well_conditioned_L(n, seed=0):
    rng = _rng(seed)
    L = _lower_offdiag(rng, n)
    L[np.arange(n), np.arange(n)] = rng.uniform(2.0, 3.0, size=n)
    return L


def rhs(n, k, seed):
    """B ~ U[-1, 1], n x k, column-major, from its own stream."""
    return _fill_uniform_f(_rng(seed), (n, k), -1.0, 1.0)


def graded_diagonal(n, k, c, seed=0):
    """(L, B) with diag(L) = permuted geomspace(1, 10^-c, n), tril ~ U[-1,1]/n."""
    rng = _rng(seed)
    L = _lower_offdiag(rng, n)
    d = np.geomspace(1.0, 10.0 ** (-c), n) if n > 1 else np.ones(n)
    d = d[rng.permutation(n)]
    L[np.arange(n), np.arange(n)] = d
    B = _fill_uniform_f(rng, (n, k), -1.0, 1.0)
    return L, B


def log_uniform_sizes(count, lo, hi, seed):
    """`count` integers round(exp(U[ln lo, ln hi]))."""
    rng = _rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
