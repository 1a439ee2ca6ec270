"""Block-size autotuner for batches of small systems.

The paper chooses n0 a priori from its cost model (Section 8; with one
processor its three-dimensional rule gives n0 ~ min(sqrt(n k), n)); on one
GPU the choice that matters is the in-launch inversion block of the
batched solve (32 or 64) per size bucket.  `tune_batch_n0` times both
candidates on synthetic systems of each bucket through the batched C ABI
and keeps the faster; `choose_n0` maps a system to its bucket's choice.
Results are cached per (dtype, bucket) for the process.
"""
import math

import numpy as np

from . import binding

# size buckets by n (log2 ranges), as in the batching workload n in [32, 1024]
BUCKETS = [(1, 64), (64, 128), (128, 256), (256, 512), (512, 1025)]
CANDIDATES = (32, 64)
_cache = {}


def paper_rule_n0(n, k):
    """The paper's a-priori block size with one processor: min(sqrt(n k), n)."""
    return int(min(math.sqrt(n * k), n))


def bucket_of(n):
    for i, (lo, hi) in enumerate(BUCKETS):
        if lo <= n < hi:
            return i
    return len(BUCKETS) - 1


def _synthetic(count, lo, hi, kmax, dtype, seed):
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    rng = np.random.default_rng(seed)
    systems = []
    for _ in range(count):
        n = int(np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi - 1)))))
        k = int(np.rint(np.exp(rng.uniform(0.0, np.log(kmax)))))
        L = torch.rand((n, n), generator=g, device="cuda", dtype=tdt).mul_(2).sub_(1).div_(n)
        L = torch.tril(L, -1)
        L.diagonal().copy_(torch.rand(n, generator=g, device="cuda", dtype=tdt).add_(2))
        L = L.t().contiguous().t()
        B = torch.rand((k, n), generator=g, device="cuda", dtype=tdt).mul_(2).sub_(1).t()
        X = torch.empty((k, n), device="cuda", dtype=tdt).t()
        systems.append({"L": L, "B": B, "X": X})
    return systems


def tune_batch_n0(dtype="f64", count=96, kmax=256, reps=3, seed=7):
    """Measures n0 = 32 and 64 per bucket; returns {bucket index: n0}."""
    import torch
    out = {}
    for bi, (lo, hi) in enumerate(BUCKETS):
        key = (dtype, bi)
        if key in _cache:
            out[bi] = _cache[key]
            continue
        systems = _synthetic(count, max(lo, 1), hi, kmax, dtype, seed + bi)
        best, best_t = None, float("inf")
        for n0 in CANDIDATES:
            for sy in systems:
                sy["n0"] = n0
            b = binding.Batch(systems, dtype=dtype)
            b.run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                b.run()
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / reps
            rc = b.status()[0]
            b.destroy()
            if rc == 0 and t < best_t:
                best, best_t = n0, t
        _cache[key] = best
        out[bi] = best
    return out


def choose_n0(n, dtype="f64", table=None):
    table = table if table is not None else {bi: v for (dt, bi), v in _cache.items() if dt == dtype}
    return table.get(bucket_of(n), 32)
