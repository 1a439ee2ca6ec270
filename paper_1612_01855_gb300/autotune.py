"""Autotuning of the batched and the single-system solve.

The paper chooses n0 a priori from its cost model (Section 8; with one
processor its three-dimensional rule gives n0 ~ min(sqrt(n k), n)).  On one
GPU the choices that matter are measured instead:

* batches (`tune_batch`): per size bucket, the in-launch inversion block
  n0 (32 or 64) and the output tile shape -- 32-wide column tiles, or tiles
  fitted to k by the library (8 for k <= 8, 16 for k <= 16, and above 32
  32-wide tiles plus one narrower tile for the remainder) -- each candidate
  timed on synthetic systems of that bucket through the batched C ABI, the
  fastest kept; `choose` maps a system to its bucket's choice;
* single systems (`tune_schedule`): the schedule of the blocked solve
  (dependency-driven kernel, right-looking loop with look-ahead, Rec-TRSM)
  timed on the system itself.

Results are cached per (dtype, bucket) for the process.
"""
import math

import numpy as np

from . import binding

# size buckets by n (log2 ranges), as in the batching workload n in [32, 1024]
BUCKETS = [(1, 64), (64, 128), (128, 256), (256, 512), (512, 1025)]
N0_CANDIDATES = (32, 64)
TILE_CANDIDATES = (0, 32)  # 0: column tiles fitted to k by the library
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


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(dtype="f64", count=96, kmax=256, reps=3, seed=7):
    """Times every (n0, tile) candidate per bucket; returns {bucket index:
    (n0, tile_cols)} with the fastest candidate that ran without error."""
    out = {}
    for bi, (lo, hi) in enumerate(BUCKETS):
        key = (dtype, bi)
        if key in _cache:
            out[bi] = _cache[key]
            continue
        systems = _synthetic(count, max(lo, 1), hi, kmax, dtype, seed + bi)
        best, best_t = (32, 0), float("inf")
        for n0 in N0_CANDIDATES:
            for tile in TILE_CANDIDATES:
                for sy in systems:
                    sy["n0"], sy["tile_cols"] = n0, tile
                b = binding.Batch(systems, dtype=dtype)
                t = _time(b.run, reps)
                rc = b.status()[0]
                b.destroy()
                if rc == 0 and t < best_t:
                    best, best_t = (n0, tile), t
        _cache[key] = best
        out[bi] = best
    return out


def tune_batch_n0(dtype="f64", **kw):
    """The block-size part of tune_batch: {bucket index: n0}."""
    return {bi: v[0] for bi, v in tune_batch(dtype, **kw).items()}


def choose(n, dtype="f64", table=None):
    """(n0, tile_cols) for a system of order n from its bucket's tuned choice."""
    table = table if table is not None else {bi: v for (dt, bi), v in _cache.items() if dt == dtype}
    return table.get(bucket_of(n), (32, 0))


def choose_n0(n, dtype="f64", table=None):
    v = choose(n, dtype, table)
    return v[0] if isinstance(v, tuple) else v


def tune_schedule(plan, B, X=None, reps=2):
    """Times the schedules of the blocked solve on this system (the sliced
    one only where the plan's block order allows it; its digit planes are
    made before the timing); returns (fastest name, {name: ms})."""
    times = {}
    for sched in binding.SCHEDULES:
        if sched == "sliced":
            try:
                binding.trsm_plan_sliced(plan)
            except binding.TrsmError:
                continue
        times[sched] = _time(lambda: binding.trsm_solve_schedule(plan, B, X=X, schedule=sched), reps)
    binding.trsm_sync_status(plan)
    return min(times, key=times.get), times
