"""Benchmark: FP64 TRSM by selective diagonal-block inversion on one GB300.

One step = the whole method on one batch of the FP64 k/n sweep workload:
for each shape (n, k) in {(16384, 256), (8192, 8192), (2048, 131072)} at its
block size n0, trsm_plan (invert the diagonal blocks) + trsm_solve (blocked
solve), inputs resident in HBM.  value = sum(n^2 k) / step time (TFLOP/s).

Prints ONE compact JSON line (rank 0).  Beside the timed step it carries the
other configurations, each measured in the same run: the block-size sweep
(`n0_sweep`), the precision configuration at c = 2, 4, 6 (`precision`), the
batches of uneven systems (`batched`), the serving loop (`serving`), the
solve schedules (`schedules_ms`) and the sliced residual's roofline.
`--details FILE` writes the full records of every study.  `--impl reference`
times the CPU oracle (forward substitution, the plain definition of
X = L^-1 B) on the host cores instead, on a bounded column sample of the
same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TRSM TFLOP/s (n²k) and roofline fraction at stated error; served solves/s, p50/p99"
SHAPES = [(16384, 256), (8192, 8192), (2048, 131072)]
# Block sizes chosen by the n0 sweep on GB300 (see the tuning table in the
# package); the paper's a-priori rule for p = 1 is n0 ~ min(sqrt(n k), n).
DEFAULT_N0 = {(16384, 256): 256, (8192, 8192): 512, (2048, 131072): 2048}
SWEEP_N0 = [64, 128, 256, 512, 1024, None]  # None = n (full inversion)
SCHEDULE_NAMES = ("dag", "right-looking", "recursive", "sliced")
# Block sizes of the sliced schedule (FP64-class products on the tensor
# cores): longer blocks mean longer, more efficient tensor-core products
# (measured, ms: 16384x256 9.7 / 7.2 / 5.8 at n0 = 256 / 512 / 1024;
# 8192x8192 26.0 / 22.0 / 20.0 at 512 / 1024 / 2048; 2048x131072 32.4 /
# 29.7 / 30.3 at 512 / 1024 / 2048)
SLICED_N0 = {(16384, 256): 2048, (8192, 8192): 2048, (2048, 131072): 2048}
SLICED_PREC_N0 = 2048  # block order of the sliced schedule's precision-configuration row
# Block size of the mixed-precision figure (n = 16384, k = 4096).  Larger
# blocks suit the mixed path: fewer, longer tensor-core updates, and the
# diagonal multiplies run in FP32 (measured: 163 / 137 / 131 / 135 ms at
# n0 = 256 / 512 / 1024 / 2048, tf32 with FP32 diagonal multiplies).
MIXED_N0 = 1024
NOMINAL_SM_MHZ = 2070.0

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one
# it_inv_solve_kernel launch per bench shape, from one 1-pass ncu capture of
# each shape in the bench's launch configuration.  They describe the
# kernel source they were taken from; once solve.cu or fp64_tile.cuh changes
# the figures no longer apply and the bench reports traffic as null.
SOLVE_TRAFFIC_SHA256 = "1b10bcd32c87a0a41972ba56e8f8083faf7da9229e5723ae1281f62ca03d8e2a"
SOLVE_TRAFFIC = {(16384, 256, 256): 1120057344 + 64409856,
                 (8192, 8192, 512): 5455504384 + 4520425216,
                 (2048, 131072, 2048): 2200583168 + 2126338304}


def solve_source_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in ("solve.cu", "fp64_tile.cuh"):  # the kernel's own sources (wait.cuh holds only the bounded wait)
        with open(os.path.join(ROOT, "paper_1612_01855_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def solve_traffic(shapes, n0s):
    """Mean DRAM bytes per solve launch over the step's shapes, the per-shape
    figures and the algorithmic bytes 8 (n^2/2 + 2 n k) beside them; None
    when the counters do not describe this kernel source or these shapes."""
    keys = [(n, k, n0) for (n, k), n0 in zip(shapes, n0s)]
    if solve_source_sha256() != SOLVE_TRAFFIC_SHA256 or any(key not in SOLVE_TRAFFIC for key in keys):
        return None, None
    by_shape = {f"{n}x{k}": {"dram_bytes": SOLVE_TRAFFIC[(n, k, n0)],
                             "algorithmic_bytes": int(8 * (n * n / 2 + 2 * n * k))} for n, k, n0 in keys}
    return sum(SOLVE_TRAFFIC[key] for key in keys) / len(keys), by_shape


def measured_peaks():
    """bf16 tensor peaks (burst, sustained) in TFLOP/s from MEASURED_PEAKS.json
    when present, else the fallback figures of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 1900.0, 1700.0, "fallback (earlier GB300 measurement)"


def sm_count():
    """Streaming multiprocessors of the current device."""
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def nominal_peaks():
    """Nominal FP64 (2 DFMA lanes per SM and clock) and FP32 (128 FFMA lanes
    per SM and clock) rates in TFLOP/s at the nominal SM clock, for the SM
    count of the current device."""
    sms = sm_count()
    return sms, sms * 2 * 2 * NOMINAL_SM_MHZ * 1e6 / 1e12, sms * 128 * 2 * NOMINAL_SM_MHZ * 1e6 / 1e12


def max_over_ranks(value, device):
    """The largest `value` over all ranks of the process group (the timing
    rule for replicas: the job lasts as long as its slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_step, world, ms_per_step):
    """Whole-job rate of `world` replicas that each process units_per_step
    per step in ms_per_step (the max over ranks): weak scaling, no exchange."""
    return units_per_step * world / (ms_per_step * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix=f"trsm_clocks_gpu{gpu_index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(shapes, seed=0):
    from paper_1612_01855_gb300 import inputs
    return [inputs.well_conditioned(n, k, seed=seed + i) for i, (n, k) in enumerate(shapes)]


def to_dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def cpu_oracle_rate(data, shapes, budget_s, max_cols=None):
    """Times the CPU oracle (forward substitution) on a column sample of each
    shape; returns (TFLOP/s counting n^2 k_sample, sample description, cores)."""
    import oracle
    flops, secs, desc = 0.0, 0.0, []
    per_shape = budget_s / len(shapes)
    cores = oracle.max_threads()
    for (L, B), (n, k) in zip(data, shapes):
        cols = max(cores, 1)
        if max_cols:
            cols = min(cols, max_cols)
        t_used, c_used = 0.0, 0
        while t_used < per_shape and c_used < k:
            c = min(cols, k - c_used)
            t0 = time.perf_counter()
            oracle.forward_subst(L, B[:, c_used:c_used + c])
            dt = time.perf_counter() - t0
            t_used += dt
            c_used += c
            cols = min(cols * 2, k)
        flops += float(n) * n * c_used
        secs += t_used
        desc.append(f"{n}:{c_used}/{k}")
    return flops / secs / 1e12, "; ".join(desc), cores


def precision_study(g, torch, n, k, n0, cs, inners, s_modes, dd_cols=4, stream=None, quick=False,
                    residuals=("sliced",), combos=None, with_sliced=False, tol=1e-11):
    """Mixed-precision refinement on the graded-diagonal workload (diagonal
    geomspace(1, 10^-c), permuted): time, iterations, forward error against
    the double-double oracle and backward error ||B - L X|| / (||L|| ||X||)
    on a seeded sample of columns, beside the FP64 solve of the same system.
    The refinement stops at max|D| <= tol max|X| (1e-11: ten times below the
    1e-10 target, above the update noise of about 1e-12 that an iterate at
    this system's FP64 error floor, about 7e-13, still shows) or when the
    updates stagnate.  s_modes: the diagonal multiply in FP64, FP32
    ("fp32"), or on the tensor cores with 3, 2 or 1 tf32 planes per factor
    ("tc", "tc2", "tc1").  A solve that stops without reaching the target
    reports its status (ENOCONV), and a non-finite result or reference
    reports None errors."""
    import oracle
    from paper_1612_01855_gb300 import binding, inputs
    out = []
    for c in cs:
        L, B = inputs.graded_diagonal(n, k, c, seed=0)
        cols = np.sort(np.random.default_rng(7).choice(k, size=min(dd_cols, k), replace=False))
        hi, lo = oracle.forward_subst_dd(L, B[:, cols])
        ref = hi + lo
        ref_ok = bool(np.all(np.isfinite(ref)))
        Ld, Bd = to_dev(L, torch), to_dev(B, torch)
        del L

        def ferr(X):
            got = X[:, torch.from_numpy(cols).cuda()].cpu().numpy()
            if not ref_ok or not np.all(np.isfinite(got)):
                return None
            return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))

        Lt_abs_rowsum = torch.tril(Ld).abs().sum(dim=1).max().item()

        def berr(X):
            """||B - L X|| / (||L|| ||X||) on the sampled columns (infinity norm)."""
            ci = torch.from_numpy(cols).cuda()
            Xs = X[:, ci]
            if not torch.isfinite(Xs).all():
                return None
            r = (Bd[:, ci] - torch.tril(Ld) @ Xs).abs().max().item()
            return r / (Lt_abs_rowsum * Xs.abs().max().item())

        plan = g.trsm_plan(Ld, n0)
        X64 = g.trsm_solve(plan, Bd)
        g.trsm_sync_status(plan)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        X64 = g.trsm_solve(plan, Bd, X=X64)
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        rec = {"c": c, "n": n, "k": k, "n0": n0, "fp64_solve_ms": round(t64, 2),
               "fp64_fwd_err": ferr(X64), "fp64_bwd_err": berr(X64), "dd_reference_finite": ref_ok,
               "sampled_columns": [int(v) for v in cols], "mixed": []}
        # (inner format, diagonal-multiply mode, residual) triples: a given
        # list, or every inner x s_mode x residual
        runs = combos or [(i, sm, r) for i in inners for sm in s_modes for r in residuals]
        cur = None
        extra = {}  # a plan at another block size, for combos that name one
        for run in runs:
            inner, smode, res = run[:3]
            rn0 = run[3] if len(run) > 3 else n0
            if rn0 != n0:
                if (rn0, inner) not in extra:
                    for p_ in extra.values():
                        p_.destroy()
                    extra = {(rn0, inner): g.trsm_plan(Ld, rn0)}
                    g.trsm_plan_mixed(extra[(rn0, inner)], Ld, inner)
                rplan = extra[(rn0, inner)]
            else:
                if inner != cur:
                    g.trsm_plan_mixed(plan, Ld, inner)
                    cur = inner
                rplan = plan
            s32 = smode in (True, "fp32")
            tc_planes = {"tc": 3, "tc2": 2, "tc1": 1}.get(smode)
            stc = tc_planes is not None
            def solve(X=None):
                try:
                    X, it, upd = g.trsm_solve_mixed(rplan, Bd, X=X, residual=res, max_iter=30, tol=tol,
                                                    raise_on_noconv=False, s_fp32=s32, s_tc=stc,
                                                    s_tc_planes=tc_planes or 3)
                    return X, it, upd, 0
                except binding.TrsmError as e:  # e.g. a non-finite working copy
                    return X, None, None, e.code
            X, it, upd, rc = solve()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            X, it, upd, rc = solve(X)
            torch.cuda.synchronize()
            tm = (time.perf_counter() - t0) * 1e3
            fe = ferr(X) if X is not None else None
            converged = bool(fe is not None and fe <= 1e-10)
            status = "ok" if converged else ("non-finite" if fe is None else "target missed")
            rec["mixed"].append({"inner": inner, "s_step": smode if stc else "fp32" if s32 else "fp64",
                                 "residual": res, "n0": rn0, "ms": round(tm, 2),
                                 "tflops_equiv": round(float(n) * n * k / (tm * 1e-3) / 1e12, 3),
                                 "iterations": it, "last_update": upd, "fwd_err": fe,
                                 "bwd_err": berr(X) if X is not None else None,
                                 "converged": converged, "status": status, "rc": rc,
                                 "speedup_vs_fp64": round(t64 / tm, 3)})
        for p_ in extra.values():
            p_.destroy()
        if with_sliced:
            # the sliced schedule: FP64-class products, one pass, no refinement,
            # on its own plan with 2048-row blocks (measured faster than 1024)
            splan = g.trsm_plan(Ld, min(SLICED_PREC_N0, n))
            g.trsm_plan_sliced(splan)
            X = g.trsm_solve_schedule(splan, Bd, schedule="sliced")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            X = g.trsm_solve_schedule(splan, Bd, X=X, schedule="sliced")
            e1.record()
            torch.cuda.synchronize()
            g.trsm_sync_status(splan)
            splan.destroy()
            tm = e0.elapsed_time(e1)
            fe = ferr(X)
            rec["mixed"].append({"inner": "sliced", "s_step": "sliced", "residual": None,
                                 "n0": min(SLICED_PREC_N0, n), "ms": round(tm, 2),
                                 "tflops_equiv": round(float(n) * n * k / (tm * 1e-3) / 1e12, 3),
                                 "iterations": 1, "last_update": None, "fwd_err": fe, "bwd_err": berr(X),
                                 "converged": bool(fe is not None and fe <= 1e-10),
                                 "status": "ok" if fe is not None and fe <= 1e-10 else (
                                     "non-finite" if fe is None else "target missed"), "rc": 0,
                                 "speedup_vs_fp64": round(t64 / tm, 3)})
        plan.destroy()
        del Ld, Bd, X64
        out.append(rec)
    return out


def compact_precision(recs):
    """Short records for the bench line: per c the FP64 solve's time and
    forward error, and per (c, inner format) the refined solve's time,
    sweeps, forward and backward errors, speed-up over FP64 and status
    ("ok": forward error <= 1e-10; "miss": finite but above; "nan": the
    solution or its reference is not finite)."""
    fp64 = {str(rec["c"]): [rec["fp64_solve_ms"], _sig(rec["fp64_fwd_err"])] for rec in recs}
    rows = []
    for rec in recs:
        for m in rec["mixed"]:
            st = "ok" if m["converged"] else ("nan" if m["fwd_err"] is None else "miss")
            rows.append([rec["c"], m["inner"], m["s_step"], m["residual"], m.get("n0", rec.get("n0")), m["ms"],
                         m["iterations"], _sig(m["fwd_err"]), _sig(m["bwd_err"]),
                         None if st == "nan" else m["speedup_vs_fp64"], st])
    return {"fp64": fp64,
            "cols": ["c", "inner", "s", "residual", "n0", "ms", "sweeps", "fwd", "bwd", "x_fp64", "status"],
            "rows": rows}


def _sig(v, digits=3):
    """A float rounded to `digits` significant digits (None stays None)."""
    if v is None:
        return None
    return float(f"{v:.{digits - 1}e}")


def n0_sweep_study(g, torch, dev_in, outs, shapes, sweep=None):
    """The block-size sweep: every shape x n0 in {64, 128, 256, 512, 1024,
    n}, plan and solve each timed once with CUDA events after one untimed
    run (n0 = n is the full inversion, Section 7.4)."""
    stream = torch.cuda.current_stream()
    res = {}
    for (n, k), (Ld, Bd), X in zip(shapes, dev_in, outs):
        rows = []
        for n0 in (sweep or SWEEP_N0):
            n0v = n if n0 is None else n0
            p = g.trsm_plan(Ld, n0v)
            g.trsm_solve(p, Bd, X=X)
            g.trsm_sync_status(p)
            p.destroy()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            p = g.trsm_plan(Ld, n0v)
            b.record(stream)
            g.trsm_solve(p, Bd, X=X)
            c.record(stream)
            g.trsm_sync_status(p)
            p.destroy()
            pm, sm_ = a.elapsed_time(b), b.elapsed_time(c)
            rows.append([n0v, round(pm, 1), round(sm_, 1), round(float(n) * n * k / ((pm + sm_) * 1e-3) / 1e12, 3)])
        res[f"{n}x{k}"] = rows
    return res


def residual_roofline(g, torch, n=16384, k=4096, reps=3):
    """The sliced FP64-class residual (the mixed path's dominant kernel) at
    n = 16384, k = 4096, as each refinement sweep runs it: L's digit planes
    come from the plan (trsm_plan_mixed), X is sliced inside the timed call,
    then the stream kernel forms R = B - L X.  bf16 MMA flops (P(P+1)/2
    plane pairs x 2 x n^2/2 x k) per call / CUDA-event time, against the bf16
    tensor peak; the slicing of X (about 1 % of the call) counts as time."""
    import ctypes
    lib = g.load_library()
    L = torch.tril(torch.rand(n, n, dtype=torch.float64, device="cuda") * 2 - 1) / n
    L.diagonal().copy_(2 + torch.rand(n, dtype=torch.float64, device="cuda"))
    L = L.t().contiguous().t()
    plan = g.trsm_plan(L, MIXED_N0)
    g.trsm_plan_mixed(plan, L, "fp16x3")
    del L
    X = (torch.rand(k, n, dtype=torch.float64, device="cuda") * 2 - 1).t()
    B = (torch.rand(k, n, dtype=torch.float64, device="cuda") * 2 - 1).t()
    R = torch.empty(k, n, dtype=torch.float64, device="cuda").t()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    burst, _, src = measured_peaks()
    out = {}
    for planes in (7, 8):
        def call():
            return lib.trsm_residual_plan(plan.handle, ctypes.c_void_p(X.data_ptr()), k, n,
                                          ctypes.c_void_p(B.data_ptr()), n, ctypes.c_void_p(R.data_ptr()), n,
                                          planes, ctypes.c_void_p(err.data_ptr()), s)
        assert call() == 0
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            call()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        flops = planes * (planes + 1) / 2 * float(n) * n * k
        achieved = flops / (ms * 1e-3) / 1e12
        out[f"planes{planes}"] = {"bound": "tensor", "kernel": "sliced stream_kernel (with the slicing of X)",
                                  "ms": round(ms, 3), "achieved": round(achieved, 1), "peak": burst,
                                  "unit": "TFLOP/s", "frac": round(achieved / burst, 4), "peak_source": src,
                                  "err_flag": int(err.item())}
    plan.destroy()
    del X, B, R
    return out


def batch_systems(torch, count, dtype, seed, choose_n0):
    """The batching workload: `count` systems, n log-uniform in [32, 1024], k
    log-uniform in [1, 256], diagonal U[2,3], strictly lower U[-1,1]/n, B
    U[-1,1], each drawn on the device from seed + index.  Returns (systems,
    sum of n^2 k)."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(32), np.log(1024), size=count))).astype(int)
    ks = np.rint(np.exp(rng.uniform(0.0, np.log(256), size=count))).astype(int)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    gen = torch.Generator(device="cuda")
    systems = []
    for i, (n, k) in enumerate(zip(ns, ks)):
        gen.manual_seed(seed + i)
        L = torch.rand((n, n), generator=gen, device="cuda", dtype=tdt).mul_(2).sub_(1).div_(int(n))
        L = torch.tril(L, -1)
        L.diagonal().copy_(torch.rand(int(n), generator=gen, device="cuda", dtype=tdt).add_(2))
        L = L.t().contiguous().t()
        B = torch.rand((int(k), int(n)), generator=gen, device="cuda", dtype=tdt).mul_(2).sub_(1).t()
        X = torch.empty((int(k), int(n)), device="cuda", dtype=tdt).t()
        c = choose_n0(int(n))
        n0, tile = c if isinstance(c, tuple) else (c, 0)
        systems.append({"L": L, "B": B, "X": X, "n0": n0, "tile_cols": tile})
    return systems, float(np.sum(ns.astype(np.float64) ** 2 * ks))


def batched_study(g, torch, count=4096, dtypes=("f64", "f32"), reps=5, seed=1000, fp64_peak=None, fp32_peak=None):
    """Batching workload: `count` independent systems, n log-uniform in
    [32, 1024], k log-uniform in [1, 256], diagonal U[2,3], strictly lower
    U[-1,1]/n, B U[-1,1] (drawn on the device from a per-system seed), all
    solved in one CUDA graph replay: FP64 by one persistent launch
    (in-launch inversion + blocked solve), FP32 by an inversion launch and a
    unit launch; n0 and tile widths per size bucket from the autotuner."""
    from paper_1612_01855_gb300 import autotune
    out = []
    for dtype in dtypes:
        table = autotune.tune_batch(dtype)
        systems, flops = batch_systems(torch, count, dtype, seed, lambda n: autotune.choose(n, dtype, table))
        batch = g.Batch(systems, dtype=dtype)
        batch.capture()
        for _ in range(2):
            batch.launch_graph()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            batch.launch_graph()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        rc = batch.status()[0]
        # spot check three systems against a plain solve of the same data
        err = 0.0
        for i in (0, count // 2, count - 1):
            sy = systems[i]
            ref = torch.linalg.solve_triangular(sy["L"].double(), sy["B"].double(), upper=False)
            err = max(err, float((sy["X"].double() - ref).abs().max() / ref.abs().max()))
        achieved = flops / (ms * 1e-3) / 1e12
        if dtype == "f64":
            peak, src = fp64_peak, "measured DFMA throughput (trsm_fp64_peak) in this run"
        else:
            peak, src = fp32_peak, "measured FFMA throughput (trsm_fp32_peak) in this run"
        out.append({"dtype": dtype, "systems": count, "ms_per_batch": round(ms, 3),
                    "tflops_n2k": round(achieved, 3), "status": rc,
                    "roofline": {"bound": "alu",
                                 "kernel": "batch_kernel" if dtype == "f64" else "inv32w_kernel + sys32_kernel",
                                 "achieved": round(achieved, 4),
                                 "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                                 "peak_source": src},
                    "n0_by_bucket": {f"{lo}-{hi - 1}": table[i][0] for i, (lo, hi) in enumerate(autotune.BUCKETS)},
                    "tile_cols_by_bucket": {f"{lo}-{hi - 1}": (table[i][1] or "by k")
                                            for i, (lo, hi) in enumerate(autotune.BUCKETS)},
                    "workspace_gb": round(batch.workspace_bytes() / 1e9, 3),
                    "spot_check_rel_err": err, "graph": True,
                    "inputs": "device-generated per-system seeds (torch Philox), config-0 distributions"})
        batch.destroy()
        del systems
    return out


def schedules_study(g, torch, dev_in, outs, shapes, n0s, reps=3, stream=None, fp64_peak=None):
    """Solve time of the three schedules of the blocked solve on the bench
    shapes (plan reused; solve only): the dependency-driven persistent kernel,
    the paper's right-looking loop with a look-ahead stream, and Rec-TRSM."""
    out = []
    for (Ld, Bd), X, (n, k), n0 in zip(dev_in, outs, shapes, n0s):
        p = g.trsm_plan(Ld, n0)
        rec = {"n": n, "k": k, "n0": n0}
        for sched in SCHEDULE_NAMES:
            g.trsm_solve_schedule(p, Bd, X=X, schedule=sched)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                g.trsm_solve_schedule(p, Bd, X=X, schedule=sched)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            ms = statistics.median(ts)
            tf = float(n) * n * k / (ms * 1e-3) / 1e12
            rec[sched] = {"solve_ms": round(ms, 3), "tflops": round(tf, 4)}
            if fp64_peak:
                rec[sched]["frac_of_measured_dfma"] = round(tf / fp64_peak, 4)
        rec["autotuned"] = min(SCHEDULE_NAMES, key=lambda x: rec[x]["solve_ms"])
        g.trsm_sync_status(p)
        p.destroy()
        out.append(rec)
    return out


def sliced_mma_flops(n, k, nb):
    """BF16 tensor-core flops of one sliced solve: 36 digit-plane pairs for
    every product; the updates W(T_{i+1}) -= L(T_{i+1}, S_i) X_i take
    2 (n - (i+1) nb) nb k each, the diagonal multiplies 2 m_i^2 k / 2 (the
    strictly lower part of each inverted block)."""
    N = -(-n // nb)
    upd = sum(2.0 * (n - (i + 1) * nb) * nb * k for i in range(N - 1))
    diag = sum(float(min(nb, n - i * nb)) ** 2 * k for i in range(N))
    return 36.0 * (upd + diag)


def sliced_study(g, torch, data, dev_in, outs, shapes, reps=3):
    """The sliced schedule (both matrix multiplies as FP64-class digit-sliced
    products on the BF16 tensor cores) on the FP64 sweep shapes at its own
    block size: plan (inversion, then digit planes) and solve times, TFLOP/s
    (n^2 k), the relative error of sampled columns against the oracle, and
    the tensor-core roofline of the solve."""
    import oracle
    burst, _, src = measured_peaks()
    rows = {}
    for (L, B), (Ld, Bd), X, (n, k) in zip(data, dev_in, outs, shapes):
        nb = SLICED_N0[(n, k)]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        p = g.trsm_plan(Ld, nb)
        ev[1].record()
        g.trsm_plan_sliced(p)
        ev[2].record()
        torch.cuda.synchronize()
        plan_ms, planes_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        g.trsm_solve_schedule(p, Bd, X=X, schedule="sliced")
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.trsm_solve_schedule(p, Bd, X=X, schedule="sliced")
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        g.trsm_sync_status(p)
        ms = statistics.median(ts)
        cols = np.array([0, k // 2, k - 1])
        want = oracle.forward_subst_columns(L, B, cols)
        got = X[:, torch.from_numpy(cols).cuda()].cpu().numpy()
        err = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
        mma = sliced_mma_flops(n, k, nb) / (ms * 1e-3) / 1e12
        rows[f"{n}x{k}"] = [nb, round(plan_ms, 2), round(planes_ms, 2), round(ms, 2),
                            round(float(n) * n * k / (ms * 1e-3) / 1e12, 2), _sig(err), round(mma / burst, 3)]
        p.destroy()
    return {"cols": ["n0", "plan_ms", "planes_ms", "solve_ms", "solve_tflops", "rel_err", "mma_frac"],
            **rows, "mma_peak": burst}


def serving_study(g, torch, nL=256, rates=(100, 300, 600, 1200, 2400), per_rate=300, seed=2000,
                  budget_gb=150.0, mixed_min_n=2048, sliced_min_flops=3e8, streams=8, mixed_s="tc2"):
    """Serving workload: nL resident L (n log-uniform in [64, 8192],
    diagonal U[2,3], strictly lower U[-1,1]/n, drawn on the device), each
    planned once; Poisson request streams at the given rates, each request a
    B with k log-uniform in [1, 2048] for a random resident L; continuous
    batching under an HBM budget.  The L with n >= mixed_min_n also carry a
    mixed-precision plan (split-fp16 updates), and half of the requests on
    them ask for the refined mixed-precision solve (tol 1e-12; diagonal
    multiplies as `mixed_s`: two tf32 planes on the tensor cores) instead of
    FP64.  The same L also carry the sliced schedule's digit planes, and an
    FP64 request of at least sliced_min_flops n^2 k flops is solved by the
    sliced schedule (FP64-class, on the tensor cores) instead of joining a
    batch.  Reports solves/s and p50/p99 latency, overall and for the mixed
    requests."""
    from paper_1612_01855_gb300.serve import Request, Server
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(64), np.log(8192), size=nL))).astype(int)
    gen = torch.Generator(device="cuda")
    plans = []
    t0 = time.perf_counter()
    for i, n in enumerate(ns):
        gen.manual_seed(seed + i)
        L = torch.rand((int(n), int(n)), generator=gen, device="cuda", dtype=torch.float64).mul_(2).sub_(1).div_(int(n))
        L = torch.tril(L, -1)
        L.diagonal().copy_(torch.rand(int(n), generator=gen, device="cuda", dtype=torch.float64).add_(2))
        L = L.t().contiguous().t()
        plans.append(g.trsm_plan(L, 256 if n >= 1024 else 64))
        if n >= mixed_min_n:
            g.trsm_plan_mixed(plans[-1], L, "fp16x3")
            g.trsm_plan_sliced(plans[-1])
        del L
    plan_s = time.perf_counter() - t0
    out = {"resident_L": nL, "plan_seconds": round(plan_s, 2),
           "mixed_plans": int(sum(1 for n in ns if n >= mixed_min_n)),
           "resident_gb": round(sum(p.device_bytes() for p in plans) / 1e9, 2), "budget_gb": budget_gb,
           "rates": []}
    for rate in rates:
        reqs = []
        t = 0.0
        for rid in range(per_rate):
            t += rng.exponential(1.0 / rate)
            lid = int(rng.integers(0, nL))
            k = int(np.rint(np.exp(rng.uniform(0.0, np.log(2048)))))
            gen.manual_seed(seed * 7 + rid)
            B = torch.rand((k, int(ns[lid])), generator=gen, device="cuda", dtype=torch.float64).mul_(2).sub_(1).t()
            mixed = bool(ns[lid] >= mixed_min_n and rng.random() < 0.5)
            reqs.append(Request(rid, lid, B, t, mixed=mixed))
        torch.cuda.synchronize()
        srv = Server(plans, budget_bytes=int(budget_gb * 1e9), streams=streams, max_batch=64,
                     sliced_min_flops=sliced_min_flops, mixed_s=mixed_s)
        st = srv.run_trace(reqs)
        st["offered_rate"] = rate
        out["rates"].append({k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()})
        # accuracy of a few served requests of each kind against a plain FP64 solve
        errs = {"fp64": 0.0, "mixed": 0.0}
        for r in [x for x in reqs if not x.mixed][:3] + [x for x in reqs if x.mixed][:3]:
            ref = g.trsm_solve(plans[r.lid], r.B)
            g.trsm_sync_status(plans[r.lid])
            e = float((r.X - ref).abs().max() / ref.abs().max())
            key = "mixed" if r.mixed else "fp64"
            errs[key] = max(errs[key], e)
        out["rates"][-1]["max_rel_diff_vs_fp64_solve"] = errs
        del reqs, srv
    for p in plans:
        p.destroy()
    return out


def run_case(args):
    """Single kernels for profiling (no JSON bench line):
    sliced:N:K[:P]   the tensor-core residual R = B - L X with P (7 or 8)
                     digit planes, twice;
    mixed:N:K:N0[:I[:S]]  one mixed-precision refined solve (graded diagonal,
                     c = 2); inner I = 0 tf32, 1 bf16, 2 split bf16, 3 split
                     fp16; S = 1 for the FP32 diagonal-block multiply, 2, 3
                     or 4 for the tensor-core one with 3, 2 or 1 tf32 planes;
    sched:N:K:N0     the sliced schedule of the FP64 solve (well-conditioned
                     L), its digit planes made first, then two solves;
    engine:M:N:K     the bf16 tensor-core GEMM self-test, twice;
    batch:COUNT:BITS[:N0] one batched launch of COUNT systems of the
                     batching workload in FP64 (BITS = 64) or FP32 (32),
                     twice; n0 = N0 for every system, else 32 below n = 256
                     and 64 above."""
    import ctypes
    import torch
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300 import build as pkg_build
    pkg_build.build()
    lib = g.load_library()
    kind, *dims = args.case.split(":")
    dims = [int(v) for v in dims]
    torch.manual_seed(0)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    if kind in ("sliced", "mixed"):
        n, k = dims[0], dims[1]
        L = torch.tril(torch.rand(n, n, dtype=torch.float64, device="cuda") * 2 - 1) / n
        if kind == "mixed":
            d = torch.from_numpy(np.geomspace(1.0, 1e-2, n)).cuda()[torch.randperm(n, device="cuda")]
        else:
            d = 2 + torch.rand(n, dtype=torch.float64, device="cuda")
        L.diagonal().copy_(d)
        L = L.t().contiguous().t()
        B = (torch.rand(k, n, dtype=torch.float64, device="cuda") * 2 - 1).t()
        if kind == "sliced":
            X = (torch.rand(k, n, dtype=torch.float64, device="cuda") * 2 - 1).t()
            R = torch.empty(k, n, dtype=torch.float64, device="cuda").t()
            for _ in range(2):
                rc = lib.trsm_residual_sliced(ctypes.c_void_p(L.data_ptr()), n, n, ctypes.c_void_p(X.data_ptr()), k,
                                              n, ctypes.c_void_p(B.data_ptr()), n, ctypes.c_void_p(R.data_ptr()),
                                              n, dims[2] if len(dims) > 2 else 7, ctypes.c_void_p(err.data_ptr()), s)
                assert rc == 0
        else:
            inner = ("tf32", "bf16", "bf16x3", "fp16x3")[dims[3]] if len(dims) > 3 else "tf32"
            plan = g.trsm_plan(L, dims[2])
            g.trsm_plan_mixed(plan, L, inner)
            sm = dims[4] if len(dims) > 4 else 0
            g.trsm_solve_mixed(plan, B, max_iter=30, tol=1e-11, raise_on_noconv=False, s_fp32=sm == 1,
                               s_tc=sm in (2, 3, 4), s_tc_planes={2: 3, 3: 2, 4: 1}.get(sm, 3))
    elif kind == "sched":
        n, k, n0 = dims
        L = torch.tril(torch.rand(n, n, dtype=torch.float64, device="cuda") * 2 - 1) / n
        L.diagonal().copy_(2 + torch.rand(n, dtype=torch.float64, device="cuda"))
        L = L.t().contiguous().t()
        B = (torch.rand(k, n, dtype=torch.float64, device="cuda") * 2 - 1).t()
        plan = g.trsm_plan(L, n0)
        g.trsm_plan_sliced(plan)
        X = torch.empty(k, n, dtype=torch.float64, device="cuda").t()
        for _ in range(2):
            g.trsm_solve_schedule(plan, B, X=X, schedule="sliced")
        g.trsm_sync_status(plan)
    elif kind == "engine":
        M, N, K = dims
        A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
        Bm = torch.randn(N, K, device="cuda").to(torch.bfloat16)
        C = torch.empty(N, M, device="cuda", dtype=torch.float32)
        for _ in range(2):
            assert lib.trsm_tc_gemm_selftest(0, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(Bm.data_ptr()),
                                             ctypes.c_void_p(C.data_ptr()), M, N, K,
                                             ctypes.c_void_p(err.data_ptr()), s) == 0
    elif kind == "batch":
        dtype = "f64" if dims[1] == 64 else "f32"
        rule = (lambda n: dims[2]) if len(dims) > 2 else (lambda n: 32 if n < 256 else 64)
        systems, _ = batch_systems(torch, dims[0], dtype, 1000, rule)
        batch = g.Batch(systems, dtype=dtype)
        for _ in range(2):
            batch.run()
        assert batch.status()[0] == 0
        batch.destroy()
    else:
        raise SystemExit(f"unknown case {kind}")
    torch.cuda.synchronize()
    assert err.item() == 0
    print(f"case {args.case} done")


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle on the host cores, bounded samples."""
    if rank != 0:
        return
    shapes = SHAPES
    data = make_inputs(shapes)
    # each step: a bounded column sample of every shape
    import oracle
    cores = oracle.max_threads()
    cols = [max(cores, 1)] * len(shapes)
    for _ in range(args.warmup):
        for (L, B), c in zip(data, cols):
            oracle.forward_subst(L, B[:, :c])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for (L, B), c in zip(data, cols):
            oracle.forward_subst(L, B[:, :c])
        times.append(time.perf_counter() - t0)
    fl = sum(float(n) * n * c for (n, k), c in zip(shapes, cols))
    t = sum(times) / len(times)
    value = fl / t / 1e12
    sample = "; ".join(f"n={n}: {c} of {k} columns" for (n, k), c in zip(shapes, cols))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded PCG64)",
        "config": {"workload": "fp64 k/n sweep shapes (16384,256),(8192,8192),(2048,131072); "
                               "CPU oracle forward substitution on a column sample per step"},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300 import build as pkg_build

    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(pkg_build.LIB):
        pkg_build.build()
    if world > 1:
        torch.distributed.barrier()
    g.load_library()
    shapes, n0s = SHAPES, [DEFAULT_N0[s] for s in SHAPES]
    if args.shapes:  # override (profiling of small cases): "n:k:n0,n:k:n0"
        trip = [tuple(int(v) for v in item.split(":")) for item in args.shapes.split(",")]
        shapes, n0s = [(a, b) for a, b, _ in trip], [c for _, _, c in trip]
    data = make_inputs(shapes)
    dev_in = [(to_dev(L, torch), to_dev(B, torch)) for L, B in data]
    outs = [torch.empty((k, n), dtype=torch.float64, device="cuda").t() for n, k in shapes]
    stream = torch.cuda.current_stream()

    def step(timers=None):
        for si, ((Ld, Bd), X, n0) in enumerate(zip(dev_in, outs, n0s)):
            if timers is not None:
                timers[si][0].record(stream)
            p = g.trsm_plan(Ld, n0)
            if timers is not None:
                timers[si][1].record(stream)
            g.trsm_solve(p, Bd, X=X)
            if timers is not None:
                timers[si][2].record(stream)
            g.trsm_sync_status(p)
            p.destroy()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    fp64_peak = g.fp64_peak(8192)
    fp32_peak = g.fp32_peak(16384)
    sms, fp64_nominal, fp32_nominal = nominal_peaks()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    g.launch_count(reset=True)
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in shapes]
          for _ in range(args.steps)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        step(ev[s])
    e1.record(stream)
    torch.cuda.synchronize()
    launches = g.launch_count()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
    ms_per_step = total_ms / args.steps
    flops_step = sum(float(n) * n * k for n, k in shapes)
    value = replica_throughput(flops_step, world, ms_per_step) / 1e12

    per_shape = []
    solve_ms_tot, solve_flops_tot = 0.0, 0.0
    for si, ((n, k), n0) in enumerate(zip(shapes, n0s)):
        plan_ms = statistics.median(ev[s][si][0].elapsed_time(ev[s][si][1]) for s in range(args.steps))
        solve_ms = statistics.median(ev[s][si][1].elapsed_time(ev[s][si][2]) for s in range(args.steps))
        solve_ms_tot += solve_ms
        solve_flops_tot += float(n) * n * k
        per_shape.append({"n": n, "k": k, "n0": n0, "plan_ms": round(plan_ms, 3),
                          "solve_ms": round(solve_ms, 3),
                          "tflops": round(float(n) * n * k / ((plan_ms + solve_ms) * 1e-3) / 1e12, 4)})
    solve_achieved = solve_flops_tot / (solve_ms_tot * 1e-3) / 1e12

    # parity check of this run's results on a few sampled columns (oracle),
    # and their backward error ||B - L X|| / (||L|| ||X||) (infinity norm)
    err, bwd = None, None
    if rank == 0 and not args.no_check:
        import oracle
        errs, bwds = [], []
        for (L, B), X, (Ld, Bd) in zip(data, outs, dev_in):
            cols = np.array([0, B.shape[1] // 2, B.shape[1] - 1])
            want = oracle.forward_subst_columns(L, B, cols)
            ci = torch.from_numpy(cols).cuda()
            got = X[:, ci].cpu().numpy()
            errs.append(float(np.max(np.abs(got - want)) / np.max(np.abs(want))))
            Lt = torch.tril(Ld)
            Xs = X[:, ci]
            r = (Bd[:, ci] - Lt @ Xs).abs().max().item()
            bwds.append(r / (Lt.abs().sum(dim=1).max().item() * Xs.abs().max().item()))
            del Lt
        err, bwd = max(errs), max(bwds)

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        pinned = []
        for (L, B), (n, k) in zip(data, shapes):
            Lh = torch.from_numpy(np.ascontiguousarray(L.T)).pin_memory()
            Bh = torch.from_numpy(np.ascontiguousarray(B.T)).pin_memory()
            Xh = torch.empty((k, n), dtype=torch.float64).pin_memory()
            pinned.append((Lh, Bh, Xh))
        sptr = stream.cuda_stream

        def e2e_step():
            for (Lh, Bh, Xh), (n, k), n0 in zip(pinned, shapes, n0s):
                g.trsm_host_ptr(Lh.data_ptr(), n, n, n0, Bh.data_ptr(), k, n, Xh.data_ptr(), n, sptr)

        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / max(1, args.steps)
        # the lower trapezoid of each block column of L, then B
        h2d = sum(8 * (sum((n - b0) * min(n0, n - b0) for b0 in range(0, n, n0)) + n * k)
                  for (n, k), n0 in zip(shapes, n0s))
        d2h = sum(8 * n * k for n, k in shapes)
        e2e = {"value": round(flops_step * world / e2e_s / 1e12, 4), "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": round(e2e_s * 1e3, 2)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, sample, cores = cpu_oracle_rate(data, shapes, args.cpu_budget)
        cpu = {"value": round(rate, 5), "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
               "sample": sample + " cols"}

    mixed = None
    residual = None
    if rank == 0 and not args.no_mixed and not args.shapes:
        residual = residual_roofline(g, torch)
    if rank == 0 and not args.no_mixed and not args.shapes:
        # config 2 at c = 2, 4, 6 at the mixed path's block size: refined
        # solves (split-fp16 updates with FP64, FP32 or two-tf32-plane
        # tensor-core diagonal multiplies, tf32 updates with tensor-core ones
        # of three planes; the adaptive residual, and eight planes throughout
        # for one of them), and the sliced schedule's direct FP64-class
        # solve.  The FP64 multiply runs on its own plan with 256-row blocks
        # (its DFMA work grows with n0: 120.7 ms at c = 2 against 236.6 at
        # n0 = 1024)
        mixed = precision_study(g, torch, 16384, 4096, MIXED_N0, [2, 4, 6], None, None,
                                combos=[("fp16x3", "fp64", "adaptive", 256), ("fp16x3", "fp32", "adaptive"),
                                        ("fp16x3", "tc2", "adaptive"), ("fp16x3", "tc2", "sliced8"),
                                        ("tf32", "tc", "adaptive")],
                                with_sliced=True)

    batched = None
    if rank == 0 and not args.no_batched and not args.shapes:
        batched = batched_study(g, torch, fp64_peak=fp64_peak, fp32_peak=fp32_peak)

    serving = None
    if rank == 0 and not args.no_serving and not args.shapes:
        serving = serving_study(g, torch)

    schedules = None
    if rank == 0 and not args.no_schedules:
        schedules = schedules_study(g, torch, dev_in, outs, shapes, n0s, fp64_peak=fp64_peak)

    sweep = None
    if rank == 0 and not args.no_sweep and not args.shapes:
        sweep = n0_sweep_study(g, torch, dev_in, outs, shapes)

    sliced = None
    if rank == 0 and not args.no_schedules and not args.shapes:
        sliced = sliced_study(g, torch, data, dev_in, outs, shapes)

    if args.precision and rank == 0:
        for rec in precision_study(g, torch, 16384, 4096, MIXED_N0, [2, 4, 6], ["tf32", "bf16", "bf16x3", "fp16x3"],
                                   [False, True], residuals=("sliced", "adaptive")):
            print(json.dumps({"precision_study": True, **rec}), flush=True)

    if rank == 0:
        traffic, traffic_by_shape = solve_traffic(shapes, n0s)
        details = {"per_shape": per_shape, "traffic_by_shape": traffic_by_shape, "mixed_precision": mixed,
                   "residual_roofline": residual, "batched": batched, "serving": serving,
                   "schedules": schedules, "n0_sweep": sweep, "fp64_sliced": sliced}
        if args.details:
            with open(args.details, "w") as fh:
                json.dump(details, fh, indent=1)
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PCG64)",
            "config": {"workload": "fp64 k/n sweep (n,k) = (16384,256),(8192,8192),(2048,131072); "
                                   "step = trsm_plan + trsm_solve per shape",
                       "n0": {f"{n}x{k}": n0 for (n, k), n0 in zip(shapes, n0s)},
                       "flops_per_step": flops_step, "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas{world}" if world > 1 else "single GPU"},
            "roofline": {"bound": "alu", "kernel": "it_inv_solve_kernel",
                         "achieved": round(solve_achieved, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                         "frac": round(solve_achieved / fp64_peak, 4),
                         "peak_source": f"measured DFMA (nominal {fp64_nominal:.3f})",
                         "traffic": traffic},
            "parity_max_rel_err": _sig(err),
            "backward_err": _sig(bwd),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clk,
            "fp32_peak": round(fp32_peak, 2),
        }
        if sweep is not None:
            line["n0_sweep"] = {"cols": ["n0", "plan_ms", "solve_ms", "tflops"], **sweep}
        if sliced is not None:
            line["fp64_sliced"] = sliced
        if mixed is not None:
            line["precision"] = compact_precision(mixed)
        if residual is not None:
            line["residual_roofline"] = {key: {"ms": round(v["ms"], 2), "frac": round(v["frac"], 3)}
                                         for key, v in residual.items()}
        if batched is not None:
            line["batched"] = [{"dtype": b["dtype"], "ms": b["ms_per_batch"], "tflops": b["tflops_n2k"],
                                "frac": b["roofline"]["frac"], "peak": b["roofline"]["peak"],
                                "status": b["status"], "err": _sig(b["spot_check_rel_err"])} for b in batched]
        if serving is not None:
            line["serving"] = {"cols": ["offered", "served", "p50_ms", "p99_ms", "fp64_p99_ms", "mixed_p99_ms",
                                        "wait_p50_ms", "wait_p99_ms", "sliced", "ok"],
                               "rates": [[r["offered_rate"], round(r["solves_per_s"], 1), round(r["p50_ms"], 1),
                                          round(r["p99_ms"], 1), round(r.get("fp64", {}).get("p99_ms", 0.0), 1),
                                          round(r.get("mixed", {}).get("p99_ms", 0.0), 1),
                                          round(r.get("wait_p50_ms", 0.0), 2), round(r.get("wait_p99_ms", 0.0), 1),
                                          r["sliced_requests"], r["statuses_ok"]]
                                         for r in serving["rates"]],
                               "slots": serving["rates"][0]["slots"] if serving["rates"] else None}
        if schedules is not None:
            line["schedules_ms"] = {f"{r['n']}x{r['k']}": {key: round(r[key]["solve_ms"], 1) for key in SCHEDULE_NAMES
                                                           if key in r} for r in schedules}
        print(json.dumps(line, separators=(",", ":")), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision refinement figure")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-systems figure")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving figure")
    ap.add_argument("--no-schedules", action="store_true", help="skip the solve-schedule comparison")
    ap.add_argument("--no-sweep", action="store_true", help="skip the n0 sweep")
    ap.add_argument("--details", default="", help="also write every study's full records to this JSON file")
    ap.add_argument("--precision", action="store_true", help="print the full c x inner x s-step study")
    ap.add_argument("--case", default="", help="profiling case: sliced:N:K[:PLANES], mixed:N:K:N0[:INNER[:S]], "
                                               "sched:N:K:N0, engine:M:N:K, batch:COUNT:BITS[:N0]")
    ap.add_argument("--shapes", default="", help="override workload, e.g. 6144:1024:256 (not a bench line)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
