"""Continuous-batching solve server over resident plans.

Each L is planned once (`trsm_plan`: its inverted diagonal blocks stay in
HBM), so a request — a right-hand side B for one of the resident L — only
pays for the blocked solve (Algorithm It-Inv-TRSM, Section 6.2).  The loop:

* requests wait in queues, each in arrival order: FP64 requests, requests
  for the refined mixed-precision solve (`mixed=True`; its plan needs
  `trsm_plan_mixed`), and large FP64 requests for the sliced schedule (below);
* whenever one of `streams` launch slots is free, it takes work: the FP64
  requests at the head of their queue, admitted while their memory (B, X and
  the batch's share of the workspace) fits in the HBM budget next to the
  resident plans, run as ONE persistent batched launch (`trsm_batch_*` with
  resident plans, laid out in an arena from torch's caching allocator: no
  device allocation by the library);
* a mixed-precision solve decides on the host when to stop refining, so it
  cannot join a persistent batch: it takes a slot alone and runs in a worker
  thread on the slot's stream (the C call releases the interpreter lock).
  At most `mixed_slots` slots hold such solves at a time, so the other slots
  always keep serving FP64 batches.  `mixed_s` picks its diagonal
  multiplies: "tc2" (default: two tf32 planes on the tensor cores), "tc",
  "fp32" or "fp64" (the DFMA pipe, which then dominates the solve);
* with `sliced_min_flops` set, an FP64 request of at least that many n^2 k
  flops whose plan carries the sliced schedule's digit planes
  (`trsm_plan_sliced`) waits in a third queue and is solved alone on a slot
  by the sliced schedule (FP64-class products on the tensor cores, 10-20x
  the DFMA rate on large systems): the largest requests, which set the
  latency tail at the DFMA rate, then take a fraction of the time;
* between the queues a free slot goes to whichever head arrived first,
  unless that head cannot start (a mixed request while every mixed slot is
  taken, or a request whose memory does not fit yet): then another queue's
  head may pass it.  No request waits behind one of another kind;
* batches run on different streams overlap on the device; a request that
  arrives while others are on the GPU is admitted as soon as a slot and
  memory free up;
* latency = completion seen by the host - arrival.

Stream order: a request's B may still be in production on the caller's
stream when it is submitted (an asynchronous copy or kernel).  `submit`
records an event on the caller's current stream; the slot stream waits on it
before reading B, and B is marked as used on the slot stream so that the
caching allocator does not hand its memory out again before the solve ends.

Memory outside the budget: the mixed and sliced solves take their scratch
from the library's workspace pool, which keeps freed memory mapped for the
next call.  The admission counts each such request's scratch while it runs;
what the pool holds afterwards (at most the largest scratch the mixed slots
needed at once) is not counted, so leave that much headroom below the
device's memory, or call `workspace_trim()` between traces.

Results do not depend on the traffic: an FP64 request's X is the same bits
whichever requests share its batch (every tile's updates are applied in a
fixed order), and a mixed request's refined solve, like a large request's
sliced solve, runs alone with its own fixed sequence of kernels.
"""
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import binding


class AdmissionError(ValueError):
    pass


class Admission:
    """HBM budget bookkeeping (host only): resident bytes are fixed, each
    admitted request holds its bytes until released."""

    def __init__(self, budget_bytes, resident_bytes=0):
        if resident_bytes > budget_bytes:
            raise AdmissionError("resident plans exceed the HBM budget")
        self.budget = int(budget_bytes)
        self.resident = int(resident_bytes)
        self.in_use = 0
        self.peak = 0

    def fits(self, nbytes):
        return self.resident + self.in_use + nbytes <= self.budget

    def check_request(self, nbytes):
        """A request larger than the whole free budget can never run."""
        if self.resident + nbytes > self.budget:
            raise AdmissionError(f"request needs {nbytes} bytes, budget leaves {self.budget - self.resident}")

    def take(self, nbytes):
        if not self.fits(nbytes):
            return False
        self.in_use += nbytes
        self.peak = max(self.peak, self.in_use)
        return True

    def release(self, nbytes):
        self.in_use -= nbytes
        if self.in_use < 0:
            raise AdmissionError("released more than admitted")


@dataclass
class Request:
    rid: int
    lid: int
    B: object            # CUDA tensor, column-major n x k, float64
    arrival: float       # seconds (host clock)
    X: object = None
    t_admit: float = None
    t_done: float = None
    cancelled: bool = False
    mixed: bool = False  # mixed-precision solve refined to `tol` (max|D| / max|X|)
    tol: float = 1e-12
    status: int = None
    iterations: int = None
    ready: object = None  # CUDA event recorded at submission on the caller's stream
    sliced: bool = False  # routed to the sliced schedule (set at submission)

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival


@dataclass
class _InFlight:
    batch: object
    event: object
    reqs: list
    nbytes: int
    arena: object = field(default=None)
    future: object = None  # a mixed-precision request's worker
    slot: int = 0
    plan: object = None    # a sliced solve's plan (its status word is read at completion)


def _has_mixed_data(plan):
    return getattr(plan, "inner", None) is not None


class Server:
    # keyword arguments of trsm_solve_mixed for each diagonal-multiply mode
    MIXED_S = {"fp64": {}, "fp32": {"s_fp32": True}, "tc": {"s_tc": True, "s_tc_planes": 3},
               "tc2": {"s_tc": True, "s_tc_planes": 2}}

    def __init__(self, plans, budget_bytes, streams=8, max_batch=64, mixed_slots=None,
                 mixed_residual="adaptive", sliced_min_flops=None, mixed_s="tc2"):
        if streams < 1:
            raise ValueError("at least one launch slot")
        if mixed_s not in self.MIXED_S:
            raise ValueError(f"mixed_s must be one of {sorted(self.MIXED_S)}, not {mixed_s!r}")
        self.mixed_s = mixed_s
        self.plans = plans
        resident = sum(self.plan_bytes(p) for p in plans)
        self.adm = Admission(budget_bytes, resident)
        self.mixed_residual = mixed_residual
        self.pool = None
        self.queue_fp64 = deque()
        self.queue_mixed = deque()
        self.queue_sliced = deque()
        self.sliced_min_flops = sliced_min_flops
        self.inflight = []
        self.done = []
        self.nstreams = streams
        # slots that may hold a mixed-precision solve at once: half of them,
        # at least one; with a single slot the two kinds take turns
        self.mixed_slots = max(1, streams // 2) if mixed_slots is None else int(mixed_slots)
        self.streams = None  # created at the first dispatch (host-side logic runs without a GPU)
        self.busy = [False] * streams
        self.mixed_busy = 0
        self.max_batch = max_batch
        self.launches = 0

    @property
    def pending(self):
        """Requests not admitted yet, in arrival order."""
        return sorted(list(self.queue_fp64) + list(self.queue_mixed) + list(self.queue_sliced),
                      key=lambda r: (r.arrival, r.rid))

    @staticmethod
    def plan_bytes(plan):
        """Device bytes a resident plan holds (the library's count when the
        plan can tell, else L~ alone)."""
        f = getattr(plan, "device_bytes", None)
        return f() if f is not None else 8 * plan.n * plan.n

    def routes_sliced(self, plan, k, mixed=False):
        """Whether an FP64 request goes to the sliced schedule."""
        return (not mixed and self.sliced_min_flops is not None and getattr(plan, "sliced", False)
                and float(plan.n) * plan.n * k >= self.sliced_min_flops)

    @staticmethod
    def request_bytes(n, k, mixed=False, sliced_block=0):
        if sliced_block:
            # X, and the sliced solve's workspace: W (FP64), the digit planes
            # of one block row of W and of X (eight bf16 planes each)
            return 16 * n * k + 2 * 16 * k * sliced_block + 4 * k + (1 << 16)
        if mixed:
            # X, and the refinement's workspace: R, D (FP64), W (FP32), the
            # eight digit planes of X (bf16), the float-float partial sums
            return (8 + 8 + 8 + 4 + 16 + 8) * n * k + (1 << 16)
        # B and X, the working copy W inside the batch workspace, counters
        return 3 * 8 * n * k + 4 * ((n + 31) // 32) * ((k + 31) // 32) * 2 + 4096

    def submit(self, req):
        plan = self.plans[req.lid]
        if req.B.shape[0] != plan.n:
            raise AdmissionError(f"request {req.rid}: B has {req.B.shape[0]} rows, L has {plan.n}")
        if req.mixed and not _has_mixed_data(plan):
            raise AdmissionError(f"request {req.rid}: mixed precision asked for, but L #{req.lid} has no "
                                 "mixed-precision plan (trsm_plan_mixed)")
        req.sliced = self.routes_sliced(plan, req.B.shape[1], req.mixed)
        self.adm.check_request(self._bytes(req))
        if getattr(req.B, "is_cuda", False):
            torch = self._torch()
            req.ready = torch.cuda.Event()
            req.ready.record(torch.cuda.current_stream(req.B.device))
        (self.queue_mixed if req.mixed else self.queue_sliced if req.sliced else self.queue_fp64).append(req)

    def _bytes(self, r):
        plan = self.plans[r.lid]
        return self.request_bytes(plan.n, r.B.shape[1], r.mixed, min(plan.n0, plan.n) if r.sliced else 0)

    def cancel(self, rid):
        """Drops a request that has not been admitted yet."""
        for q in (self.queue_fp64, self.queue_mixed, self.queue_sliced):
            for r in q:
                if r.rid == rid:
                    r.cancelled = True
                    q.remove(r)
                    return True
        return False

    def poll(self):
        still = []
        for f in self.inflight:
            if f.future is not None:
                if not f.future.done():
                    still.append(f)
                    continue
                r = f.reqs[0]
                r.t_done = time.perf_counter()
                try:
                    r.status, r.iterations = f.future.result()
                except Exception:  # a failure outside the library (e.g. the runtime): report, keep serving
                    r.status, r.iterations = binding.TRSM_ECUDA, None
                self.done.append(r)
                self.adm.release(f.nbytes)
                self.busy[f.slot] = False
                self.mixed_busy -= 1
                continue
            if f.event.query():
                now = time.perf_counter()
                if f.batch is None:  # a sliced solve: the plan's status word (the stream has completed)
                    try:
                        with self._torch().cuda.stream(self.streams[f.slot]):
                            binding.trsm_sync_status(f.plan)
                        rc = 0
                    except binding.TrsmError as e:
                        rc = e.code
                    r = f.reqs[0]
                    r.t_done = now
                    r.status = rc
                    self.done.append(r)
                    self.adm.release(f.nbytes)
                    self.busy[f.slot] = False
                    continue
                with self._torch().cuda.stream(self.streams[f.slot]):
                    rc = f.batch.status()[0]  # the stream has completed: no wait
                for r in f.reqs:
                    r.t_done = now
                    r.status = rc
                    self.done.append(r)
                f.batch.destroy()
                self.adm.release(f.nbytes)
                self.busy[f.slot] = False
            else:
                still.append(f)
        self.inflight = still

    @staticmethod
    def _torch():
        import torch
        return torch

    @staticmethod
    def _order_after_submission(r, stream):
        """The slot stream waits for B's producer; B stays allocated until
        the slot stream's work on it is done."""
        if r.ready is not None:
            stream.wait_event(r.ready)
        if getattr(r.B, "is_cuda", False):
            r.B.record_stream(stream)

    def mixed_kwargs(self):
        """The diagonal-multiply flags the server's mixed solves use."""
        return dict(self.MIXED_S[self.mixed_s])

    def _solve_mixed(self, slot, r):
        """Worker: one refined mixed-precision solve on the slot's stream.
        Returns (status, iterations)."""
        import torch
        with torch.cuda.stream(self.streams[slot]):
            try:
                _, it, _ = binding.trsm_solve_mixed(self.plans[r.lid], r.B, X=r.X, residual=self.mixed_residual,
                                                    tol=r.tol, **self.mixed_kwargs())
                return 0, it
            except binding.TrsmError as e:
                return e.code, None

    def _next_kind(self):
        """Which queue a free slot serves: "fp64", "mixed", "sliced" or None
        (the arrival-order rule of the module docstring)."""
        heads = []
        if self.queue_mixed and self.mixed_busy < self.mixed_slots:
            heads.append(("mixed", self.queue_mixed[0]))
        if self.queue_fp64:
            heads.append(("fp64", self.queue_fp64[0]))
        if self.queue_sliced:
            heads.append(("sliced", self.queue_sliced[0]))
        ready = [(r.arrival, r.rid, kind) for kind, r in heads if self.adm.fits(self._bytes(r))]
        return min(ready)[2] if ready else None

    def _take_fp64(self):
        """FP64 requests from the head of their queue that fit together."""
        take, nbytes = [], 0
        while self.queue_fp64 and len(take) < self.max_batch:
            r = self.queue_fp64[0]
            b = self._bytes(r)
            if not self.adm.fits(nbytes + b):
                break
            take.append(self.queue_fp64.popleft())
            nbytes += b
        return take, nbytes

    def dispatch(self):
        import torch
        if self.streams is None:
            self.streams = [torch.cuda.Stream() for _ in range(self.nstreams)]
        for slot in range(len(self.streams)):
            if self.busy[slot]:
                continue
            kind = self._next_kind()
            if kind is None:
                break
            stream = self.streams[slot]
            if kind == "sliced":
                r = self.queue_sliced.popleft()
                b = self._bytes(r)
                self.adm.take(b)
                n, k = r.B.shape
                plan = self.plans[r.lid]
                with torch.cuda.stream(stream):
                    self._order_after_submission(r, stream)
                    r.X = torch.empty((k, n), dtype=torch.float64, device="cuda").t()
                    r.t_admit = time.perf_counter()
                    binding.trsm_solve_schedule(plan, r.B, X=r.X, schedule="sliced")
                    ev = torch.cuda.Event()
                    ev.record(stream)
                self.busy[slot] = True
                self.inflight.append(_InFlight(None, ev, [r], b, slot=slot, plan=plan))
                self.launches += 1
                continue
            if kind == "mixed":
                r = self.queue_mixed.popleft()
                b = self._bytes(r)
                self.adm.take(b)
                n, k = r.B.shape
                with torch.cuda.stream(stream):
                    self._order_after_submission(r, stream)
                    r.X = torch.empty((k, n), dtype=torch.float64, device="cuda").t()
                r.t_admit = time.perf_counter()
                if self.pool is None:
                    self.pool = ThreadPoolExecutor(max_workers=self.mixed_slots)
                f = _InFlight(None, None, [r], b, future=self.pool.submit(self._solve_mixed, slot, r), slot=slot)
                self.busy[slot] = True
                self.mixed_busy += 1
                self.inflight.append(f)
                self.launches += 1
                continue
            take, nbytes = self._take_fp64()
            self.adm.take(nbytes)
            with torch.cuda.stream(stream):
                systems = []
                for r in take:
                    self._order_after_submission(r, stream)
                    n, k = r.B.shape
                    r.X = torch.empty((k, n), dtype=torch.float64, device="cuda").t()
                    r.t_admit = time.perf_counter()
                    systems.append({"plan": self.plans[r.lid], "B": r.B, "X": r.X})
                ws = binding.Batch.workspace_size(systems)
                arena = torch.empty(ws + 256, dtype=torch.uint8, device="cuda")
                off = (-arena.data_ptr()) % 256
                batch = binding.Batch(systems, arena=arena[off:off + ws])
                batch.run()
                ev = torch.cuda.Event()
                ev.record(stream)
            f = _InFlight(batch, ev, take, nbytes, arena, slot=slot)
            self.busy[slot] = True
            self.inflight.append(f)
            self.launches += 1

    def drain(self):
        while self.queue_fp64 or self.queue_mixed or self.queue_sliced or self.inflight:
            self.poll()
            self.dispatch()

    def run_trace(self, requests, idle_sleep=20e-6):
        """Feeds requests at their arrival times (seconds from now) and runs
        the loop until all are done.  Returns a stats dict."""
        t0 = time.perf_counter()
        order = sorted(requests, key=lambda r: r.arrival)
        for r in order:
            r.arrival += t0
        i = 0
        while i < len(order) or self.queue_fp64 or self.queue_mixed or self.queue_sliced or self.inflight:
            now = time.perf_counter()
            while i < len(order) and order[i].arrival <= now:
                self.submit(order[i])
                i += 1
            self.poll()
            self.dispatch()
            if i < len(order) and not self.inflight:
                time.sleep(max(0.0, min(idle_sleep, order[i].arrival - time.perf_counter())))
        t1 = time.perf_counter()
        if self.pool is not None:
            self.pool.shutdown(wait=True)
            self.pool = None
        lat = np.array([r.latency for r in order if r.latency is not None])
        flops = float(sum(self.plans[r.lid].n ** 2 * r.B.shape[1] for r in order))
        out = {"requests": len(order), "seconds": t1 - t0, "solves_per_s": len(order) / (t1 - t0),
               "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
               "mean_ms": float(lat.mean() * 1e3), "tflops_n2k": flops / (t1 - t0) / 1e12,
               "batches": self.launches, "slots": self.nstreams, "mixed_slots": self.mixed_slots,
               "peak_inflight_gb": self.adm.peak / 1e9,
               "statuses_ok": all(r.status == 0 for r in order)}
        # queueing delay (arrival to dispatch): head-of-line blocking shows
        # here, apart from the spread of the requests' own solve times
        wait = np.array([r.t_admit - r.arrival for r in order if r.t_admit is not None])
        if wait.size:
            out["wait_p50_ms"] = float(np.percentile(wait, 50) * 1e3)
            out["wait_p99_ms"] = float(np.percentile(wait, 99) * 1e3)
        out["sliced_requests"] = sum(1 for r in order if r.sliced)
        for kind, sel in (("fp64", lambda r: not r.mixed), ("mixed", lambda r: r.mixed)):
            part = [r for r in order if sel(r) and r.latency is not None]
            if part:
                pl = np.array([r.latency for r in part])
                out[kind] = {"requests": len(part), "p50_ms": float(np.percentile(pl, 50) * 1e3),
                             "p99_ms": float(np.percentile(pl, 99) * 1e3)}
                pw = np.array([r.t_admit - r.arrival for r in part if r.t_admit is not None])
                if pw.size:
                    out[kind]["wait_p99_ms"] = float(np.percentile(pw, 99) * 1e3)
                if kind == "mixed":
                    out[kind]["mean_iterations"] = float(np.mean([r.iterations or 0 for r in part]))
        return out
