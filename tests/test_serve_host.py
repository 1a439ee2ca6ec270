"""Host-side logic of the solve server (no GPU): HBM-budget admission,
malformed and oversized requests, cancellation."""
import pytest

from paper_1612_01855_gb300.serve import Admission, AdmissionError, Request, Server


class _Plan:
    def __init__(self, n):
        self.n = n


class _B:
    def __init__(self, n, k):
        self.shape = (n, k)


def test_admission_budget_accounting():
    a = Admission(1000, resident_bytes=400)
    assert a.take(300) and a.in_use == 300
    assert not a.take(301)          # would exceed 1000
    assert a.take(300) and a.peak == 600
    a.release(300)
    assert a.fits(300) and not a.fits(301)
    with pytest.raises(AdmissionError):
        a.release(10_000)


def test_admission_rejects_impossible_requests():
    with pytest.raises(AdmissionError):
        Admission(100, resident_bytes=200)
    a = Admission(1000, resident_bytes=900)
    with pytest.raises(AdmissionError):
        a.check_request(200)


def test_server_validates_and_cancels_without_gpu():
    plans = [_Plan(64), _Plan(128)]
    srv = Server(plans, budget_bytes=10**9)
    srv.submit(Request(0, 1, _B(128, 4), 0.0))
    srv.submit(Request(1, 0, _B(64, 2), 0.0))
    with pytest.raises(AdmissionError):          # wrong number of rows for L #0
        srv.submit(Request(2, 0, _B(65, 2), 0.0))
    tight = Server(plans, budget_bytes=8 * (64 * 64 + 128 * 128) + 1000)
    with pytest.raises(AdmissionError):          # can never fit next to the plans
        tight.submit(Request(3, 1, _B(128, 1000), 0.0))
    assert srv.cancel(0) and not srv.cancel(0)
    assert [r.rid for r in srv.pending] == [1]


def test_mixed_requests_need_a_mixed_plan():
    plans = [_Plan(64), _Plan(128)]
    plans[1].inner = "bf16x3"  # as set by trsm_plan_mixed
    srv = Server(plans, budget_bytes=10**9)
    with pytest.raises(AdmissionError):
        srv.submit(Request(0, 0, _B(64, 4), 0.0, mixed=True))
    srv.submit(Request(1, 1, _B(128, 4), 0.0, mixed=True))
    assert [r.rid for r in srv.pending] == [1]
    # the refinement's workspace is larger than the FP64 batch share
    assert Server.request_bytes(128, 4, mixed=True) > Server.request_bytes(128, 4)


def test_autotune_buckets_and_paper_rule():
    from paper_1612_01855_gb300 import autotune
    assert [autotune.bucket_of(n) for n in (1, 63, 64, 255, 256, 1024, 5000)] == [0, 0, 1, 2, 3, 4, 4]
    assert autotune.paper_rule_n0(16384, 256) == 2048 and autotune.paper_rule_n0(100, 10000) == 100
    table = {0: (32, 0), 1: (64, 32)}
    assert autotune.choose(100, table=table) == (64, 32) and autotune.choose(900, table=table) == (32, 0)


def test_queues_have_no_head_of_line_blocking():
    """A free slot serves the earlier of the two queue heads, unless that head
    cannot start: an FP64 request passes a mixed one while every mixed slot
    is taken, and a mixed one passes an FP64 request that does not fit."""
    plans = [_Plan(64), _Plan(128)]
    plans[1].inner = "fp16x3"
    srv = Server(plans, budget_bytes=10**9, streams=4)
    assert srv.mixed_slots == 2
    srv.submit(Request(0, 1, _B(128, 8), 0.0, mixed=True))
    srv.submit(Request(1, 0, _B(64, 8), 1.0))
    assert [r.rid for r in srv.pending] == [0, 1]
    assert srv._next_kind() == "mixed"           # earlier head, a mixed slot is free
    srv.mixed_busy = srv.mixed_slots
    assert srv._next_kind() == "fp64"            # the mixed head must wait; FP64 passes it
    srv.mixed_busy = 0
    take, nbytes = srv._take_fp64()
    assert [r.rid for r in take] == [1] and nbytes == Server.request_bytes(64, 8)
    assert srv._next_kind() == "mixed"
    # an FP64 head that does not fit the budget is passed by a mixed request that does
    tight = Server(plans, budget_bytes=8 * (64 * 64 + 128 * 128) + Server.request_bytes(64, 2000) + 10,
                   streams=2)
    tight.submit(Request(2, 0, _B(64, 2000), 0.0))
    tight.submit(Request(3, 1, _B(128, 8), 1.0, mixed=True))
    assert Server.request_bytes(64, 2000) > Server.request_bytes(128, 8, True)
    tight.adm.take(tight.adm.budget - tight.adm.resident - Server.request_bytes(128, 8, True))
    assert not tight.adm.fits(Server.request_bytes(64, 2000))
    assert tight._next_kind() == "mixed"
    assert tight.cancel(2) and tight.cancel(3) and not tight.pending


def test_single_slot_serves_both_kinds():
    plans = [_Plan(64)]
    plans[0].inner = "bf16x3"
    srv = Server(plans, budget_bytes=10**9, streams=1)
    assert srv.mixed_slots == 1
    srv.submit(Request(0, 0, _B(64, 2), 0.0))
    srv.submit(Request(1, 0, _B(64, 2), 0.5, mixed=True))
    assert srv._next_kind() == "fp64"
    srv.queue_fp64.clear()
    assert srv._next_kind() == "mixed"


def test_large_fp64_requests_route_to_the_sliced_schedule():
    """With sliced_min_flops set, an FP64 request of at least that many n^2 k
    flops on a plan with the sliced schedule's planes waits in its own queue;
    smaller ones, mixed ones and those on plans without planes do not."""
    plans = [_Plan(4096), _Plan(4096), _Plan(256)]
    for p in plans:
        p.n0 = 256
    plans[0].sliced = True
    plans[2].sliced = True
    plans[1].inner = "fp16x3"
    srv = Server(plans, budget_bytes=10**12, streams=4, sliced_min_flops=1e10)
    srv.submit(Request(0, 0, _B(4096, 1000), 0.0))            # 1.7e10 flops, sliced planes: sliced
    srv.submit(Request(1, 0, _B(4096, 100), 1.0))             # 1.7e9: batched
    srv.submit(Request(2, 1, _B(4096, 1000), 2.0))            # no sliced planes: batched
    srv.submit(Request(3, 1, _B(4096, 1000), 3.0, mixed=True))
    srv.submit(Request(4, 2, _B(256, 2000), 4.0))             # 1.3e8: batched
    assert [r.rid for r in srv.queue_sliced] == [0]
    assert [r.rid for r in srv.queue_fp64] == [1, 2, 4] and [r.rid for r in srv.queue_mixed] == [3]
    assert [r.rid for r in srv.pending] == [0, 1, 2, 3, 4]
    assert srv._next_kind() == "sliced"                       # the earliest head
    # its bytes: X and W (16 n k), one block row of digit planes of W and of X
    assert srv._bytes(srv.queue_sliced[0]) == Server.request_bytes(4096, 1000, sliced_block=256)
    assert Server.request_bytes(4096, 1000, sliced_block=256) > 16 * 4096 * 1000
    srv.queue_sliced.clear()
    assert srv._next_kind() == "fp64"
    off = Server(plans, budget_bytes=10**12, streams=4)     # routing off by default
    off.submit(Request(5, 0, _B(4096, 1000), 0.0))
    assert not off.queue_sliced and [r.rid for r in off.queue_fp64] == [5]


def test_mixed_diagonal_multiply_modes():
    """The mixed requests' diagonal multiply: two tf32 planes on the tensor
    cores by default, any of the library's modes by name, and the same
    keyword arguments for the served solve and for a solve alone."""
    plans = [_Plan(64)]
    assert Server(plans, budget_bytes=10**9).mixed_kwargs() == {"s_tc": True, "s_tc_planes": 2}
    assert Server(plans, budget_bytes=10**9, mixed_s="fp32").mixed_kwargs() == {"s_fp32": True}
    assert Server(plans, budget_bytes=10**9, mixed_s="fp64").mixed_kwargs() == {}
    assert Server(plans, budget_bytes=10**9, mixed_s="tc").mixed_kwargs() == {"s_tc": True, "s_tc_planes": 3}
    srv = Server(plans, budget_bytes=10**9)
    kw = srv.mixed_kwargs()
    kw["s_tc_planes"] = 1  # a copy: the server's own mode is unchanged
    assert srv.mixed_kwargs()["s_tc_planes"] == 2
    with pytest.raises(ValueError):
        Server(plans, budget_bytes=10**9, mixed_s="tf32")
