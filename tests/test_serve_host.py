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
