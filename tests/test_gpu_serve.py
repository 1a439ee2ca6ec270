"""The continuous-batching server on the GPU: every served result equals
the single-request solve of the same right-hand side (the result does not
depend on the batch it shared), and memory admission holds."""
import numpy as np
import pytest

import oracle
from paper_1612_01855_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda().t()


def _setup(nL=5, seed=0):
    import paper_1612_01855_gb300 as g
    rng = np.random.default_rng(seed)
    Ls, plans = [], []
    for i in range(nL):
        n = int(rng.integers(40, 700))
        L = inputs.well_conditioned_L(n, seed=100 + i)
        Ls.append(L)
        plans.append(g.trsm_plan(_dev(L), [32, 64, 128][i % 3]))
    return Ls, plans


def _requests(Ls, count, rate, seed):
    from paper_1612_01855_gb300.serve import Request
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs, host = [], []
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        lid = int(rng.integers(0, len(Ls)))
        k = int(np.rint(np.exp(rng.uniform(0, np.log(96)))))
        B = inputs.rhs(Ls[lid].shape[0], k, seed=seed * 1000 + rid)
        reqs.append(Request(rid, lid, _dev(B), t))
        host.append(B)
    return reqs, host


def test_served_results_match_single_solves(cuda_lib):
    import torch
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300.serve import Server
    Ls, plans = _setup()
    reqs, host = _requests(Ls, 48, rate=4000.0, seed=1)
    srv = Server(plans, budget_bytes=40 * 2**30, streams=2, max_batch=16)
    stats = srv.run_trace(reqs)
    assert stats["statuses_ok"] and stats["requests"] == 48
    assert stats["batches"] < 48  # requests shared launches
    for r, B in zip(reqs, host):
        alone = g.trsm_solve(plans[r.lid], r.B)
        g.trsm_sync_status(plans[r.lid])
        assert torch.equal(alone, r.X), r.rid                  # same alone and in the mix
        want = oracle.forward_subst(Ls[r.lid], B)
        assert np.max(np.abs(r.X.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want))


def test_server_respects_tight_budget(cuda_lib):
    from paper_1612_01855_gb300.serve import Server
    Ls, plans = _setup(3, seed=2)
    reqs, _ = _requests(Ls, 30, rate=10000.0, seed=3)
    resident = sum(8 * p.n * p.n for p in plans)
    budget = resident + 3 * max(Server.request_bytes(p.n, 96) for p in plans)
    srv = Server(plans, budget_bytes=budget, streams=2, max_batch=64)
    stats = srv.run_trace(reqs)
    assert stats["statuses_ok"]
    assert srv.adm.peak + resident <= budget
    assert all(r.X is not None and r.t_done is not None for r in reqs)


def test_server_mixes_fp64_and_refined_requests(cuda_lib):
    """Half the requests ask for the mixed-precision solve (split-bf16
    updates, refined on the tensor cores): they run alone on a slot's worker
    thread next to the FP64 batches; every result matches the oracle and is
    the same bits as the request's solve run alone."""
    import torch
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300.serve import Server
    Ls, plans = _setup(4, seed=7)
    for L, p in zip(Ls, plans):
        g.trsm_plan_mixed(p, _dev(L), "bf16x3")
    reqs, host = _requests(Ls, 40, rate=3000.0, seed=9)
    for r in reqs:
        r.mixed = r.rid % 2 == 1
    srv = Server(plans, budget_bytes=40 * 2**30, streams=2, max_batch=16)
    stats = srv.run_trace(reqs)
    assert stats["statuses_ok"] and stats["requests"] == 40
    assert stats["mixed"]["requests"] == 20 and stats["mixed"]["mean_iterations"] >= 2
    for r, B in zip(reqs, host):
        want = oracle.forward_subst(Ls[r.lid], B)
        assert np.max(np.abs(r.X.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want)), (r.rid, r.mixed)
        # same bits alone and in the mix, for both kinds of request
        if r.mixed:
            alone, _, _ = g.trsm_solve_mixed(plans[r.lid], r.B, residual=srv.mixed_residual, tol=r.tol,
                                             **srv.mixed_kwargs())
        else:
            alone = g.trsm_solve(plans[r.lid], r.B)
            g.trsm_sync_status(plans[r.lid])
        assert torch.equal(alone, r.X), (r.rid, r.mixed)
    assert all(p.device_bytes() > 8 * p.n * p.n for p in plans)  # L~ plus the mixed data


def test_server_waits_for_b_produced_on_the_callers_stream(cuda_lib):
    """B is still being written by a kernel on the caller's stream when it is
    submitted (the stream first sleeps, then copies B in): the slot streams
    must wait for it, for FP64 batches and for mixed solves alike."""
    import torch
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300.serve import Request, Server
    Ls, plans = _setup(3, seed=11)
    for L, p in zip(Ls, plans):
        g.trsm_plan_mixed(p, _dev(L), "fp16x3")
    srv = Server(plans, budget_bytes=40 * 2**30, streams=4, max_batch=8)
    producer = torch.cuda.Stream()
    reqs, host = [], []
    rng = np.random.default_rng(12)
    for rid in range(12):
        lid = rid % len(Ls)
        n, k = Ls[lid].shape[0], int(rng.integers(1, 40))
        Bh = inputs.rhs(n, k, seed=500 + rid)
        src = torch.from_numpy(np.ascontiguousarray(Bh.T)).pin_memory()
        with torch.cuda.stream(producer):
            B = torch.full((k, n), float("nan"), dtype=torch.float64, device="cuda").t()
            torch.cuda._sleep(20_000_000)  # about 10 ms of device time before B is written
            B.t().copy_(src, non_blocking=True)
            r = Request(rid, lid, B, 0.0, mixed=rid % 3 == 0)
            srv.submit(r)  # the event is recorded on `producer`, before B is complete
        reqs.append(r)
        host.append(Bh)
    srv.drain()
    for r, B in zip(reqs, host):
        assert r.status == 0, r.rid
        want = oracle.forward_subst(Ls[r.lid], B)
        assert np.max(np.abs(r.X.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want)), (r.rid, r.mixed)


def test_server_routes_large_requests_to_the_sliced_schedule(cuda_lib):
    """Large FP64 requests go to the sliced schedule alone on a slot, the
    rest to batches: every result matches the oracle, and a sliced request
    equals its own sliced solve bit for bit."""
    import torch
    import paper_1612_01855_gb300 as g
    from paper_1612_01855_gb300.serve import Server
    Ls, plans = _setup(4, seed=21)
    for p in plans:
        if p.n0 % 64 == 0 and p.n0 <= 2048:
            g.trsm_plan_sliced(p)
    reqs, host = _requests(Ls, 40, rate=3000.0, seed=23)
    srv = Server(plans, budget_bytes=40 * 2**30, streams=4, max_batch=16, sliced_min_flops=2e6)
    stats = srv.run_trace(reqs)
    assert stats["statuses_ok"] and stats["requests"] == 40
    assert 0 < stats["sliced_requests"] < 40
    for r, B in zip(reqs, host):
        want = oracle.forward_subst(Ls[r.lid], B)
        assert np.max(np.abs(r.X.cpu().numpy() - want)) <= 1e-12 * np.max(np.abs(want)), (r.rid, r.sliced)
        if r.sliced:
            alone = g.trsm_solve_schedule(plans[r.lid], r.B, schedule="sliced")
            g.trsm_sync_status(plans[r.lid])
            assert torch.equal(alone, r.X), r.rid
