"""The multi-process path of bench.py on CPU: replicas only (the method
shards over independent right-hand-side columns, so ranks never exchange
data), timing is the maximum over ranks and the value counts every rank's
work.  Two gloo ranks, no GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        local_ms = 100.0 + 37.0 * rank           # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, "cpu")
        value = bench.replica_throughput(2.0e12, world, ms)
        if rank != 0:  # the reference arm does its work on rank 0 only: others return at once
            assert bench.run_reference(None, rank, world) is None
        out.put((rank, ms, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == pytest.approx(137.0)             # max over ranks
        assert value == pytest.approx(2 * 2.0e12 / 0.137)  # both replicas' work
