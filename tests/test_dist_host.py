"""The multi-rank host logic of bench.py on two gloo ranks (CPU): the barrier, the max over ranks
of the step time, the whole-job rate of weak-scaling replicas, and the reference arm's rule that
rank 0 alone runs it (the other ranks return without work).  The replicas share no data-path
collective, so these are the only cross-rank operations."""
import multiprocessing as mp
import os
import socket
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), PWA_DIST_BACKEND="gloo")
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_init(world)
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.5 + rank, w)  # rank r took 1.5 + r seconds
    rate = bench.job_rate(1000, w, slowest)
    ref = bench.run_reference(SimpleNamespace(workload="scale", warmup=3, steps=1), w, r) if r != 0 else "rank 0"
    q.put((r, slowest, rate, ref))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_job_rate_and_reference_rule():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, slowest, rate, ref in out:
        assert slowest == 2.5  # the max over ranks, seen by every rank
        assert rate == pytest.approx(2 * 1000 / 2.5)  # all ranks' units over the slowest time
    assert out[1][3] is None  # the reference arm: only rank 0 runs it
