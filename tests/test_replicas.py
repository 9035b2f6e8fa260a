"""The replica bookkeeping of runs on several GPUs, as two gloo ranks on CPU.

A relit frame does not shard, so N GPUs run N independent replicas; the
ranks share only a barrier, the max-over-ranks elapsed time and the
whole-job rate computed from it.  This runs that host logic in two
processes (world size 2, 127.0.0.1) without a GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2410_11419_gb300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = replicas.rank_env()
        replicas.barrier()
        slowest = replicas.max_over_ranks(1.5 + rank)      # rank 1 is the slower one
        views = [replicas.view_index(s, r, w, offset=5) for s in range(30)]
        rate = replicas.whole_job_rate(30, slowest, w)
        replicas.barrier()
        out.put((r, w, lr, slowest, views, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_only_bookkeeping():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, v0, rate0), (r1, w1, l1, s1, v1, rate1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert s0 == s1 == pytest.approx(2.5)                  # every rank sees the slowest time
    assert rate0 == rate1 == pytest.approx(2 * 30 / 2.5)   # all units over the slowest time
    assert not set(v0) & set(v1)                           # disjoint views
    assert v0[:3] == [5, 7, 9] and v1[:3] == [6, 8, 10]


def test_single_process_defaults():
    assert replicas.rank_env() == (1, 0, 0) or "WORLD_SIZE" in os.environ
    assert replicas.max_over_ranks(3.25) == 3.25
    assert [replicas.view_index(s, 0, 1, offset=5) for s in range(3)] == [5, 6, 7]
    assert replicas.whole_job_rate(30, 0.5, 1) == pytest.approx(60.0)
