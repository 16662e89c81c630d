"""The multi-GPU path is replicas (the rays are independent, Sec. 2): the
host-side pieces -- the maximum of the ranks' times, the whole-job rate and
the split of work items over ranks -- checked with two gloo processes on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1303_5057_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    me = replicas.from_env()
    dist = replicas.init(me, "gloo")
    ms = 10.0 + 5.0 * me.rank  # rank 1 is the slowest
    top = replicas.max_over_ranks(dist, ms)
    first, count = replicas.shard(11, me.rank, me.world)
    mine = replicas.route(list(range(7)), me.rank, me.world)
    out.put((me.rank, top, replicas.job_rate(1000, top, me.world), first, count, mine))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]             # the max over ranks, on both
    assert res[0][2] == pytest.approx(2 * 1000 / 0.015)    # whole-job units/s
    shards = [(r[3], r[4]) for r in res]
    assert shards == [(0, 6), (6, 5)]                      # 11 items, every one exactly once
    assert res[0][5] + res[1][5] == [0, 2, 4, 6, 1, 3, 5]


def test_single_rank_needs_no_group():
    me = replicas.Rank()
    assert replicas.init(me, "gloo") is None
    assert replicas.max_over_ranks(None, 3.5) == 3.5
    assert replicas.shard(5, 0, 1) == (0, 5)
    for n in (0, 1, 7, 100):
        for w in (1, 2, 3, 8):
            parts = [replicas.shard(n, r, w) for r in range(w)]
            assert sum(c for _, c in parts) == n
            assert all(parts[r][0] + parts[r][1] == parts[r + 1][0] for r in range(w - 1))
