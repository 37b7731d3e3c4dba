"""Replica (N > 1) host logic on CPU with the gloo backend, world size 2: sharding of right-
hand sides and the max/sum reductions the bench uses for its whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1801_08655_gb300 import replicas


def test_shard_covers_items_once():
    items = list(range(11))
    parts = [replicas.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, rk, lr = replicas.env_ranks()
    mine = replicas.shard(list(range(10)), rk, ws)
    secs = 1.0 + rk                      # rank 1 is the slow one
    rate = replicas.whole_job_rate(len(mine), secs)
    replicas.barrier()
    q.put((rk, ws, mine, replicas.max_over_ranks(secs), replicas.sum_over_ranks(len(mine)), rate))
    dist.destroy_process_group()


def test_gloo_two_ranks_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][2] == [0, 1, 2, 3, 4] and out[1][2] == [5, 6, 7, 8, 9]
    for rk, ws, mine, mx, sm, rate in out:
        assert ws == 2 and mx == 2.0 and sm == 10.0 and rate == pytest.approx(5.0)
