"""Multi-GPU replicas, host side, on CPU ranks (gloo, world size 2): each rank
takes a disjoint share of every step's blocks, the shares cover the step, and
the step time reported is the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, k, bps, steps, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [bench.rank_blocks(k, rank, world, s, bps) for s in range(steps)]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = torch.tensor([0.5 + rank], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        if rank == 0:
            q.put((gathered, float(t.item())))
    finally:
        dist.destroy_process_group()


def test_two_replicas_split_each_step():
    world, k, bps, steps = 2, 8, 8, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, k, bps, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 1.5
    seen = []
    for s in range(steps):
        a, b = set(gathered[0][s]), set(gathered[1][s])
        assert len(a) == bps and len(b) == bps and not (a & b)
        seen += list(a | b)
    # consecutive steps walk the row-major block sequence without gaps or repeats
    assert len(seen) >= k * k
    assert len(set(seen[:k * k])) == k * k == len(set(bench.block_list(k, 0, k * k)))
