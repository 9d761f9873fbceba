"""The multi-GPU host logic on CPU: two gloo ranks (127.0.0.1) run bench.py's
rank reductions and the batched sweep's sharding.  The 64-instance sweep
splits into independent shards (no data-path collective), so what needs
checking is that every rank computes the same split on its own, that the
shards cover every instance exactly once with balanced work, and that the
max/sum reductions the bench uses for its timing and totals are correct."""
import os
import socket
from math import comb

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2606_05297_gb300 import batched
        from paper_2606_05297_gb300 import workloads as W
        mx = bench.max_over_ranks(float(rank + 1), world)
        sm = bench.sum_over_ranks(float(rank + 1), world)
        dims = [comb(m.N + m.L - 1, m.L - 1) for m in W.c4_instances(0, 64)]
        mine = batched.shard(dims, rank, world)
        every = [None] * world
        dist.all_gather_object(every, mine)
        q.put((rank, mx, sm, every, dims))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_rank_reductions_and_sweep_shards(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm, every, dims in out:
        assert mx == float(world) and sm == world * (world + 1) / 2
        assert every == out[0][3]  # every rank computed the same split
    shards = out[0][3]
    dims = out[0][4]
    flat = sorted(i for sh in shards for i in sh)
    assert flat == list(range(64))
    loads = [sum(dims[i] for i in sh) for sh in shards]
    # longest-first greedy is within 4/3 of the best split; the largest instance bounds it from below
    assert max(loads) <= max(sum(loads) / world * 4 / 3, max(dims) + sum(loads) / world)
