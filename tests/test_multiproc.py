"""World-size-2 gloo check of the bench's multi-GPU host logic: every rank
owns a disjoint block of Monte Carlo runs and the reported time is the maximum
over ranks (weak scaling, no collective on the data path)."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ids = bench.shard_mc_ids(rank, world, 5)
    gathered = [None] * world
    dist.all_gather_object(gathered, ids)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (gathered, float(t.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_shards_disjoint_and_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        gathered, tmax = out[r]
        flat = [i for ids in gathered for i in ids]
        assert sorted(flat) == list(range(10)) and len(set(flat)) == 10
        assert tmax == 2.0
