"""Multi-rank logic of bench.py on CPU (gloo, world size 2): the ensemble is
sharded by member with disjoint seeds, the job time is the slowest rank's,
and the throughput counts every rank's updates (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed = 1.0 + rank  # rank 1 is the slow one
    out[rank] = bench.max_over_ranks(elapsed)
    seeds = [bench.member_seed(1000, rank, 64, m) for m in range(64)]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    if rank == 0:
        allseeds = [s for g in gathered for s in g]
        out[10] = len(set(allseeds)) == len(allseeds) == 128
        out[11] = bench.aggregate_glups(world, 64 * 512 * 512 * 200, 5, out[0])
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 2.0          # max over ranks
    assert out[10] is True                  # disjoint member seeds
    lu = 2 * 64 * 512 * 512 * 200 * 5
    assert abs(out[11] - lu / 2.0 / 1e9) < 1e-9
