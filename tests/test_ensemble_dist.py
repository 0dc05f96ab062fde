"""Ensemble sharding over ranks on CPU (gloo, world size 2): the member
partition covers every member once in contiguous balanced blocks, and the
per-member statistics gathered once per diagnostic event come back in global
member order on every rank, uneven shards and an empty shard included."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1809_06735_gb300.ensemble import gather_member_stats, shard  # noqa: E402

NL = 4  # box sizes per member in the synthetic statistics


def _stats_of(members):
    """Statistics that name their member: [n, NL, 15, 2] with entry
    (member, L, q, k) = member + L / 10 + q / 1000 + k / 1e5."""
    m = np.asarray(list(members), dtype=np.float64)[:, None, None, None]
    L = np.arange(NL)[None, :, None, None] / 10.0
    q = np.arange(15)[None, None, :, None] / 1000.0
    k = np.arange(2)[None, None, None, :] / 1e5
    return m + L + q + k + np.zeros((len(m), NL, 15, 2))


def test_shard_partitions_every_member_once():
    for n in (0, 1, 5, 64, 67):
        for ws in (1, 2, 3, 8):
            parts = [shard(n, ws, r) for r in range(ws)]
            assert [i for p in parts for i in p] == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def test_gather_without_process_group_is_identity():
    s = _stats_of(range(3))
    assert np.array_equal(gather_member_stats(s), s)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    for n in (5, 1, 64):  # uneven (3 + 2), one empty shard (1 + 0), even
        mine = shard(n, world, rank)
        got = gather_member_stats(_stats_of(mine))
        out[(rank, n)] = bool(np.array_equal(got, _stats_of(range(n))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_in_member_order():
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
    assert all(out[(r, n)] for r in range(2) for n in (5, 1, 64))
