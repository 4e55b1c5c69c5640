"""The N > 1 host path on CPU: two gloo ranks (world_size 2) run the multi-GPU helpers the
bench uses under torchrun -- per-rank seeds and shards, the timing barrier, the max over
ranks of the timed region and the weak-scaling value.  No GPU is touched."""
import os
import socket

import pytest

from paper_0806_3121_gb300 import multigpu as mg

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank          # rank 1 is the slower one
        mg.barrier()
        mx = mg.max_over_ranks(ms)
        value = mg.weak_scaling_value(2e12, world, mx)
        items = list(mg.shard(41, rank, world))
        gathered = [None] * world
        dist.all_gather_object(gathered, (mg.rank_seed(7, rank), items))
        out.put((rank, mx, value, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, value, gathered in res:
        assert mx == 15.0                                  # the slowest rank's time
        assert value == pytest.approx(2e12 * 2 / 15e-3 / 1e12)
        seeds = [g[0] for g in gathered]
        shards = [g[1] for g in gathered]
        assert seeds == [7, 8]                             # distinct problems per rank
        assert sorted(shards[0] + shards[1]) == list(range(41))
        assert len(shards[0]) == 21 and len(shards[1]) == 20


def test_single_process_helpers():
    assert mg.max_over_ranks(3.5) == 3.5
    mg.barrier()
    assert list(mg.shard(5, 0, 1)) == [0, 1, 2, 3, 4]
    assert [len(mg.shard(10, r, 4)) for r in range(4)] == [3, 3, 2, 2]
    with pytest.raises(ValueError):
        mg.shard(4, 2, 2)
    with pytest.raises(ValueError):
        mg.weak_scaling_value(1.0, 1, 0.0)
