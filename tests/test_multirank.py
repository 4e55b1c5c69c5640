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


# --------------------------------------------------------------------------- grid split
def test_block_row_grid_partition():
    g = mg.BlockRowGrid(22, 4)
    assert [len(g.rows(r)) for r in range(4)] == [6, 6, 5, 5]
    assert g.owner == 3
    assert [g.rank_of(I) for I in (0, 5, 6, 11, 12, 16, 17, 21)] == [0, 0, 1, 1, 2, 2, 3, 3]
    assert [g.local(I) for I in (0, 5, 6, 12, 21)] == [0, 5, 0, 0, 4]
    with pytest.raises(ValueError):
        mg.BlockRowGrid(2, 3)
    with pytest.raises(ValueError):
        g.rank_of(22)


def _grid_worker(rank, world, port, out):
    """One rank of a split problem.  The oracle stands in for the rank's GPU arithmetic
    (local encode, product and share); the partition, the two reductions and where they
    land are the product's host code under test."""
    import numpy as np
    import torch.distributed as dist

    import oracle
    from paper_0806_3121_gb300 import workloads as wl
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, q, bs, bc, k = 5, 3, 8, 6, 12
        m, n = p * bs, q * bc
        A = wl.rng(31, 1).integers(-4, 5, (m, k)).astype(np.float64)  # every rank draws the
        B = wl.rng(31, 2).integers(-4, 5, (k, n)).astype(np.float64)  # same global problem
        grid = mg.BlockRowGrid(p, world)
        rows = grid.rows(rank)
        A_loc = A[rows.start * bs:rows.stop * bs]
        C_loc = oracle.gemm(A_loc, B)
        # encode: the local block sum, reduced into the owner -> the grid's S_A
        acs = oracle.encode_A(A_loc, bs, p=len(rows))
        S_A = torch.from_numpy(np.ascontiguousarray(acs[2 * len(rows):]))
        mg.reduce_block_checksum(grid, S_A)
        S = oracle.gemm(S_A.numpy(), B) if rank == grid.owner else None
        # lose a block on its rank, rebuild it from the shares: block (1, 0) on rank 0,
        # then block (3, 2) on rank 1 beside the checksum rows
        results = []
        for bi, bj in ((1, 0), (3, 2)):
            saved = None
            if grid.rank_of(bi) == rank:
                lb = grid.local(bi)
                saved = C_loc[lb * bs:(lb + 1) * bs, bj * bc:(bj + 1) * bc].copy()
                C_loc[lb * bs:(lb + 1) * bs, bj * bc:(bj + 1) * bc] = np.nan
            buf = torch.empty((bs, bc), dtype=torch.float64)

            def share(skip, col, with_checksum, outbuf):
                v = S[:, col * bc:(col + 1) * bc].copy() if with_checksum else np.zeros((bs, bc))
                for I in range(len(rows)):
                    if I != skip:
                        v -= C_loc[I * bs:(I + 1) * bs, col * bc:(col + 1) * bc]
                outbuf.copy_(torch.from_numpy(v))

            def restore(lb, col, total):
                C_loc[lb * bs:(lb + 1) * bs, col * bc:(col + 1) * bc] = total.numpy()
                return "restored"

            res = mg.rebuild_block(grid, rank, bi, bj, share, restore, buf)
            ok = None
            if saved is not None:
                lb = grid.local(bi)
                ok = bool(np.array_equal(C_loc[lb * bs:(lb + 1) * bs, bj * bc:(bj + 1) * bc],
                                         saved))
            results.append((res, ok))
        full_S_A = A.reshape(p, bs, k).sum(0)
        out.put((rank, results, bool(np.array_equal(S_A.numpy(), full_S_A))
                 if rank == grid.owner else None))
    finally:
        dist.destroy_process_group()


def test_grid_split_rebuild_two_gloo_ranks():
    """A 5 x 3 grid split over two ranks (block rows 0-2 and 3-4; the checksum rows on rank
    1): the reduced S_A on the owner equals the grid's sum of A blocks, and a lost block
    on either rank -- (1, 0) on rank 0, (3, 2) on rank 1 beside the checksum -- is
    rebuilt exactly (integer data) from the reduction of both ranks' shares."""
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grid_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, out0, s0), (r1, out1, s1) = res
    assert out0 == [("restored", True), (None, None)]   # block row 1 is rank 0's
    assert out1 == [(None, None), ("restored", True)]   # block row 3 is rank 1's
    assert s0 is None and s1 is True
