"""Host-side logic of multi-GPU runs: one process per GPU.

Independent problems: the method shards naturally, so N ranks run N problems (weak
scaling) and the only collectives are the timing barrier and the max over ranks of the
timed region.

One problem split over GPUs (BlockRowGrid, GridShard): the block rows of its erasure grid
are spread over the ranks (section 3.1), B is replicated, and each rank runs the local
ABFT product, verify and correction of its rows.  Two steps cross ranks, each one
reduction: the block checksum S_A = sum_I A_I is reduced into the rank that holds the
checksum rows before its product, and a lost block is rebuilt from the reduction of
every rank's share over its block column (section 3.3).  The arithmetic of both runs in
the C-ABI library; this module only decides who sends what where.

The functions work with any torch.distributed backend: gloo on CPU tensors (tests), NCCL
on CUDA tensors (under torchrun).
"""
from __future__ import annotations


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s problem: distinct per rank, reproducible."""
    return int(seed) + int(rank)


def shard(count: int, rank: int, world: int) -> range:
    """Contiguous share of `count` independent items for `rank` (the first count % world
    ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(int(count), int(world))
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def _device_for_backend():
    import torch
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(value: float) -> float:
    """The maximum of `value` over all ranks (the slowest rank's time); the value itself
    without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device_for_backend())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def weak_scaling_value(useful_flops_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput in TFLOP/s: every rank's useful flops over the slowest time."""
    if max_ms <= 0:
        raise ValueError("max_ms must be positive")
    return useful_flops_per_rank * world / (max_ms * 1e-3) / 1e12


# --------------------------------------------------------------------------- grid split
class BlockRowGrid:
    """The block rows of one problem's p x q erasure grid spread over `world` ranks
    (section 3.1: the process grid holds the blocks of the matrices).  Rank r owns the
    contiguous block rows rows(r) of A and C; B is replicated on every rank.  The block
    checksum rows S = sum_I C_I (and the S_A = sum_I A_I rows that produce them) live on
    `owner`, by default the last rank, like the paper's extra checksum processes."""

    def __init__(self, p: int, world: int, owner: int | None = None):
        if p < world or world < 1:
            raise ValueError("need at least one block row per rank")
        self.p, self.world = int(p), int(world)
        self.owner = self.world - 1 if owner is None else int(owner)
        if not 0 <= self.owner < self.world:
            raise ValueError("owner must be a rank")

    def rows(self, rank: int) -> range:
        return shard(self.p, rank, self.world)

    def rank_of(self, I: int) -> int:
        for r in range(self.world):
            if I in self.rows(r):
                return r
        raise ValueError(f"block row {I} outside the grid")

    def local(self, I: int) -> int:
        """Index of global block row I among its rank's block rows."""
        return I - self.rows(self.rank_of(I)).start


def dist_reduce(t, dst: int) -> None:
    """Sum of `t` over all ranks into rank dst's `t` (one collective)."""
    import torch.distributed as dist
    dist.reduce(t, dst=dst, op=dist.ReduceOp.SUM)


def reduce_block_checksum(grid: BlockRowGrid, local_sum, reduce=dist_reduce) -> None:
    """Encode step of the split: each rank's sum of its own A blocks (`local_sum`,
    bs x k) is reduced into the owner's, which then holds S_A = sum_I A_I over the whole
    grid; the owner's product turns it into the block checksum rows S = S_A B."""
    reduce(local_sum, grid.owner)


def rebuild_block(grid: BlockRowGrid, rank: int, bi: int, bj: int, share, restore, buf,
                  reduce=dist_reduce):
    """Rebuild of lost block (bi, bj) of the split problem (section 3.3: the checksum minus
    the survivors, one reduction over the processes of the block column).

    Every rank calls it.  share(skip, bj, with_checksum, out) writes this rank's share
    into buf -- the owner's block checksum (with_checksum) minus its local blocks of the
    column, skipping local block row `skip` (-1: the lost block is elsewhere); the
    reduction sums the shares into the rank of block row bi, whose restore(local_bi, bj,
    total) writes the block and re-checks it.  Returns restore's result on that rank,
    None elsewhere."""
    r_bi = grid.rank_of(bi)
    skip = grid.local(bi) if rank == r_bi else -1
    share(skip, bj, rank == grid.owner, buf)
    reduce(buf, r_bi)
    if rank == r_bi:
        return restore(grid.local(bi), bj, buf)
    return None


class GridShard:
    """One rank's part of a binary64 ABFT product whose block rows are spread over GPUs:
    the local problem (this rank's block rows of A and C, all of B), its workspace, and
    the C-ABI calls of the split's encode and rebuild.  The element checksums, the verify
    and the location / correction of single errors are local to each rank; only the
    block checksum and the block rebuild cross ranks."""

    def __init__(self, grid: BlockRowGrid, rank: int, m: int, n: int, k: int, vb_r: int,
                 vb_c: int, q: int, device):
        import torch
        from paper_0806_3121_gb300 import abft
        if m % grid.p or n % q:
            raise ValueError("the grid must divide m and n")
        self.grid, self.rank = grid, rank
        self.bs, self.bc = m // grid.p, n // q
        if self.bs % vb_r:
            raise ValueError("verify blocks must not straddle block rows")
        self.rows = grid.rows(rank)
        self.m = len(self.rows) * self.bs
        self.n, self.k = n, k
        self.desc = abft.make_desc(self.m, n, k, "f64", vb_r, vb_c, len(self.rows), q)
        self.layout = abft.abft_workspace_layout(self.desc)
        self.ws = torch.zeros(self.layout.total, dtype=torch.uint8, device=device)
        self.buf = torch.empty((self.bs, self.bc), dtype=torch.float64, device=device)
        self.C = None

    def s_rows(self):
        """The workspace's S_A rows (bs x k binary64): the local block sum after the
        local encode, the grid's S_A on the owner after reduce_block_checksum."""
        L = self.layout
        off = L.acs + 2 * L.nvr * self.k * 8
        return self.ws[off:off + self.bs * self.k * 8].view(torch_f64()).view(self.bs, self.k)

    def encode(self, A_local, B, reduce=dist_reduce, stream=None):
        from paper_0806_3121_gb300 import abft
        abft.abft_encode(self.desc, A_local, B, self.ws, stream=stream)
        reduce_block_checksum(self.grid, self.s_rows(), reduce)

    def gemm(self, A_local, B, C, stream=None):
        """The local ABFT product; the owner's carries the grid's block checksum rows."""
        from paper_0806_3121_gb300 import abft
        abft.abft_gemm(self.desc, A_local, B, C, self.ws, stream=stream)
        self.C = C

    def local_blocks(self, blocks):
        """The blocks of a global (bi, bj) list that lie on this rank, in local indices."""
        return [(self.grid.local(bi), bj) for bi, bj in blocks
                if self.grid.rank_of(bi) == self.rank]

    def verify(self, erased=(), stream=None):
        """Local detect / locate / correct, skipping the lines of the erased blocks
        (global indices) that lie on this rank."""
        from paper_0806_3121_gb300 import abft
        return abft.abft_verify_correct(self.desc, self.C, self.ws,
                                        erased=self.local_blocks(erased), stream=stream)

    def rebuild(self, bi, bj, reduce=dist_reduce):
        """Every rank calls this for lost block (bi, bj) (global indices)."""
        return rebuild_block(self.grid, self.rank, bi, bj, self.share, self.restore, self.buf,
                             reduce)

    def share(self, skip, bj, with_checksum, out, stream=None):
        from paper_0806_3121_gb300 import abft
        abft.abft_block_partial(self.desc, self.C, self.ws, skip, bj, with_checksum, out,
                                stream=stream)

    def restore(self, bi_local, bj, total, stream=None):
        from paper_0806_3121_gb300 import abft
        return abft.abft_block_restore(self.desc, self.C, self.ws, bi_local, bj, total,
                                       stream=stream)


def torch_f64():
    import torch
    return torch.float64
