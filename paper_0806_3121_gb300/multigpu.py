"""Host-side logic of multi-GPU runs: one process per GPU, each rank an independent ABFT
problem (or group of problems), no collective on the data path.

The method shards naturally: independent problems need no exchange, so N ranks run N
problems (weak scaling) and the only collectives are the timing barrier and the max over
ranks of the timed region.  (A grid split of ONE problem across GPUs, with the block rebuild
as a reduce over the GPUs of a block column, is not built: it needs several GPUs in one run.)
The functions below work with any torch.distributed backend: gloo on CPU tensors (tests),
NCCL on CUDA tensors (bench under torchrun).
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
