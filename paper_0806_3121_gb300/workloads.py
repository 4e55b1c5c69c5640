"""Seeded synthetic workloads: operands, fault lists and erased blocks.

This module only draws random inputs (numpy PCG64 streams keyed by a seed) and holds
none of the ABFT method's arithmetic.  Both the CUDA path (tests, bench) and the CPU
oracle consume what it produces.  The paper's matrices were random (section 4.3 stress
test); the shapes and distributions below are the ones each workload names.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    dtype: str            # "f64" | "bf16" | "bf16x3" | "fp8"
    m: int
    n: int
    k: int
    vb_r: int             # verify block rows
    vb_c: int             # verify block columns
    p: int = 0            # erasure grid (0 = none)
    q: int = 0
    dist: str = "normal"  # "uniform" U[-1,1] | "normal" N(0,1) | "fp8rows"
    n_flips: int = 0
    n_erased: int = 0
    note: str = ""


# The paper's workload shapes, restated per dtype.
F64_512 = Workload("f64_512", "f64", 512, 512, 512, 512, 512, dist="uniform", n_flips=1,
                   note="FP64 512^3, U[-1,1], one bit-flip in C before verify")
F64_11264_GRID22 = Workload("f64_11264_grid22", "f64", 11264, 11264, 11264, 512, 512, 22, 22,
                            dist="normal", n_flips=3, n_erased=1,
                            note="FP64 11264^3 as a 22x22 grid of 512-blocks (484 'processes'); "
                                 "one block erased to NaN plus 3 bit-flips in distinct blocks")
# Smaller cases of the same kernels, for profiling captures that must stay a few GB.
F64_4096_GRID8 = Workload("f64_4096_grid8", "f64", 4096, 4096, 4096, 512, 512, 8, 8,
                          dist="normal", n_flips=3, n_erased=1,
                          note="FP64 4096^3 as an 8x8 grid of 512-blocks (profiling size)")
BF16_8192 = Workload("bf16_8192", "bf16", 8192, 8192, 8192, 256, 256, dist="normal", n_flips=3,
                     note="BF16 8192^3 (profiling size)")
# Verify blocks of 256: half the checksum tiles of 128-blocks at the same detection power
# (the threshold is dominated by the sqrt(k) accumulation term).
BF16_16384 = Workload("bf16_16384", "bf16", 16384, 16384, 16384, 256, 256, dist="normal",
                      n_flips=3, note="BF16 16384^3, N(0,1) rounded to BF16, FP32 accumulate")
BF16X3_16384 = Workload("bf16x3_16384", "bf16x3", 16384, 16384, 16384, 256, 256,
                        dist="normal", n_flips=3,
                        note="FP32 16384^3 inputs N(0,1), split bf16x3 product, FP32 accumulate")
BF16X3_8192 = Workload("bf16x3_8192", "bf16x3", 8192, 8192, 8192, 256, 256, dist="normal",
                       n_flips=3, note="split bf16x3 8192^3 (profiling size)")
BF16X6_16384 = Workload("bf16x6_16384", "bf16x6", 16384, 16384, 16384, 256, 256,
                        dist="normal", n_flips=3,
                        note="FP32 16384^3 inputs N(0,1), split bf16x6 product (three bf16 "
                             "pieces, six products), FP32-level accuracy")
FP8_16384 = Workload("fp8_16384", "fp8", 16384, 16384, 16384, 256, 256, dist="fp8rows",
                     n_flips=5, note="FP8 E4M3 16384^3: A, B iid U[-1,1] x 10^U(-2,2) per row, "
                                     "quantised with one power-of-two binary32 scale per 128x128 "
                                     "block; fp32 accumulate; 5 seeded faults")
FP8_4096 = Workload("fp8_4096", "fp8", 4096, 4096, 4096, 256, 256, dist="fp8rows", n_flips=5,
                    note="the FP8 recipe at 4096^3 (profiling size)")
FP8_8192 = Workload("fp8_8192", "fp8", 8192, 8192, 8192, 256, 256, dist="fp8rows", n_flips=5,
                    note="the FP8 recipe at 8192^3 (profiling size)")
BF16X6_8192 = Workload("bf16x6_8192", "bf16x6", 8192, 8192, 8192, 256, 256, dist="normal",
                       n_flips=3, note="split bf16x6 8192^3 (profiling size)")
WORKLOADS = {w.name: w for w in (F64_512, F64_11264_GRID22, F64_4096_GRID8, BF16_16384,
                                 BF16_8192, BF16X3_16384, BF16X3_8192, BF16X6_16384, BF16X6_8192,
                                 FP8_16384, FP8_4096, FP8_8192)}


def fp8_quantize_dev(x, blk=128):
    """The FP8 input recipe on the device: one power-of-two binary32 scale per blk x blk
    block, 2^ceil(log2(max|x| / 448)), codes rounded to nearest-even E4M3.  Returns
    (uint8 codes, float32 scales [rows/blk x cols/blk])."""
    import torch
    r, c = x.shape
    amax = x.abs().reshape(r // blk, blk, c // blk, blk).amax(dim=(1, 3))
    e = torch.where(amax > 0, torch.ceil(torch.log2(amax / 448.0)), torch.zeros_like(amax))
    s = torch.exp2(e).float()
    full = s.repeat_interleave(blk, 0).repeat_interleave(blk, 1)
    q = (x / full).to(torch.float8_e4m3fn).view(torch.uint8)
    return q.contiguous(), s.contiguous()


def device_operands(w: Workload, seed: int, dev):
    """Operands of a tensor-core workload drawn on the device (torch.Generator(seed)):
    (A, B, a_scale, b_scale).  bf16: N(0,1) rounded to bf16; bf16x3 / bf16x6: the binary32
    N(0,1) values; fp8: U[-1,1] x 10^U(-2,2) per row, quantised by fp8_quantize_dev
    (scales returned, None otherwise)."""
    import torch
    g = torch.Generator(device=dev).manual_seed(seed)
    if w.dtype == "fp8":
        out = []
        for rows, cols in ((w.m, w.k), (w.k, w.n)):
            x = torch.rand(rows, cols, generator=g, device=dev) * 2 - 1
            x *= 10.0 ** (torch.rand(rows, 1, generator=g, device=dev) * 4 - 2)
            out.append(fp8_quantize_dev(x))
            del x
        (qa, sa), (qb, sb) = out
        return qa, qb, sa, sb
    A = torch.randn(w.m, w.k, generator=g, device=dev)
    B = torch.randn(w.k, w.n, generator=g, device=dev)
    if w.dtype == "bf16":
        A, B = A.to(torch.bfloat16), B.to(torch.bfloat16)
    return A, B, None, None


@dataclass(frozen=True)
class GroupWorkload:
    """Many independent bf16 problems: m, n, k uniform over multiples of `step` in
    [lo, hi]; one accumulator bit flip in a `fault_frac` share of the instances."""
    name: str
    count: int
    lo: int = 64
    hi: int = 2048
    step: int = 64
    fault_frac: float = 0.01
    note: str = ""


BF16_GROUPED_4096 = GroupWorkload(
    "bf16_grouped_4096", 4096,
    note="4096 independent BF16 GEMMs, m, n, k uniform over multiples of 64 in [64, 2048], "
         "N(0,1) rounded to BF16, FP32 accumulate; one fp32 accumulator flip in 1% (41) of the "
         "instances at seeded positions")
BF16_GROUPED_512 = GroupWorkload("bf16_grouped_512", 512, note="the same recipe, 512 problems")
GROUP_WORKLOADS = {w.name: w for w in (BF16_GROUPED_4096, BF16_GROUPED_512)}


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Independent PCG64 stream per (seed, stream)."""
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def operand(shape, dist: str, seed: int, stream: int) -> np.ndarray:
    """A float64 matrix with the named distribution."""
    g = rng(seed, stream)
    if dist == "uniform":
        return g.uniform(-1.0, 1.0, size=shape)
    if dist == "normal":
        return g.standard_normal(size=shape)
    if dist == "int":
        return g.integers(-4, 5, size=shape).astype(np.float64)
    if dist == "fp8rows":  # U[-1,1] times 10^U(-2,2), one magnitude per row
        x = g.uniform(-1.0, 1.0, size=shape)
        return x * 10.0 ** g.uniform(-2.0, 2.0, size=(shape[0], 1))
    raise ValueError(dist)


def operands(w: Workload, seed: int, m=None, n=None, k=None):
    """(A, B) as float64 for workload w (optionally at a reduced shape)."""
    m, n, k = m or w.m, n or w.n, k or w.k
    return operand((m, k), w.dist, seed, 1), operand((k, n), w.dist, seed, 2)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round-to-nearest-even, via torch on the CPU) and
    return the raw 16-bit patterns."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16).copy()


def bit_flips(seed: int, m: int, n: int, count: int, bits: int = 64, stream: int = 7,
              distinct_blocks=None, avoid_blocks=()):
    """count (row, col, bit) triples, uniform positions and bits.

    distinct_blocks=(bs_r, bs_c) forces the flips into distinct blocks of that size,
    none of them in avoid_blocks.
    """
    g = rng(seed, stream)
    out, used = [], set(tuple(b) for b in avoid_blocks)
    if distinct_blocks is not None:
        nb = -(-m // distinct_blocks[0]) * -(-n // distinct_blocks[1])
        free = nb - len({b for b in used
                         if 0 <= b[0] < -(-m // distinct_blocks[0])
                         and 0 <= b[1] < -(-n // distinct_blocks[1])})
        if count > free:
            raise ValueError(f"{count} flips in distinct blocks, but only {free} blocks are free")
    while len(out) < count:
        i, j, b = int(g.integers(0, m)), int(g.integers(0, n)), int(g.integers(0, bits))
        if distinct_blocks is not None:
            blk = (i // distinct_blocks[0], j // distinct_blocks[1])
            if blk in used:
                continue
            used.add(blk)
        elif any((i, j) == (r, c) for r, c, _ in out):
            continue
        out.append((i, j, b))
    return out


def erased_blocks(seed: int, p: int, q: int, count: int, stream: int = 8):
    """count distinct (bi, bj) grid positions, at most one per block column."""
    g = rng(seed, stream)
    out, cols = [], set()
    while len(out) < count:
        bi, bj = int(g.integers(0, p)), int(g.integers(0, q))
        if bj in cols:
            continue
        cols.add(bj)
        out.append((bi, bj))
    return out


def flip_f64(C: np.ndarray, flips) -> np.ndarray:
    """XOR the given bits of float64 elements (in place on a copy)."""
    C = np.array(C, dtype=np.float64, copy=True)
    u = C.view(np.uint64)
    for i, j, b in flips:
        u[i, j] ^= np.uint64(1) << np.uint64(b)
    return C


def flip_f32(C: np.ndarray, flips) -> np.ndarray:
    C = np.array(C, dtype=np.float32, copy=True)
    u = C.view(np.uint32)
    for i, j, b in flips:
        u[i, j] ^= np.uint32(1) << np.uint32(b)
    return C


def group_shapes(seed: int, w: GroupWorkload):
    """(m, n, k) of every problem of a grouped workload."""
    g = rng(seed, 20)
    v = w.step * g.integers(w.lo // w.step, w.hi // w.step + 1, size=(w.count, 3))
    return [tuple(int(x) for x in row) for row in v]


def group_operand_bits(seed: int, p: int, which: int, rows: int, cols: int, ld: int = 0):
    """bf16 bit patterns (rows x ld, zero padding past cols) of iid N(0,1) values for
    operand `which` (0 = A, 1 = B) of problem p (stream 100000 + 2p + which)."""
    ld = ld or (cols + 7) // 8 * 8
    x = rng(seed, 100000 + 2 * p + which).standard_normal(size=(rows, cols), dtype=np.float32)
    out = np.zeros((rows, ld), np.uint16)
    out[:, :cols] = bf16_bits(x)
    return out


def faulty_instances(seed: int, count: int, frac: float):
    """Sorted indices of the instances that receive a flip (sampled without replacement)."""
    nf = max(1, int(round(frac * count)))
    return sorted(int(i) for i in rng(seed, 21).choice(count, size=nf, replace=False))


E4M3_MAX = 448.0


def quantize_e4m3(x: np.ndarray, blk: int = 128):
    """Quantise to OCP FP8 E4M3 with one binary32 scale per blk x blk block: the scale is
    the power of two 2^ceil(log2(max|x_block| / 448)) (1 for an all-zero block), the codes
    are x / scale rounded to nearest-even E4M3 (torch's conversion on the CPU).  Returns
    (codes uint8, scales float32 of shape ceil(rows/blk) x ceil(cols/blk))."""
    import torch
    x = np.asarray(x, dtype=np.float64)
    rows, cols = x.shape
    br, bc = -(-rows // blk), -(-cols // blk)
    pad = np.zeros((br * blk, bc * blk))
    pad[:rows, :cols] = np.abs(x)
    amax = pad.reshape(br, blk, bc, blk).max(axis=(1, 3))
    with np.errstate(divide="ignore"):
        e = np.where(amax > 0, np.ceil(np.log2(amax / E4M3_MAX)), 0.0)
    scales = np.exp2(e).astype(np.float32)
    full = np.repeat(np.repeat(scales.astype(np.float64), blk, 0), blk, 1)[:rows, :cols]
    t = torch.from_numpy(np.ascontiguousarray(x / full, dtype=np.float32))
    codes = t.to(torch.float8_e4m3fn).view(torch.uint8).numpy().copy()
    return codes, scales
