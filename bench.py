#!/usr/bin/env python3
"""Benchmark of the ABFT GEMM hot path on GB300: prints ONE JSON line.

A step is one pass of the whole path over one synthetic problem: checksum encoding of A
and B, the ABFT product (data + checksum tiles), bit-flips (and, with an erasure grid, one
erased block) injected into C, detect / locate / correct, and the block rebuild.  The
default workload is the paper's 484-process grid restated on one GPU: FP64
m = n = k = 11264 as a 22 x 22 grid of 512 x 512 blocks.  The same run also measures the
bf16 tensor-core workloads (16384^3: bf16 inputs, and fp32 inputs in the split bf16x3
product) and attaches them as "bf16_16384" and "bf16x3_16384".

value       useful TFLOP/s (2mnk per step / step time), operands resident in HBM
overhead    product-only and whole-step time over the checksum-free product of the same
            kernel, minus one
e2e         the same metric through the C ABI with host buffers: every step's pinned
            host -> device copy of A and B and device -> host copy of C inside the timed
            region, pipelined over two device buffer sets (the next step's inputs are
            copied, and the previous step's result read back, while a step computes)
roofline    the product kernel: algorithmic FLOPs per launch / measured launch time
cpu_baseline the CPU oracle on a bounded sample of the workload, on the host cores

--impl reference times the CPU oracle alone (the reference arm of this benchmark).
Multi-GPU (torchrun): each rank runs its own independent problem (weak scaling, no
collective on the data path); value = all ranks' useful FLOPs / max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0806_3121_gb300 import multigpu as mg  # noqa: E402
from paper_0806_3121_gb300 import workloads as wl  # noqa: E402

METRIC = "ABFT GEMM TFLOPS (useful 2mnk) and % overhead vs checksum-free GEMM, same GPU/dtype"
# FP64 peak of GB300 (the DFMA pipe, no FP64 tensor path): 152 SMs x 2 DFMA/clk/SM
# (measured rate) x 2 flop x 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# Measured DRAM read + write per launch of the product kernel at the bench workloads (ncu
# dram__bytes_read.sum + dram__bytes_write.sum, one launch after three warm-up products; the
# counters take one pass, see profiles/), or None when the kernel changed since it was
# captured.  f64: 34.22 + 1.10 GB; bf16 (256-row tiles): 6.77 + 1.17 GB; fp8 (e4m3 data
# tiles): 5.72 + 1.63 GB; bf16x6: 59.96 + 1.58 GB; grouped 4096 (ABFT product after the
# autotuner, default tuning): 19.06 + 20.58 GB.
TRAFFIC_BYTES = {"f64_11264_grid22": 35.32e9, "bf16_16384": 7.95e9, "fp8_16384": 7.35e9,
                 "bf16x6_16384": 61.54e9, "bf16_grouped_4096": 39.64e9}


def bf16_peak():
    """Dense bf16 tensor peak: the measured burst figure, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops (burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s (no MEASURED_PEAKS.json)"


def fp8_peak():
    """Dense FP8 tensor peak: the measured bf16 burst peak times the nominal FP8 / bf16
    ratio (4.5 / 2.25 PFLOP/s dense)."""
    p, src = bf16_peak()
    return 2.0 * p, src + " x 2 (nominal FP8 / bf16 dense ratio)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="f64_11264_grid22")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the bf16_16384 summary")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the dtype peaks (cuBLAS DGEMM, FP8 _scaled_mm, bf16 GEMM at "
                         "8192^3, and a DFMA throughput probe) and print them as one JSON line")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- oracle timing
def oracle_pipeline(A, B, w, blocks: int, seed: int):
    """The CPU oracle's whole path on a leading sub-problem of the workload (full k): for a
    grid workload the leading blocks x blocks blocks with one erasure, else a
    (blocks*128)^2 corner; three flips.  Returns (useful flops, seconds, corner size, seconds
    of the product C = A B alone)."""
    import oracle
    if w.p:
        bs = w.m // w.p
        ms = ns = blocks * bs
        p = q = blocks
    else:
        bs = 128
        ms = ns = blocks * bs
        p = q = 0
    As, Bs = np.ascontiguousarray(A[:ms]), np.ascontiguousarray(B[:, :ns])
    t0 = time.perf_counter()
    enc = oracle.Encoded(As, Bs, w.vb_r, w.vb_c, p, q, dtype=w.dtype)
    tg = time.perf_counter()
    C = oracle.gemm(As, Bs)
    dt_gemm = time.perf_counter() - tg
    flips = wl.bit_flips(seed, ms, ns, 3, distinct_blocks=(bs, bs))
    erased = []
    if p:
        (bi, bj), = wl.erased_blocks(seed, p, q, 1)
        flips = wl.bit_flips(seed, ms, ns, 3, distinct_blocks=(bs, bs), avoid_blocks=[(bi, bj)])
        erased = [(bi, bj)]
    C = wl.flip_f64(C, [(i, j, 62) for i, j, _ in flips])
    for bi, bj in erased:
        C[bi * bs:(bi + 1) * bs, bj * bs:(bj + 1) * bs] = np.nan
    st, rep, C, _ = enc.verify_correct(C, erased=erased)
    for bi, bj in erased:
        enc.recover_block(C, bi, bj)
    dt = time.perf_counter() - t0
    return 2.0 * ms * ns * w.k, dt, ms, dt_gemm


def oracle_group_pipeline(w, seed: int, budget_flops: float = 6e10):
    """The CPU oracle's whole path on the leading problems of a grouped workload (in the
    workload's order, until `budget_flops` useful FLOPs): encode, product, one graded
    flip in each problem the workload marks faulty, verify / correct.  Returns (useful
    flops, seconds, problems)."""
    import oracle
    shapes = wl.group_shapes(seed, w)
    faulty = set(wl.faulty_instances(seed, w.count, w.fault_frac))
    ops, flops = [], 0.0
    for p, (m, n, k) in enumerate(shapes):
        if flops >= budget_flops:
            break
        a = oracle.bf16_to_f64(wl.group_operand_bits(seed, p, 0, m, k)[:, :k])
        b = oracle.bf16_to_f64(wl.group_operand_bits(seed, p, 1, k, n)[:, :n])
        ops.append((p, a, b))
        flops += 2.0 * m * n * k
    t0 = time.perf_counter()
    for p, a, b in ops:
        enc = oracle.Encoded(a, b, 128, 256, dtype="bf16")
        C = oracle.gemm(a, b)
        if p in faulty:
            C[0, 0] = C[0, 0] * 2.0 ** 64
        enc.verify_correct(C)
    return flops, time.perf_counter() - t0, len(ops)


def oracle_cores() -> int:
    """Threads the oracle's GEMM loop runs on (OpenMP; the rest of the oracle is serial)."""
    import oracle
    return oracle.threads()


def cpu_baseline(A, B, w, blocks, seed):
    flops, dt, ms, dt_gemm = oracle_pipeline(A, B, w, blocks, seed)
    what = "erased block + 3 flips" if w.p else "3 flips"
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": oracle_cores(),
            "kind": "oracle", "gemm_only_value": flops / dt_gemm / 1e12,
            "sample": f"oracle encode+gemm+verify/correct{'+recover' if w.p else ''} on a "
                      f"{ms}x{ms} corner of the workload with full k={w.k}, {what}; gemm "
                      f"loop OpenMP over {oracle_cores()} threads, the rest serial; {dt:.1f} s"}


# --------------------------------------------------------------------------- reference arm
def run_reference_grouped(args, w):
    for _ in range(args.warmup):
        oracle_group_pipeline(w, args.seed)
    tot_f, tot_t, npr = 0.0, 0.0, 0
    for _ in range(args.steps):
        f, t, npr = oracle_group_pipeline(w, args.seed)
        tot_f += f
        tot_t += t
    v = tot_f / tot_t / 1e12
    sample = (f"oracle encode+gemm+verify/correct of the first {npr} of the {w.count} problems "
              f"of {w.name} per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic", "config": {"workload": w.name, "problems": w.count, "sample": npr},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": oracle_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    if world > 1:  # the other ranks exit at once: the oracle may use every host core
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
    if args.workload in wl.GROUP_WORKLOADS:
        return run_reference_grouped(args, wl.GROUP_WORKLOADS[args.workload])
    w = wl.WORKLOADS[args.workload]
    if w.dtype == "f64":
        A, B = wl.operands(w, args.seed)
        blocks = 2
    else:
        import oracle
        A = oracle.bf16_to_f64(wl.bf16_bits(wl.operand((1024, w.k), w.dist, args.seed, 1)))
        B = oracle.bf16_to_f64(wl.bf16_bits(wl.operand((w.k, 1024), w.dist, args.seed, 2)))
        blocks = 4
    for _ in range(args.warmup):
        oracle_pipeline(A, B, w, blocks, args.seed)
    tot_f, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        f, t, ms, _ = oracle_pipeline(A, B, w, blocks, args.seed)
        tot_f += f
        tot_t += t
    v = tot_f / tot_t / 1e12
    sample = (f"oracle encode+gemm+verify/correct on a {ms}x{ms} corner of {w.name} "
              f"(k={w.k}) per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": w.dtype,
        "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k,
                   "grid": f"{w.p}x{w.q}" if w.p else None, "sample": f"{ms}x{ms}"},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": oracle_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------------- our arm
def library_context(w, A, B, scales, dev, useful, reps=None):
    """cuBLAS on the same operands, for context (not a baseline of the method): FP64
    DGEMM, bf16 GEMM (bf16 output), binary32 SGEMM with TF32 off for the split dtypes (their
    accuracy class), FP8 torch._scaled_mm with unit per-tensor scales.  Timed with CUDA
    events on torch's current stream after one warm-up; any library error is reported, not
    raised."""
    import torch
    reps = reps or (1 if w.dtype == "f64" else 3)  # an FP64 DGEMM of 11264^3 takes seconds
    try:
        if w.dtype == "fp8":
            a = A.view(torch.float8_e4m3fn)
            b = B.view(torch.float8_e4m3fn).t().contiguous().t()
            one = torch.ones((), dtype=torch.float32, device=dev)
            op, fn = "torch._scaled_mm e4m3 (unit per-tensor scales, fp32 out)", \
                lambda: torch._scaled_mm(a, b, one, one, out_dtype=torch.float32)
        elif w.dtype in ("bf16x3", "bf16x6"):
            torch.backends.cuda.matmul.allow_tf32 = False
            op, fn = "torch.matmul fp32 (SGEMM, TF32 off)", lambda: torch.matmul(A, B)
        else:
            op, fn = f"torch.matmul {w.dtype} ({'bf16' if w.dtype == 'bf16' else 'fp64'} out)", \
                lambda: torch.matmul(A, B)
        out = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        del out
        ms = e0.elapsed_time(e1) / reps
        return {"op": op, "ms": ms, "tflops": useful / (ms * 1e-3) / 1e12}
    except Exception as exc:  # context only: the line stands without it
        return {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}


def run_workload(w, args, dev, rank, world, secondary=False):
    """Measure one workload; returns the JSON dict (without the driver's wrapper keys)."""
    import torch
    from paper_0806_3121_gb300 import abft

    seed = mg.rank_seed(args.seed, rank)
    scales = {}
    if w.dtype == "f64":
        A_np, B_np = wl.operands(w, seed)
        A, B = torch.from_numpy(A_np).to(dev), torch.from_numpy(B_np).to(dev)
    else:
        A_np = B_np = None
        A, B, sa, sb = wl.device_operands(w, seed, dev)
        if sa is not None:
            scales = dict(a_scale=sa, b_scale=sb)
    lp = w.dtype != "f64"
    desc = abft.make_desc(w.m, w.n, w.k, w.dtype, w.vb_r, w.vb_c, w.p, w.q)
    L = abft.abft_workspace_layout(desc)
    stream = torch.cuda.Stream(device=dev)
    C = torch.empty((w.m, w.n), dtype=torch.float32 if lp else torch.float64, device=dev)
    ws = torch.zeros(L.total, dtype=torch.uint8, device=dev)
    # torch's side streams do not wait for its default stream, where the operands were
    # drawn and the workspace zeroed
    stream.wait_stream(torch.cuda.current_stream(dev))
    erased = []
    bs = w.m // w.p if w.p else 512
    if w.n_erased:
        erased = wl.erased_blocks(seed, w.p, w.q, w.n_erased)
    pos = wl.bit_flips(seed, w.m, w.n, w.n_flips, distinct_blocks=(bs, bs), avoid_blocks=erased)
    # graded flips by construction: exponent bits that move the value by many orders
    abft.abft_encode(desc, A, B, ws, stream=stream, **scales)
    abft.abft_gemm(desc, A, B, C, ws, stream=stream)
    torch.cuda.synchronize()
    flips = []
    for t, (i, j, _) in enumerate(pos):
        if lp:
            flips.append((i, j, 29 if abs(C[i, j].item()) >= 2.0 else 30))
        else:
            flips.append((i, j, 62 - t))
    if lp:
        # compute faults: flips of the accumulator outputs, applied in the product's epilogue
        # before C and its fused observed checksums are formed; verify reads those sums
        abft.abft_set_epilogue_faults(desc, ws, flips, stream=stream)

    barrier = mg.barrier

    gemm_ms = []

    def step(timed_gemm=False, bufs=None):
        A_, B_, C_, ws_ = bufs if bufs is not None else (A, B, C, ws)
        abft.abft_encode(desc, A_, B_, ws_, stream=stream, **scales)
        if timed_gemm:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        abft.abft_gemm(desc, A_, B_, C_, ws_, stream=stream)
        if timed_gemm:
            e1.record(stream)
        if not lp:  # memory faults in the stored C
            abft.abft_inject_bitflips(desc, C_, flips, stream=stream)
        for bi, bj in erased:
            abft.abft_erase_block(desc, C_, bi, bj, stream=stream)
        st, rep, n = abft.abft_verify_correct(desc, C_, ws_, erased=erased, stream=stream,
                                              reread_C=0 if lp else 1)
        st2 = abft.OK
        for bi, bj in erased:
            st2, _ = abft.abft_recover_block(desc, C_, ws_, bi, bj, stream=stream)
        if timed_gemm:
            gemm_ms.append(e0.elapsed_time(e1))
        return st, st2, rep

    for _ in range(args.warmup):
        st, st2, rep = step()
    assert st == abft.OK and st2 == abft.OK, (st, st2)
    assert sorted((e["row"], e["col"]) for e in rep) == sorted((i, j) for i, j, _ in flips), rep

    launches0 = abft.abft_kernel_launches()
    with ClockSampler(dev.index) as clk:
        barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(timed_gemm=True)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = abft.abft_kernel_launches() - launches0
    step_ms = t0.elapsed_time(t1) / args.steps
    clocks = clk.summary()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # product-only overhead: checksum-free and ABFT products launched alternately, so
    # both see the same clock and power state; medians of the pairs
    pairs = max(2, min(args.steps, 3)) if not lp else 10
    t_plain, t_abft = [], []
    for _ in range(pairs):
        t_plain.append(timed(lambda: abft.abft_gemm_plain(desc, A, B, C, ws=ws, stream=stream),
                             1))
        t_abft.append(timed(lambda: abft.abft_gemm(desc, A, B, C, ws, stream=stream), 1))
    plain_ms = statistics.median(t_plain)
    abft_pair_ms = statistics.median(t_abft)
    encode_ms = timed(lambda: abft.abft_encode(desc, A, B, ws, stream=stream, **scales), 5)
    gemm_avg = sum(gemm_ms) / len(gemm_ms)

    e2e = None
    if not args.no_e2e and not secondary:
        # Two device buffer sets: step i computes on set i % 2 while the host -> device
        # copy of step i + 1's inputs (copy stream) and the device -> host read of step
        # i - 1's result (read-back stream) run on the copy engines.  Every step's copies
        # are inside the timed region.
        A_h = A.cpu().pin_memory()
        B_h = B.cpu().pin_memory()
        C_h = [torch.empty(C.shape, dtype=C.dtype).pin_memory() for _ in range(2)]
        A2, B2, C2 = torch.empty_like(A), torch.empty_like(B), torch.empty_like(C)
        ws2 = torch.zeros_like(ws)
        stream.wait_stream(torch.cuda.current_stream(dev))
        if lp:  # the armed epilogue faults live in the workspace
            abft.abft_encode(desc, A, B, ws2, stream=stream, **scales)
            abft.abft_set_epilogue_faults(desc, ws2, flips, stream=stream)
        sets = [(A, B, C, ws), (A2, B2, C2, ws2)]
        h2d_s, d2h_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        ev = lambda: torch.cuda.Event()  # noqa: E731
        loaded = [ev(), ev()]     # a set's inputs are on the device
        computed = [ev(), ev()]   # a set's step is done (its C may be read back)
        freed = [ev(), ev()]      # a set's result has been read back (the set may be reused)
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)

        def load(x):
            h2d_s.wait_event(a)
            if used[x]:
                h2d_s.wait_event(freed[x])
            with torch.cuda.stream(h2d_s):
                sets[x][0].copy_(A_h, non_blocking=True)
                sets[x][1].copy_(B_h, non_blocking=True)
            loaded[x].record(h2d_s)
            used[x] = True

        used = [False, False]
        load(0)
        for i in range(args.steps):
            x = i % 2
            if i + 1 < args.steps:
                load(1 - x)
            stream.wait_event(loaded[x])
            step(bufs=sets[x])
            computed[x].record(stream)
            d2h_s.wait_event(computed[x])
            with torch.cuda.stream(d2h_s):
                C_h[x].copy_(sets[x][2], non_blocking=True)
            freed[x].record(d2h_s)
        stream.wait_event(freed[(args.steps - 1) % 2])
        if args.steps > 1:
            stream.wait_event(freed[args.steps % 2])
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = a.elapsed_time(b) / args.steps
        del A2, B2, C2, ws2
        e2e_ms = mg.max_over_ranks(e2e_ms)
        e2e = {"value": 2.0 * w.m * w.n * w.k * world / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": A_h.numel() * A_h.element_size() +
                                     B_h.numel() * B_h.element_size(),
               "d2h_bytes_per_step": C_h[0].numel() * C_h[0].element_size()}

    step_ms = mg.max_over_ranks(step_ms)

    useful = 2.0 * w.m * w.n * w.k
    if lp:
        nseg = {"bf16x3": 3, "bf16x6": 6}.get(w.dtype, 1)  # split products: 3 or 6 bf16 products
        kernel_flops = nseg * 2.0 * w.k * ((w.m + L.acs_rows) * w.n + w.m * L.bcs_cols)
        peak, peak_src = fp8_peak() if w.dtype == "fp8" else bf16_peak()
        roof = {"kernel": "k_gemm_bf16", "bound": "tensor", "peak_source": peak_src}
    else:
        kernel_flops = 2.0 * w.k * ((w.m + L.R) * w.n + w.m * L.Cc)
        peak, peak_src = FP64_PEAK_TFLOPS, "152 SMs x 2 DFMA/clk/SM (measured) x 2 flop x 2070 MHz"
        roof = {"kernel": "k_gemm_f64", "bound": "alu", "peak_source": peak_src}
    achieved = kernel_flops / (gemm_avg * 1e-3) / 1e12
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "traffic": TRAFFIC_BYTES.get(w.name), "algorithmic_flops_per_launch": kernel_flops})
    value = mg.weak_scaling_value(useful, world, step_ms)
    cfg = {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "verify_block": [w.vb_r, w.vb_c],
           "dist": {"fp8": "U[-1,1] x 10^U(-2,2) per row, e4m3 with power-of-two binary32 "
                           "scales per 128x128 block (product of the exact dequantised values "
                           "on the bf16 tensor path)"}.get(
                w.dtype, "N(0,1)" + {"bf16": " rounded to bf16", "bf16x3": " in fp32, split "
                                     "into bf16 hi+lo", "bf16x6": " in fp32, split into three "
                                     "bf16 pieces"}.get(w.dtype, "")),
           "faults_per_step": (f"{w.n_erased} erased block + " if w.n_erased else "") +
                              f"{w.n_flips} exponent bit-flips in distinct blocks" +
                              (" of the accumulator outputs (epilogue), verified from the "
                               "fused observed checksums" if lp else " of the stored C, "
                               "verified by re-reading C"),
           "l2": "operands larger than L2 (129 MB)",
           "parallelism": f"{world} independent problems (one per GPU)"}
    if w.p:
        cfg.update({"grid": f"{w.p}x{w.q}", "block": bs})
    out = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": w.dtype, "data": "synthetic", "config": cfg,
        "overhead_pct": {
            "gemm_only": 100.0 * (abft_pair_ms / plain_ms - 1.0),
            "step_without_encode": 100.0 * ((step_ms - encode_ms) / plain_ms - 1.0),
            "end_to_end_step": 100.0 * (step_ms / plain_ms - 1.0)},
        "times_ms": {"step": step_ms, "abft_gemm_in_step": gemm_avg,
                     "abft_gemm_paired": abft_pair_ms, "plain_gemm_paired": plain_ms,
                     "encode": encode_ms},
        "useful_frac_of_peak": (useful / (step_ms * 1e-3) / 1e12) / peak,
        "roofline": roof, "gpu_launches": launches, "clocks": clocks, "e2e": e2e,
        "library_context": library_context(w, A, B, scales, dev, useful),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not secondary:
        if A_np is None:
            # the leading 1024 rows of A and columns of B, as exact binary64 values
            import oracle
            if w.dtype == "bf16":
                A_np = oracle.bf16_to_f64(A[:1024].cpu().view(torch.int16).numpy().view(np.uint16))
                B_np = oracle.bf16_to_f64(B[:, :1024].contiguous().cpu().view(torch.int16).numpy()
                                          .view(np.uint16))
            elif w.dtype == "fp8":
                A_np = oracle.dequant_e4m3(A[:1024].cpu().numpy(), scales["a_scale"][:8].cpu().numpy())
                B_np = oracle.dequant_e4m3(B[:, :1024].contiguous().cpu().numpy(),
                                           scales["b_scale"][:, :8].contiguous().cpu().numpy())
            else:  # the split dtypes take binary32 inputs
                A_np = A[:1024].double().cpu().numpy()
                B_np = B[:, :1024].double().cpu().numpy()
            out["cpu_baseline"] = cpu_baseline(A_np, B_np, w, 8, seed)
        else:
            out["cpu_baseline"] = cpu_baseline(A_np, B_np, w, 4, seed)
    if w.p and not secondary:
        out["multi_erasure"] = multi_erasure_leg(w, A, B, dev, stream, seed)
    del A, B, C, ws
    torch.cuda.empty_cache()
    return out


def multi_erasure_leg(w, A, B, dev, stream, seed, f=2):
    """Two block checksums (grid_f = 2) on the same operands: two erased blocks of one block
    column rebuilt from the checksums and the survivors by the binary64 2 x 2 solve.  One
    encode + product (not timed), then the rebuild timed with CUDA events and its error
    against the values before the erasure.  Returns the dict attached to the JSON line."""
    import torch
    from paper_0806_3121_gb300 import abft
    desc = abft.make_desc(w.m, w.n, w.k, w.dtype, w.vb_r, w.vb_c, w.p, w.q, grid_f=f)
    L = abft.abft_workspace_layout(desc)
    ws = torch.zeros(L.total, dtype=torch.uint8, device=dev)
    C = torch.empty((w.m, w.n), dtype=torch.float64, device=dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    abft.abft_encode(desc, A, B, ws, stream=stream)
    abft.abft_gemm(desc, A, B, C, ws, stream=stream)
    bs, bc = w.m // w.p, w.n // w.q
    g = wl.rng(seed, 9)
    bj = int(g.integers(0, w.q))
    rows = sorted(int(x) for x in g.choice(w.p, size=f, replace=False))
    blocks = [(bi, bj) for bi in rows]
    torch.cuda.synchronize()
    saved = [C[bi * bs:(bi + 1) * bs, bj * bc:(bj + 1) * bc].clone() for bi, _ in blocks]
    for bi, _ in blocks:
        abft.abft_erase_block(desc, C, bi, bj, stream=stream)
    st, rep, n = abft.abft_verify_correct(desc, C, ws, erased=blocks, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st2, ents = abft.abft_recover_blocks(desc, C, ws, blocks, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    err = max(((C[bi * bs:(bi + 1) * bs, bj * bc:(bj + 1) * bc] - sv).norm() / sv.norm()).item()
              for (bi, _), sv in zip(blocks, saved))
    # algorithmic bytes: the survivors of the block column, the f checksum blocks, the
    # rebuilt blocks written and read back by the re-check
    nbytes = 8 * bs * bc * ((w.p - f) + f + 2 * f)
    out = {"grid_f": f, "erased_blocks": blocks, "verify_status": st, "recover_status": st2,
           "recover_ms": ms, "recover_GBps": nbytes / (ms * 1e-3) / 1e9,
           "max_rel_err_rebuilt_block": err}
    del ws, C
    return out


def run_grouped(w, args, dev, rank, world, secondary=False):
    """The grouped workload: `w.count` independent bf16 problems in one persistent product
    launch; a step is the captured graph (ABFT product of every problem with one armed
    accumulator flip in each faulty instance, fused verify, locate / correct) plus the
    report read.  Returns the JSON dict."""
    import torch
    from paper_0806_3121_gb300 import abft

    seed = mg.rank_seed(args.seed, rank)
    shapes = wl.group_shapes(seed, w)
    g = torch.Generator(device=dev).manual_seed(seed)
    As, Bs, Cs, probs = [], [], [], []
    for (m, n, k) in shapes:
        As.append(torch.randn(m, k, generator=g, device=dev).to(torch.bfloat16))
        Bs.append(torch.randn(k, n, generator=g, device=dev).to(torch.bfloat16))
        Cs.append(torch.empty((m, n), dtype=torch.float32, device=dev))
        probs.append(dict(m=m, n=n, k=k, A=As[-1], B=Bs[-1], C=Cs[-1]))
    stream = torch.cuda.Stream(device=dev)
    grp = abft.abft_group_create(probs, "bf16")
    ws = torch.zeros(abft.abft_group_workspace_bytes(grp), dtype=torch.uint8, device=dev)
    stream.wait_stream(torch.cuda.current_stream(dev))  # operands and ws on the default stream
    abft.abft_group_bind(grp, ws, stream=stream)
    tuning, tune_ms = abft.abft_group_autotune(grp, reps=3, stream=stream)
    abft.abft_group_encode(grp, stream=stream)
    abft.abft_group_gemm(grp, True, stream=stream)
    torch.cuda.synchronize()
    faulty = wl.faulty_instances(seed, w.count, w.fault_frac)
    gr = wl.rng(seed, 22)
    flips = []
    for p in faulty:
        m, n, _ = shapes[p]
        i, j = int(gr.integers(0, m)), int(gr.integers(0, n))
        # a graded flip by construction: an exponent bit that moves the value by >= 2^64
        flips.append((p, i, j, 29 if abs(Cs[p][i, j].item()) >= 2.0 else 30))
    abft.abft_group_set_epilogue_faults(grp, flips, stream=stream)
    abft.abft_group_capture(grp, True, stream=stream)

    def step():
        abft.abft_group_launch(grp, stream=stream)
        return abft.abft_group_report(grp, max_reports=4 * len(flips) + 16, stream=stream)

    for _ in range(args.warmup):
        st, rep, nrep = step()
    assert st == abft.OK, st
    assert sorted((e["problem"], e["row"], e["col"]) for e in rep) == \
        sorted((p, i, j) for p, i, j, _ in flips), rep

    barrier = mg.barrier

    launches0 = abft.abft_kernel_launches()
    with ClockSampler(dev.index) as clk:
        barrier()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step()
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = abft.abft_kernel_launches() - launches0
    step_ms = t0.elapsed_time(t1) / args.steps
    clocks = clk.summary()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    t_plain, t_abft = [], []
    for _ in range(10):
        t_plain.append(timed(lambda: abft.abft_group_gemm(grp, False, stream=stream), 1))
        t_abft.append(timed(lambda: abft.abft_group_gemm(grp, True, stream=stream), 1))
    plain_ms, abft_ms = statistics.median(t_plain), statistics.median(t_abft)
    verify_ms = timed(lambda: abft.abft_group_verify_enqueue(grp, stream=stream), 5)
    encode_ms = timed(lambda: abft.abft_group_encode(grp, stream=stream), 3)
    abft.abft_group_set_epilogue_faults(grp, [], stream=stream)

    useful = sum(2.0 * m * n * k for m, n, k in shapes)
    cs_flops = sum(2.0 * k * (4 * -(-m // 128) * n + m * 4 * -(-n // 256)) for m, n, k in shapes)
    peak, peak_src = bf16_peak()
    achieved = (useful + cs_flops) / (abft_ms * 1e-3) / 1e12
    step_ms = mg.max_over_ranks(step_ms)
    out = {
        "metric": METRIC, "value": mg.weak_scaling_value(useful, world, step_ms), "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": w.name, "problems": w.count,
                   "shapes": f"m, n, k uniform over multiples of {w.step} in [{w.lo}, {w.hi}]",
                   "verify_block": [128, 256], "dist": "N(0,1) rounded to bf16",
                   "faults_per_step": f"one exponent flip of an accumulator output in each of "
                                      f"{len(flips)} instances ({w.fault_frac:.0%})",
                   "tuning": tuning, "step": "CUDA graph: grouped ABFT product + fused "
                                             "verify + locate/correct, then the report read "
                                             "(operands encoded once, outside the step)",
                   "l2": "operands larger than L2 (129 MB)",
                   "parallelism": f"{world} independent groups (one per GPU)"},
        # the step re-uses the encoded operands; end_to_end_step adds the group's encode
        # (timed alone) to it, as the single-problem lines' steps include theirs
        "overhead_pct": {"gemm_only": 100.0 * (abft_ms / plain_ms - 1.0),
                         "step_without_encode": 100.0 * (step_ms / plain_ms - 1.0),
                         "end_to_end_step": 100.0 * ((step_ms + encode_ms) / plain_ms - 1.0)},
        "times_ms": {"step": step_ms, "abft_gemm_paired": abft_ms, "plain_gemm_paired": plain_ms,
                     "verify": verify_ms, "encode": encode_ms,
                     "autotune_best": tune_ms},
        "useful_frac_of_peak": (useful / (step_ms * 1e-3) / 1e12) / peak,
        "plain_useful_tflops": useful / (plain_ms * 1e-3) / 1e12,
        "roofline": {"kernel": "k_gemm_grouped", "bound": "tensor", "peak_source": peak_src,
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": TRAFFIC_BYTES.get(w.name),
                     "algorithmic_flops_per_launch": useful + cs_flops},
        "library_context": {"unavailable": "torch has no grouped GEMM of uneven shapes"},
        "gpu_launches": launches, "clocks": clocks, "e2e": None,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not secondary:
        f, dt, npr = oracle_group_pipeline(w, seed)
        out["cpu_baseline"] = {
            "value": f / dt / 1e12, "unit": "TFLOP/s", "cores": oracle_cores(), "kind": "oracle",
            "sample": f"oracle encode+gemm+verify/correct of the first {npr} problems of the "
                      f"recipe (host-drawn operands of the same shapes and distribution); "
                      f"{dt:.1f} s"}
    abft.abft_group_destroy(grp)
    del As, Bs, Cs, ws
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world):
    import torch
    from paper_0806_3121_gb300 import abft, build

    build.build()
    abft.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    if args.workload in wl.GROUP_WORKLOADS:
        out = run_grouped(wl.GROUP_WORKLOADS[args.workload], args, dev, rank, world)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    w = wl.WORKLOADS[args.workload]
    secondary = {}
    keys = ("value", "unit", "ms_per_step", "overhead_pct", "times_ms", "useful_frac_of_peak",
            "roofline", "gpu_launches", "clocks", "config", "library_context")
    if w.name == "f64_11264_grid22" and not args.no_secondary:
        # the tensor-core workloads first: the FP64 run is a minute of full-power load
        for name in ("bf16_16384", "bf16x3_16384", "bf16x6_16384", "fp8_16384"):
            sec = run_workload(wl.WORKLOADS[name], args, dev, rank, world, secondary=True)
            secondary[name] = {k: sec[k] for k in keys}
        sec = run_grouped(wl.BF16_GROUPED_4096, args, dev, rank, world, secondary=True)
        secondary[wl.BF16_GROUPED_4096.name] = {k: sec[k] for k in keys + ("plain_useful_tflops",)}
    out = run_workload(w, args, dev, rank, world)
    out.update(secondary)
    out["summary"] = summary(out, secondary)
    if rank == 0:
        print(json.dumps(out), flush=True)


def summary(main, secondary):
    """One short row per workload, the last key of the line (a reader of the line's tail
    sees every workload): useful TF/s per step, product-only and whole-step overhead over
    the checksum-free product, roofline fraction of the product kernel, encode ms and the
    median SM clock under load."""
    rows = {"cols": "useful TF/s | product ovh % | step ovh % | roofline frac | encode ms | "
                    "SM MHz"}
    for name, d in [(main["config"]["workload"], main)] + list(secondary.items()):
        ov, tm = d.get("overhead_pct", {}), d.get("times_ms", {})
        rows[name] = [round(d["value"], 3), round(ov.get("gemm_only", float("nan")), 2),
                      round(ov.get("end_to_end_step", ov.get("step", float("nan"))), 2),
                      round(d["roofline"]["frac"], 3), round(tm.get("encode", float("nan")), 3),
                      (d.get("clocks") or {}).get("sm_mhz")]
    return rows


# --------------------------------------------------------------------------- peaks
DFMA_PROBE = r"""
#include <cuda_runtime.h>
// Independent chains of binary64 fused multiply-adds: each thread runs 8 chains of
// `iters` steps (16 flops per step); enough warps per SM to hide the pipe latency.
__global__ void k_dfma(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5,
         x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
extern "C" double dfma_tflops(int iters, int reps) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 512, blocks = sms * 4;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    k_dfma<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaFree(out);
  if (err != cudaSuccess) return -2.0;
  return 16.0 * iters * (double)threads * blocks / (best * 1e-3) / 1e12;
}
"""


def run_peaks(args):
    """Dtype peaks on this GPU, for the roofline denominators: best of 10 at 8192^3 of
    cuBLAS DGEMM (torch.matmul float64), FP8 torch._scaled_mm (e4m3, unit scales, bf16 and
    fp32 out) and bf16 torch.matmul, plus a DFMA throughput probe (independent fma chains,
    best of 10).  nvidia-smi clocks are sampled during the measurements."""
    import ctypes
    import torch
    dev = torch.device("cuda", 0)
    n = 8192
    out = {"what": "dtype peaks, best of 10 at 8192^3 (2 n^3 flops), CUDA events"}

    def best(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return 2.0 * n ** 3 / (min(ts) * 1e-3) / 1e12

    src = os.path.join(ROOT, "paper_0806_3121_gb300", "_build", "dfma_probe.cu")
    lib = src[:-3] + ".so"
    os.makedirs(os.path.dirname(src), exist_ok=True)
    with open(src, "w") as f:
        f.write(DFMA_PROBE)
    from paper_0806_3121_gb300 import build
    subprocess.run([build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                    "-Xcompiler", "-fPIC", src, "-o", lib], check=True)
    with ClockSampler(0) as clk:
        x = torch.randn(n, n, device=dev, dtype=torch.float64)
        out["fp64_dgemm_tflops"] = best(lambda: torch.matmul(x, x))
        del x
        probe = ctypes.CDLL(lib)
        probe.dfma_tflops.restype = ctypes.c_double
        probe.dfma_tflops.argtypes = [ctypes.c_int, ctypes.c_int]
        out["fp64_dfma_probe_tflops"] = probe.dfma_tflops(20000, 10)
        a = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn).t().contiguous().t()
        one = torch.ones((), dtype=torch.float32, device=dev)
        out["fp8_scaled_mm_bf16out_tflops"] = best(
            lambda: torch._scaled_mm(a, b, one, one, out_dtype=torch.bfloat16))
        out["fp8_scaled_mm_fp32out_tflops"] = best(
            lambda: torch._scaled_mm(a, b, one, one, out_dtype=torch.float32))
        del a, b
        x = torch.randn(n, n, device=dev, dtype=torch.bfloat16)
        out["bf16_matmul_tflops"] = best(lambda: torch.matmul(x, x))
    out["clocks"] = clk.summary()
    out["gpu"] = torch.cuda.get_device_name(dev)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.peaks:
        run_peaks(args)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if world > 1 and args.impl == "ours":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
