#!/usr/bin/env python3
"""Benchmark of the ABFT GEMM hot path on GB300: prints ONE JSON line.

A step is one pass of the whole path over one synthetic problem: checksum encoding of A
and B, the ABFT product (data + checksum tiles), three bit-flips and one erased block
injected into C, detect / locate / correct, and rebuilding the erased block.  The
workload is the paper's 484-process grid restated on one GPU: FP64 m = n = k = 11264 as a
22 x 22 grid of 512 x 512 blocks.

value       useful TFLOP/s (2mnk per step / step time), operands resident in HBM
overhead    step (and product-only) time over the checksum-free product of the same
            kernel, minus one
e2e         the same metric through the C ABI with host buffers: pinned host -> device
            copy of A and B and device -> host copy of C inside the timed region
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

from paper_0806_3121_gb300 import workloads as wl  # noqa: E402

METRIC = "ABFT GEMM TFLOPS (useful 2mnk) and % overhead vs checksum-free GEMM, same GPU/dtype"
# FP64 peak of GB300 (the DFMA pipe, no FP64 tensor path): 152 SMs x 2 DFMA/clk/SM
# (measured rate) x 2 flop x 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# Measured DRAM traffic of one k_gemm_f64 launch at this workload (ncu, see profiles/),
# or None when the kernel changed since it was captured.
GEMM_TRAFFIC_BYTES = None


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
    """The CPU oracle's whole path on the leading blocks x blocks sub-grid of the workload
    (full k).  Returns (useful flops, seconds)."""
    import oracle
    bs = w.m // w.p
    ms = ns = blocks * bs
    As, Bs = np.ascontiguousarray(A[:ms]), np.ascontiguousarray(B[:, :ns])
    t0 = time.perf_counter()
    enc = oracle.Encoded(As, Bs, w.vb_r, w.vb_c, blocks, blocks)
    C = oracle.gemm(As, Bs)
    (bi, bj), = wl.erased_blocks(seed, blocks, blocks, 1)
    flips = wl.bit_flips(seed, ms, ns, 3, distinct_blocks=(bs, bs), avoid_blocks=[(bi, bj)])
    C = wl.flip_f64(C, flips)
    C[bi * bs:(bi + 1) * bs, bj * bs:(bj + 1) * bs] = np.nan
    st, rep, C, _ = enc.verify_correct(C, erased=[(bi, bj)])
    st2, C, _ = enc.recover_block(C, bi, bj)
    dt = time.perf_counter() - t0
    return 2.0 * ms * ns * w.k, dt


def cpu_baseline(A, B, w, blocks, seed):
    flops, dt = oracle_pipeline(A, B, w, blocks, seed)
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"oracle encode+gemm+verify/correct+recover on the leading {blocks}x{blocks} "
                      f"blocks of the grid ({blocks * (w.m // w.p)}^2 x k={w.k}), 3 flips + 1 "
                      f"erased block; gemm loop OpenMP over all cores, the rest serial; "
                      f"{dt:.1f} s"}


# --------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    w = wl.WORKLOADS[args.workload]
    A, B = wl.operands(w, args.seed)
    blocks = 2
    for _ in range(args.warmup):
        oracle_pipeline(A, B, w, blocks, args.seed)
    tot_f, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        f, t = oracle_pipeline(A, B, w, blocks, args.seed)
        tot_f += f
        tot_t += t
    v = tot_f / tot_t / 1e12
    sample = (f"oracle encode+gemm+verify/correct+recover on the leading {blocks}x{blocks} blocks "
              f"of the grid ({blocks * 512}^2 x k={w.k}) per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "grid": f"{w.p}x{w.q}",
                   "block": w.m // w.p, "sample_blocks": blocks},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------------- our arm
def run_ours(args, rank, world):
    import torch
    from paper_0806_3121_gb300 import abft, build

    build.build()
    lib = abft.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = wl.WORKLOADS[args.workload]
    assert w.dtype == "f64"
    seed = args.seed + rank
    A_np, B_np = wl.operands(w, seed)
    desc = abft.make_desc(w.m, w.n, w.k, "f64", w.vb_r, w.vb_c, w.p, w.q)
    (bi, bj), = wl.erased_blocks(seed, w.p, w.q, w.n_erased)
    bs = w.m // w.p
    flips = wl.bit_flips(seed, w.m, w.n, w.n_flips, distinct_blocks=(bs, bs),
                         avoid_blocks=[(bi, bj)])
    flips = [(i, j, 62 - t) for t, (i, j, _) in enumerate(flips)]  # graded exponent flips

    stream = torch.cuda.Stream(device=dev)
    A = torch.from_numpy(A_np).to(dev)
    B = torch.from_numpy(B_np).to(dev)
    C = torch.empty((w.m, w.n), dtype=torch.float64, device=dev)
    ws = torch.zeros(abft.abft_workspace_bytes(desc), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    gemm_ms = []

    def step(timed_gemm=False):
        abft.abft_encode(desc, A, B, ws, stream=stream)
        if timed_gemm:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        abft.abft_gemm(desc, A, B, C, ws, stream=stream)
        if timed_gemm:
            e1.record(stream)
        abft.abft_inject_bitflips(desc, C, flips, stream=stream)
        abft.abft_erase_block(desc, C, bi, bj, stream=stream)
        st, rep, n = abft.abft_verify_correct(desc, C, ws, erased=[(bi, bj)], stream=stream)
        st2, _ = abft.abft_recover_block(desc, C, ws, bi, bj, stream=stream)
        if timed_gemm:
            gemm_ms.append(e0.elapsed_time(e1))
        return st, st2, rep

    for _ in range(args.warmup):
        st, st2, rep = step()
    assert st == abft.OK and st2 == abft.OK, (st, st2)
    assert sorted((e["row"], e["col"]) for e in rep) == sorted((i, j) for i, j, _ in flips), rep

    # ---- timed: the whole path
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

    # ---- checksum-free product of the same kernel, and the encode alone
    def timed(fn, reps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    reps = max(2, min(args.steps, 3))
    plain_ms = timed(lambda: abft.abft_gemm_plain(desc, A, B, C, stream=stream), reps)
    encode_ms = timed(lambda: abft.abft_encode(desc, A, B, ws, stream=stream), 5)
    gemm_avg = sum(gemm_ms) / len(gemm_ms)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        A_h = torch.from_numpy(A_np).pin_memory()
        B_h = torch.from_numpy(B_np).pin_memory()
        C_h = torch.empty((w.m, w.n), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                A.copy_(A_h, non_blocking=True)
                B.copy_(B_h, non_blocking=True)
            step()
            with torch.cuda.stream(stream):
                C_h.copy_(C, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = a.elapsed_time(b) / args.steps
        e2e = {"value": 2.0 * w.m * w.n * w.k / (e2e_ms * 1e-3) / 1e12 * world, "unit": "TFLOP/s",
               "h2d_bytes_per_step": A_h.numel() * 8 + B_h.numel() * 8,
               "d2h_bytes_per_step": C_h.numel() * 8 + 4}
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e["value"] = 2.0 * w.m * w.n * w.k * world / (t.item() * 1e-3) / 1e12

    # ---- max over ranks
    if world > 1:
        t = torch.tensor([step_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        step_ms = t.item()

    useful = 2.0 * w.m * w.n * w.k
    L = abft.abft_workspace_layout(desc)
    kernel_flops = 2.0 * w.k * ((w.m + L.R) * w.n + w.m * L.Cc)
    achieved = kernel_flops / (gemm_avg * 1e-3) / 1e12
    out = {
        "metric": METRIC,
        "value": useful * world / (step_ms * 1e-3) / 1e12,
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "grid": f"{w.p}x{w.q}",
                   "block": bs, "verify_block": w.vb_r, "dist": "N(0,1)",
                   "faults_per_step": "1 erased block + 3 exponent bit-flips in distinct blocks",
                   "l2": "inputs larger than L2 (A, B, C 1.0 GB each)",
                   "parallelism": f"{world} independent problems (one per GPU)"},
        "overhead_pct": {
            "gemm_only": 100.0 * (gemm_avg / plain_ms - 1.0),
            "step_without_encode": 100.0 * ((step_ms - encode_ms) / plain_ms - 1.0),
            "end_to_end_step": 100.0 * (step_ms / plain_ms - 1.0)},
        "times_ms": {"step": step_ms, "abft_gemm": gemm_avg, "plain_gemm": plain_ms,
                     "encode": encode_ms},
        "fraction_of_fp64_peak": (useful / (step_ms * 1e-3) / 1e12) / FP64_PEAK_TFLOPS,
        "roofline": {"kernel": "k_gemm_f64", "bound": "alu", "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": GEMM_TRAFFIC_BYTES,
                     "algorithmic_flops_per_launch": kernel_flops,
                     "peak_source": "152 SMs x 2 DFMA/clk/SM (measured) x 2 flop x 2070 MHz"},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(A_np, B_np, w, 4, seed)
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse()
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
