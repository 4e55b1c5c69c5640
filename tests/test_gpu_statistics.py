"""Seeded statistics of the workloads' fault recipes on the GPU, against the CPU oracle.

* fault-free runs report nothing, over 100 seeds each: the FP64 512^3 workload (config 1),
  the bf16 product at 2048^3 (config 3 scaled down) and groups of 64 problems of the
  grouped recipe (config 5 scaled down);
* the accumulator-flip rate of the bf16 workload, 1e-9 per element of the full 16384^2
  output, drawn over 100 seeds (about 27 flips in all, uniform positions and fp32 bits):
  each flip is classified by the oracle from its own rows and columns (graded: must be
  located; benign: must stay silent; guard band: either), and nothing else is reported;
* the 4096-problem grouped workload at the bench's size and recipe, seeds 0..4 (device
  operands from the seeded generator, one graded flip in 41 instances): for every faulty
  instance the
  decisions (positions and kinds) equal the oracle's on the same C, and the other 4055
  instances report nothing.

The single-flip parity of config 1 over seeds 0..99 is in test_gpu_f64.py."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


def bf16_randn(rows, cols, g):
    return torch.randn(rows, cols, generator=g, device="cuda").to(torch.bfloat16)


def to_f64(t):
    """Exact binary64 values of a bf16 device tensor (through the oracle's decoder)."""
    return oracle.bf16_to_f64(t.contiguous().cpu().view(torch.int16).numpy().view(np.uint16))


# --------------------------------------------------------------- fault-free, 100 seeds
def test_config1_fault_free_100_seeds():
    w = wl.F64_512
    desc = abft.make_desc(w.m, w.n, w.k, "f64", w.vb_r, w.vb_c)
    ws = torch.zeros(abft.abft_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
    C = torch.empty((w.m, w.n), dtype=torch.float64, device="cuda")
    for seed in range(100):
        A, B = (torch.from_numpy(x).cuda() for x in wl.operands(w, seed))
        abft.abft_encode(desc, A, B, ws)
        abft.abft_gemm(desc, A, B, C, ws)
        st, rep, n = abft.abft_verify_correct(desc, C, ws)
        assert st == abft.OK and n == 0, (seed, rep)


def test_config3_scaled_fault_free_100_seeds():
    m = n = k = 2048
    desc = abft.make_desc(m, n, k, "bf16", 256, 256)
    ws = torch.zeros(abft.abft_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    for seed in range(100):
        g = torch.Generator(device="cuda").manual_seed(seed)
        A, B = bf16_randn(m, k, g), bf16_randn(k, n, g)
        abft.abft_encode(desc, A, B, ws)
        abft.abft_gemm(desc, A, B, C, ws)
        for reread in (0, 1):
            st, rep, nrep = abft.abft_verify_correct(desc, C, ws, reread_C=reread)
            assert st == abft.OK and nrep == 0, (seed, reread, rep)


def test_config5_scaled_fault_free_100_seeds():
    w = wl.GroupWorkload("bf16_grouped_64", 64, note="64 problems of the grouped recipe")
    for seed in range(100):
        shapes = wl.group_shapes(seed, w)
        g = torch.Generator(device="cuda").manual_seed(seed)
        probs = []
        keep = []
        for (m, n, k) in shapes:
            A, B = bf16_randn(m, k, g), bf16_randn(k, n, g)
            C = torch.empty((m, n), dtype=torch.float32, device="cuda")
            keep += [A, B, C]
            probs.append(dict(m=m, n=n, k=k, A=A, B=B, C=C))
        grp = abft.abft_group_create(probs, "bf16")
        try:
            ws = torch.zeros(abft.abft_group_workspace_bytes(grp), dtype=torch.uint8,
                             device="cuda")
            abft.abft_group_bind(grp, ws)
            abft.abft_group_encode(grp)
            abft.abft_group_gemm(grp, True)
            st, rep, nrep = abft.abft_group_verify_correct(grp)
            assert st == abft.OK and nrep == 0, (seed, rep)
        finally:
            abft.abft_group_destroy(grp)


# ------------------------------------------------ rate 1e-9 at full size, 100 seeds
def test_rate_1e9_full_size_100_seeds():
    """bf16 16384^3, verify blocks 256: per seed, Poisson(1e-9 m n) accumulator flips at
    uniform positions (distinct verify blocks) and uniform fp32 bits, armed in the
    epilogue; the fused verify's decisions against the oracle's class of each flip."""
    m = n = k = 16384
    vb = 256
    desc = abft.make_desc(m, n, k, "bf16", vb, vb)
    ws = torch.zeros(abft.abft_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    total = graded = 0
    for seed in range(100):
        g = torch.Generator(device="cuda").manual_seed(seed)
        A, B = bf16_randn(m, k, g), bf16_randn(k, n, g)
        count = int(wl.rng(seed, 11).poisson(1e-9 * m * n))
        abft.abft_encode(desc, A, B, ws)
        flips = wl.bit_flips(seed, m, n, count, bits=32, distinct_blocks=(vb, vb)) if count else []
        clean = []
        if flips:
            abft.abft_gemm(desc, A, B, C, ws)
            torch.cuda.synchronize()
            clean = [C[i, j].item() for i, j, _ in flips]
        abft.abft_set_epilogue_faults(desc, ws, flips)
        abft.abft_gemm(desc, A, B, C, ws)
        abft.abft_set_epilogue_faults(desc, ws, [])
        torch.cuda.synchronize()
        faulty = [C[i, j].item() for i, j, _ in flips]
        st, rep, nrep = abft.abft_verify_correct(desc, C, ws, reread_C=0)
        got = {(e["row"], e["col"]): e["kind"] for e in rep if e["kind"] in (1, 2)}
        allowed = set()
        for (i, j, b), c0, c1 in zip(flips, clean, faulty):
            I, J = i // vb, j // vb
            enc = oracle.Encoded(to_f64(A[I * vb:(I + 1) * vb]), to_f64(B[:, J * vb:(J + 1) * vb]),
                                 vb, vb, dtype="bf16", products=False)
            with np.errstate(invalid="ignore"):
                cls = enc.classify(i - I * vb, j - J * vb, c1 - c0)
            total += 1
            if cls == "graded":
                graded += 1
                kind = abft.KIND_CORRECTED if np.isfinite(c1) else abft.KIND_NONFINITE_CORRECTED
                assert got.get((i, j)) == kind, (seed, i, j, b, rep)
            elif cls == "benign":
                assert (i, j) not in got, (seed, i, j, b)
            allowed.add((i, j))
        assert set(got) <= allowed, (seed, rep)
        assert st == abft.OK or any(e["kind"] == abft.KIND_UNCORRECTABLE for e in rep)
    print(f"rate 1e-9 over 100 seeds: {total} flips, {graded} graded")
    assert total >= 10 and graded >= 1


# ------------------------------------------- the grouped workload at the bench's size
@pytest.mark.parametrize("seed", range(5))
def test_grouped_4096_bench_size_decisions_like_oracle(seed):
    """The 4096-problem bench recipe (seeds 0..4): one graded accumulator flip in each of the
    41 faulty instances, every problem's decisions against the oracle's on its faulty C."""
    w = wl.BF16_GROUPED_4096
    shapes = wl.group_shapes(seed, w)
    g = torch.Generator(device="cuda").manual_seed(seed)
    As, Bs, Cs, probs = [], [], [], []
    for (m, n, k) in shapes:  # the bench's recipe, in its order
        As.append(bf16_randn(m, k, g))
        Bs.append(bf16_randn(k, n, g))
        Cs.append(torch.empty((m, n), dtype=torch.float32, device="cuda"))
        probs.append(dict(m=m, n=n, k=k, A=As[-1], B=Bs[-1], C=Cs[-1]))
    grp = abft.abft_group_create(probs, "bf16")
    try:
        ws = torch.zeros(abft.abft_group_workspace_bytes(grp), dtype=torch.uint8, device="cuda")
        abft.abft_group_bind(grp, ws)
        abft.abft_group_encode(grp)
        abft.abft_group_gemm(grp, True)
        torch.cuda.synchronize()
        faulty = wl.faulty_instances(seed, w.count, w.fault_frac)
        assert len(faulty) == 41
        gr = wl.rng(seed, 22)
        flips = []
        for p in faulty:
            m, n, _ = shapes[p]
            i, j = int(gr.integers(0, m)), int(gr.integers(0, n))
            flips.append((p, i, j, 29 if abs(Cs[p][i, j].item()) >= 2.0 else 30))
        abft.abft_group_set_epilogue_faults(grp, flips)
        abft.abft_group_gemm(grp, True)
        abft.abft_group_set_epilogue_faults(grp, [])
        torch.cuda.synchronize()
        Cf = {p: Cs[p].cpu().numpy().astype(np.float64) for p in faulty}
        st, rep, nrep = abft.abft_group_verify_correct(grp, max_reports=4096)
        assert st == abft.OK, rep
        mine = {}
        for e in rep:
            mine.setdefault(e["problem"], []).append((e["row"], e["col"], e["kind"]))
        assert set(mine) == set(faulty)
        for p, i, j, b in flips:
            m, n, k = shapes[p]
            enc = oracle.Encoded(to_f64(As[p]), to_f64(Bs[p]), 128, 256, dtype="bf16")
            ost, orep, oC, on = enc.verify_correct(Cf[p])
            assert ost == oracle.ST_OK
            theirs = sorted((r["row"], r["col"], r["kind"]) for r in orep)
            # bit 30 of a value in [1, 2) makes it non-finite
            kind = abft.KIND_CORRECTED if np.isfinite(Cf[p][i, j]) else abft.KIND_NONFINITE_CORRECTED
            assert sorted(mine[p]) == theirs == [(i, j, kind)], (p, mine[p], theirs)
    finally:
        abft.abft_group_destroy(grp)
