"""Parity of the grouped bf16 ABFT path (many independent problems per launch: one
persistent tcgen05 product, one encode and one verify pass) with the CPU oracle, through the
C ABI.

Every problem is checked like a single bf16 problem (the bounds of test_gpu_bf16): its
product values against the oracle's binary64 product of the bf16 inputs, its expected
checksums (hi + lo products folded in binary64) and threshold norms against the oracle's
encode with verify blocks of 128 rows x 256 columns, and its decisions (bit-exact fault
positions and kinds) against the oracle run on the GPU's C.  The shapes cover ragged sizes,
problems whose checksum rows / columns share the last data tile and problems that need a
tile of checksums of their own, a 1 x 1 x 1 problem, and both tile widths of the tuner."""
import os

import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
VB_R, VB_C = 128, 256


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


def rel_fro(x, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def check_fp32_product(C, A, B, ref, extra_rel=0.0):
    k = A.shape[1]
    mag = np.abs(A) @ np.abs(B)
    bound = (2 * k * U32 + extra_rel) * mag + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    assert rel_fro(C, ref) <= 4 * np.sqrt(max(k, 1)) * U32 + 4 * extra_rel


def positions(rep):
    return sorted((e["problem"], e["row"], e["col"], e["kind"]) for e in rep if e["kind"] in (1, 2))


class Group:
    """A group of problems with seeded bf16 operands; host copies kept for small ones."""

    def __init__(self, shapes, seed=0, keep_host=True, tuning=None):
        self.shapes = shapes
        self.A, self.B, self.C, self.A64, self.B64, probs = [], [], [], [], [], []
        for p, (m, n, k) in enumerate(shapes):
            a = wl.group_operand_bits(seed, p, 0, m, k)
            b = wl.group_operand_bits(seed, p, 1, k, n)
            self.A.append(torch.from_numpy(a.view(np.int16)).view(torch.bfloat16).cuda())
            self.B.append(torch.from_numpy(b.view(np.int16)).view(torch.bfloat16).cuda())
            self.C.append(torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda"))
            if keep_host:
                self.A64.append(oracle.bf16_to_f64(a[:, :k]))
                self.B64.append(oracle.bf16_to_f64(b[:, :n]))
            probs.append(dict(m=m, n=n, k=k, A=self.A[-1], B=self.B[-1], C=self.C[-1],
                              lda=a.shape[1], ldb=b.shape[1], ldc=n))
        self.g = abft.abft_group_create(probs, "bf16")
        self.ws = torch.zeros(abft.abft_group_workspace_bytes(self.g), dtype=torch.uint8,
                              device="cuda")
        abft.abft_group_bind(self.g, self.ws)
        if tuning:
            abft.abft_group_set_tuning(self.g, *tuning)
        abft.abft_group_encode(self.g)
        abft.abft_group_gemm(self.g, True)
        torch.cuda.synchronize()

    def __del__(self):
        if getattr(self, "g", None):
            abft.abft_group_destroy(self.g)

    def region(self, off, shape, dtype):
        nb = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
        return self.ws[off:off + nb].view(dtype).reshape(shape).cpu().numpy()

    def E(self, p):
        """Expected column checksums (2 nvr x n): hi + lo products folded in binary64."""
        L = abft.abft_group_problem_layout(self.g, p)
        e16 = self.region(L.E16, (L.R16, self.shapes[p][1]), torch.float32).astype(np.float64)
        return e16[0::2] + e16[1::2]

    def F(self, p):
        L = abft.abft_group_problem_layout(self.g, p)
        f16 = self.region(L.F16, (self.shapes[p][0], L.C16), torch.float32).astype(np.float64)
        return f16[:, 0::2] + f16[:, 1::2]

    def norms(self, p):
        L = abft.abft_group_problem_layout(self.g, p)
        m, n, _ = self.shapes[p]
        return [self.region(L.nArow, (m,), torch.float64), self.region(L.nAblk, (4 * L.nvr,),
                torch.float64), self.region(L.nBcol, (n,), torch.float64),
                self.region(L.nBblk, (4 * L.nvc,), torch.float64)]


SMALL = [(64, 64, 64), (128, 256, 64), (192, 320, 136), (1, 1, 1), (100, 37, 9),
         (256, 512, 128), (320, 448, 200), (640, 1000, 64), (129, 257, 65), (384, 768, 512),
         (64, 1536, 96), (1088, 64, 128),
         # tiles of checksum columns only, with an odd number of k-steps (the last stage
         # holds one): data + checksum rows in the tile row (130), whole data tiles (256)
         (130, 256, 136), (256, 768, 320)]


@pytest.mark.parametrize("tuning", [(4, 1), (4, 0), (2, 1), (2, 0)])
def test_group_products_checksums_vs_oracle(tuning):
    G = Group(SMALL, seed=5, tuning=tuning)
    for p, (m, n, k) in enumerate(SMALL):
        A, B = G.A64[p], G.B64[p]
        enc = oracle.Encoded(A, B, VB_R, VB_C, dtype="bf16")
        check_fp32_product(G.C[p].cpu().numpy(), A, B, oracle.gemm(A, B))
        check_fp32_product(G.E(p), np.abs(enc.acs), B, enc.E, extra_rel=2.0 ** -17 + 256 * U32)
        check_fp32_product(G.F(p), A, np.abs(enc.bcs), enc.F, extra_rel=2.0 ** -17 + 256 * U32)
        for got, ref in zip(G.norms(p), (enc.nArow, enc.nAblk, enc.nBcol, enc.nBblk)):
            assert np.allclose(got, ref, rtol=1e-5), p
    st, rep, nrep = abft.abft_group_verify_correct(G.g)
    assert st == abft.OK and nrep == 0


def test_group_plain_product_matches_abft_data():
    G = Group(SMALL, seed=6)
    ref = [c.clone() for c in G.C]
    for c in G.C:
        c.fill_(float("nan"))
    abft.abft_group_gemm(G.g, False)
    torch.cuda.synchronize()
    for p, (m, n, k) in enumerate(SMALL):
        got = G.C[p].cpu().numpy()
        assert np.all(np.isfinite(got))
        check_fp32_product(got, G.A64[p], G.B64[p], oracle.gemm(G.A64[p], G.B64[p]))
        assert np.allclose(got, ref[p].cpu().numpy(), rtol=1e-6, atol=1e-6)


def graded_bits(C, i, j):
    """An exponent bit that moves the fp32 value by >= 2^64 (always graded)."""
    return 29 if abs(float(C[i, j])) >= 2.0 else 30


def inject_and_verify(G, flips_by_problem, capture=False):
    """Arms one flip per listed problem, multiplies, verifies; returns (status, report)."""
    flips = [(p, i, j, b) for p, (i, j, b) in flips_by_problem.items()]
    abft.abft_group_set_epilogue_faults(G.g, flips)
    torch.cuda.synchronize()
    if capture:
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            abft.abft_group_capture(G.g, True, stream=s)
            abft.abft_group_launch(G.g, stream=s)
            st, rep, nrep = abft.abft_group_report(G.g, stream=s)
    else:
        abft.abft_group_gemm(G.g, True)
        st, rep, nrep = abft.abft_group_verify_correct(G.g)
    abft.abft_group_set_epilogue_faults(G.g, [])
    return st, rep


@pytest.mark.parametrize("capture", [False, True])
def test_group_epilogue_faults_located_like_oracle(capture):
    """Accumulator flips armed in several problems are located from the fused sums at the
    same positions the oracle finds on the GPU's faulty C of each problem, and corrected."""
    G = Group(SMALL, seed=7)
    clean = [c.cpu().numpy().astype(np.float64) for c in G.C]
    g = wl.rng(7, 30)
    flips = {}
    for p, (m, n, k) in enumerate(SMALL):
        if p % 2 == 0:
            i, j = int(g.integers(0, m)), int(g.integers(0, n))
            flips[p] = (i, j, graded_bits(clean[p], i, j))
    # the faulty C of each problem, as the oracle sees it
    for p, (i, j, b) in flips.items():
        assert i < SMALL[p][0] and j < SMALL[p][1]
    faulty = {}
    abft.abft_group_set_epilogue_faults(G.g, [(p, i, j, b) for p, (i, j, b) in flips.items()])
    abft.abft_group_gemm(G.g, True)
    abft.abft_group_set_epilogue_faults(G.g, [])
    torch.cuda.synchronize()
    for p in flips:
        faulty[p] = G.C[p].cpu().numpy().astype(np.float64)
    st, rep = inject_and_verify(G, flips, capture=capture)
    assert st == abft.OK
    got = positions(rep)
    want = []
    for p, Cf in faulty.items():
        enc = oracle.Encoded(G.A64[p], G.B64[p], VB_R, VB_C, dtype="bf16")
        ost, orep, oC, on = enc.verify_correct(Cf)
        assert ost == oracle.ST_OK
        want += [(p, e["row"], e["col"], e["kind"]) for e in orep if e["kind"] in (1, 2)]
        i, j, _ = flips[p]
        assert [(e["row"], e["col"]) for e in orep if e["kind"] in (1, 2)] == [(i, j)]
    assert got == sorted(want)
    for p, (m, n, k) in enumerate(SMALL):
        check_corrected(G.C[p].cpu().numpy().astype(np.float64), G.A64[p], G.B64[p],
                        [(i, j) for q, i, j, _ in got if q == p])


def check_corrected(C, A, B, fixed):
    """Values after correction: untouched elements within the product bound; a recomputed
    element carries the error of its line's expected checksum (bf16 hi + lo pieces, 2^-17
    relative, plus the fp32 accumulation of the checksum product and of the other elements
    of the line), bounded by (2^-16 + 4 k u32 + 256 u32) (e^T |A_I|) |B_j|."""
    ref = oracle.gemm(A, B)
    k = A.shape[1]
    mag = np.abs(A) @ np.abs(B)
    ok = np.abs(C - ref) <= 2 * k * U32 * mag + 1e-30
    for i, j in fixed:
        i0 = (i // VB_R) * VB_R
        colmag = float(np.abs(A[i0:i0 + VB_R]).sum(axis=0) @ np.abs(B[:, j]))
        assert abs(C[i, j] - ref[i, j]) <= (2.0 ** -16 + (4 * k + 256) * U32) * colmag
        ok[i, j] = True
    assert ok.all()
    assert rel_fro(C, ref) <= 4 * np.sqrt(k) * U32 + 1e-7


def test_group_graph_replays():
    """The captured step (product + verify) replays with the same results as direct calls,
    and each replay counts its kernels."""
    G = Group(SMALL[:6], seed=8)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        abft.abft_group_capture(G.g, True, stream=s)
        n0 = abft.abft_kernel_launches()
        for _ in range(3):
            abft.abft_group_launch(G.g, stream=s)
        st, rep, nrep = abft.abft_group_report(G.g, stream=s)
    assert st == abft.OK and nrep == 0
    assert abft.abft_kernel_launches() - n0 == 3 * 4  # product, column, row, locate
    for p, (m, n, k) in enumerate(SMALL[:6]):
        check_fp32_product(G.C[p].cpu().numpy(), G.A64[p], G.B64[p],
                           oracle.gemm(G.A64[p], G.B64[p]))


def test_group_autotune_and_cache(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("ABFT_TUNE_CACHE", str(cache))
    G = Group(SMALL, seed=9)
    t, ms = abft.abft_group_autotune(G.g, reps=2)
    assert t["boxes_per_tile"] in (2, 4) and t["order"] in (0, 1) and ms > 0
    assert cache.exists() and len(cache.read_text().splitlines()) == 1
    # a second group of the same shapes takes the recorded choice without measuring
    G2 = Group(SMALL, seed=10)
    t2, ms2 = abft.abft_group_autotune(G2.g, reps=2)
    assert t2 == t and ms2 == -1.0 and abft.abft_group_get_tuning(G2.g) == t
    # after tuning the group still computes and verifies correctly
    abft.abft_group_encode(G.g)
    abft.abft_group_gemm(G.g, True)
    st, rep, nrep = abft.abft_group_verify_correct(G.g)
    assert st == abft.OK and nrep == 0
    for p in (0, 7, 9):
        check_fp32_product(G.C[p].cpu().numpy(), G.A64[p], G.B64[p],
                           oracle.gemm(G.A64[p], G.B64[p]))


def test_group_invalid_problems_rejected():
    a = torch.zeros((8, 8), dtype=torch.bfloat16, device="cuda")
    c = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    bad = [dict(m=8, n=8, k=8, A=a, B=a, C=c, lda=4),           # lda < k
           dict(m=0, n=8, k=8, A=a, B=a, C=c),                  # empty
           dict(m=8, n=8, k=8, A=a.data_ptr() + 2, B=a, C=c)]   # misaligned A
    for q in bad:
        with pytest.raises(abft.AbftError) as e:
            abft.abft_group_create([q], "bf16")
        assert e.value.status == abft.ERR_INVALID
    with pytest.raises(abft.AbftError) as e:
        abft.abft_group_create([dict(m=8, n=8, k=8, A=a, B=a, C=c)], "f64")
    assert e.value.status == abft.ERR_UNSUPPORTED


def test_grouped_workload_sampled():
    """The grouped workload recipe at 512 problems (m, n, k uniform over multiples of 64 in
    [64, 2048]): one flip in 1% of the instances at a uniform position and a uniform fp32
    bit, classified by the oracle.  Graded flips are located exactly, benign ones stay
    silent, fault-free problems report nothing; sampled problems' values match the oracle."""
    w = wl.BF16_GROUPED_512
    seed = 3
    shapes = wl.group_shapes(seed, w)
    G = Group(shapes, seed=seed, keep_host=False)
    st, rep, nrep = abft.abft_group_verify_correct(G.g)
    assert st == abft.OK and nrep == 0
    faulty = wl.faulty_instances(seed, w.count, w.fault_frac)
    g = wl.rng(seed, 22)
    flips = {}
    for p in faulty:
        m, n, _ = shapes[p]
        flips[p] = (int(g.integers(0, m)), int(g.integers(0, n)), int(g.integers(0, 32)))
    clean = {p: G.C[p].cpu().numpy().astype(np.float64) for p in faulty}
    abft.abft_group_set_epilogue_faults(G.g, [(p, i, j, b) for p, (i, j, b) in flips.items()])
    abft.abft_group_gemm(G.g, True)
    abft.abft_group_set_epilogue_faults(G.g, [])
    torch.cuda.synchronize()
    classes = {}
    for p, (i, j, b) in flips.items():
        m, n, k = shapes[p]
        a = wl.group_operand_bits(seed, p, 0, m, k)
        bb = wl.group_operand_bits(seed, p, 1, k, n)
        enc = oracle.Encoded(oracle.bf16_to_f64(a[:, :k]), oracle.bf16_to_f64(bb[:, :n]), VB_R,
                             VB_C, dtype="bf16")
        Cf = G.C[p].cpu().numpy().astype(np.float64)
        with np.errstate(invalid="ignore"):
            classes[p] = enc.classify(i, j, Cf[i, j] - clean[p][i, j])
    st, rep, nrep = abft.abft_group_verify_correct(G.g)
    guard = {p for p, c in classes.items() if c == "guard"}
    # a guard-band flip may be flagged without a located position (uncorrectable line)
    assert st == abft.OK or (st == abft.ERR_UNCORRECTABLE and guard)
    assert all(e["problem"] in guard for e in rep if e["kind"] == abft.KIND_UNCORRECTABLE)
    got = {(e["problem"], e["row"], e["col"]) for e in rep if e["kind"] in (1, 2)}
    for p, (i, j, b) in flips.items():
        if classes[p] == "graded":
            assert (p, i, j) in got
        elif classes[p] == "benign":
            assert all(q != p for q, _, _ in got)
    assert all(q in flips for q, _, _ in got)
    assert sum(c == "graded" for c in classes.values()) >= 1
    # sampled values of three problems against the oracle's dot products
    for p in (0, int(np.argmax([m * n * k for m, n, k in shapes])), faulty[0]):
        m, n, k = shapes[p]
        a = oracle.bf16_to_f64(wl.group_operand_bits(seed, p, 0, m, k)[:, :k])
        bb = oracle.bf16_to_f64(wl.group_operand_bits(seed, p, 1, k, n)[:, :n])
        gs = wl.rng(seed, 40 + p)
        rows, cols = gs.integers(0, m, 64), gs.integers(0, n, 64)
        Cg = G.C[p].cpu().numpy().astype(np.float64)
        for i, j in zip(rows, cols):
            ref = float(oracle.gemm(a[i:i + 1], bb[:, j:j + 1])[0, 0])
            mag = float(np.abs(a[i]) @ np.abs(bb[:, j]))
            assert abs(Cg[i, j] - ref) <= 2 * k * U32 * mag + 1e-30
