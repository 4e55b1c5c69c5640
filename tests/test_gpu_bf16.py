"""Parity of the bf16 tensor-core path (tcgen05 / TMEM / TMA, fp32 accumulation and fp32 C)
with the CPU oracle, through the C ABI.

The oracle works in binary64 on the exact values of the bf16 inputs.  Values: elementwise
|C - C*| <= 2 k u32 (|A||B|) (u32 = 2^-24; the products of bf16 values are exact in fp32 and
each of at most k additions errs by at most 2 u32 of the partial sum's magnitude, which holds
for round-to-nearest and for truncation alike), and relative Frobenius <= 4 sqrt(k) u32 as a
check of the observed scale (about 2.4 sqrt(k) u32 at k = 16384).  The checksum products also
carry the bf16 hi+lo representation error (2^-17 relative) of the checksum operand.
Decisions: bit-exact fault positions and kinds for graded and benign flips (bits of the fp32
elements of C)."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


def bf16_matrix(rows, cols, dist, seed, stream, ld=None):
    """(device tensor rows x ld of bf16, exact float64 values rows x cols)."""
    ld = ld or (cols + 7) // 8 * 8
    bits = np.zeros((rows, ld), np.uint16)
    bits[:, :cols] = wl.bf16_bits(wl.operand((rows, cols), dist, seed, stream))
    dev = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()
    return dev, oracle.bf16_to_f64(bits[:, :cols]), ld


class Run:
    def __init__(self, m, n, k, vb_r, vb_c, p=0, q=0, seed=0, dist="normal", plain=False):
        self.m, self.n, self.k = m, n, k
        self.A, self.A64, lda = bf16_matrix(m, k, dist, seed, 1)
        self.B, self.B64, ldb = bf16_matrix(k, n, dist, seed, 2)
        self.desc = abft.make_desc(m, n, k, "bf16", vb_r, vb_c, p, q, lda=lda, ldb=ldb)
        self.L = abft.abft_workspace_layout(self.desc)
        self.C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        if plain:
            abft.abft_gemm_plain(self.desc, self.A, self.B, self.C)
        else:
            self.ws = torch.zeros(self.L.total, dtype=torch.uint8, device="cuda")
            abft.abft_encode(self.desc, self.A, self.B, self.ws)
            abft.abft_gemm(self.desc, self.A, self.B, self.C, self.ws)
        torch.cuda.synchronize()

    def region(self, off, shape, dtype=torch.float64):
        nb = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
        return self.ws[off:off + nb].view(dtype).reshape(shape).cpu().numpy()

    def E(self):
        return self.region(self.L.E, (self.L.R, self.n))

    def F(self):
        return self.region(self.L.F, (self.m, self.L.Cc))


def rel_fro(x, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def check_fp32_product(C, A, B, ref, extra_rel=0.0):
    k = A.shape[1]
    mag = np.abs(A) @ np.abs(B)
    bound = (2 * k * U32 + extra_rel) * mag + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    assert rel_fro(C, ref) <= 4 * np.sqrt(max(k, 1)) * U32 + 4 * extra_rel


def test_plain_product_one_tile_column():
    r = Run(256, 256, 128, 128, 128, plain=True)
    check_fp32_product(r.C.cpu().numpy(), r.A64, r.B64, oracle.gemm(r.A64, r.B64))


@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (200, 300, 100), (384, 512, 1000),
                                   (1, 8, 8), (130, 700, 520)])
def test_plain_product_shapes(m, n, k):
    r = Run(m, n, k, min(128, m), min(128, n), seed=m + n + k, plain=True)
    check_fp32_product(r.C.cpu().numpy(), r.A64, r.B64, oracle.gemm(r.A64, r.B64))


SHAPES = [  # (m, n, k, vb_r, vb_c, p, q)
    (256, 512, 256, 128, 128, 0, 0),
    (384, 256, 200, 128, 64, 3, 2),
    (200, 300, 136, 40, 30, 0, 0),
    (512, 512, 128, 64, 128, 4, 4),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_abft_product_and_checksums_vs_oracle(shape):
    m, n, k, vbr, vbc, p, q = shape
    r = Run(m, n, k, vbr, vbc, p, q, seed=7)
    enc = oracle.Encoded(r.A64, r.B64, vbr, vbc, p, q, dtype="bf16")
    check_fp32_product(r.C.cpu().numpy(), r.A64, r.B64, oracle.gemm(r.A64, r.B64))
    # E / F: fp32 sums of bf16 data fed as bf16 hi+lo pieces, products summed in binary64
    check_fp32_product(r.E(), np.abs(enc.acs), r.B64, enc.E, extra_rel=2.0 ** -17 + 256 * U32)
    check_fp32_product(r.F(), r.A64, np.abs(enc.bcs), enc.F, extra_rel=2.0 ** -17 + 256 * U32)
    for off, ref in ((r.L.nArow, enc.nArow), (r.L.nAblk, enc.nAblk), (r.L.nBcol, enc.nBcol),
                     (r.L.nBblk, enc.nBblk)):
        assert np.allclose(r.region(off, ref.shape), ref, rtol=1e-5)


def test_plain_equals_abft_data_block():
    r = Run(256, 512, 192, 128, 128, seed=3)
    C2 = torch.empty_like(r.C)
    abft.abft_gemm_plain(r.desc, r.A, r.B, C2)
    torch.cuda.synchronize()
    assert torch.equal(C2, r.C)


@pytest.mark.parametrize("seed", range(4))
def test_fault_free_no_false_positives(seed):
    r = Run(512, 768, 1024, 128, 128, 4, 3, seed=seed)
    C0 = r.C.clone()
    st, rep, n = abft.abft_verify_correct(r.desc, r.C, r.ws)
    assert st == abft.OK and n == 0 and torch.equal(C0, r.C)


@pytest.mark.parametrize("shape", [(1024, 1024, 2048, 128, 128), (512, 640, 4096, 128, 64)])
def test_residual_margin_below_thresholds(shape):
    """Fault-free residuals of the GPU product, computed by the oracle on the GPU's C, stay
    far below the thresholds (the margin the detection rests on)."""
    m, n, k, vbr, vbc = shape
    r = Run(m, n, k, vbr, vbc, seed=5)
    enc = oracle.Encoded(r.A64, r.B64, vbr, vbc, dtype="bf16")
    C = r.C.cpu().numpy().astype(np.float64)
    re, rw, te, tw, _ = enc.col_residuals(C)
    ratio_c = max(np.max(np.abs(re) / te), np.max(np.abs(rw) / tw))
    re, rw, te, tw, _ = enc.row_residuals(C)
    ratio_r = max(np.max(np.abs(re) / te), np.max(np.abs(rw) / tw))
    print(f"max |r|/tau: column checks {ratio_c:.3e}, row checks {ratio_r:.3e}")
    assert ratio_c < 0.25 and ratio_r < 0.25


def positions(rep):
    return sorted((e["row"], e["col"], e["kind"]) for e in rep if e["kind"] in (1, 2))


@pytest.mark.parametrize("seed", range(16))
def test_single_fp32_flip_parity(seed):
    """Scaled-down bf16 workload (1024 x 1024 x 2048, verify blocks 128): one flip of a
    uniform bit of an fp32 element of C."""
    m = n = 1024
    k = 2048
    r = Run(m, n, k, 128, 128, seed=seed)
    enc = oracle.Encoded(r.A64, r.B64, 128, 128, dtype="bf16")
    C_clean = r.C.cpu().numpy().astype(np.float64)
    (i, j, b), = wl.bit_flips(seed, m, n, 1, bits=32)
    abft.abft_inject_bitflips(r.desc, r.C, [(i, j, b)])
    Cf = r.C.cpu().numpy().astype(np.float64)
    with np.errstate(invalid="ignore"):
        cls = enc.classify(i, j, Cf[i, j] - C_clean[i, j])
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws)
    ost, orep, oC, on = enc.verify_correct(Cf)
    if cls == "graded":
        kind = abft.KIND_CORRECTED if np.isfinite(Cf[i, j]) else abft.KIND_NONFINITE_CORRECTED
        assert st == abft.OK and positions(rep) == [(i, j, kind)] == positions(orep)
    elif cls == "benign":
        assert st == abft.OK and nrep == 0 and on == 0
    else:
        assert all((e["row"], e["col"]) == (i, j) for e in rep if e["kind"] in (1, 2))
    if cls != "guard":
        Cg = r.C.cpu().numpy().astype(np.float64)
        assert rel_fro(Cg, oracle.gemm(r.A64, r.B64)) <= 4 * np.sqrt(k) * U32 + 1e-7


def test_forced_exponent_flips_and_erasure():
    m = n = 512
    k = 384
    r = Run(m, n, k, 128, 128, 4, 4, seed=21)
    enc = oracle.Encoded(r.A64, r.B64, 128, 128, 4, 4, dtype="bf16")
    C_clean = r.C.cpu().numpy().astype(np.float64)
    flips = [(5, 300, 30), (200, 17, 29), (450, 450, 31)]  # blocks (0,2), (1,0), (3,3)
    abft.abft_inject_bitflips(r.desc, r.C, flips)
    abft.abft_erase_block(r.desc, r.C, 2, 1)
    Cf = r.C.cpu().numpy().astype(np.float64)
    for i, j, _ in flips:
        with np.errstate(invalid="ignore"):
            assert enc.classify(i, j, Cf[i, j] - C_clean[i, j]) == "graded"
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, erased=[(2, 1)])
    ost, orep, oC, on = enc.verify_correct(Cf, erased=[(2, 1)])
    assert st == abft.OK and ost == oracle.ST_OK
    assert [(a, b) for a, b, _ in positions(rep)] == sorted((i, j) for i, j, _ in flips)
    assert positions(rep) == positions(orep)
    st, ent = abft.abft_recover_block(r.desc, r.C, r.ws, 2, 1)
    assert st == abft.OK
    Cg = r.C.cpu().numpy().astype(np.float64)
    Cstar = oracle.gemm(r.A64, r.B64)
    blk = np.s_[256:384, 128:256]
    assert rel_fro(Cg[blk], Cstar[blk]) <= 8 * np.sqrt(k) * U32
    assert rel_fro(Cg, Cstar) <= 4 * np.sqrt(k) * U32


def test_bf16_16384_full_size_sampled():
    """The 16384^3 bf16 workload in the benchmark's launch configuration: sampled outputs
    against the oracle, the section 4.3 residual check on all of C, and located flips."""
    w = wl.BF16_16384
    m, n, k = w.m, w.n, w.k
    r = Run(m, n, k, w.vb_r, w.vb_c, seed=0)
    g = wl.rng(0, 99)
    rows = np.sort(g.choice(m, 32, replace=False))
    cols = np.sort(g.choice(n, 32, replace=False))
    Cs = r.C[rows][:, cols].cpu().numpy().astype(np.float64)
    check_fp32_product(Cs, r.A64[rows], r.B64[:, cols], oracle.gemm(r.A64[rows], r.B64[:, cols]))
    C = r.C.cpu().numpy().astype(np.float64)
    x = wl.operand((n,), "uniform", 0, 5)
    # binary32 accumulation: the ratio is scaled by eps32 / eps64
    assert oracle.residual_check(r.A64, r.B64, C, x) * 2.0 ** -29 < 1.0
    flips = [(100, 200, 30), (9000, 16000, 29), (16383, 5, 28), (4242, 777, 26)]
    abft.abft_inject_bitflips(r.desc, r.C, flips)
    Cf = r.C.cpu().numpy().astype(np.float64)
    enc = oracle.Encoded(r.A64, r.B64, w.vb_r, w.vb_c, dtype="bf16", products=False)
    with np.errstate(invalid="ignore"):
        cls = {(i, j): enc.classify(i, j, Cf[i, j] - C[i, j]) for i, j, _ in flips}
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws)
    assert st == abft.OK
    found = [(a, b) for a, b, _ in positions(rep)]
    graded = sorted(p for p, c in cls.items() if c == "graded")
    assert len(graded) >= 3, cls
    assert all(p in found for p in graded)
    assert all(cls[p] != "benign" for p in found) and all(p in cls for p in found)
    for i, j in found:
        assert abs(r.C[i, j].item() - C[i, j]) <= 1e-3 * max(1.0, abs(C[i, j]))


# --------------------------------------------------------------------------- fused checksums
def graded_bits(C, positions):
    """An exponent bit per position that moves the fp32 value by >= 2^64 (always graded)."""
    return [(i, j, 29 if abs(float(C[i, j])) >= 2.0 else 30) for i, j in positions]


@pytest.mark.parametrize("shape", [(1024, 1024, 2048, 128, 128), (640, 700, 520, 128, 64),
                                   (512, 1024, 256, 256, 512), (384, 300, 128, 128, 32)])
def test_fused_verify_epilogue_faults(shape):
    """Accumulator-output flips armed in the epilogue (compute faults) are located from the
    epilogue's observed sums (no re-read of C) at the same positions as the oracle finds on
    the GPU's C; fault-free runs give no flags in either mode."""
    m, n, k, vbr, vbc = shape
    r = Run(m, n, k, vbr, vbc, seed=31)
    assert r.L.fused == 1
    enc = oracle.Encoded(r.A64, r.B64, vbr, vbc, dtype="bf16")
    for reread in (0, 1):
        st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=reread)
        assert st == abft.OK and nrep == 0
    C_clean = r.C.cpu().numpy().astype(np.float64)
    pos = [(p[0], p[1]) for p in wl.bit_flips(9, m, n, 3, bits=32,
                                              distinct_blocks=(vbr, max(vbc, 64)))]
    flips = graded_bits(C_clean, pos)
    abft.abft_set_epilogue_faults(r.desc, r.ws, flips)
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    abft.abft_set_epilogue_faults(r.desc, r.ws, [])
    Cf = r.C.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isnan(Cf), np.isnan(wl.flip_f32(C_clean.astype(np.float32), flips)))
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    ost, orep, oC, on = enc.verify_correct(Cf)
    assert st == abft.OK and ost == oracle.ST_OK
    assert [(a, b) for a, b, _ in positions(rep)] == sorted(pos)
    assert positions(rep) == positions(orep)
    Cg = r.C.cpu().numpy().astype(np.float64)
    assert rel_fro(Cg, oracle.gemm(r.A64, r.B64)) <= 4 * np.sqrt(k) * U32 + 1e-7


def test_fused_sums_do_not_see_faults_after_the_product():
    """The fused observed sums describe C as the product wrote it: a memory fault in C
    after the product is found by the re-reading verify, not by the fused one."""
    r = Run(512, 512, 256, 128, 128, seed=41)
    abft.abft_inject_bitflips(r.desc, r.C, [(10, 20, 29)])
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    assert st == abft.OK and nrep == 0
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=1)
    assert st == abft.OK and [(e["row"], e["col"]) for e in rep] == [(10, 20)]


def test_rate_1e9_epilogue_injection_seeded():
    """The accumulator-flip workload: flips at rate 1e-9 per element of a seeded draw
    (at least one guaranteed), located from the fused sums."""
    m, n, k = 2048, 2048, 1024
    r = Run(m, n, k, 128, 128, seed=51)
    C_clean = r.C.cpu().numpy().astype(np.float64)
    g = wl.rng(51, 11)
    count = max(1, int(g.poisson(1e-9 * m * n)))
    pos = [(p[0], p[1]) for p in wl.bit_flips(51, m, n, count, bits=32,
                                              distinct_blocks=(128, 128))]
    flips = graded_bits(C_clean, pos)
    abft.abft_set_epilogue_faults(r.desc, r.ws, flips)
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    abft.abft_set_epilogue_faults(r.desc, r.ws, [])
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    assert st == abft.OK and [(a, b) for a, b, _ in positions(rep)] == sorted(pos)


def test_bounded_wait_timeout_is_reported(monkeypatch):
    """Failure detection without a GPU fault: with the test hook set, the producer of the
    single data tile never fills its stages, the MMA warp's bounded wait runs out (0.2 s),
    the kernel drains and frees TMEM, and the verify on that workspace reports
    ABFT_ERR_TIMEOUT (writing nothing into C) until the next product; a problem on
    another workspace is not affected.  The context stays usable: the same problem then
    runs normally."""
    r = Run(128, 256, 64, 128, 256, seed=61)  # 1 data tile + 1 checksum-row + 1 checksum-col tile
    other = Run(256, 256, 128, 128, 256, seed=62)  # a problem on another workspace
    monkeypatch.setenv("ABFT_TEST_STALL_PRODUCER", "1")
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    monkeypatch.delenv("ABFT_TEST_STALL_PRODUCER")
    # the status belongs to r's workspace: the other problem verifies clean
    abft.abft_gemm(other.desc, other.A, other.B, other.C, other.ws)
    st, rep, nrep = abft.abft_verify_correct(other.desc, other.C, other.ws)
    assert st == abft.OK and nrep == 0
    torch.cuda.synchronize()
    before = r.C.clone()
    for _ in range(2):  # reported on every verify until the next product; C untouched
        with pytest.raises(abft.AbftError) as e:
            abft.abft_verify_correct(r.desc, r.C, r.ws)
        assert e.value.status == abft.ERR_TIMEOUT
        assert torch.equal(r.C.view(torch.int32), before.view(torch.int32))
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws)
    assert st == abft.OK and nrep == 0
    check_fp32_product(r.C.cpu().numpy(), r.A64, r.B64, oracle.gemm(r.A64, r.B64))


def test_two_erasures_in_a_block_column_bf16():
    """bf16 product with 2 block checksums: two erased blocks of one block column rebuilt
    from the first two checksums (binary64 solve), against the oracle's rebuild."""
    m = n = 512
    k = 256
    desc_kw = dict(p=4, q=4)
    A, A64, lda = bf16_matrix(m, k, "normal", 23, 1)
    B, B64, ldb = bf16_matrix(k, n, "normal", 23, 2)
    desc = abft.make_desc(m, n, k, "bf16", 128, 128, 4, 4, lda=lda, ldb=ldb, grid_f=2)
    L = abft.abft_workspace_layout(desc)
    assert L.acs_rows == 4 * 4 + 2 * 2 * 128
    ws = torch.zeros(L.total, dtype=torch.uint8, device="cuda")
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    abft.abft_encode(desc, A, B, ws)
    abft.abft_gemm(desc, A, B, C, ws)
    enc = oracle.Encoded(A64, B64, 128, 128, 4, 4, dtype="bf16", f=2)
    ref = oracle.gemm(A64, B64)
    blocks = [(1, 3), (2, 3)]
    for bi, bj in blocks:
        abft.abft_erase_block(desc, C, bi, bj)
    st, rep, nrep = abft.abft_verify_correct(desc, C, ws, erased=blocks)
    assert st == abft.OK and nrep == 0
    st, ents = abft.abft_recover_blocks(desc, C, ws, blocks)
    assert st == abft.OK
    Cg = C.cpu().numpy().astype(np.float64)
    blk = np.s_[128:384, 384:512]
    # the rebuilt blocks carry the errors of the checksums and of the survivors,
    # amplified by the 2 x 2 solve (nodes 2/8 and 3/8)
    assert rel_fro(Cg[blk], ref[blk]) <= 8 * (4 * np.sqrt(k) * U32 + 2.0 ** -17)


@pytest.mark.parametrize("m,n,k,vbr,vbc,ldc", [
    (256, 301, 192, 128, 32, 301),   # C and E16 rows not 16-byte multiples: plain stores
    (256, 320, 192, 128, 64, 323),   # C plain stores, E16 / F16 by TMA
    (384, 300, 136, 128, 64, 304),   # TMA stores clipped at n inside a wider C
])
def test_outputs_with_any_row_pitch(m, n, k, vbr, vbc, ldc):
    """C with a leading dimension beyond n: the product writes exactly the m x n data block
    (the padding keeps its NaNs), by TMA stores when the row pitch allows and plain stores
    otherwise; fused checksums and located epilogue faults are the oracle's either way."""
    A, A64, lda = bf16_matrix(m, k, "normal", 61, 1)
    B, B64, ldb = bf16_matrix(k, n, "normal", 61, 2)
    desc = abft.make_desc(m, n, k, "bf16", vbr, vbc, lda=lda, ldb=ldb, ldc=ldc)
    L = abft.abft_workspace_layout(desc)
    assert L.fused == 1
    ws = torch.zeros(L.total, dtype=torch.uint8, device="cuda")
    Cbuf = torch.full((m, ldc), float("nan"), dtype=torch.float32, device="cuda")
    abft.abft_encode(desc, A, B, ws)
    abft.abft_gemm(desc, A, B, Cbuf, ws)
    torch.cuda.synchronize()
    full = Cbuf.cpu().numpy().astype(np.float64)
    assert np.isnan(full[:, n:]).all()
    ref = oracle.gemm(A64, B64)
    check_fp32_product(full[:, :n], A64, B64, ref)
    st, rep, nrep = abft.abft_verify_correct(desc, Cbuf, ws, reread_C=0)
    assert st == abft.OK and nrep == 0
    enc = oracle.Encoded(A64, B64, vbr, vbc, dtype="bf16")
    pos = [(p[0], p[1]) for p in wl.bit_flips(13, m, n, 2, bits=32, distinct_blocks=(vbr, 64))]
    flips = graded_bits(full[:, :n], pos)
    abft.abft_set_epilogue_faults(desc, ws, flips)
    abft.abft_gemm(desc, A, B, Cbuf, ws)
    abft.abft_set_epilogue_faults(desc, ws, [])
    Cf = Cbuf.cpu().numpy().astype(np.float64)
    assert np.isnan(Cf[:, n:]).all()
    st, rep, nrep = abft.abft_verify_correct(desc, Cbuf, ws, reread_C=0)
    ost, orep, oC, on = enc.verify_correct(Cf[:, :n])
    assert st == abft.OK and ost == oracle.ST_OK
    assert [(a, b) for a, b, _ in positions(rep)] == sorted(pos)
    assert positions(rep) == positions(orep)
    assert rel_fro(Cbuf.cpu().numpy().astype(np.float64)[:, :n], ref) <= 4 * np.sqrt(k) * U32


# --------------------------------------------------------------------------- tile heights
@pytest.mark.parametrize("tall", ["0", "1"])
@pytest.mark.parametrize("shape", [(200, 300, 136, 128, 64), (640, 700, 520, 128, 256),
                                   (320, 256, 2048, 256, 256), (1000, 264, 72, 128, 32),
                                   (400, 320, 200, 128, 64)])  # last tall tile: 3 halves
def test_tile_heights_agree(shape, tall, monkeypatch):
    """128-row and 256-row tiles (ABFT_TALL_TILES forces the choice): ragged rows, tiles
    holding one, two or three 64-row halves, checksum-row tiles of 256 rows; products,
    expected checksums and fused-verify decisions against the oracle, and the plain
    product equal to the ABFT product's data bit for bit."""
    monkeypatch.setenv("ABFT_TALL_TILES", tall)
    m, n, k, vbr, vbc = shape
    r = Run(m, n, k, vbr, vbc, seed=61)
    enc = oracle.Encoded(r.A64, r.B64, vbr, vbc, dtype="bf16")
    C = r.C.cpu().numpy().astype(np.float64)
    check_fp32_product(C, r.A64, r.B64, oracle.gemm(r.A64, r.B64))
    check_fp32_product(r.E(), np.abs(enc.acs), r.B64, enc.E, extra_rel=2.0 ** -17 + 256 * U32)
    check_fp32_product(r.F(), r.A64, np.abs(enc.bcs), enc.F, extra_rel=2.0 ** -17 + 256 * U32)
    for reread in (0, 1):
        st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=reread)
        assert st == abft.OK and nrep == 0
    plain = Run(m, n, k, vbr, vbc, seed=61, plain=True)
    assert torch.equal(plain.C, r.C)
    blocks = (vbr, max(vbc, 64))
    nflip = min(3, -(-m // blocks[0]) * -(-n // blocks[1]))
    pos = [(p[0], p[1]) for p in wl.bit_flips(62, m, n, nflip, bits=32, distinct_blocks=blocks)]
    flips = graded_bits(C, pos)
    abft.abft_set_epilogue_faults(r.desc, r.ws, flips)
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    abft.abft_set_epilogue_faults(r.desc, r.ws, [])
    Cf = r.C.cpu().numpy().astype(np.float64)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    ost, orep, oC, on = enc.verify_correct(Cf)
    assert st == abft.OK and ost == oracle.ST_OK
    assert [(a, b) for a, b, _ in positions(rep)] == sorted(pos)
    assert positions(rep) == positions(orep)


@pytest.mark.parametrize("reread", [0, 1])
def test_non_finite_operand_decided_like_oracle(reread):
    """A NaN in a bf16 operand: the non-finite row of C is located element by element,
    recomputed to non-finite values and its lines reported uncorrectable, as the oracle
    decides on the GPU's C, from the fused sums or from a re-read of C."""
    m, n, k = 256, 384, 192
    bits_a = wl.bf16_bits(wl.operand((m, k), "normal", 7, 1))
    bits_a[37, 11] = 0x7FC0  # bf16 quiet NaN
    bits_b = wl.bf16_bits(wl.operand((k, n), "normal", 7, 2))
    A = torch.from_numpy(bits_a.view(np.int16)).view(torch.bfloat16).cuda()
    B = torch.from_numpy(bits_b.view(np.int16)).view(torch.bfloat16).cuda()
    A64, B64 = oracle.bf16_to_f64(bits_a), oracle.bf16_to_f64(bits_b)
    desc = abft.make_desc(m, n, k, "bf16", 128, 128)
    ws = torch.zeros(abft.abft_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    abft.abft_encode(desc, A, B, ws)
    abft.abft_gemm(desc, A, B, C, ws)
    torch.cuda.synchronize()
    Cg = C.cpu().numpy().astype(np.float64)
    assert np.isnan(Cg[37]).all() and np.isfinite(np.delete(Cg, 37, axis=0)).all()
    enc = oracle.Encoded(A64, B64, 128, 128, dtype="bf16")
    st, rep, nrep = abft.abft_verify_correct(desc, C, ws, reread_C=reread, max_reports=4096)
    ost, orep, oC, on = enc.verify_correct(Cg, max_reports=4096)
    assert st == abft.ERR_UNCORRECTABLE and ost == oracle.ST_UNCORRECTABLE
    key = lambda e: (e["row"], e["col"], e["kind"])
    assert nrep == on and sorted(map(key, rep)) == sorted(map(key, orep))
    assert np.array_equal(np.delete(C.cpu().numpy(), 37, axis=0), np.delete(Cg, 37, axis=0))


@pytest.mark.parametrize("tall", ["0", "1"])
def test_flip_near_binary32_max_located(tall, monkeypatch):
    """A flip of exponent bit 30 of an element in [0.5, 1) gives a value in [2^127, 2^128):
    finite, near the binary32 maximum.  The fused weighted sums scale every term by a weight
    in (0, 1], so they stay finite like the element itself and the fault is located and
    corrected (an unscaled weight of 31 overflowed to inf and left it uncorrectable)."""
    monkeypatch.setenv("ABFT_TALL_TILES", tall)
    m, n, k = 512, 512, 256
    r = Run(m, n, k, 128, 128, seed=71)
    C = r.C.cpu().numpy().astype(np.float64)
    enc = oracle.Encoded(r.A64, r.B64, 128, 128, dtype="bf16")
    # an element in [0.5, 1) at row and column offsets 29..31 of its 32 x 32 chunk
    cand = [(i, j) for i in range(29, m, 32) for j in range(29, n, 32) if 0.5 <= abs(C[i, j]) < 1.0]
    assert cand
    i, j = cand[len(cand) // 2]
    abft.abft_set_epilogue_faults(r.desc, r.ws, [(i, j, 30)])
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    abft.abft_set_epilogue_faults(r.desc, r.ws, [])
    Cf = r.C.cpu().numpy().astype(np.float64)
    assert np.isfinite(Cf[i, j]) and abs(Cf[i, j]) >= 2.0 ** 127
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    ost, orep, oC, on = enc.verify_correct(Cf)
    assert st == abft.OK and positions(rep) == [(i, j, abft.KIND_CORRECTED)] == positions(orep)
    check_fp32_product(r.C.cpu().numpy().astype(np.float64), r.A64, r.B64, oracle.gemm(r.A64, r.B64))
