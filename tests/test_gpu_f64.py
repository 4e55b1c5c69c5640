"""Parity of the binary64 CUDA path (through the C ABI) with the CPU oracle.

Values: relative Frobenius error <= 1e-12 and an elementwise rounding bound.
Decisions: fault positions, kinds and recovered blocks bit-exact, for every injected
flip the oracle classifies as graded or benign (guard-band flips may go either way)."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_F64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


class Run:
    """One problem on the GPU: operands, workspace, encode + ABFT product."""

    def __init__(self, A, B, vb_r, vb_c, p=0, q=0, plain=False, f=0):
        self.A_np, self.B_np = np.ascontiguousarray(A), np.ascontiguousarray(B)
        m, k = A.shape
        n = B.shape[1]
        self.m, self.n, self.k = m, n, k
        self.desc = abft.make_desc(m, n, k, "f64", vb_r, vb_c, p, q, grid_f=f)
        self.L = abft.abft_workspace_layout(self.desc)
        self.A = torch.from_numpy(self.A_np).cuda()
        self.B = torch.from_numpy(self.B_np).cuda()
        self.C = torch.empty((m, n), dtype=torch.float64, device="cuda")
        self.ws = torch.zeros(self.L.total, dtype=torch.uint8, device="cuda")
        abft.abft_encode(self.desc, self.A, self.B, self.ws)
        abft.abft_gemm(self.desc, self.A, self.B, self.C, self.ws)
        torch.cuda.synchronize()

    def region(self, off, shape):
        nb = int(np.prod(shape)) * 8
        return self.ws[off:off + nb].view(torch.float64).reshape(shape).cpu().numpy()

    def E(self):
        return self.region(self.L.E, (self.L.R, self.n))

    def F(self):
        return self.region(self.L.F, (self.m, self.L.Cc))

    def acs(self):
        return self.region(self.L.acs, (self.L.R, self.k))

    def bcs(self):
        return self.region(self.L.bcs, (self.k, self.L.Cc))


def rel_fro(x, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def check_product(C, A, B, ref):
    """Elementwise |C - ref| <= 2 k u (|A||B|) and relative Frobenius <= 1e-12."""
    k = A.shape[1]
    bound = 2 * k * 2.0 ** -53 * (np.abs(A) @ np.abs(B)) + 1e-300
    assert np.all(np.abs(C - ref) <= bound)
    assert rel_fro(C, ref) <= TOL_F64


SHAPES = [  # (m, n, k, vb_r, vb_c, p, q): several tiles and ragged tails
    (150, 130, 77, 32, 16, 0, 0),
    (64, 64, 64, 64, 64, 2, 2),
    (1, 1, 1, 1, 1, 0, 0),
    (200, 3, 300, 7, 3, 0, 0),
    (3, 257, 129, 3, 100, 0, 0),
    (192, 256, 40, 32, 64, 3, 4),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_encode_and_product_vs_oracle(shape):
    m, n, k, vbr, vbc, p, q = shape
    A = wl.operand((m, k), "normal", 1, 1)
    B = wl.operand((k, n), "uniform", 1, 2)
    r = Run(A, B, vbr, vbc, p, q)
    enc = oracle.Encoded(A, B, vbr, vbc, p, q)
    # encode: the unweighted sums run in the oracle's order (bitwise); weighted
    # sums differ only by fused multiply-add rounding
    acs, bcs = r.acs(), r.bcs()
    assert np.allclose(acs, enc.acs, rtol=1e-14, atol=1e-14 * np.abs(enc.acs).max())
    assert np.allclose(bcs, enc.bcs, rtol=1e-14, atol=1e-14 * np.abs(enc.bcs).max())
    assert np.array_equal(acs[0::2][:r.L.nvr], enc.acs[0::2][:r.L.nvr])
    for off, ref in ((r.L.nArow, enc.nArow), (r.L.nAblk, enc.nAblk), (r.L.nBcol, enc.nBcol),
                     (r.L.nBblk, enc.nBblk)):
        assert np.allclose(r.region(off, ref.shape), ref, rtol=1e-12)
    C = r.C.cpu().numpy()
    check_product(C, A, B, oracle.gemm(A, B))
    check_product(r.E(), enc.acs, B, enc.E)
    check_product(r.F(), A, enc.bcs, enc.F)


def test_plain_gemm_equals_abft_data_block():
    A = wl.operand((130, 90), "normal", 2, 1)
    B = wl.operand((90, 70), "normal", 2, 2)
    r = Run(A, B, 32, 32)
    C2 = torch.empty_like(r.C)
    abft.abft_gemm_plain(r.desc, r.A, r.B, C2)
    torch.cuda.synchronize()
    assert torch.equal(C2, r.C)


def test_k_zero_gives_zero_product_and_no_flags():
    A = np.zeros((40, 0))
    B = np.zeros((0, 24))
    r = Run(A, B, 8, 8)
    assert torch.count_nonzero(r.C).item() == 0
    st, rep, n = abft.abft_verify_correct(r.desc, r.C, r.ws)
    assert st == abft.OK and n == 0


@pytest.mark.parametrize("seed", range(6))
def test_fault_free_no_false_positives(seed):
    A = wl.operand((256, 192), "uniform", seed, 1)
    B = wl.operand((192, 320), "normal", seed, 2)
    r = Run(A, B, 64, 32, 4, 5)
    C0 = r.C.clone()
    st, rep, n = abft.abft_verify_correct(r.desc, r.C, r.ws)
    assert st == abft.OK and n == 0 and torch.equal(C0, r.C)


def verify_both(r, enc, Cf_np, erased=()):
    """Run the GPU verify on the current C and the oracle verify on the same C."""
    st, rep, n = abft.abft_verify_correct(r.desc, r.C, r.ws, erased=erased)
    ost, orep, oC, on = enc.verify_correct(Cf_np, erased=erased)
    return (st, rep, n), (ost, orep, oC, on)


def positions(rep, kinds=(abft.KIND_CORRECTED, abft.KIND_NONFINITE_CORRECTED)):
    return sorted((e["row"], e["col"], e["kind"]) for e in rep if e["kind"] in kinds)


@pytest.mark.parametrize("seed", range(100))
def test_f64_512_single_flip_parity(seed):
    """512^3 U[-1,1], one seeded flip (uniform position and bit) in C before verify."""
    w = wl.F64_512
    A, B = wl.operands(w, seed)
    r = Run(A, B, w.vb_r, w.vb_c)
    enc = oracle.Encoded(A, B, w.vb_r, w.vb_c)
    Cstar = oracle.gemm(A, B)
    C_clean = r.C.cpu().numpy()
    (i, j, b), = wl.bit_flips(seed, w.m, w.n, 1)
    abft.abft_inject_bitflips(r.desc, r.C, [(i, j, b)])
    Cf = r.C.cpu().numpy()
    assert np.array_equal(Cf, wl.flip_f64(C_clean, [(i, j, b)]), equal_nan=True)
    cls = enc.classify(i, j, Cf[i, j] - C_clean[i, j])
    (st, rep, n), (ost, orep, oC, on) = verify_both(r, enc, Cf)
    Cg = r.C.cpu().numpy()
    if cls == "graded":
        kind = abft.KIND_CORRECTED if np.isfinite(Cf[i, j]) else abft.KIND_NONFINITE_CORRECTED
        assert st == abft.OK and positions(rep) == [(i, j, kind)] and n == 1
        assert ost == oracle.ST_OK and positions(orep) == [(i, j, kind)]
    elif cls == "benign":
        assert st == abft.OK and n == 0 and on == 0
    else:  # guard band: any outcome, but a correction must be at the right place
        assert all((e["row"], e["col"]) == (i, j) for e in rep if e["kind"] in (1, 2))
    if cls != "guard":
        assert rel_fro(Cg, oC) <= TOL_F64
        assert rel_fro(Cg, Cstar) <= TOL_F64


@pytest.mark.parametrize("bit", [62, 61, 60, 55, 63])
def test_f64_512_forced_graded_flips(bit):
    """Exponent and sign flips are always graded; bit 62 on an element in [1, 2)
    produces a NaN, located by the non-finite scan."""
    w = wl.F64_512
    A, B = wl.operands(w, 1000 + bit)
    r = Run(A, B, w.vb_r, w.vb_c)
    enc = oracle.Encoded(A, B, w.vb_r, w.vb_c)
    C_clean = r.C.cpu().numpy()
    cand = np.argwhere((np.abs(C_clean) >= 1) & (np.abs(C_clean) < 2))
    i, j = (int(v) for v in cand[len(cand) // 3])
    abft.abft_inject_bitflips(r.desc, r.C, [(i, j, bit)])
    Cf = r.C.cpu().numpy()
    with np.errstate(invalid="ignore"):
        assert enc.classify(i, j, Cf[i, j] - C_clean[i, j]) == "graded"
    (st, rep, n), (ost, orep, oC, on) = verify_both(r, enc, Cf)
    kind = abft.KIND_CORRECTED if np.isfinite(Cf[i, j]) else abft.KIND_NONFINITE_CORRECTED
    if bit == 62:
        assert kind == abft.KIND_NONFINITE_CORRECTED
    assert st == abft.OK and positions(rep) == [(i, j, kind)] == positions(orep)
    assert rel_fro(r.C.cpu().numpy(), oracle.gemm(A, B)) <= TOL_F64


@pytest.mark.parametrize("seed", range(10))
def test_grid_erasure_and_flips_parity(seed):
    """Scaled-down grid workload: 6x6 blocks of 64, one block erased to NaN and three
    graded flips in distinct other blocks; verify (skipping the erased block) then
    rebuild the block from the block checksum."""
    m = n = k = 384
    A = wl.operand((m, k), "normal", seed, 1)
    B = wl.operand((k, n), "normal", seed, 2)
    r = Run(A, B, 64, 64, 6, 6)
    enc = oracle.Encoded(A, B, 64, 64, 6, 6)
    Cstar = oracle.gemm(A, B)
    (bi, bj), = wl.erased_blocks(seed, 6, 6, 1)
    flips = [(i, j, 62 - (t % 3)) for t, (i, j, _) in enumerate(
        wl.bit_flips(seed, m, n, 3, distinct_blocks=(64, 64), avoid_blocks=[(bi, bj)]))]
    C_clean = r.C.cpu().numpy()
    abft.abft_inject_bitflips(r.desc, r.C, flips)
    abft.abft_erase_block(r.desc, r.C, bi, bj)
    Cf = r.C.cpu().numpy()
    assert np.isnan(Cf[64 * bi:64 * bi + 64, 64 * bj:64 * bj + 64]).all()
    for i, j, _ in flips:
        assert enc.classify(i, j, Cf[i, j] - C_clean[i, j]) == "graded"
    (st, rep, n_), (ost, orep, oC, on) = verify_both(r, enc, Cf, erased=[(bi, bj)])
    assert st == abft.OK and ost == oracle.ST_OK
    assert [(a, b) for a, b, _ in positions(rep)] == sorted((i, j) for i, j, _ in flips)
    assert positions(rep) == positions(orep)
    st, ent = abft.abft_recover_block(r.desc, r.C, r.ws, bi, bj)
    ost, oCr, onfl = enc.recover_block(oC, bi, bj)
    assert st == abft.OK and ost == oracle.ST_OK and onfl == 0
    assert ent["kind"] == abft.KIND_BLOCK_RECOVERED and (ent["row"], ent["col"]) == (64 * bi, 64 * bj)
    Cg = r.C.cpu().numpy()
    blk = np.s_[64 * bi:64 * bi + 64, 64 * bj:64 * bj + 64]
    assert rel_fro(Cg[blk], Cstar[blk]) <= TOL_F64
    assert rel_fro(Cg[blk], oCr[blk]) <= TOL_F64
    assert rel_fro(Cg, Cstar) <= TOL_F64


def test_errors_sharing_lines_are_uncorrectable_like_oracle():
    A = wl.operand((64, 48), "int", 3, 1)
    B = wl.operand((48, 64), "int", 3, 2)
    r = Run(A, B, 64, 64)
    enc = oracle.Encoded(A, B, 64, 64)
    abft.abft_inject_bitflips(r.desc, r.C, [(1, 1, 62), (1, 5, 61), (4, 1, 60)])
    Cf = r.C.cpu().numpy()
    (st, rep, n), (ost, orep, oC, on) = verify_both(r, enc, Cf)
    assert st == abft.ERR_UNCORRECTABLE and ost == oracle.ST_UNCORRECTABLE
    key = lambda rr: sorted((e["row"], e["col"], e["kind"]) for e in rr)
    assert key(rep) == key(orep)


def test_two_errors_in_one_column_line_integer_exact():
    """Two errors share a column line; each is alone in its row line, so both are
    corrected from their row lines and the exact integer product comes back."""
    A = wl.operand((64, 40), "int", 4, 1)
    B = wl.operand((40, 64), "int", 4, 2)
    r = Run(A, B, 64, 16)
    enc = oracle.Encoded(A, B, 64, 16)
    C_clean = r.C.clone()
    abft.abft_inject_bitflips(r.desc, r.C, [(3, 7, 61), (50, 7, 58)])
    Cf = r.C.cpu().numpy()
    (st, rep, n), (ost, orep, oC, on) = verify_both(r, enc, Cf)
    assert st == abft.OK and ost == oracle.ST_OK
    key = lambda rr: [(e["row"], e["col"], e["kind"], e["side"]) for e in rr]
    assert key(rep) == key(orep) and [(e[0], e[1]) for e in key(rep)] == [(3, 7), (50, 7)]
    assert torch.equal(r.C, C_clean)


def test_unlisted_erasure_is_reported_uncorrectable():
    A = wl.operand((128, 64), "normal", 5, 1)
    B = wl.operand((64, 128), "normal", 5, 2)
    r = Run(A, B, 32, 32, 4, 4)
    abft.abft_erase_block(r.desc, r.C, 1, 2)
    st, rep, n = abft.abft_verify_correct(r.desc, r.C, r.ws, max_reports=4)
    assert st == abft.ERR_UNCORRECTABLE and n > 4 and len(rep) == 4


def test_f64_11264_grid22_full_size():
    """The benchmark workload at full size (11264^3, 22x22 grid of 512, one erased
    block, three flips in distinct blocks), in the benchmark's launch configuration.
    The oracle checks sampled outputs; the section 4.3 residual check covers all of C."""
    w = wl.F64_11264_GRID22
    seed = 0
    A, B = wl.operands(w, seed)
    r = Run(A, B, w.vb_r, w.vb_c, w.p, w.q)
    enc = oracle.Encoded(A, B, w.vb_r, w.vb_c, w.p, w.q, products=False)
    g = wl.rng(seed, 99)
    rows = np.sort(g.choice(w.m, 48, replace=False))
    cols = np.sort(g.choice(w.n, 48, replace=False))
    Cs = r.C[rows][:, cols].cpu().numpy()
    check_product(Cs, A[rows], B[:, cols], oracle.gemm(A[rows], B[:, cols]))
    Es = r.E()[:, cols]
    check_product(Es, enc.acs, B[:, cols], oracle.gemm(enc.acs, B[:, cols]))
    Fs = r.F()[rows]
    check_product(Fs, A[rows], enc.bcs, oracle.gemm(A[rows], enc.bcs))
    x = wl.operand((w.n,), "uniform", seed, 5)
    C_clean = r.C.cpu().numpy()
    assert oracle.residual_check(A, B, C_clean, x) < 1.0

    (bi, bj), = wl.erased_blocks(seed, w.p, w.q, 1)
    flips = wl.bit_flips(seed, w.m, w.n, 3, distinct_blocks=(512, 512), avoid_blocks=[(bi, bj)])
    flips = [(i, j, 62 - t) for t, (i, j, _) in enumerate(flips)]
    abft.abft_inject_bitflips(r.desc, r.C, flips)
    abft.abft_erase_block(r.desc, r.C, bi, bj)
    st, rep, n = abft.abft_verify_correct(r.desc, r.C, r.ws, erased=[(bi, bj)])
    assert st == abft.OK
    assert [(a, b) for a, b, _ in positions(rep)] == sorted((i, j) for i, j, _ in flips)
    st, ent = abft.abft_recover_block(r.desc, r.C, r.ws, bi, bj)
    assert st == abft.OK
    Cg = r.C.cpu().numpy()
    blk = np.s_[512 * bi:512 * bi + 512, 512 * bj:512 * bj + 512]
    ref_blk = oracle.gemm(A[512 * bi:512 * bi + 512], B[:, 512 * bj:512 * bj + 512])
    assert rel_fro(Cg[blk], ref_blk) <= TOL_F64
    for i, j, _ in flips:
        assert abs(Cg[i, j] - C_clean[i, j]) <= 1e-12 * np.abs(C_clean[i]).max()
    assert oracle.residual_check(A, B, Cg, x) < 1.0


@pytest.mark.parametrize("f,nerase", [(2, 2), (3, 3), (3, 2)])
def test_multiple_erasures_per_block_column(f, nerase):
    """f block checksums (section 2.1): nerase erased blocks in one block column, one more in
    another column, and a flip elsewhere -- verified (erased blocks skipped), the flip
    corrected, every erased block rebuilt; values against the oracle's rebuild and the
    binary64 product, block checksum rows against the oracle's encode."""
    m = n = 384
    k = 256
    p = q = 6
    bs = m // p
    A = wl.operand((m, k), "normal", 40 + f, 1)
    B = wl.operand((k, n), "normal", 40 + f, 2)
    r = Run(A, B, 64, 64, p, q, f=f)
    enc = oracle.Encoded(A, B, 64, 64, p, q, f=f)
    assert r.L.R == 2 * (m // 64) + f * bs
    E = r.E()
    assert rel_fro(E, enc.E) <= TOL_F64
    Cstar = oracle.gemm(A, B)
    blocks = [(bi, 2) for bi in (0, 3, 5)[:nerase]] + [(4, 0)]
    flip = (20, 300, 61)  # block (0, 4)
    abft.abft_inject_bitflips(r.desc, r.C, [flip])
    for bi, bj in blocks:
        abft.abft_erase_block(r.desc, r.C, bi, bj)
    Cf = r.C.cpu().numpy()
    (st, rep, n_), (ost, orep, oC, on) = verify_both(r, enc, Cf, erased=blocks)
    assert st == abft.OK and ost == oracle.ST_OK
    assert positions(rep) == positions(orep) == [(20, 300, abft.KIND_CORRECTED)]
    st, ents = abft.abft_recover_blocks(r.desc, r.C, r.ws, blocks)
    ost, oCr, onfl = enc.recover_blocks(oC, blocks)
    assert st == abft.OK and ost == oracle.ST_OK and onfl == 0
    assert [(e["row"], e["col"], e["kind"]) for e in ents] == \
        [(bs * bi, 64 * bj, abft.KIND_BLOCK_RECOVERED) for bi, bj in blocks]
    Cg = r.C.cpu().numpy()
    for bi, bj in blocks:
        blk = np.s_[bs * bi:bs * (bi + 1), 64 * bj:64 * (bj + 1)]
        assert rel_fro(Cg[blk], Cstar[blk]) <= 1e-11
        assert rel_fro(Cg[blk], oCr[blk]) <= 1e-11
    assert rel_fro(Cg, Cstar) <= 1e-11


def test_more_erasures_than_block_checksums_refused():
    A = wl.operand((256, 128), "normal", 50, 1)
    B = wl.operand((128, 256), "normal", 50, 2)
    r = Run(A, B, 64, 64, 4, 4, f=2)
    for bi in (0, 1, 2):
        abft.abft_erase_block(r.desc, r.C, bi, 1)
    st, ents = abft.abft_recover_blocks(r.desc, r.C, r.ws, [(0, 1), (1, 1), (2, 1)])
    assert st == abft.ERR_UNCORRECTABLE
    assert np.isnan(r.C.cpu().numpy()[0:192, 64:128]).all()      # nothing launched
    st, ents = abft.abft_recover_blocks(r.desc, r.C, r.ws, [(0, 1), (1, 1)])
    assert st == abft.ERR_UNCORRECTABLE                            # block (2, 1) still NaN


@pytest.mark.parametrize("where", ["A", "B"])
@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_non_finite_operand_decided_like_oracle(where, value):
    """A NaN or Inf in an operand (a degenerate input of the method): a whole row (A) or
    column (B) of C is non-finite and so are the checksums that cover it.  Every such
    element is located by the non-finite scan and recomputed -- to a non-finite value --
    and its lines stay flagged: the verify reports them uncorrectable, exactly as the
    oracle does, and leaves every finite element alone."""
    g = wl.rng(5)
    m, n, k = 256, 192, 128
    A, B = g.standard_normal((m, k)), g.standard_normal((k, n))
    if where == "A":
        A[37, 11] = value
    else:
        B[5, 100] = value
    r = Run(A, B, 64, 64)
    enc = oracle.Encoded(A, B, 64, 64)
    C = r.C.cpu().numpy()
    with np.errstate(invalid="ignore", over="ignore"):
        ref = oracle.gemm(A, B)
    assert np.array_equal(np.isfinite(C), np.isfinite(ref))
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, max_reports=4096)
    ost, orep, oC, on = enc.verify_correct(C, max_reports=4096)
    assert st == abft.ERR_UNCORRECTABLE and ost == oracle.ST_UNCORRECTABLE
    key = lambda e: (e["row"], e["col"], e["kind"])
    assert nrep == on and sorted(map(key, rep)) == sorted(map(key, orep))
    fin = np.isfinite(ref)
    assert np.array_equal(r.C.cpu().numpy()[fin], C[fin])


@pytest.mark.parametrize("f,start", [(2, 0), (2, 10), (4, 0), (4, 9)])
def test_adjacent_erasures_on_the_22_block_grid(f, start):
    """The 22-block-row grid of the 11264^3 workload with 64-row blocks: f adjacent lost
    blocks of one block column are rebuilt by the binary64 solve with centred Vandermonde
    nodes (condition number 45 for two adjacent blocks, 1.6e4 for four).  Two come back
    within 1e-12 and pass the re-check; four come back within cond(M) times the rounding
    of a line, above the element checksums' threshold, and the re-check reports them
    uncorrectable -- the same status as the oracle's rebuild of the same C."""
    p, bs, q, bc, k = 22, 64, 2, 64, 512
    A = wl.operand((p * bs, k), "normal", 70 + f, 1)
    B = wl.operand((k, q * bc), "normal", 70 + f, 2)
    r = Run(A, B, bs, bc, p, q, f=f)
    enc = oracle.Encoded(A, B, bs, bc, p, q, f=f)
    Cstar = oracle.gemm(A, B)
    blocks = [(bi, 1) for bi in range(start, start + f)]
    for bi, bj in blocks:
        abft.abft_erase_block(r.desc, r.C, bi, bj)
    Cf = r.C.cpu().numpy()
    st, rep, n_ = abft.abft_verify_correct(r.desc, r.C, r.ws, erased=blocks)
    assert st == abft.OK and n_ == 0
    st, ents = abft.abft_recover_blocks(r.desc, r.C, r.ws, blocks)
    ost, oCr, onfl = enc.recover_blocks(Cf, blocks)
    Cg = r.C.cpu().numpy()
    err = max(rel_fro(Cg[bs * bi:bs * (bi + 1), bc:], Cstar[bs * bi:bs * (bi + 1), bc:])
              for bi, _ in blocks)
    if f == 2:
        assert st == abft.OK and ost == oracle.ST_OK and err <= TOL_F64
    else:
        assert st == abft.ERR_UNCORRECTABLE and ost == oracle.ST_UNCORRECTABLE
        assert err <= 1e-10


@pytest.mark.parametrize("f,start", [(2, 6), (4, 6)])
def test_adjacent_erasures_on_the_22_block_grid_bf16(f, start):
    """The same on the bf16 tensor-core path (binary32 C): two adjacent lost blocks are
    rebuilt within 8 cond(M) times the fp32 rounding of the lines and pass the re-check;
    four adjacent ones are reported uncorrectable by the re-check (their rebuilt values
    carry cond(M) ~ 1e4 times the binary32 rounding), never silently accepted."""
    p, bs, q, bc, k = 22, 128, 2, 128, 256
    m, n = p * bs, q * bc
    U32 = 2.0 ** -24
    bits_a = wl.bf16_bits(wl.operand((m, k), "normal", 80 + f, 1))
    bits_b = wl.bf16_bits(wl.operand((k, n), "normal", 80 + f, 2))
    A64, B64 = oracle.bf16_to_f64(bits_a), oracle.bf16_to_f64(bits_b)
    A = torch.from_numpy(bits_a.view(np.int16)).view(torch.bfloat16).cuda()
    B = torch.from_numpy(bits_b.view(np.int16)).view(torch.bfloat16).cuda()
    desc = abft.make_desc(m, n, k, "bf16", 128, 128, p, q, grid_f=f)
    ws = torch.zeros(abft.abft_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
    C = torch.empty((m, n), dtype=torch.float32, device="cuda")
    abft.abft_encode(desc, A, B, ws)
    abft.abft_gemm(desc, A, B, C, ws)
    blocks = [(bi, 1) for bi in range(start, start + f)]
    for bi, bj in blocks:
        abft.abft_erase_block(desc, C, bi, bj)
    st, rep, n_ = abft.abft_verify_correct(desc, C, ws, erased=blocks, reread_C=0)
    assert st == abft.OK and n_ == 0
    st, ents = abft.abft_recover_blocks(desc, C, ws, blocks)
    Cstar = oracle.gemm(A64, B64)
    Cg = C.cpu().numpy().astype(np.float64)
    rows = [bi for bi, _ in blocks]
    M = np.array([[oracle.block_coef(l, I, p) for I in rows] for l in range(f)])
    err = max(rel_fro(Cg[bs * bi:bs * (bi + 1), bc:], Cstar[bs * bi:bs * (bi + 1), bc:])
              for bi in rows)
    if f == 2:
        assert st == abft.OK
        assert err <= 8 * np.linalg.cond(M) * (4 * np.sqrt(k) * U32 + 2.0 ** -17)
    else:
        assert st == abft.ERR_UNCORRECTABLE
