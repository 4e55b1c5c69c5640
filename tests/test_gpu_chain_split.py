"""Chained split-precision products on the GPU (section 3.2: stacked ABFT calls carry the
checksums instead of recomputing them) for the binary32-accuracy dtypes bf16x3 / bf16x6,
through the C ABI, against the CPU oracle.

The earlier product (bf16, bf16x3 or bf16x6) leaves binary32 C and binary64 expected
checksums; the chained product takes them as its checksum operand, split into bf16 pieces
(two for bf16x3, three for bf16x6).  Checked: the pieces add up to the carried values
within the split's representation bound, norms and carried deviation bounds against the
oracle's (the GPU sums the norms in binary32: 1e-5), fault decisions equal to the oracle's,
faults at rest caught, erased blocks rebuilt from the carried block checksums."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
# representation error of a binary64 value held as bf16 pieces (relative)
PIECES_REL = {"bf16x3": 2.0 ** -16, "bf16x6": 2.0 ** -25}
# relative Frobenius error of a product against binary64 on the same binary32 inputs
PROD_TOL = {"bf16x3": 1e-4, "bf16x6": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


def _dev(X, dtype):
    if torch.is_tensor(X):
        return X
    t = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    return t.to(torch.bfloat16) if dtype == "bf16" else t


class Prod:
    """One tensor-core ABFT product (binary32 C); left / right: earlier Prods whose
    outputs are this product's A / B."""

    def __init__(self, A, B, dtype, vb_r, vb_c, p=0, q=0, f=0, left=None, right=None,
                 s=0.0):
        self.dtype = dtype
        self.A, self.B = _dev(A, dtype), _dev(B, dtype)
        m, k = self.A.shape
        n = self.B.shape[1]
        self.m, self.n, self.k = m, n, k
        self.desc = abft.make_desc(m, n, k, dtype, vb_r, vb_c, p, q, grid_f=f, tau_safety=s)
        self.L = abft.abft_workspace_layout(self.desc)
        self.ws = torch.zeros(self.L.total, dtype=torch.uint8, device="cuda")
        self.C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        abft.abft_encode_chained(self.desc, self.A, self.B, self.ws,
                                 left=(left.desc, left.ws) if left else None,
                                 right=(right.desc, right.ws) if right else None)
        abft.abft_gemm(self.desc, self.A, self.B, self.C, self.ws)
        torch.cuda.synchronize()

    def region(self, off, shape):
        nb = int(np.prod(shape)) * 8
        return self.ws[off:off + nb].view(torch.float64).reshape(shape).cpu().numpy()

    def E(self):
        return self.region(self.L.E, (self.L.R, self.n))

    def F(self):
        return self.region(self.L.F, (self.m, self.L.Cc))

    def nAblk(self):
        return self.region(self.L.nAblk, (4 * self.L.nvr,))

    def nBblk(self):
        return self.region(self.L.nBblk, (4 * self.L.nvc,))

    def car(self):
        return self.region(self.L.car_a, (2 * self.L.nvr,)), \
            self.region(self.L.car_b, (2 * self.L.nvc,))

    def pieces(self, off, plane_bytes, rows, ld):
        """Sum of the bf16 checksum planes (rows x ld), in binary64."""
        tot = np.zeros((rows, ld), np.float64)
        for i in range(self.L.planes):
            o = off + i * plane_bytes
            pl = self.ws[o:o + rows * ld * 2].view(torch.bfloat16).reshape(rows, ld)
            tot += pl.float().cpu().numpy().astype(np.float64)
        return tot

    def acs_sum(self):
        return self.pieces(self.L.acs, self.L.acs_plane, self.L.R, self.L.acs_ld)

    def bcs_sum(self):
        return self.pieces(self.L.bcs, self.L.bcs_plane, self.k, self.L.bcs_ld)

    def Cf64(self):
        return self.C.cpu().numpy().astype(np.float64)


def _f64(X):
    if torch.is_tensor(X):
        return X.float().cpu().numpy().astype(np.float64)
    return np.asarray(X, np.float64)


def rel_fro(x, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def positions(rep, kinds=(abft.KIND_CORRECTED, abft.KIND_NONFINITE_CORRECTED)):
    return sorted((e["row"], e["col"], e["kind"]) for e in rep if e["kind"] in kinds)


def _operands(g, shape, dtype):
    X = g.standard_normal(shape).astype(np.float32)
    if dtype == "bf16":  # the values the bf16 product actually multiplies
        X = torch.from_numpy(X).to(torch.bfloat16).float().numpy()
    return X


@pytest.mark.parametrize("first,then", [("bf16x6", "bf16x6"), ("bf16", "bf16x3"),
                                        ("bf16x3", "bf16x6")])
def test_carried_pieces_norms_and_bounds(first, then):
    g = wl.rng(11)
    m, k, n, n2, r2 = 160, 72, 136, 96, 80
    A, B = _operands(g, (m, k), first), _operands(g, (k, n), first)
    D = g.standard_normal((n, n2)).astype(np.float32)
    G = g.standard_normal((r2, m)).astype(np.float32)
    p1 = Prod(A, B, first, 32, 16)
    left = Prod(p1.C, D, then, 32, 16, left=p1)      # C D
    right = Prod(G, p1.C, then, 16, 16, right=p1)    # G C
    rel = PIECES_REL[then]
    E1, F1 = p1.E(), p1.F()
    acs = left.acs_sum()
    assert np.all(np.abs(acs[:, :n] - E1) <= rel * np.abs(E1))   # left.k == n
    assert not acs[:, n:].any()
    bcs = right.bcs_sum()
    assert np.all(np.abs(bcs[:, :right.L.Cc] - F1) <= rel * np.abs(F1))
    assert not bcs[:, right.L.Cc:].any()
    # norms: the carried rows' own, and the stored operand's rows
    C1 = p1.Cf64()
    e1 = oracle.Encoded(_f64(A), _f64(B), 32, 16, dtype=first)
    o_left = oracle.Encoded(C1, D, 32, 16, dtype=then, left=e1)
    o_right = oracle.Encoded(G, C1, 16, 16, dtype=then, right=e1)
    nA = left.nAblk().reshape(-1, 4)
    want = o_left.nAblk.reshape(-1, 4)
    assert np.allclose(nA[:, :2], want[:, :2], rtol=1e-5, atol=0)
    assert np.allclose(nA[:, 2], np.linalg.norm(E1[0::2], axis=1), rtol=1e-5, atol=0)
    assert np.allclose(nA[:, 3], np.linalg.norm(E1[1::2], axis=1), rtol=1e-5, atol=0)
    nB = right.nBblk().reshape(-1, 4)
    assert np.allclose(nB[:, :2], o_right.nBblk.reshape(-1, 4)[:, :2], rtol=1e-5, atol=0)
    assert np.allclose(nB[:, 2], np.linalg.norm(F1[:, 0::2], axis=0), rtol=1e-5, atol=0)
    # carried deviation bounds: the oracle's formula on the earlier product's norms
    car_a, car_b = left.car()
    assert np.allclose(car_a, o_left.car_a, rtol=1e-5, atol=0) and car_a.min() > 0
    assert not car_b.any()
    car_a, car_b = right.car()
    assert np.allclose(car_b, o_right.car_b, rtol=1e-5, atol=0) and not car_a.any()
    # the chained products are the plain products; fault-free verifies stay silent
    assert rel_fro(left.Cf64(), oracle.gemm(C1, D)) <= PROD_TOL[then]
    assert rel_fro(right.Cf64(), oracle.gemm(G, C1)) <= PROD_TOL[then]
    for p in (p1, left, right):
        for reread in (0, 1):
            st, rep, nrep = abft.abft_verify_correct(p.desc, p.C, p.ws, reread_C=reread)
            assert st == abft.OK and nrep == 0


@pytest.mark.parametrize("seed", range(3))
def test_split_chain_faults_located_like_oracle(seed):
    """A B -> C (bf16x6), C D left-chained (bf16x6): accumulator flips in the chained
    product's epilogue are located and corrected exactly where the oracle puts them."""
    g = wl.rng(500 + seed)
    m, k, n, n2, vb_r, vb_c = 384, 256, 320, 512, 128, 128
    A, B = _operands(g, (m, k), "bf16x6"), _operands(g, (k, n), "bf16x6")
    D = g.standard_normal((n, n2)).astype(np.float32)
    p1 = Prod(A, B, "bf16x6", vb_r, vb_c)
    p2 = Prod(p1.C, D, "bf16x6", vb_r, vb_c, left=p1)
    e1 = oracle.Encoded(_f64(A), _f64(B), vb_r, vb_c, dtype="bf16x6")
    C1 = p1.Cf64()
    o2 = oracle.Encoded(C1, D, vb_r, vb_c, dtype="bf16x6", left=e1)
    clean = p2.Cf64()
    pos = [(a, b) for a, b, _ in wl.bit_flips(seed, m, n2, 3, bits=32,
                                             distinct_blocks=(vb_r, vb_c))]
    flips = [(i, j, 29 if abs(clean[i, j]) >= 2.0 else 30) for i, j in pos]
    abft.abft_set_epilogue_faults(p2.desc, p2.ws, flips)
    abft.abft_gemm(p2.desc, p2.A, p2.B, p2.C, p2.ws)
    abft.abft_set_epilogue_faults(p2.desc, p2.ws, [])
    Cf = p2.Cf64()
    for i, j in pos:
        assert o2.classify(i, j, Cf[i, j] - clean[i, j]) == "graded"
    st, rep, nrep = abft.abft_verify_correct(p2.desc, p2.C, p2.ws, reread_C=0)
    ost, orep, oC, on = o2.verify_correct(Cf)
    assert st == abft.OK and ost == oracle.ST_OK
    assert positions(rep) == positions(orep)
    assert [(a, b) for a, b, _ in positions(rep)] == sorted(pos)
    assert rel_fro(p2.Cf64(), oracle.gemm(C1, D)) <= PROD_TOL["bf16x6"]


def _ints(g, shape, lo, hi):
    return g.integers(lo, hi, shape).astype(np.float32)


# Small integers keep every sum exact in binary32: |C| <= 72, verify blocks of 16 rows
# (weights j/16), D in 1..4 over 32 columns: the largest expected checksum needs 22 bits.
@pytest.mark.parametrize("side", ["left", "right"])
def test_split_fault_at_rest_like_oracle(side):
    """A value of C changed between the calls: the chained split product's verify restores
    the spoiled output line from the carried checksums (exactly, on integer data) and reports
    the other side's lines uncorrectable, as the oracle does."""
    g = wl.rng(61 if side == "left" else 62)
    m, k, n = 48, 8, 32
    A, B = _ints(g, (m, k), -3, 4), _ints(g, (k, n), -3, 4)
    p1 = Prod(A, B, "bf16x6", 16, 16)
    e1 = oracle.Encoded(_f64(A), _f64(B), 16, 16, dtype="bf16x6")
    C = oracle.gemm(_f64(A), _f64(B))
    assert np.array_equal(p1.Cf64(), C)
    st, rep, nrep = abft.abft_verify_correct(p1.desc, p1.C, p1.ws)
    assert st == abft.OK and nrep == 0
    i, j = (37, 11) if side == "left" else (21, 29)
    assert abs(C[i, j]) >= 2
    # the lowest exponent bit of binary32 doubles or halves the value
    abft.abft_inject_bitflips(p1.desc, p1.C, [(i, j, 23)])
    Cbad = p1.Cf64()
    assert Cbad[i, j] in (2 * C[i, j], C[i, j] / 2)
    if side == "left":
        D = _ints(g, (n, 40), 1, 5)
        p2 = Prod(p1.C, D, "bf16x6", 16, 16, left=p1)
        o2 = oracle.Encoded(Cbad, _f64(D), 16, 16, dtype="bf16x6", left=e1)
        want = oracle.gemm(C, _f64(D))
        line = [(i, l, abft.KIND_CORRECTED) for l in range(40)]
        unc = [(i, -1)] * 3
    else:
        G = _ints(g, (40, m), 1, 5)
        p2 = Prod(G, p1.C, "bf16x6", 16, 16, right=p1)
        o2 = oracle.Encoded(_f64(G), Cbad, 16, 16, dtype="bf16x6", right=e1)
        want = oracle.gemm(_f64(G), C)
        line = [(l, j, abft.KIND_CORRECTED) for l in range(40)]
        unc = [(-1, j)] * 3
    bad = p2.Cf64()
    st, rep, nrep = abft.abft_verify_correct(p2.desc, p2.C, p2.ws, max_reports=4096)
    ost, orep, oC, on = o2.verify_correct(bad, max_reports=4096)
    assert st == abft.ERR_UNCORRECTABLE and ost == oracle.ST_UNCORRECTABLE
    key = lambda r: (r["row"], r["col"], r["kind"])
    assert sorted(map(key, rep)) == sorted(map(key, orep))
    assert positions(rep) == line
    assert sorted((r["row"], r["col"]) for r in rep
                  if r["kind"] == abft.KIND_UNCORRECTABLE) == unc
    assert np.array_equal(p2.Cf64(), want)
    # re-encoding the changed operand hides the change
    fresh = Prod(p2.A, p2.B, "bf16x6", 16, 16)
    st, rep, nrep = abft.abft_verify_correct(fresh.desc, fresh.C, fresh.ws)
    assert st == abft.OK and nrep == 0


@pytest.mark.parametrize("then", ["bf16x3", "bf16x6"])
def test_split_chain_erasure_rebuilt_from_carried_block_checksums(then):
    """The carried block checksum rows rebuild an erased block of the chained product's
    output; the rebuilt block carries the earlier product's rounding in its sums."""
    g = wl.rng(71)
    m, k, n, n2, p, q = 512, 256, 512, 512, 4, 4
    A, B = _operands(g, (m, k), "bf16x6"), _operands(g, (k, n), "bf16x6")
    D = g.standard_normal((n, n2)).astype(np.float32)
    p1 = Prod(A, B, "bf16x6", 128, 128, p, q, f=1)
    p2 = Prod(p1.C, D, then, 128, 128, p, q, f=1, left=p1)
    ref = oracle.gemm(p1.Cf64(), D)
    abft.abft_erase_block(p2.desc, p2.C, 2, 1)
    st, rep, nrep = abft.abft_verify_correct(p2.desc, p2.C, p2.ws, erased=[(2, 1)])
    assert st == abft.OK and nrep == 0
    st, ent = abft.abft_recover_block(p2.desc, p2.C, p2.ws, 2, 1)
    assert st == abft.OK
    Cg = p2.Cf64()
    blk = np.s_[256:384, 128:256]
    err = rel_fro(Cg[blk], ref[blk])
    print(f"{then}: rebuilt block rel Frobenius error {err:.2e}")
    assert err <= 4 * PROD_TOL[then]
    other = np.ones(Cg.shape, bool)
    other[blk] = False
    assert rel_fro(Cg[other], ref[other]) <= PROD_TOL[then]
