"""Chained binary64 products on the GPU (section 3.2: stacked ABFT calls carry the
checksums instead of recomputing them), through the C ABI, against the CPU oracle.

Carried rows / columns are the earlier product's expected checksums bit for bit; norms and
deviation bounds match the oracle's; decisions (fault positions and kinds) match the
oracle's; values within 1e-12 relative Frobenius of the oracle's chain."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


class Prod:
    """One binary64 ABFT product on the GPU; left / right: earlier Prods whose outputs are
    this product's A / B (their workspaces supply the carried checksums)."""

    def __init__(self, A, B, vb_r, vb_c, p=0, q=0, f=0, left=None, right=None, s=0.0):
        self.A = A if torch.is_tensor(A) else torch.from_numpy(np.ascontiguousarray(A)).cuda()
        self.B = B if torch.is_tensor(B) else torch.from_numpy(np.ascontiguousarray(B)).cuda()
        m, k = self.A.shape
        n = self.B.shape[1]
        self.m, self.n, self.k = m, n, k
        self.desc = abft.make_desc(m, n, k, "f64", vb_r, vb_c, p, q, grid_f=f, tau_safety=s)
        self.L = abft.abft_workspace_layout(self.desc)
        self.ws = torch.zeros(self.L.total, dtype=torch.uint8, device="cuda")
        self.C = torch.empty((m, n), dtype=torch.float64, device="cuda")
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

    def acs(self):
        return self.region(self.L.acs, (self.L.R, self.k))

    def bcs(self):
        return self.region(self.L.bcs, (self.k, self.L.Cc))

    def nAblk(self):
        return self.region(self.L.nAblk, (4 * self.L.nvr,))

    def nBblk(self):
        return self.region(self.L.nBblk, (4 * self.L.nvc,))

    def car(self):
        return self.region(self.L.car_a, (2 * self.L.nvr,)), \
            self.region(self.L.car_b, (2 * self.L.nvc,))


def rel_fro(x, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def positions(rep, kinds=(abft.KIND_CORRECTED, abft.KIND_NONFINITE_CORRECTED)):
    return sorted((e["row"], e["col"], e["kind"]) for e in rep if e["kind"] in kinds)


def test_carried_checksums_norms_and_bounds():
    g = wl.rng(7)
    m, k, n, n2, r2 = 150, 77, 130, 96, 70
    A, B = g.standard_normal((m, k)), g.standard_normal((k, n))
    D, G = g.standard_normal((n, n2)), g.standard_normal((r2, m))
    p1 = Prod(A, B, 32, 16)
    e1 = oracle.Encoded(A, B, 32, 16)
    C1 = oracle.gemm(A, B)
    left = Prod(p1.C, D, 32, 16, left=p1)       # C D
    right = Prod(G, p1.C, 16, 16, right=p1)     # G C
    assert np.array_equal(left.acs(), p1.E())   # carried, bit for bit
    assert np.array_equal(right.bcs(), p1.F())
    o_left = oracle.Encoded(C1, D, 32, 16, left=e1)
    o_right = oracle.Encoded(G, C1, 16, 16, right=e1)
    assert np.allclose(left.nAblk(), o_left.nAblk, rtol=1e-12, atol=0)
    assert np.allclose(right.nBblk(), o_right.nBblk, rtol=1e-12, atol=0)
    car_a, car_b = left.car()
    assert np.allclose(car_a, o_left.car_a, rtol=1e-12, atol=0) and car_a.min() > 0
    assert not car_b.any()                      # B = D was encoded afresh
    car_a, car_b = right.car()
    assert np.allclose(car_b, o_right.car_b, rtol=1e-12, atol=0) and not car_a.any()
    # a fresh encode clears a workspace's carried bounds
    abft.abft_encode(left.desc, left.A, left.B, left.ws)
    torch.cuda.synchronize()
    assert not left.car()[0].any()
    # the chained products are the plain products, their checksums the oracle's
    assert rel_fro(left.C.cpu().numpy(), oracle.gemm(C1, D)) <= TOL
    assert rel_fro(right.C.cpu().numpy(), oracle.gemm(G, C1)) <= TOL
    assert rel_fro(left.E(), o_left.E) <= TOL and rel_fro(right.F(), o_right.F) <= TOL


@pytest.mark.parametrize("seed", range(4))
def test_three_chained_products_with_faults(seed):
    """A B -> C (left-chained) C D -> E, then G E (right-chained).  Graded flips in each
    output are located and corrected like the oracle; the final product is the oracle's."""
    g = wl.rng(100 + seed)
    m, k, n, n2, r3 = 160, 96, 144, 112, 72
    A, B = g.standard_normal((m, k)), g.standard_normal((k, n))
    D, G = g.standard_normal((n, n2)), g.standard_normal((r3, m))
    vb_r, vb_c = 32, 16
    o1 = oracle.Encoded(A, B, vb_r, vb_c)
    C_or = oracle.gemm(A, B)
    p1 = Prod(A, B, vb_r, vb_c)
    stages = [(p1, o1, C_or)]
    for stage in range(3):
        p, o, ref = stages[-1]
        mm, nn = p.C.shape
        flips = [(i, j, 62 - (t % 2)) for t, (i, j, _) in
                 enumerate(wl.bit_flips(seed * 10 + stage, mm, nn, 2,
                                        distinct_blocks=(vb_r, vb_c)))]
        C_clean = p.C.cpu().numpy()
        abft.abft_inject_bitflips(p.desc, p.C, flips)
        Cf = p.C.cpu().numpy()
        for i, j, _ in flips:
            with np.errstate(invalid="ignore"):
                assert o.classify(i, j, Cf[i, j] - C_clean[i, j]) == "graded"
        st, rep, nrep = abft.abft_verify_correct(p.desc, p.C, p.ws)
        ost, orep, oC, on = o.verify_correct(Cf)
        assert st == abft.OK and ost == oracle.ST_OK
        assert positions(rep) == positions(orep)
        assert sorted((i, j) for i, j, _ in flips) == [(a, b) for a, b, _ in positions(rep)]
        assert rel_fro(p.C.cpu().numpy(), ref) <= TOL
        if stage == 0:      # C D, left chain
            nxt = Prod(p.C, D, vb_r, vb_c, left=p)
            onxt = oracle.Encoded(ref, D, vb_r, vb_c, left=o)
            stages.append((nxt, onxt, oracle.gemm(ref, D)))
        elif stage == 1:    # G E: E is the right operand; chain its row checksums
            nxt = Prod(G, p.C, vb_c, vb_c, right=p)
            onxt = oracle.Encoded(G, ref, vb_c, vb_c, right=o)
            stages.append((nxt, onxt, oracle.gemm(G, ref)))
    last, olast, ref = stages[-1]
    assert rel_fro(last.C.cpu().numpy(), ref) <= TOL
    assert last.car()[1].min() > 0 and not last.car()[0].any()


def test_fault_free_chain_stays_silent_where_carry_dominates():
    """k1 >> n: the carried deviation dominates the next product's own rounding; with its
    bound the chained verify raises no flag even at safety factor 1."""
    for seed in range(3):
        g = wl.rng(200 + seed)
        m, k1, n, n2 = 256, 8192, 16, 192
        A, B, D = g.standard_normal((m, k1)), g.standard_normal((k1, n)), \
            g.standard_normal((n, n2))
        p1 = Prod(A, B, 32, 8, s=1.0)
        st, rep, nrep = abft.abft_verify_correct(p1.desc, p1.C, p1.ws)
        assert st == abft.OK and nrep == 0
        p2 = Prod(p1.C, D, 32, 8, left=p1, s=1.0)
        st, rep, nrep = abft.abft_verify_correct(p2.desc, p2.C, p2.ws)
        assert st == abft.OK and nrep == 0


def _ints(g, shape, lo=-8, hi=9):
    return g.integers(lo, hi, shape).astype(np.float64)


def test_fault_at_rest_left_operand_like_oracle():
    """C changed between the calls (integer data: exact).  The chained product's verify
    recomputes the spoiled output row from the carried checksums and reports the row lines
    uncorrectable, exactly as the oracle; a fresh encode of the changed C stays silent."""
    g = wl.rng(44)
    m, k, n, n2, vb_r, vb_c = 64, 24, 40, 48, 32, 16
    A, B = _ints(g, (m, k)), _ints(g, (k, n))
    D = g.integers(1, 9, (n, n2)).astype(np.float64)
    p1 = Prod(A, B, vb_r, vb_c)
    e1 = oracle.Encoded(A, B, vb_r, vb_c)
    st, rep, nrep = abft.abft_verify_correct(p1.desc, p1.C, p1.ws)
    assert st == abft.OK and nrep == 0
    C = oracle.gemm(A, B)
    assert np.array_equal(p1.C.cpu().numpy(), C)
    i, j = 37, 11
    assert abs(C[i, j]) >= 2
    # the lowest exponent bit doubles or halves the value: every sum stays exact
    abft.abft_inject_bitflips(p1.desc, p1.C, [(i, j, 52)])
    Cbad = p1.C.cpu().numpy()
    assert Cbad[i, j] in (2 * C[i, j], C[i, j] / 2)
    p2 = Prod(p1.C, D, vb_r, vb_c, left=p1)
    o2 = oracle.Encoded(Cbad, D, vb_r, vb_c, left=e1)
    Ebad = p2.C.cpu().numpy()
    st, rep, nrep = abft.abft_verify_correct(p2.desc, p2.C, p2.ws, max_reports=4096)
    ost, orep, oE, on = o2.verify_correct(Ebad, max_reports=4096)
    assert st == abft.ERR_UNCORRECTABLE and ost == oracle.ST_UNCORRECTABLE
    key = lambda r: (r["row"], r["col"], r["kind"])
    assert sorted(map(key, rep)) == sorted(map(key, orep))
    assert positions(rep) == [(i, l, abft.KIND_CORRECTED) for l in range(n2)]
    assert np.array_equal(p2.C.cpu().numpy(), oracle.gemm(C, D))
    fresh = Prod(p1.C, D, vb_r, vb_c)
    st, rep, nrep = abft.abft_verify_correct(fresh.desc, fresh.C, fresh.ws)
    assert st == abft.OK and nrep == 0


def test_fault_at_rest_right_operand_like_oracle():
    g = wl.rng(45)
    m, k, n, r_, vb_r, vb_c = 48, 20, 40, 56, 16, 16
    A, B = _ints(g, (m, k)), _ints(g, (k, n))
    G = g.integers(1, 9, (r_, m)).astype(np.float64)
    p1 = Prod(A, B, vb_r, vb_c)
    e1 = oracle.Encoded(A, B, vb_r, vb_c)
    C = oracle.gemm(A, B)
    i, j = 21, 33
    assert abs(C[i, j]) >= 2
    abft.abft_inject_bitflips(p1.desc, p1.C, [(i, j, 52)])
    Cbad = p1.C.cpu().numpy()
    assert Cbad[i, j] in (2 * C[i, j], C[i, j] / 2)
    p2 = Prod(G, p1.C, 32, vb_c, right=p1)
    o2 = oracle.Encoded(G, Cbad, 32, vb_c, right=e1)
    Hbad = p2.C.cpu().numpy()
    st, rep, nrep = abft.abft_verify_correct(p2.desc, p2.C, p2.ws, max_reports=4096)
    ost, orep, oH, on = o2.verify_correct(Hbad, max_reports=4096)
    assert st == abft.ERR_UNCORRECTABLE and ost == oracle.ST_UNCORRECTABLE
    key = lambda r: (r["row"], r["col"], r["kind"])
    assert sorted(map(key, rep)) == sorted(map(key, orep))
    assert positions(rep) == [(l, j, abft.KIND_CORRECTED) for l in range(r_)]
    assert np.array_equal(p2.C.cpu().numpy(), oracle.gemm(G, C))


@pytest.mark.parametrize("f,blocks", [(1, [(2, 1)]), (2, [(0, 3), (3, 3)])])
def test_chained_output_erasures_rebuilt_from_carried_block_checksums(f, blocks):
    """The block checksum rows travel with the column checksums: erased blocks of a chained
    product's output are rebuilt (the paper's recovery, section 2.1) to 1e-12."""
    g = wl.rng(300 + f)
    m, k, n, n2, p, q = 512, 192, 256, 384, 4, 4
    A, B, D = g.standard_normal((m, k)), g.standard_normal((k, n)), g.standard_normal((n, n2))
    p1 = Prod(A, B, 64, 64, p, q, f=f)
    p2 = Prod(p1.C, D, 64, 64, p, q, f=f, left=p1)
    e1 = oracle.Encoded(A, B, 64, 64, p, q, f=f)
    C = oracle.gemm(A, B)
    e2 = oracle.Encoded(C, D, 64, 64, p, q, f=f, left=e1)
    E = oracle.gemm(C, D)
    bs, bc = m // p, n2 // q
    for bi, bj in blocks:
        abft.abft_erase_block(p2.desc, p2.C, bi, bj)
    st, rep, nrep = abft.abft_verify_correct(p2.desc, p2.C, p2.ws, erased=blocks)
    assert st == abft.OK and nrep == 0
    Ef = p2.C.cpu().numpy()
    st, ents = abft.abft_recover_blocks(p2.desc, p2.C, p2.ws, blocks)
    ost, oE, onfl = e2.recover_blocks(Ef, blocks)
    assert st == abft.OK and ost == oracle.ST_OK and onfl == 0
    assert [(e["row"], e["col"]) for e in ents] == [(bi * bs, bj * bc) for bi, bj in blocks]
    Eg = p2.C.cpu().numpy()
    for bi, bj in blocks:
        blk = np.s_[bi * bs:(bi + 1) * bs, bj * bc:(bj + 1) * bc]
        assert rel_fro(Eg[blk], E[blk]) <= TOL
        assert rel_fro(Eg[blk], oE[blk]) <= TOL
