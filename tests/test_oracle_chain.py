"""Pins for the oracle's chained calls (section 3.2: ABFT BLAS calls stacked one after the
other carry the checksums instead of recomputing them).  Each test checks the oracle against
something other than itself: exact integer arithmetic, numpy norms, the measured deviation of
the carried checksums, and the behaviour that distinguishes carrying from re-encoding."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import workloads as wl

cdiv = oracle.cdiv


def _ints(g, shape, lo=-8, hi=9):
    return g.integers(lo, hi, shape).astype(np.float64)


def _chain_left(A, B, D, vb_r, vb_c, **kw):
    e1 = oracle.Encoded(A, B, vb_r, vb_c, **kw)
    C = oracle.gemm(A, B)
    e2 = oracle.Encoded(C, D, vb_r, vb_c, left=e1, **kw)
    return e1, C, e2


def test_carried_rows_equal_fresh_encoding_on_integers():
    """On exact (integer) data the product's expected checksums ARE the checksums of its
    output: the carried rows, block checksum rows included, equal a fresh encoding of C."""
    g = wl.rng(41)
    m, k, n, n2, vb_r, vb_c, p, f = 96, 40, 56, 24, 32, 16, 3, 2
    A, B, D = _ints(g, (m, k)), _ints(g, (k, n)), _ints(g, (n, n2))
    e1, C, e2 = _chain_left(A, B, D, vb_r, vb_c, p=p, q=2, f=f)
    assert np.array_equal(e2.acs, oracle.encode_A(C, vb_r, p, f))
    # the right side: C as the right operand of G C
    G = _ints(g, (20, m))
    e3 = oracle.Encoded(G, C, 16, vb_c, right=e1)
    assert np.array_equal(e3.bcs, oracle.encode_B(C, vb_c))
    # fault-free exact chains leave exactly zero residuals
    E = oracle.gemm(C, D)
    re, rw, te, tw, nf = e2.col_residuals(E)
    assert not re.any() and not rw.any() and not nf.any()
    H = oracle.gemm(G, C)
    re, rw, te, tw, nf = e3.row_residuals(H)
    assert not re.any() and not rw.any()


def test_carried_norms_are_those_of_the_carried_rows():
    g = wl.rng(42)
    A, B, D = g.standard_normal((70, 33)), g.standard_normal((33, 45)), g.standard_normal((45, 12))
    e1, C, e2 = _chain_left(A, B, D, 32, 16)
    nrow, nblk = oracle.norms_A(C, 32)
    assert np.allclose(e2.nArow, np.linalg.norm(C, axis=1), rtol=1e-14)
    for I in range(cdiv(70, 32)):
        assert e2.nAblk[4 * I] == pytest.approx(nblk[4 * I], rel=1e-14)
        assert e2.nAblk[4 * I + 1] == pytest.approx(nblk[4 * I + 1], rel=1e-14)
        assert e2.nAblk[4 * I + 2] == pytest.approx(np.linalg.norm(e1.E[2 * I]), rel=1e-14)
        assert e2.nAblk[4 * I + 3] == pytest.approx(np.linalg.norm(e1.E[2 * I + 1]), rel=1e-14)
    G = g.standard_normal((9, 70))
    e3 = oracle.Encoded(G, C, 16, 16, right=e1)
    for J in range(cdiv(45, 16)):
        assert e3.nBblk[4 * J + 2] == pytest.approx(np.linalg.norm(e1.F[:, 2 * J]), rel=1e-14)
        assert e3.nBblk[4 * J + 3] == pytest.approx(np.linalg.norm(e1.F[:, 2 * J + 1]), rel=1e-14)


def test_carry_bound_by_hand():
    """car_e(I) = max_j ||B_j|| (f1 ||A_I||_F + f2 ||e^T A_I|| + car_prev), written out."""
    g = wl.rng(43)
    m, k, n, vb = 50, 27, 31, 16
    A, B = g.standard_normal((m, k)), g.standard_normal((k, n))
    e1 = oracle.Encoded(A, B, vb, 8)
    u = 2.0 ** -53
    f1 = np.sqrt(k) * u + np.sqrt(vb) * 2 * u + u
    f2 = np.sqrt(k) * u + u
    mx = np.linalg.norm(B, axis=0).max()
    car = oracle.carry_rows(e1)
    for I in range(cdiv(m, vb)):
        blk = A[I * vb:(I + 1) * vb]
        w = (np.arange(blk.shape[0]) + 1) / 16.0
        want_e = mx * (f1 * np.linalg.norm(blk) + f2 * np.linalg.norm(blk.sum(0)))
        want_w = mx * (f1 * np.linalg.norm(w[:, None] * blk) + f2 * np.linalg.norm(w @ blk))
        assert car[2 * I] == pytest.approx(want_e, rel=1e-12)
        assert car[2 * I + 1] == pytest.approx(want_w, rel=1e-12)
    mr = np.linalg.norm(A, axis=1).max()
    carb = oracle.carry_cols(e1)
    for J in range(cdiv(n, 8)):
        blk = B[:, J * 8:(J + 1) * 8]
        f1r = np.sqrt(k) * u + np.sqrt(8) * 2 * u + u
        want = mr * (f1r * np.linalg.norm(blk) + f2 * np.linalg.norm(blk.sum(1)))
        assert carb[2 * J] == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_carry_bound_covers_measured_deviation_over_a_chain(seed):
    """The deviation of carried rows from the sums of the stored product stays under the
    bound, for one and for two chained products (the recursion carries the earlier bound)."""
    g = wl.rng(300 + seed)
    m, k1, n, n2, n3, vb = 64, 2048, 16, 24, 20, 32
    A, B = g.standard_normal((m, k1)), g.standard_normal((k1, n))
    D, G = g.standard_normal((n, n2)), g.standard_normal((n2, n3))
    e1, C, e2 = _chain_left(A, B, D, vb, 8)
    E = oracle.gemm(C, D)
    e3 = oracle.Encoded(E, G, vb, 8, left=e2)
    nr = 2 * cdiv(m, vb)
    for enc, out, nxt in ((e1, C, e2), (e2, E, e3)):
        dev = np.abs(enc.E[:nr] - oracle.encode_A(out, vb))
        for r in range(nr):
            assert dev[r].max() <= nxt.car_a[r]
    # the second bound contains the first: dropping car_prev would undercut it
    assert np.all(e3.car_a > e2.car_a * np.linalg.norm(D, axis=0).max() * 0.999)


@pytest.mark.parametrize("seed", range(3))
def test_uncarried_threshold_gives_false_flags_carried_does_not(seed):
    """With k1 >> n the carried deviation dominates the fresh rounding of the next
    product: without its term (s = 1) fault-free chains are flagged, with it they are not."""
    g = wl.rng(200 + seed)
    m, k1, n, n2, vb = 64, 8192, 8, 40, 32
    A, B, D = g.standard_normal((m, k1)), g.standard_normal((k1, n)), g.standard_normal((n, n2))
    e1, C, e2 = _chain_left(A, B, D, vb, 8, s=1.0)
    E = oracle.gemm(C, D)
    st, rep, _, nrep = e2.verify_correct(E)
    assert st == oracle.ST_OK and nrep == 0
    e2.car_a[:] = 0.0
    st0, rep0, _, nrep0 = e2.verify_correct(E)
    assert st0 == oracle.ST_UNCORRECTABLE and nrep0 > 0


def test_fault_at_rest_left_operand_is_caught_only_when_carried():
    """A value of C changed between the calls: the next product's row i is wrong in every
    column.  Carried checksums flag every column line, restore the whole output row exactly
    (integer data) and report the row lines, whose expectations came from the changed
    operand, uncorrectable.  Re-encoding the changed C would hide the change."""
    g = wl.rng(44)
    m, k, n, n2, vb_r, vb_c = 64, 24, 40, 48, 32, 16
    A, B = _ints(g, (m, k)), _ints(g, (k, n))
    D = g.integers(1, 9, (n, n2)).astype(np.float64)  # positive: every line sum moves
    e1 = oracle.Encoded(A, B, vb_r, vb_c)
    C = oracle.gemm(A, B)
    i, j, delta = 37, 11, 4096.0
    Cbad = C.copy()
    Cbad[i, j] += delta
    # the next call sees the changed operand; only its checksum rows are carried
    e2 = oracle.Encoded(Cbad, D, vb_r, vb_c, left=e1)
    Etrue = oracle.gemm(C, D)
    Ebad = oracle.gemm(Cbad, D)
    st, rep, Efix, nrep = e2.verify_correct(Ebad)
    assert st == oracle.ST_UNCORRECTABLE
    corr = [(r["row"], r["col"], r["delta"]) for r in rep if r["kind"] == oracle.KIND_CORRECTED]
    assert corr == [(i, l, delta * D[j, l]) for l in range(n2)]
    unc = [(r["row"], r["col"]) for r in rep if r["kind"] == oracle.KIND_UNCORRECTABLE]
    assert unc == [(i, -1)] * cdiv(n2, vb_c)
    assert np.array_equal(Efix, Etrue)
    # re-encoding the changed operand: consistent, silent
    fresh = oracle.Encoded(Cbad, D, vb_r, vb_c)
    st, rep, _, nrep = fresh.verify_correct(Ebad)
    assert st == oracle.ST_OK and nrep == 0


def test_fault_at_rest_right_operand_is_caught_only_when_carried():
    g = wl.rng(45)
    m, k, n, r_, vb_r, vb_c = 48, 20, 40, 56, 16, 16
    A, B = _ints(g, (m, k)), _ints(g, (k, n))
    G = g.integers(1, 9, (r_, m)).astype(np.float64)
    e1 = oracle.Encoded(A, B, vb_r, vb_c)
    C = oracle.gemm(A, B)
    i, j, delta = 21, 33, -2048.0
    Cbad = C.copy()
    Cbad[i, j] += delta
    e2 = oracle.Encoded(G, Cbad, 32, vb_c, right=e1)
    Htrue, Hbad = oracle.gemm(G, C), oracle.gemm(G, Cbad)
    st, rep, Hfix, nrep = e2.verify_correct(Hbad)
    assert st == oracle.ST_UNCORRECTABLE
    corr = sorted((r["row"], r["col"], r["delta"]) for r in rep
                  if r["kind"] == oracle.KIND_CORRECTED)
    assert corr == [(l, j, delta * G[l, i]) for l in range(r_)]
    unc = sorted((r["row"], r["col"]) for r in rep if r["kind"] == oracle.KIND_UNCORRECTABLE)
    assert unc == [(-1, j)] * cdiv(r_, 32)
    assert np.array_equal(Hfix, Htrue)
    fresh = oracle.Encoded(G, Cbad, 32, vb_c)
    assert fresh.verify_correct(Hbad)[0] == oracle.ST_OK


def test_chain_compute_faults_and_erasures_exact_on_integers():
    """Faults of the chained product itself are located and corrected as in a fresh one,
    and erased blocks of its output are rebuilt from the carried block checksums."""
    g = wl.rng(46)
    m, k, n, n2, vb, p, q, f = 96, 16, 48, 64, 16, 3, 4, 2
    A, B, D = _ints(g, (m, k), -4, 5), _ints(g, (k, n), -4, 5), _ints(g, (n, n2), -4, 5)
    e1, C, e2 = _chain_left(A, B, D, vb, vb, p=p, q=q, f=f)
    E = oracle.gemm(C, D)
    bad = E.copy()
    bad[5, 7] += 1000.0
    bad[70, 40] = np.inf
    st, rep, fixed, _ = e2.verify_correct(bad)
    assert st == oracle.ST_OK
    assert [(r["row"], r["col"]) for r in rep] == [(5, 7), (70, 40)]
    assert np.array_equal(fixed, E)
    lost = E.copy()
    bs, bc = m // p, n2 // q
    for bi in (0, 2):
        lost[bi * bs:(bi + 1) * bs, 1 * bc:2 * bc] = np.nan
    st, rebuilt, nfl = e2.recover_blocks(lost, [(0, 1), (2, 1)])
    assert st == oracle.ST_OK and nfl == 0
    assert np.array_equal(rebuilt, E)
