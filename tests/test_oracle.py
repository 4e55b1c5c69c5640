"""Pins for the CPU oracle: each test checks it against something other than itself --
hand-worked values, numpy (library special cases), exact integer arithmetic, closed
forms and invariants of Eq. (1), brute force on tiny matrices.  No GPU needed."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    """Parse a golden file: '# comment' lines, 'key v...' lines and 'key r c' matrix headers."""
    out, lines = {}, [l.strip() for l in open(os.path.join(GOLDEN, name))]
    lines = [l for l in lines if l and not l.startswith("#")]
    t = 0
    while t < len(lines):
        parts = lines[t].split()
        key = parts[0]
        vals = [float(v) for v in parts[1:]]
        if len(vals) == 2 and key not in ("col_residual", "row_residual") and t + 1 < len(lines) \
                and not lines[t + 1].split()[0][0].isalpha():
            r, c = int(vals[0]), int(vals[1])
            out[key] = np.array([[float(v) for v in lines[t + 1 + i].split()] for i in range(r)])
            assert out[key].shape == (r, c)
            t += 1 + r
        else:
            out[key] = vals
            t += 1
    return out


# --------------------------------------------------------------------------- GEMM
def test_gemm_matches_numpy():
    g = wl.rng(1)
    A, B = g.standard_normal((37, 29)), g.standard_normal((29, 53))
    C = oracle.gemm(A, B)
    bound = 29 * 2.0 ** -52 * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(C - A @ B) <= bound)


def test_gemm_exact_on_integers():
    g = wl.rng(2)
    A = g.integers(-50, 51, (23, 31))
    B = g.integers(-50, 51, (31, 17))
    C = oracle.gemm(A, B)
    assert np.array_equal(C, (A @ B).astype(np.float64))


def test_gemm_identity_and_rank_one():
    g = wl.rng(3)
    B = g.standard_normal((12, 9))
    assert np.array_equal(oracle.gemm(np.eye(12), B), B)
    u = g.integers(-9, 10, 7).astype(float)
    v = g.integers(-9, 10, 12).astype(float)
    Bi = g.integers(-9, 10, (12, 9)).astype(float)
    C = oracle.gemm(np.outer(u, v), Bi)
    vB = np.array([sum(v[l] * Bi[l, j] for l in range(12)) for j in range(9)])
    assert np.array_equal(C, np.outer(u, vB))


# --------------------------------------------------------------------------- encode
def test_weights_hand_values():
    assert oracle.weight(0, 512) == 1 / 512 and oracle.weight(511, 512) == 1.0
    assert [oracle.weight(t, 3) for t in range(3)] == [0.25, 0.5, 0.75]
    assert oracle.weight(0, 1) == 1.0


def test_encode_golden():
    gd = read_golden("encode_small.txt")
    A = np.array([[1, 2], [3, 4], [5, 6], [7, 8]], float)
    B = np.array([[1, 2, 3, 4], [5, 6, 7, 8]], float)
    assert np.array_equal(oracle.encode_A(A, 2, p=2), gd["A_vb2_p2"])
    assert np.array_equal(oracle.encode_A(A, 3), gd["A_vb3"])
    assert np.array_equal(oracle.encode_B(B, 2), gd["B_vb2"])


@pytest.mark.parametrize("m,n,k,vbr,vbc,p,q", [(12, 10, 7, 4, 5, 3, 2), (11, 13, 5, 4, 3, 0, 0),
                                               (8, 8, 8, 8, 8, 1, 1)])
def test_consistency_invariants_exact(m, n, k, vbr, vbc, p, q):
    """Eq. (1): the product of the encoded operands carries the checksums of the
    product.  With small integers every sum is exact, so equality is bitwise:
    (e^T A_I) B = e^T C_I, (w^T A_I) B = w^T C_I, A (B_J e) = C_J e, S_A B = sum_I C_I."""
    g = wl.rng(4)
    A = g.integers(-4, 5, (m, k))
    B = g.integers(-4, 5, (k, n))
    C = A @ B  # exact int64 product (numpy)
    enc = oracle.Encoded(A, B, vbr, vbc, p, q)
    er, ew = 2 ** math.ceil(math.log2(vbr)), 2 ** math.ceil(math.log2(vbc))
    for I in range(-(-m // vbr)):
        blk = C[I * vbr:(I + 1) * vbr]
        w = np.arange(1, blk.shape[0] + 1)[:, None]
        assert np.array_equal(enc.E[2 * I], blk.sum(0))
        assert np.array_equal(enc.E[2 * I + 1] * er, (w * blk).sum(0))
    for J in range(-(-n // vbc)):
        blk = C[:, J * vbc:(J + 1) * vbc]
        w = np.arange(1, blk.shape[1] + 1)[None, :]
        assert np.array_equal(enc.F[:, 2 * J], blk.sum(1))
        assert np.array_equal(enc.F[:, 2 * J + 1] * ew, (w * blk).sum(1))
    if p:
        bs = m // p
        S = sum(C[I * bs:(I + 1) * bs] for I in range(p))
        assert np.array_equal(enc.E[2 * (-(-m // vbr)):], S)


def test_norms_vs_numpy():
    g = wl.rng(5)
    A, B = g.standard_normal((10, 7)), g.standard_normal((7, 9))
    nrow, nblk = oracle.norms_A(A, 4)
    assert np.allclose(nrow, np.linalg.norm(A, axis=1), rtol=1e-14)
    ncol, nbb = oracle.norms_B(B, 4)
    assert np.allclose(ncol, np.linalg.norm(B, axis=0), rtol=1e-14)
    for I in range(3):
        blk = A[4 * I:4 * I + 4]
        w = np.arange(1, blk.shape[0] + 1)[:, None] / 4.0
        ref = [np.linalg.norm(blk), np.linalg.norm(w * blk), np.linalg.norm(blk.sum(0)),
               np.linalg.norm((w * blk).sum(0))]
        assert np.allclose(nblk[4 * I:4 * I + 4], ref, rtol=1e-14)
    for J in range(3):
        blk = B[:, 4 * J:4 * J + 4]
        w = np.arange(1, blk.shape[1] + 1)[None, :] / 4.0
        ref = [np.linalg.norm(blk), np.linalg.norm(w * blk), np.linalg.norm(blk.sum(1)),
               np.linalg.norm((w * blk).sum(1))]
        assert np.allclose(nbb[4 * J:4 * J + 4], ref, rtol=1e-14)


# --------------------------------------------------------------------------- verify
def test_locate_golden():
    gd = read_golden("locate_small.txt")
    A = np.array([[1, 0], [0, 1], [1, 1], [2, 1]], float)
    B = np.array([[1, 2, 3, 4], [0, 1, 0, 1]], float)
    enc = oracle.Encoded(A, B, 4, 4, 2, 2)
    C = oracle.gemm(A, B)
    i, j, val = (int(v) if t < 2 else v for t, v in enumerate(gd["fault"]))
    Cf = C.copy()
    Cf[i, j] = val
    re, rw, *_ = enc.col_residuals(Cf)
    assert (re[0, j], rw[0, j]) == tuple(gd["col_residual"])
    re, rw, *_ = enc.row_residuals(Cf)
    assert (re[i, 0], rw[i, 0]) == tuple(gd["row_residual"])
    st, rep, Cc, _ = enc.verify_correct(Cf)
    assert st == oracle.ST_OK
    assert [(r["row"], r["col"], r["kind"]) for r in rep] == [(i, j, oracle.KIND_CORRECTED)]
    assert Cc[i, j] == gd["corrected"][0] and rep[0]["delta"] == val - gd["corrected"][0]
    # erasure recovery
    assert np.array_equal(enc.E[2:], gd["S"])
    Ce = C.copy()
    Ce[2:4, 0:2] = np.nan
    st, rep, Cv, _ = enc.verify_correct(Ce, erased=[(1, 0)])
    assert st == oracle.ST_OK and rep == []
    st, Cr, nfl = enc.recover_block(Cv, 1, 0)
    assert st == oracle.ST_OK and nfl == 0
    assert np.array_equal(Cr[2:4, 0:2], gd["recovered"])


@pytest.mark.parametrize("seed", range(6))
def test_fault_free_no_flags(seed):
    """False-positive invariant: a fault-free product is never flagged, and the
    residuals sit far below the thresholds."""
    A, B = wl.operand((96, 64), "uniform", seed, 1), wl.operand((64, 80), "normal", seed, 2)
    enc = oracle.Encoded(A, B, 32, 16, 3, 5)
    C = oracle.gemm(A, B)
    st, rep, Cc, n = enc.verify_correct(C)
    assert st == oracle.ST_OK and n == 0 and np.array_equal(Cc, C)
    re, rw, te, tw, nf = enc.col_residuals(C)
    assert np.max(np.abs(re) / te) < 0.05 and np.max(np.abs(rw) / tw) < 0.05
    re, rw, te, tw, nf = enc.row_residuals(C)
    assert np.max(np.abs(re) / te) < 0.05 and np.max(np.abs(rw) / tw) < 0.05


def _tau_at(enc, i, j):
    """Smaller of the column-check and row-check thresholds at element (i, j)."""
    C0 = np.zeros((enc.m, enc.n))
    _, _, te, _, _ = enc.col_residuals(C0)
    _, _, te2, _, _ = enc.row_residuals(C0)
    return min(te[i // enc.cfg.vb_r, j], te2[i, j // enc.cfg.vb_c])


def test_brute_force_every_position_every_bit_integer_data():
    """Tiny integer product (exact): every element x every one of the 64 bits.
    A flip that is non-finite or exceeds 8 tau must be located at exactly its
    position and the original bit pattern restored; a flip below tau/2 must not be
    flagged.  Flips in between (the guard band) may go either way."""
    g = wl.rng(6)
    A = g.integers(-4, 5, (8, 6)).astype(float)
    B = g.integers(-4, 5, (6, 8)).astype(float)
    enc = oracle.Encoded(A, B, 4, 4)
    C = oracle.gemm(A, B)
    located = silent = 0
    for i in range(8):
        for j in range(8):
            tau = _tau_at(enc, i, j)
            for b in range(64):
                Cf = wl.flip_f64(C, [(i, j, b)])
                d = Cf[i, j] - C[i, j]
                st, rep, Cc, n = enc.verify_correct(Cf)
                if not np.isfinite(Cf[i, j]) or abs(d) >= 8 * tau:
                    assert st == oracle.ST_OK, (i, j, b)
                    assert [(r["row"], r["col"]) for r in rep] == [(i, j)], (i, j, b, rep)
                    kind = oracle.KIND_CORRECTED if np.isfinite(Cf[i, j]) else oracle.KIND_NONFINITE
                    assert rep[0]["kind"] == kind
                    assert Cc.view(np.uint64)[i, j] == C.view(np.uint64)[i, j]
                    located += 1
                elif abs(d) <= tau / 2:
                    assert n == 0, (i, j, b)
                    silent += 1
    assert located > 8 * 8 * 12 and silent > 0


def test_brute_force_random_data_graded_bits():
    """Random FP64 data: every position, the 12 top bits (sign + exponent): located
    exactly and restored to within rounding of the recomputation."""
    A, B = wl.operand((16, 24), "uniform", 7, 1), wl.operand((24, 12), "uniform", 7, 2)
    enc = oracle.Encoded(A, B, 8, 6)
    C = oracle.gemm(A, B)
    for i in range(16):
        for j in range(12):
            tau = _tau_at(enc, i, j)
            for b in range(52, 64):
                Cf = wl.flip_f64(C, [(i, j, b)])
                if np.isfinite(Cf[i, j]) and abs(Cf[i, j] - C[i, j]) < 8 * tau:
                    continue
                st, rep, Cc, n = enc.verify_correct(Cf)
                assert st == oracle.ST_OK and [(r["row"], r["col"]) for r in rep] == [(i, j)]
                assert abs(Cc[i, j] - C[i, j]) <= 1e-13 * np.abs(C).max()


def test_two_errors_in_one_column_line_use_row_checks():
    g = wl.rng(8)
    A = g.integers(-4, 5, (8, 5)).astype(float)
    B = g.integers(-4, 5, (5, 8)).astype(float)
    enc = oracle.Encoded(A, B, 8, 4)
    C = oracle.gemm(A, B)
    Cf = C.copy()
    Cf[1, 3] += 100.0
    Cf[6, 3] -= 37.0
    st, rep, Cc, n = enc.verify_correct(Cf)
    assert st == oracle.ST_OK
    assert [(r["row"], r["col"], r["side"]) for r in rep] == [(1, 3, 1), (6, 3, 1)]
    assert np.array_equal(Cc, C)


def test_three_errors_sharing_lines_are_uncorrectable():
    g = wl.rng(9)
    A = g.integers(-4, 5, (8, 5)).astype(float)
    B = g.integers(-4, 5, (5, 8)).astype(float)
    enc = oracle.Encoded(A, B, 8, 8)
    C = oracle.gemm(A, B)
    Cf = C.copy()
    Cf[1, 1] += 100.0
    Cf[1, 5] += 30.0
    Cf[4, 1] -= 70.0
    st, rep, Cc, n = enc.verify_correct(Cf)
    assert st == oracle.ST_UNCORRECTABLE
    assert any(r["kind"] == oracle.KIND_UNCORRECTABLE for r in rep)


def test_erasure_exact_on_integers():
    g = wl.rng(10)
    A = g.integers(-4, 5, (12, 7)).astype(float)
    B = g.integers(-4, 5, (7, 9)).astype(float)
    enc = oracle.Encoded(A, B, 2, 3, 3, 3)
    C = oracle.gemm(A, B)
    for bi in range(3):
        for bj in range(3):
            Ce = C.copy()
            Ce[4 * bi:4 * bi + 4, 3 * bj:3 * bj + 3] = np.nan
            st, rep, Cv, n = enc.verify_correct(Ce, erased=[(bi, bj)])
            assert st == oracle.ST_OK and n == 0
            st, Cr, nfl = enc.recover_block(Cv, bi, bj)
            assert st == oracle.ST_OK and nfl == 0 and np.array_equal(Cr, C)


def test_erasure_plus_flips_random():
    """Scaled-down grid workload: one block erased, three flips in distinct other blocks."""
    w = wl.Workload("t", "f64", 96, 96, 64, 16, 16, 6, 6, dist="normal")
    A, B = wl.operands(w, 11)
    enc = oracle.Encoded(A, B, 16, 16, 6, 6)
    C = oracle.gemm(A, B)
    (bi, bj), = wl.erased_blocks(11, 6, 6, 1)
    flips = [(i, j, 62) for i, j, _ in wl.bit_flips(11, 96, 96, 3, distinct_blocks=(16, 16),
                                                      avoid_blocks=[(bi, bj)])]
    Cf = wl.flip_f64(C, flips)
    Cf[16 * bi:16 * bi + 16, 16 * bj:16 * bj + 16] = np.nan
    st, rep, Cv, n = enc.verify_correct(Cf, erased=[(bi, bj)])
    assert st == oracle.ST_OK
    assert sorted((r["row"], r["col"]) for r in rep) == sorted((i, j) for i, j, _ in flips)
    st, Cr, nfl = enc.recover_block(Cv, bi, bj)
    assert st == oracle.ST_OK and nfl == 0
    assert np.linalg.norm(Cr - C) / np.linalg.norm(C) < 1e-14


def test_residual_check_section_4_3():
    A, B = wl.operand((40, 30), "normal", 12, 1), wl.operand((30, 50), "normal", 12, 2)
    x = wl.operand((50,), "uniform", 12, 3)
    C = oracle.gemm(A, B)
    assert oracle.residual_check(A, B, C, x) < 1.0
    assert oracle.residual_check(A, B, A @ B, x) < 1.0
    Cbad = C.copy()
    Cbad[7, 11] += 1e-6
    assert oracle.residual_check(A, B, Cbad, x) > 1e3


# --------------------------------------------------------------------------- formats
def test_bf16_decode():
    bits = np.array([0x3F80, 0xC000, 0x7F80, 0x0001, 0x4049], np.uint16)
    v = oracle.bf16_to_f64(bits)
    assert v[0] == 1.0 and v[1] == -2.0 and np.isinf(v[2]) and v[3] == 2.0 ** -133
    assert v[4] == 3.140625
    import torch
    allb = np.arange(0, 65536, dtype=np.uint16)
    ref = torch.from_numpy(allb.view(np.int16)).view(torch.bfloat16).double().numpy()
    got = oracle.bf16_to_f64(allb)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin]) and np.all(np.isnan(got[np.isnan(ref)]))


def test_e4m3_decode():
    assert oracle.e4m3_value(0x7E) == 448.0 and oracle.e4m3_value(0xFE) == -448.0
    assert oracle.e4m3_value(0x08) == 2.0 ** -6 and oracle.e4m3_value(0x01) == 2.0 ** -9
    assert oracle.e4m3_value(0x38) == 1.0 and math.isnan(oracle.e4m3_value(0x7F))
    import torch
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8)
    ref = codes.view(torch.float8_e4m3fn).double().numpy()
    got = np.array([oracle.e4m3_value(b) for b in range(256)])
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin]) and np.all(np.isnan(got[~fin]))


# ---- several block checksums (section 2.1: f checksums recover f lost blocks)

def test_block_coefficients_vandermonde():
    """c_{l,I} = x_I^l with distinct dyadic nodes x_I = (2I+1-p)/2^e, 2^e > p (symmetric
    about 0): l = 0 is the plain sum, values are exact, and every f x f minor is
    nonsingular."""
    import itertools
    p = 22
    for I in range(p):
        assert oracle.block_coef(0, I, p) == 1.0
        assert oracle.block_coef(1, I, p) == (2 * I + 1 - 22) / 32.0
        assert oracle.block_coef(3, I, p) == ((2 * I + 1 - 22) / 32.0) ** 3   # exact: dyadic
    assert oracle.block_coef(1, 0, 1) == 0.0 and oracle.block_coef(1, 1, 3) == 0.0
    p = 7
    for f in (2, 3, 4):
        Mfull = np.array([[oracle.block_coef(l, I, p) for I in range(p)] for l in range(f)])
        for cols in itertools.combinations(range(p), f):
            assert abs(np.linalg.det(Mfull[:, cols])) > 0


def _int_problem(seed, m, k, n):
    g = wl.rng(seed)
    return (g.integers(-4, 5, (m, k)).astype(float), g.integers(-4, 5, (k, n)).astype(float))


def test_block_checksum_rows_invariant_exact():
    """S^(l) B = sum_I c_{l,I} C_I exactly on integer data, for every l < f."""
    A, B = _int_problem(20, 12, 7, 9)
    f, p = 3, 4
    enc = oracle.Encoded(A, B, 3, 3, p, 3, f=f)
    C = oracle.gemm(A, B)
    bs, nvr = 12 // p, 4
    for l in range(f):
        S = enc.acs[2 * nvr + l * bs: 2 * nvr + (l + 1) * bs]
        ref = sum(oracle.block_coef(l, I, p) * C[I * bs:(I + 1) * bs] for I in range(p))
        assert np.array_equal(oracle.gemm(S, B), ref)
        assert np.array_equal(enc.E[2 * nvr + l * bs: 2 * nvr + (l + 1) * bs], ref)


def test_multi_erasure_every_subset_integer_data():
    """Every subset of up to f = 3 erased block rows of a block column (and one more block
    in another column) is rebuilt to the exact integer product."""
    import itertools
    A, B = _int_problem(21, 16, 7, 9)
    p, q, f = 4, 3, 3
    enc = oracle.Encoded(A, B, 4, 3, p, q, f=f)
    C = oracle.gemm(A, B)
    for J in range(q):
        other = (0, (J + 1) % q)
        for t in (1, 2, 3):
            for rows in itertools.combinations(range(p), t):
                blocks = [(r, J) for r in rows] + [other]
                Ce = C.copy()
                for bi, bj in blocks:
                    Ce[4 * bi:4 * bi + 4, 3 * bj:3 * bj + 3] = np.nan
                st, rep, Cv, n = enc.verify_correct(Ce, erased=blocks)
                assert st == oracle.ST_OK and n == 0
                st, Cr, nfl = enc.recover_blocks(Cv, blocks)
                assert st == oracle.ST_OK and nfl == 0
                assert np.allclose(Cr, C, rtol=0, atol=1e-9) and np.array_equal(np.rint(Cr), C)


def test_multi_erasure_random_data_and_single_block_agrees():
    w = wl.Workload("t", "f64", 96, 96, 64, 16, 16, 6, 6, dist="normal")
    A, B = wl.operands(w, 12)
    enc2 = oracle.Encoded(A, B, 16, 16, 6, 6, f=2)
    enc1 = oracle.Encoded(A, B, 16, 16, 6, 6)
    C = oracle.gemm(A, B)
    Ce = C.copy()
    Ce[32:48, 16:32] = np.nan
    Ce[80:96, 16:32] = np.nan          # two blocks of block column 1
    st, Cr, nfl = enc2.recover_blocks(Ce, [(2, 1), (5, 1)])
    assert st == oracle.ST_OK and nfl == 0
    blk = np.s_[32:48, 16:32], np.s_[80:96, 16:32]
    for b in blk:
        assert np.linalg.norm(Cr[b] - C[b]) <= 1e-12 * np.linalg.norm(C[b])
    # one erased block: the first checksum (the plain sum) alone, as with f = 1
    Ce = C.copy()
    Ce[32:48, 16:32] = np.nan
    st2, Cr2, _ = enc2.recover_blocks(Ce, [(2, 1)])
    st1, Cr1, _ = enc1.recover_block(Ce, 2, 1)
    assert st1 == st2 == oracle.ST_OK
    assert np.allclose(Cr2, Cr1, rtol=1e-13, atol=1e-13)


def test_more_erasures_than_checksums_is_uncorrectable():
    A, B = _int_problem(22, 12, 7, 9)
    enc = oracle.Encoded(A, B, 3, 3, 4, 3, f=2)
    C = oracle.gemm(A, B)
    Ce = C.copy()
    for bi in (0, 1, 3):
        Ce[3 * bi:3 * bi + 3, 0:3] = np.nan
    st, Cr, nfl = enc.recover_blocks(Ce, [(0, 0), (1, 0), (3, 0)])
    assert st == oracle.ST_UNCORRECTABLE and np.isnan(Cr[0:3, 0:3]).all()


def test_multi_erasure_conditioning_p22():
    """Several adjacent lost blocks of the 22-block-row grid (binary64, N(0,1) data): the
    rebuild solves the Vandermonde system of their nodes, whose condition number bounds
    the amplification of the survivors' and checksums' rounding (centred nodes: at most
    45, 1.1e3 and 1.6e4 for 2, 3 and 4 adjacent blocks).  Two adjacent blocks come back
    within 1e-12 and pass the re-check; three or four come back within cond(M) times the
    rounding of a line (1e-11 relative here), which the element checksums' re-check does
    flag: the status is uncorrectable, never a silently wrong block."""
    p, bs, q, bc, k = 22, 32, 2, 32, 512
    g = wl.rng(5)
    A = g.standard_normal((p * bs, k))
    B = g.standard_normal((k, q * bc))
    C = oracle.gemm(A, B)
    for f, start in ((2, 0), (2, 10), (3, 0), (4, 0), (4, 9)):
        rows = list(range(start, start + f))
        M = np.array([[oracle.block_coef(l, I, p) for I in rows] for l in range(f)])
        assert np.linalg.cond(M) <= {2: 45, 3: 1.1e3, 4: 1.7e4}[f]
        enc = oracle.Encoded(A, B, bs, bc, p, q, f=f)
        Ce = C.copy()
        for I in rows:
            Ce[I * bs:(I + 1) * bs, bc:] = np.nan
        st, Cr, nfl = enc.recover_blocks(Ce, [(I, 1) for I in rows])
        err = max(np.linalg.norm(Cr[I * bs:(I + 1) * bs, bc:] - C[I * bs:(I + 1) * bs, bc:])
                  / np.linalg.norm(C[I * bs:(I + 1) * bs, bc:]) for I in rows)
        if f == 2:
            assert st == oracle.ST_OK and nfl == 0 and err <= 1e-12
        else:
            assert err <= 1e-11
            assert st == oracle.ST_UNCORRECTABLE and nfl > 0
