"""Pins of the oracle's detection thresholds and chained-call carry bounds.

The paper only says that the rounding of floating-point checksums is of the same order
as the rounding of the method itself (section 2.1), and that stacked ABFT calls keep
their checksums instead of recomputing them (section 3.2).  The oracle turns that into
a threshold formula (a probabilistic rounding model with Cauchy-Schwarz magnitudes) and
a bound on the deviation of carried checksums.  These tests pin both against things
other than the oracle:

* hand-worked values of the formula on a tiny integer case (tests/golden/threshold_small.txt);
* the rigorous worst-case rounding bound of each residual, written out here from |A|, |B|,
  |C| and the encoded operands with gamma_n = n u / (1 - n u) (Higham's bound for sums and
  dot products): every fault-free residual must lie inside it (a theorem), and the
  threshold must not exceed it (a threshold above the worst case would only lose
  detection power);
* the rounding model's own prediction of the fault-free residual size for N(0, 1) data:
  the largest residual over the lines of a product sits at a predictable fraction of the
  threshold, so a threshold several times too loose (or too tight) fails.

Binary64 throughout (the oracle's products are binary64).  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import workloads as wl
from test_oracle import read_golden

U = 2.0 ** -53


def gamma(n):
    return n * U / (1.0 - n * U)


A1 = np.array([[1, 2, 0], [2, 1, 1], [0, 1, 3], [1, 0, 2]], float)
B1 = np.array([[1, 0, 2, 1], [0, 1, 1, 2], [2, 1, 0, 1]], float)
B2 = np.array([[1, 0], [0, 1], [1, 1], [1, -1]], float)


# --------------------------------------------------------------------------- golden
def test_threshold_norms_golden():
    gd = read_golden("threshold_small.txt")
    enc = oracle.Encoded(A1, B1, 2, 4)
    # squared norms of the blocks worked by hand: ||A_I||_F, ||diag(w) A_I||_F,
    # ||e^T A_I||, ||w^T A_I|| per block
    assert np.allclose(enc.nAblk ** 2, gd["norms_A_blk"], rtol=1e-14, atol=0)
    assert np.allclose(enc.nBblk ** 2, gd["norms_B_blk"], rtol=1e-14, atol=0)
    assert np.allclose(enc.nArow ** 2, [5, 6, 10, 5], rtol=1e-14)
    assert np.allclose(enc.nBcol ** 2, [5, 2, 5, 6], rtol=1e-14)


@pytest.mark.parametrize("dtype,key", [("f64", "tau_f64"), ("bf16", "tau_bf16")])
def test_thresholds_golden(dtype, key):
    """The four thresholds of an element (column line e / w, row line e / w) against the
    hand-worked values; the two lines of each dtype have different block sizes (vb_r = 2,
    vb_c = 4), so a swapped f1 / f2, a dropped term or a wrong unit changes them."""
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                 "threshold_small.txt"))
            if l.startswith(key + " ")]
    assert len(rows) == 2
    enc = oracle.Encoded(A1, B1, 2, 4, dtype=dtype)
    for r in rows:
        i, j = int(r[1]), int(r[2])
        want = np.array([float(v) for v in r[3:7]])
        got = enc.thresholds_at(i, j)
        assert np.allclose(got, want, rtol=2e-10, atol=0), (i, j, got, want)


def test_carry_golden():
    """Carried-row deviation bounds out of product 1, and the thresholds of a product
    that takes product 1's output as its A (left chain), against hand-worked values."""
    gd = read_golden("threshold_small.txt")
    enc1 = oracle.Encoded(A1, B1, 2, 4)
    assert np.allclose(oracle.carry_rows(enc1), gd["car_rows"], rtol=2e-10, atol=0)
    C1 = oracle.gemm(A1, B1)
    assert np.array_equal(C1, A1 @ B1)
    enc2 = oracle.Encoded(C1, B2, 2, 2, left=enc1)
    assert np.array_equal(enc2.acs, enc1.E[:4])
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                 "threshold_small.txt"))
            if l.startswith("tau_chain ")]
    assert len(rows) == 2
    for r in rows:
        I, j = int(r[1]), int(r[2])
        want = np.array([float(v) for v in r[3:5]])
        got = enc2.thresholds_at(2 * I, j)[:2]
        assert np.allclose(got, want, rtol=2e-10, atol=0), (I, j, got, want)


# ------------------------------------------------------------- rigorous worst case
def col_bounds(enc, C):
    """Worst-case |residual| of every column line of a fault-free binary64 product.

    r_e = fl(fl(sum_i C_ij) - E_j) with C_ij = fl(sum_l a_il b_lj), acs_l = fl(sum_i a_il)
    and E_j = fl(sum_l acs_l b_lj).  In exact arithmetic sum_i C*_ij = sum_l acs*_l b_lj,
    so r_e is the sum of four rounding errors, each bounded by gamma_n times the sum of
    the magnitudes it adds: the observed sum (vb terms), the products of the block's
    elements (k terms each), the encoding (vb terms), and the checksum's product (k
    terms); the final subtraction adds a factor 1 + u.  The weighted line is the same
    with w_i |C_ij| and w_i |a_il|."""
    A, B = enc.A, enc.B
    m, k = A.shape
    n = B.shape[1]
    vb = enc.cfg.vb_r
    aA, aB, aC = np.abs(A), np.abs(B), np.abs(C)
    nvr = -(-m // vb)
    De, Dw = np.empty((nvr, n)), np.empty((nvr, n))
    for I in range(nvr):
        i0, i1 = I * vb, min(m, (I + 1) * vb)
        w = np.array([(t + 1) / 2.0 ** math.ceil(math.log2(vb)) for t in range(i1 - i0)])
        L = i1 - i0
        De[I] = (gamma(L) * aC[i0:i1].sum(0) + (gamma(k) + gamma(L)) * (aA[i0:i1].sum(0) @ aB)
                 + gamma(k) * (np.abs(enc.acs[2 * I]) @ aB)) * (1 + U)
        Dw[I] = (gamma(L) * (w[:, None] * aC[i0:i1]).sum(0)
                 + (gamma(k) + gamma(L)) * ((w[:, None] * aA[i0:i1]).sum(0) @ aB)
                 + gamma(k) * (np.abs(enc.acs[2 * I + 1]) @ aB)) * (1 + U)
    return De, Dw


def row_bounds(enc, C):
    """The transpose of col_bounds for the row lines (row i, column block J)."""
    A, B = enc.A, enc.B
    m, k = A.shape
    n = B.shape[1]
    vb = enc.cfg.vb_c
    aA, aB, aC = np.abs(A), np.abs(B), np.abs(C)
    nvc = -(-n // vb)
    De, Dw = np.empty((m, nvc)), np.empty((m, nvc))
    for J in range(nvc):
        j0, j1 = J * vb, min(n, (J + 1) * vb)
        w = np.array([(t + 1) / 2.0 ** math.ceil(math.log2(vb)) for t in range(j1 - j0)])
        L = j1 - j0
        De[:, J] = (gamma(L) * aC[:, j0:j1].sum(1) + (gamma(k) + gamma(L)) * (aA @ aB[:, j0:j1].sum(1))
                    + gamma(k) * (aA @ np.abs(enc.bcs[:, 2 * J]))) * (1 + U)
        Dw[:, J] = (gamma(L) * (aC[:, j0:j1] * w[None, :]).sum(1)
                    + (gamma(k) + gamma(L)) * (aA @ (aB[:, j0:j1] * w[None, :]).sum(1))
                    + gamma(k) * (aA @ np.abs(enc.bcs[:, 2 * J + 1]))) * (1 + U)
    return De, Dw


def operands(dist, seed, m, n, k):
    g = wl.rng(700 + seed)
    if dist == "normal":
        return g.standard_normal((m, k)), g.standard_normal((k, n))
    if dist == "uniform01":  # all positive: Cauchy-Schwarz is nearly tight
        return g.random((m, k)), g.random((k, n))
    # rows of very different magnitude (as in the FP8 recipe)
    sa = 10.0 ** g.uniform(-2, 2, (m, 1))
    sb = 10.0 ** g.uniform(-2, 2, (k, 1))
    return g.uniform(-1, 1, (m, k)) * sa, g.uniform(-1, 1, (k, n)) * sb


@pytest.mark.parametrize("dist", ["normal", "uniform01", "scaled_rows"])
@pytest.mark.parametrize("m,n,k,vbr,vbc", [(192, 160, 256, 64, 32), (96, 128, 512, 32, 64)])
def test_residuals_within_worst_case_and_threshold_below_it(dist, m, n, k, vbr, vbc):
    """Theorem: every fault-free residual lies inside its rigorous worst-case bound.
    Looseness: the threshold never exceeds that bound (measured: at most 0.2 of it for
    N(0, 1) and U[0, 1] data, 0.5 with rows of very different magnitude), and
    soundness: no fault-free residual reaches the threshold."""
    for seed in range(3):
        A, B = operands(dist, seed, m, n, k)
        enc = oracle.Encoded(A, B, vbr, vbc)
        C = oracle.gemm(A, B)
        re, rw, te, tw, nf = enc.col_residuals(C)
        De, Dw = col_bounds(enc, C)
        assert np.all(np.abs(re) <= De) and np.all(np.abs(rw) <= Dw)
        assert np.all(te <= De) and np.all(tw <= Dw)
        assert np.all(np.abs(re) < te) and np.all(np.abs(rw) < tw)
        re, rw, te, tw, nf = enc.row_residuals(C)
        De, Dw = row_bounds(enc, C)
        assert np.all(np.abs(re) <= De) and np.all(np.abs(rw) <= Dw)
        assert np.all(te <= De) and np.all(tw <= Dw)
        assert np.all(np.abs(re) < te) and np.all(np.abs(rw) < tw)


def test_worst_case_bound_catches_planted_errors():
    """The worst-case bound is not vacuous: an error of a few times the bound in one
    element of C breaks it on that element's lines (and only there)."""
    A, B = operands("normal", 9, 64, 64, 128)
    enc = oracle.Encoded(A, B, 16, 16)
    C = oracle.gemm(A, B)
    De, _ = col_bounds(enc, C)
    C[37, 11] += 3 * De[37 // 16, 11]
    re, rw, te, tw, nf = enc.col_residuals(C)
    out = np.argwhere(np.abs(re) > De)
    assert out.tolist() == [[37 // 16, 11]]


@pytest.mark.parametrize("m,n,k,vb", [(256, 256, 256, 64), (128, 192, 512, 32)])
def test_threshold_not_loose_for_gaussian_data(m, n, k, vb):
    """The rounding model predicts the fault-free residual of N(0, 1) data: the error of
    a recursive dot product of k terms is a random walk over partial sums of size
    sqrt(t), about u k / sqrt(6), and a line adds vb of them plus the checksum's
    product, so sigma_r ~ u k sqrt(vb / 3); the threshold is about
    s ||B_j|| (f1 + f2) sqrt(vb k) ~ 8 u k^(3/2) sqrt(vb), and the largest of the
    n * m / vb lines is about 3 sigma_r, so max |r| / tau ~ 3 / (8 sqrt(3 k)).  The pin
    asks for at least a quarter of that: a threshold more than about four times too
    loose fails, while the soundness pins above fail a threshold that is too tight."""
    pred = 3.0 / (8.0 * math.sqrt(3 * k))
    worst = []
    for seed in range(4):
        A, B = operands("normal", 20 + seed, m, n, k)
        enc = oracle.Encoded(A, B, vb, vb)
        C = oracle.gemm(A, B)
        re, rw, te, tw, _ = enc.col_residuals(C)
        worst.append(max(np.max(np.abs(re) / te), np.max(np.abs(rw) / tw)))
        re, rw, te, tw, _ = enc.row_residuals(C)
        worst.append(max(np.max(np.abs(re) / te), np.max(np.abs(rw) / tw)))
    assert min(worst) >= pred / 4, (min(worst), pred)
    assert max(worst) <= 4 * pred, (max(worst), pred)


# -------------------------------------------------------------------- carry bound
@pytest.mark.parametrize("dist", ["normal", "uniform01", "scaled_rows"])
def test_carry_bound_between_actual_deviation_and_worst_case(dist):
    """A carried checksum row E_I = fl((e^T A_I) B) differs from the exact sum of the
    stored rows of C = fl(A B) by d_I(j); the theorem bounds it by gamma_k of the
    checksum's product, gamma_vb of the encoding and gamma_k of the products of the
    block's elements.  The oracle's carried bound (section 3.2 reading) must cover the
    actual deviation and stay below the worst case."""
    m, n, k, vb = 128, 96, 384, 32
    for seed in range(3):
        A, B = operands(dist, 40 + seed, m, n, k)
        enc = oracle.Encoded(A, B, vb, vb)
        C = oracle.gemm(A, B)
        car = oracle.carry_rows(enc)
        aA, aB = np.abs(A), np.abs(B)
        for I in range(m // vb):
            i0, i1 = I * vb, (I + 1) * vb
            w = np.array([(t + 1) / 2.0 ** math.ceil(math.log2(vb)) for t in range(vb)])
            exact_e = np.array([math.fsum(C[i0:i1, j]) for j in range(n)])
            exact_w = np.array([math.fsum((w * C[i0:i1, j]).tolist()) for j in range(n)])
            d_e = np.abs(enc.E[2 * I] - exact_e)
            d_w = np.abs(enc.E[2 * I + 1] - exact_w)
            D_e = ((gamma(k) + gamma(vb)) * (aA[i0:i1].sum(0) @ aB)
                   + gamma(k) * (np.abs(enc.acs[2 * I]) @ aB)) * (1 + 2 * U)
            D_w = ((gamma(k) + gamma(vb)) * ((w[:, None] * aA[i0:i1]).sum(0) @ aB)
                   + gamma(k) * (np.abs(enc.acs[2 * I + 1]) @ aB)) * (1 + 2 * U)
            assert np.all(d_e <= D_e) and np.all(d_w <= D_w)
            assert d_e.max() <= car[2 * I] <= D_e.max()
            assert d_w.max() <= car[2 * I + 1] <= D_w.max()
        # the column side (carried row-checksum columns F) is the transpose
        carc = oracle.carry_cols(enc)
        for J in range(n // vb):
            j0, j1 = J * vb, (J + 1) * vb
            exact_e = np.array([math.fsum(C[i, j0:j1]) for i in range(m)])
            d_e = np.abs(enc.F[:, 2 * J] - exact_e)
            D_e = ((gamma(k) + gamma(vb)) * (aA @ aB[:, j0:j1].sum(1))
                   + gamma(k) * (aA @ np.abs(enc.bcs[:, 2 * J]))) * (1 + 2 * U)
            assert np.all(d_e <= D_e)
            assert d_e.max() <= carc[2 * J] <= D_e.max()
