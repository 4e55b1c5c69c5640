"""The tensor-core workloads at their full size (16384^3) in the benchmark's launch
configuration: operands drawn on the device by the benchmark's generator, verify blocks of
256, compute faults armed as accumulator-output flips in the product's epilogue and located
from the fused observed sums (no re-read of C).

What the oracle can compute one by one is compared element by element: a 32 x 32 sample of
C, the expected checksums of 32 sampled columns (rows) against the oracle's encoding times
those columns of B (rows of A), the threshold norms of every line; decisions are compared
exactly (every armed flip located at its position, nothing else reported), and every flip
is graded by the oracle's classification of the GPU's error."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24
# per dtype: extra relative error of the product (split residual) and of the checksum
# operand (bf16 pieces of the binary32 sums)
EXTRA = {"fp8": (0.0, 2.0 ** -17), "bf16x3": (2.0 ** -16, 2.0 ** -16),
         "bf16x6": (2.0 ** -25, 2.0 ** -25)}


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


def host_f64(w, X, scale):
    """Binary64 values of a device operand: dequantised codes (fp8) or binary32 values."""
    if w.dtype == "fp8":
        return oracle.dequant_e4m3(X.cpu().numpy(), scale.cpu().numpy())
    return X.cpu().numpy().astype(np.float64)


def within(val, ref, mag, rel):
    bound = rel * mag + 1e-30
    assert np.all(np.abs(val - ref) <= bound), np.max(np.abs(val - ref) / bound)


def region(ws, off, shape):
    nb = int(np.prod(shape)) * 8
    return ws[off:off + nb].view(torch.float64).reshape(shape).cpu().numpy()


@pytest.mark.parametrize("w", [wl.FP8_16384, wl.BF16X3_16384, wl.BF16X6_16384],
                         ids=lambda w: w.name)
def test_full_size_sampled(w):
    m, n, k, vbr, vbc = w.m, w.n, w.k, w.vb_r, w.vb_c
    A, B, sa, sb = wl.device_operands(w, 0, "cuda")
    scales = dict(a_scale=sa, b_scale=sb) if sa is not None else {}
    desc = abft.make_desc(m, n, k, w.dtype, vbr, vbc)
    L = abft.abft_workspace_layout(desc)
    assert L.fused == 1
    ws = torch.zeros(L.total, dtype=torch.uint8, device="cuda")
    C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    abft.abft_encode(desc, A, B, ws, **scales)
    abft.abft_gemm(desc, A, B, C, ws)
    torch.cuda.synchronize()
    for reread in (0, 1):
        st, rep, nrep = abft.abft_verify_correct(desc, C, ws, reread_C=reread)
        assert st == abft.OK and nrep == 0
    A64, B64 = host_f64(w, A, sa), host_f64(w, B, sb)
    ex_c, ex_cs = EXTRA[w.dtype]
    g = wl.rng(0, 98)
    rows = np.sort(g.choice(m, 32, replace=False))
    cols = np.sort(g.choice(n, 32, replace=False))
    # products
    clean = C.cpu().numpy().astype(np.float64)
    Ar, Bc = A64[rows], B64[:, cols]
    within(clean[np.ix_(rows, cols)], Ar @ Bc, np.abs(Ar) @ np.abs(Bc), 2 * k * U32 + ex_c)
    # expected checksums: the oracle's encoding (sums in binary64) times sampled columns /
    # rows; the GPU's sums run in binary32 over a verify block (vb u32 of the magnitudes)
    acs, acs_mag = oracle.encode_A(A64, vbr), oracle.encode_A(np.abs(A64), vbr)
    E = region(ws, L.E, (L.R, n))[:, cols]
    within(E, acs @ Bc, acs_mag @ np.abs(Bc), 2 * k * U32 + vbr * U32 + ex_cs + ex_c)
    bcs, bcs_mag = oracle.encode_B(B64, vbc), oracle.encode_B(np.abs(B64), vbc)
    F = region(ws, L.F, (m, L.Cc))[rows]
    within(F, Ar @ bcs, np.abs(Ar) @ bcs_mag, 2 * k * U32 + vbc * U32 + ex_cs + ex_c)
    # threshold norms of every line and verify block (binary32 partial sums)
    enc = oracle.Encoded(A64, B64, vbr, vbc, dtype=w.dtype, products=False)
    for off, ref in ((L.nArow, enc.nArow), (L.nAblk, enc.nAblk), (L.nBcol, enc.nBcol),
                     (L.nBblk, enc.nBblk)):
        assert np.allclose(region(ws, off, ref.shape), ref, rtol=1e-5, atol=0)
    # compute faults: the benchmark's flips, armed in the epilogue
    pos = [(i, j) for i, j, _ in wl.bit_flips(0, m, n, w.n_flips, distinct_blocks=(512, 512))]
    flips = [(i, j, 29 if abs(clean[i, j]) >= 2.0 else 30) for i, j in pos]
    abft.abft_set_epilogue_faults(desc, ws, flips)
    abft.abft_gemm(desc, A, B, C, ws)
    abft.abft_set_epilogue_faults(desc, ws, [])
    torch.cuda.synchronize()
    bad = np.array([C[i, j].item() for i, j in pos], np.float64)
    with np.errstate(invalid="ignore"):
        for (i, j), v in zip(pos, bad):
            assert enc.classify(i, j, v - clean[i, j]) == "graded"
    st, rep, nrep = abft.abft_verify_correct(desc, C, ws, reread_C=0)
    assert st == abft.OK and nrep == len(pos)
    found = sorted((e["row"], e["col"]) for e in rep
                   if e["kind"] in (abft.KIND_CORRECTED, abft.KIND_NONFINITE_CORRECTED))
    assert found == sorted(pos)
    # corrected by recomputation from the checksums: within the line's threshold
    for i, j in pos:
        te_c, tw_c, te_r, tw_r = enc.thresholds_at(i, j)
        assert abs(C[i, j].item() - clean[i, j]) <= max(te_c, te_r) + 4 * U32 * abs(clean[i, j])
    # every other element is the clean product, bit for bit
    fixed = C.cpu().numpy().astype(np.float64)
    idx = tuple(np.array(pos).T)
    fixed[idx] = clean[idx]
    assert np.array_equal(fixed, clean)
