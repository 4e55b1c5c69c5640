"""Parity of the split bf16x3 path (binary32 inputs split into bf16 hi+lo planes, product
A_hi B_hi + A_hi B_lo + A_lo B_hi on the tensor cores, fp32 accumulation) with the CPU
oracle, through the C ABI.

The oracle works in binary64 on the exact binary32 inputs.  Values: elementwise
|C - C*| <= (2 k u32 + 2^-16)(|A||B|) -- fp32 accumulation plus the split's dropped A_lo B_lo
term and the hi+lo representation of the inputs.  Accuracy: the product promotes its tensor-core
accumulator into round-to-nearest fp32 registers every 4 k-steps, so the accumulation error is
small next to the split's own (inputs kept to ~16 significant bits, the A_lo B_lo term
dropped): the relative Frobenius error against binary64 stays below 2^-17 and at least 500x
below that of a plain bf16 product of the rounded inputs; the binary32 FMA GEMM (cuBLAS SGEMM,
TF32 off) error is printed for comparison.  The looser 4 sqrt(3k) u32 + 2^-17 scale bounds
the other cases."""
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


class Run:
    def __init__(self, m, n, k, vb_r, vb_c, p=0, q=0, seed=0, lda=None, ldb=None):
        self.m, self.n, self.k = m, n, k
        lda, ldb = lda or k, ldb or n
        A = np.zeros((m, lda), np.float32)
        B = np.zeros((k, ldb), np.float32)
        A[:, :k] = wl.operand((m, k), "normal", seed, 1)
        B[:, :n] = wl.operand((k, n), "normal", seed, 2)
        self.A64, self.B64 = A[:, :k].astype(np.float64), B[:, :n].astype(np.float64)
        self.A, self.B = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        self.desc = abft.make_desc(m, n, k, "bf16x3", vb_r, vb_c, p, q, lda=lda, ldb=ldb)
        self.L = abft.abft_workspace_layout(self.desc)
        self.ws = torch.zeros(self.L.total, dtype=torch.uint8, device="cuda")
        self.C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        abft.abft_encode(self.desc, self.A, self.B, self.ws)
        abft.abft_gemm(self.desc, self.A, self.B, self.C, self.ws)
        torch.cuda.synchronize()

    def region(self, off, shape):
        nb = int(np.prod(shape)) * 8
        return self.ws[off:off + nb].view(torch.float64).reshape(shape).cpu().numpy()


def rel_fro(x, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def x3_tol(k):
    """Relative Frobenius scale of the split product: fp32 accumulation of 3k products on
    the tensor cores plus the split's 2^-17."""
    return 4 * np.sqrt(3 * k) * U32 + 2.0 ** -17


def check_x3(C, A, B, ref, extra=0.0):
    k = A.shape[1]
    bound = (2 * k * U32 + 2.0 ** -16 + extra) * (np.abs(A) @ np.abs(B)) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)


@pytest.mark.parametrize("shape", [(256, 256, 128, 128, 128, 0, 0), (200, 300, 136, 40, 30, 0, 0),
                                   (384, 512, 520, 128, 64, 3, 4), (130, 264, 72, 130, 88, 0, 0)])
def test_x3_product_and_checksums_vs_oracle(shape):
    m, n, k, vbr, vbc, p, q = shape
    r = Run(m, n, k, vbr, vbc, p, q, seed=3)
    enc = oracle.Encoded(r.A64, r.B64, vbr, vbc, p, q, dtype="bf16x3")
    check_x3(r.C.cpu().numpy().astype(np.float64), r.A64, r.B64, oracle.gemm(r.A64, r.B64))
    E = r.region(r.L.E, (r.L.R, n))
    F = r.region(r.L.F, (m, r.L.Cc))
    check_x3(E, np.abs(enc.acs), r.B64, enc.E, extra=2.0 ** -16 + 256 * U32)
    check_x3(F, r.A64, np.abs(enc.bcs), enc.F, extra=2.0 ** -16 + 256 * U32)
    for off, ref in ((r.L.nArow, enc.nArow), (r.L.nAblk, enc.nAblk), (r.L.nBcol, enc.nBcol),
                     (r.L.nBblk, enc.nBblk)):
        assert np.allclose(r.region(off, ref.shape), ref, rtol=1e-5)


def test_x3_accuracy_fp32_level():
    """Split bf16x3 recovers binary32-level accuracy against binary64."""
    m = n = 1024
    k = 4096
    r = Run(m, n, k, 128, 128, seed=5)
    ref = oracle.gemm(r.A64, r.B64)
    e_x3 = rel_fro(r.C.cpu().numpy().astype(np.float64), ref)
    torch.backends.cuda.matmul.allow_tf32 = False
    c32 = torch.matmul(r.A, r.B).cpu().numpy().astype(np.float64)
    e_32 = rel_fro(c32, ref)
    cb = torch.matmul(r.A.to(torch.bfloat16), r.B.to(torch.bfloat16)).float().cpu().numpy()
    e_bf = rel_fro(cb.astype(np.float64), ref)
    print(f"rel Frobenius error vs binary64: bf16x3 {e_x3:.2e}, fp32 SGEMM {e_32:.2e}, "
          f"bf16 {e_bf:.2e}")
    assert e_x3 <= 2.0 ** -17 and e_x3 * 500 < e_bf


@pytest.mark.parametrize("seed", range(3))
def test_x3_fault_free_and_flips(seed):
    m, n, k = 512, 768, 1024
    r = Run(m, n, k, 128, 256, 4, 3, seed=seed)
    enc = oracle.Encoded(r.A64, r.B64, 128, 256, 4, 3, dtype="bf16x3")
    for reread in (0, 1):
        st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=reread)
        assert st == abft.OK and nrep == 0
    C_clean = r.C.cpu().numpy().astype(np.float64)
    pos = [(p_[0], p_[1]) for p_ in wl.bit_flips(seed, m, n, 3, bits=32,
                                                 distinct_blocks=(128, 256))]
    flips = [(i, j, 29 if abs(C_clean[i, j]) >= 2.0 else 30) for i, j in pos]
    abft.abft_set_epilogue_faults(r.desc, r.ws, flips)
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    abft.abft_set_epilogue_faults(r.desc, r.ws, [])
    Cf = r.C.cpu().numpy().astype(np.float64)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    ost, orep, oC, on = enc.verify_correct(np.nan_to_num(Cf, nan=np.nan))
    key = lambda rr: sorted((e["row"], e["col"], e["kind"]) for e in rr if e["kind"] in (1, 2))
    assert st == abft.OK and ost == oracle.ST_OK
    assert [(a, b) for a, b, _ in key(rep)] == sorted(pos) and key(rep) == key(orep)
    assert rel_fro(r.C.cpu().numpy().astype(np.float64), oracle.gemm(r.A64, r.B64)) <= x3_tol(k)


def test_x3_erasure_rebuild():
    m = n = 512
    k = 256
    r = Run(m, n, k, 128, 128, 4, 4, seed=9)
    abft.abft_erase_block(r.desc, r.C, 1, 3)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, erased=[(1, 3)])
    assert st == abft.OK and nrep == 0
    st, ent = abft.abft_recover_block(r.desc, r.C, r.ws, 1, 3)
    assert st == abft.OK
    ref = oracle.gemm(r.A64, r.B64)
    blk = np.s_[128:256, 384:512]
    # the rebuilt block carries the errors of S and of the p - 1 other blocks
    assert rel_fro(r.C.cpu().numpy().astype(np.float64)[blk], ref[blk]) <= np.sqrt(5) * x3_tol(k)


def test_x3_plain_equals_abft_data_block():
    r = Run(256, 512, 192, 128, 128, seed=11)
    C2 = torch.empty_like(r.C)
    abft.abft_gemm_plain(r.desc, r.A, r.B, C2, ws=r.ws)
    torch.cuda.synchronize()
    assert torch.equal(C2, r.C)
