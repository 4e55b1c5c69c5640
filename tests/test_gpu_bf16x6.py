"""Parity of the split bf16x6 path (binary32 inputs split into three bf16 planes,
x = p0 + p1 + p2 with 24 significant bits; the six products p_a q_b with a + b <= 2 on the
tensor cores; the accumulator promoted into round-to-nearest fp32 registers every 8 k-steps)
with the CPU oracle, through the C ABI.

The oracle works in binary64 on the exact binary32 inputs.  Values: elementwise
|C - C*| <= (2 k u32 + 2^-25)(|A||B|) (fp32 accumulation plus the dropped products and the
pieces' residual).  Accuracy (the bar for "FP32-level"): the relative Frobenius error
against binary64 is at most 4x that of the binary32 FMA GEMM (cuBLAS SGEMM, TF32 off) on the
same inputs, at k = 4096 and k = 16384.  Decisions: bit-exact fault positions and kinds."""
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
    def __init__(self, m, n, k, vb_r, vb_c, p=0, q=0, seed=0):
        self.m, self.n, self.k = m, n, k
        A = wl.operand((m, k), "normal", seed, 1).astype(np.float32)
        B = wl.operand((k, n), "normal", seed, 2).astype(np.float32)
        self.A64, self.B64 = A.astype(np.float64), B.astype(np.float64)
        self.A, self.B = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        self.desc = abft.make_desc(m, n, k, "bf16x6", vb_r, vb_c, p, q)
        self.L = abft.abft_workspace_layout(self.desc)
        assert self.L.planes == 3
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


def check_x6(C, A, B, ref, extra=0.0):
    k = A.shape[1]
    bound = (2 * k * U32 + 2.0 ** -25 + extra) * (np.abs(A) @ np.abs(B)) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)


@pytest.mark.parametrize("shape", [(256, 256, 128, 128, 128, 0, 0), (200, 300, 136, 40, 30, 0, 0),
                                   (384, 512, 520, 128, 64, 3, 4)])
def test_x6_product_and_checksums_vs_oracle(shape):
    m, n, k, vbr, vbc, p, q = shape
    r = Run(m, n, k, vbr, vbc, p, q, seed=4)
    enc = oracle.Encoded(r.A64, r.B64, vbr, vbc, p, q, dtype="bf16x6")
    check_x6(r.C.cpu().numpy().astype(np.float64), r.A64, r.B64, oracle.gemm(r.A64, r.B64))
    E = r.region(r.L.E, (r.L.R, n))
    F = r.region(r.L.F, (m, r.L.Cc))
    check_x6(E, np.abs(enc.acs), r.B64, enc.E, extra=2.0 ** -25 + 256 * U32)
    check_x6(F, r.A64, np.abs(enc.bcs), enc.F, extra=2.0 ** -25 + 256 * U32)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=1)
    assert st == abft.OK and nrep == 0


@pytest.mark.parametrize("m,k", [(1024, 4096), (512, 16384)])
def test_x6_accuracy_within_4x_sgemm(m, k):
    """FP32-level accuracy (G7): within 4x the binary32 FMA GEMM's error against binary64."""
    r = Run(m, m, k, 128, 128, seed=6)
    ref = oracle.gemm(r.A64, r.B64)
    e_x6 = rel_fro(r.C.cpu().numpy().astype(np.float64), ref)
    torch.backends.cuda.matmul.allow_tf32 = False
    e_32 = rel_fro(torch.matmul(r.A, r.B).cpu().numpy().astype(np.float64), ref)
    print(f"k={k}: rel Frobenius error vs binary64: bf16x6 {e_x6:.2e}, fp32 SGEMM {e_32:.2e}")
    assert e_x6 <= 4 * e_32


def test_x6_faults_located_like_oracle():
    m, n, k = 512, 768, 1024
    r = Run(m, n, k, 128, 256, 4, 3, seed=2)
    enc = oracle.Encoded(r.A64, r.B64, 128, 256, 4, 3, dtype="bf16x6")
    for reread in (0, 1):
        st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=reread)
        assert st == abft.OK and nrep == 0
    C_clean = r.C.cpu().numpy().astype(np.float64)
    pos = [(p_[0], p_[1]) for p_ in wl.bit_flips(2, m, n, 3, bits=32,
                                                 distinct_blocks=(128, 256))]
    flips = [(i, j, 29 if abs(C_clean[i, j]) >= 2.0 else 30) for i, j in pos]
    abft.abft_set_epilogue_faults(r.desc, r.ws, flips)
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    abft.abft_set_epilogue_faults(r.desc, r.ws, [])
    Cf = r.C.cpu().numpy().astype(np.float64)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    ost, orep, oC, on = enc.verify_correct(Cf)
    key = lambda rr: sorted((e["row"], e["col"], e["kind"]) for e in rr if e["kind"] in (1, 2))
    assert st == abft.OK and ost == oracle.ST_OK
    assert [(a, b) for a, b, _ in key(rep)] == sorted(pos) and key(rep) == key(orep)


def test_x6_erasure_rebuild():
    m = n = 512
    k = 256
    r = Run(m, n, k, 128, 128, 4, 4, seed=9)
    ref = oracle.gemm(r.A64, r.B64)
    abft.abft_erase_block(r.desc, r.C, 2, 0)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, erased=[(2, 0)])
    assert st == abft.OK and nrep == 0
    st, ent = abft.abft_recover_block(r.desc, r.C, r.ws, 2, 0)
    assert st == abft.OK
    blk = np.s_[256:384, 0:128]
    Cg = r.C.cpu().numpy().astype(np.float64)
    # the rebuilt block carries the errors of S and of the p - 1 other blocks
    assert rel_fro(Cg[blk], ref[blk]) <= np.sqrt(5) * (4 * np.sqrt(k) * U32 + 2.0 ** -25)
