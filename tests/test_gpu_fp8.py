"""Parity of the FP8 E4M3 path (e4m3 operands with one power-of-two binary32 scale per
128 x 128 block) with the CPU oracle, through the C ABI.

The oracle dequantises the same codes and scales in binary64 (e4m3 decoding pinned in
test_oracle) and runs the same checks as for bf16.  The GPU's data tiles multiply the e4m3
codes on the 8-bit tensor path (kind::f8f6f4), one TMEM accumulator per run of k-steps with
the same block-scale product, each scaled exactly by that power of two in the epilogue
("native"), or the dequantised values (exact in bf16 for power-of-two scales) on the bf16
path ("planes", ABFT_FP8_NATIVE=0); the checksum tiles always use the bf16 planes.  Either
way the products are exact and accumulate in fp32, so the product bound is the bf16 one,
elementwise 2 k u32 (|A||B|) and relative Frobenius 4 sqrt(k) u32, against the oracle's
product of the dequantised operands.  The quantisation error against the binary64
product of the unquantised inputs is stated (printed) and bounded loosely.  Decisions:
bit-exact fault positions and kinds."""
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


@pytest.fixture(params=["native", "planes"])
def mode(request, monkeypatch):
    """Data tiles on the e4m3 codes (native) or on the dequantised bf16 planes."""
    monkeypatch.setenv("ABFT_FP8_NATIVE", "1" if request.param == "native" else "0")
    return request.param


def rel_fro(x, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (den if den > 0 else 1.0)


def check_fp32_product(C, A, B, ref, extra_rel=0.0):
    k = A.shape[1]
    mag = np.abs(A) @ np.abs(B)
    bound = (2 * k * U32 + extra_rel) * mag + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    assert rel_fro(C, ref) <= 4 * np.sqrt(max(k, 1)) * U32 + 4 * extra_rel


def positions(rep):
    return sorted((e["row"], e["col"], e["kind"]) for e in rep if e["kind"] in (1, 2))


class Run:
    def __init__(self, m, n, k, vb_r, vb_c, p=0, q=0, seed=0, scale_fix=None, scale_fix_b=None):
        self.m, self.n, self.k = m, n, k
        self.A_src, self.B_src = wl.operands(wl.FP8_4096, seed, m, n, k)
        qa, sa = wl.quantize_e4m3(self.A_src)
        qb, sb = wl.quantize_e4m3(self.B_src)
        if scale_fix:
            scale_fix(sa)
        if scale_fix_b:
            scale_fix_b(sb)
        self.A64, self.B64 = oracle.dequant_e4m3(qa, sa), oracle.dequant_e4m3(qb, sb)
        self.A = torch.from_numpy(qa).cuda()
        self.B = torch.from_numpy(qb).cuda()
        self.sA = torch.from_numpy(sa).cuda()
        self.sB = torch.from_numpy(sb).cuda()
        self.desc = abft.make_desc(m, n, k, "fp8", vb_r, vb_c, p, q)
        self.L = abft.abft_workspace_layout(self.desc)
        self.C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        self.ws = torch.zeros(self.L.total, dtype=torch.uint8, device="cuda")
        abft.abft_encode(self.desc, self.A, self.B, self.ws, a_scale=self.sA, b_scale=self.sB)
        abft.abft_gemm(self.desc, self.A, self.B, self.C, self.ws)
        torch.cuda.synchronize()

    def region(self, off, shape, dtype=torch.float64):
        nb = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
        return self.ws[off:off + nb].view(dtype).reshape(shape).cpu().numpy()


SHAPES = [  # (m, n, k, vb_r, vb_c, p, q)
    (256, 512, 256, 128, 128, 0, 0),
    (384, 256, 200, 128, 64, 3, 2),
    (200, 300, 136, 40, 30, 0, 0),
    (640, 700, 520, 128, 256, 0, 0),
    (256, 264, 250, 128, 64, 0, 0),   # rows of A not 8-byte aligned: separate dequantisation
    # 16-byte aligned rows (native data tiles) with ragged m, n and k
    (200, 272, 144, 40, 136, 0, 0),
    (640, 704, 528, 128, 256, 0, 0),
    (384, 512, 1040, 128, 128, 3, 4),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_fp8_product_and_checksums_vs_oracle(shape, mode):
    m, n, k, vbr, vbc, p, q = shape
    r = Run(m, n, k, vbr, vbc, p, q, seed=3)
    enc = oracle.Encoded(r.A64, r.B64, vbr, vbc, p, q, dtype="fp8")
    C = r.C.cpu().numpy()
    ref = oracle.gemm(r.A64, r.B64)
    check_fp32_product(C, r.A64, r.B64, ref)
    E = r.region(r.L.E, (r.L.R, n))
    F = r.region(r.L.F, (m, r.L.Cc))
    check_fp32_product(E, np.abs(enc.acs), r.B64, enc.E, extra_rel=2.0 ** -17 + 256 * U32)
    check_fp32_product(F, r.A64, np.abs(enc.bcs), enc.F, extra_rel=2.0 ** -17 + 256 * U32)
    # the stated error of the FP8 product against the unquantised binary64 product
    err = rel_fro(C, oracle.gemm(r.A_src, r.B_src))
    print(f"fp8 {m}x{n}x{k}: rel Frobenius vs dequantised oracle {rel_fro(C, ref):.3e}, "
          f"vs unquantised binary64 {err:.3e}")
    assert err < 0.1
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=1)
    assert st == abft.OK and nrep == 0


@pytest.mark.parametrize("seed", [11] + list(range(10)))
def test_fp8_five_seeded_faults_located_like_oracle(mode, seed):
    """Five accumulator-output flips (graded exponent bits) in distinct verify blocks, armed
    in the epilogue: located from the fused sums at the oracle's positions and corrected
    (operands and positions of seeds 0..9, and 11)."""
    m, n, k = 1024, 1024, 512
    r = Run(m, n, k, 256, 256, seed=seed)
    assert r.L.fused == 1
    enc = oracle.Encoded(r.A64, r.B64, 256, 256, dtype="fp8")
    clean = r.C.cpu().numpy().astype(np.float64)
    pos = [(i, j) for i, j, _ in wl.bit_flips(seed, m, n, 5, bits=32, distinct_blocks=(256, 256))]
    flips = [(i, j, 29 if abs(clean[i, j]) >= 2.0 else 30) for i, j in pos]
    abft.abft_set_epilogue_faults(r.desc, r.ws, flips)
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    abft.abft_set_epilogue_faults(r.desc, r.ws, [])
    Cf = r.C.cpu().numpy().astype(np.float64)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    ost, orep, oC, on = enc.verify_correct(Cf)
    assert st == abft.OK and ost == oracle.ST_OK
    assert [(a, b) for a, b, _ in positions(rep)] == sorted(pos)
    assert positions(rep) == positions(orep)
    Cg = r.C.cpu().numpy().astype(np.float64)
    assert rel_fro(Cg, oracle.gemm(r.A64, r.B64)) <= 4 * np.sqrt(k) * U32 + 1e-7


def test_fp8_fault_free_runs_report_nothing(mode):
    for seed in range(4):
        r = Run(512, 384, 640, 128, 128, seed=100 + seed)
        for reread in (0, 1):
            st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=reread)
            assert st == abft.OK and nrep == 0


def test_fp8_plain_product_matches(mode):
    r = Run(384, 512, 256, 128, 128, seed=5)
    C2 = torch.full_like(r.C, float("nan"))
    abft.abft_gemm_plain(r.desc, r.A, r.B, C2, ws=r.ws)
    torch.cuda.synchronize()
    check_fp32_product(C2.cpu().numpy(), r.A64, r.B64, oracle.gemm(r.A64, r.B64))


def test_fp8_non_power_of_two_scale_is_rejected():
    """A block scale that is not a power of two (so the dequantised values need not be
    exact in bf16) is rejected: the next verify reports ABFT_ERR_INVALID, and a correct call
    afterwards succeeds."""
    def bad(sa):
        sa[0, 0] *= 1.1
    r = Run(256, 256, 256, 128, 128, seed=7, scale_fix=bad)
    with pytest.raises(abft.AbftError) as e:
        abft.abft_verify_correct(r.desc, r.C, r.ws)
    assert e.value.status == abft.ERR_INVALID and "power" in str(e.value)
    r2 = Run(256, 256, 256, 128, 128, seed=7)
    st, rep, nrep = abft.abft_verify_correct(r2.desc, r2.C, r2.ws)
    assert st == abft.OK and nrep == 0


def test_fp8_varying_block_scales_several_scale_groups(mode):
    """Block scales that change along k (powers of two times the recipe's: A's scales x4
    on every second k-block, B's x1/2 on every third) split each native data tile's K loop
    into several scale groups, each accumulated in its own TMEM accumulator and scaled in
    the epilogue: the product and the checks still match the oracle, with one graded
    fault located."""
    def fa(sa):
        sa[:, ::2] *= 4.0

    def fb(sb):
        sb[1::3, :] *= 0.5
    m, n, k = 512, 768, 1280
    r = Run(m, n, k, 256, 256, seed=21, scale_fix=fa, scale_fix_b=fb)
    ref = oracle.gemm(r.A64, r.B64)
    C = r.C.cpu().numpy()
    check_fp32_product(C, r.A64, r.B64, ref)
    enc = oracle.Encoded(r.A64, r.B64, 256, 256, dtype="fp8")
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=1)
    assert st == abft.OK and nrep == 0
    i, j = 300, 517
    flips = [(i, j, 29 if abs(C[i, j]) >= 2.0 else 30)]
    abft.abft_set_epilogue_faults(r.desc, r.ws, flips)
    abft.abft_gemm(r.desc, r.A, r.B, r.C, r.ws)
    abft.abft_set_epilogue_faults(r.desc, r.ws, [])
    Cf = r.C.cpu().numpy().astype(np.float64)
    st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=0)
    ost, orep, oC, on = enc.verify_correct(Cf)
    assert st == abft.OK and positions(rep) == positions(orep) == [(i, j, abft.KIND_CORRECTED)]
    check_fp32_product(r.C.cpu().numpy().astype(np.float64), r.A64, r.B64, ref)


def test_fp8_native_and_planes_agree():
    """The same codes through both data-tile paths: both within the product bound of the
    oracle's product, and within twice that bound of each other."""
    import os
    out = {}
    for mode_ in ("1", "0"):
        os.environ["ABFT_FP8_NATIVE"] = mode_
        try:
            r = Run(512, 512, 2048, 128, 128, seed=9)
        finally:
            del os.environ["ABFT_FP8_NATIVE"]
        out[mode_] = r.C.cpu().numpy().astype(np.float64)
    ref = oracle.gemm(r.A64, r.B64)
    for C in out.values():
        check_fp32_product(C, r.A64, r.B64, ref)
    mag = np.abs(r.A64) @ np.abs(r.B64)
    assert np.all(np.abs(out["1"] - out["0"]) <= 4 * 2048 * U32 * mag + 1e-30)
