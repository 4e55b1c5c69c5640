"""The tile schedules of the single-problem tensor-core product give the same results.

* regular: 128 x 256 tiles on one CTA, two alternating TMEM accumulators;
* tall: 256 x 256 tiles on one CTA, two M = 128 MMAs per K step (products without
  promotion only; the promoted and FP8 products fall back to regular tiles);
* pair: 256 x 256 tiles on a CTA pair (a cluster of two), one M = 256 MMA per K step
  (cta_group::2) reading 128 rows of A and 128 columns of B from each CTA's shared memory,
  each CTA holding its 128 rows of the accumulator in its own TMEM.

Each mode is forced with ABFT_PAIR_TILES / ABFT_TALL_TILES, for bf16, bf16x3, bf16x6 and
FP8 (native data tiles, block scales that vary along k, so several scale groups per tile),
on shapes whose tile rows and columns are ragged (pair tiles with no rows for the second
CTA, tiles with 1-3 B boxes, checksum tiles of a few rows).  Checks: C within the dtype's
product bound of the oracle's product; the checksum products E and F against the
oracle's; fault-free verify reports nothing; flips armed in the epilogue are located at
the oracle's positions with its kinds."""
import numpy as np
import pytest

import oracle
from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U32 = 2.0 ** -24

MODES = {
    "regular": {"ABFT_PAIR_TILES": "0", "ABFT_TALL_TILES": "0"},
    "tall": {"ABFT_PAIR_TILES": "0", "ABFT_TALL_TILES": "1"},
    "pair": {"ABFT_PAIR_TILES": "1", "ABFT_TALL_TILES": "0"},
}


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


@pytest.fixture(params=list(MODES))
def mode(request, monkeypatch):
    for k, v in MODES[request.param].items():
        monkeypatch.setenv(k, v)
    return request.param


def operands(dtype, m, n, k, seed):
    """(device A, device B, scales or {}, binary64 A, binary64 B) of the dtype."""
    if dtype == "fp8":
        A_src, B_src = wl.operands(wl.FP8_4096, seed, m, n, k)
        qa, sa = wl.quantize_e4m3(A_src)
        qb, sb = wl.quantize_e4m3(B_src)
        sa[:, ::2] *= 4.0   # scales that change along k: several scale groups per tile
        sb[1::3, :] *= 0.5
        A64, B64 = oracle.dequant_e4m3(qa, sa), oracle.dequant_e4m3(qb, sb)
        sc = dict(a_scale=torch.from_numpy(sa).cuda(), b_scale=torch.from_numpy(sb).cuda())
        return torch.from_numpy(qa).cuda(), torch.from_numpy(qb).cuda(), sc, A64, B64
    A = wl.operand((m, k), "normal", seed, 1).astype(np.float32)
    B = wl.operand((k, n), "normal", seed, 2).astype(np.float32)
    if dtype == "bf16":
        ba, bb = wl.bf16_bits(A), wl.bf16_bits(B)
        dA = torch.from_numpy(ba.view(np.int16)).view(torch.bfloat16).cuda()
        dB = torch.from_numpy(bb.view(np.int16)).view(torch.bfloat16).cuda()
        return dA, dB, {}, oracle.bf16_to_f64(ba), oracle.bf16_to_f64(bb)
    return (torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), {},
            A.astype(np.float64), B.astype(np.float64))


# elementwise bound of C (and of E, F with their extra representation error): the fp32
# accumulation's 2 k u32 plus what the split drops (bf16x3: A_lo B_lo and the hi+lo
# rounding; bf16x6: the three-piece rounding)
EXTRA = {"bf16": 0.0, "fp8": 0.0, "bf16x3": 2.0 ** -16, "bf16x6": 2.0 ** -25}
CS_EXTRA = {"bf16": 2.0 ** -17, "fp8": 2.0 ** -17, "bf16x3": 2.0 ** -16, "bf16x6": 2.0 ** -16}


def within(C, A, B, ref, extra):
    k = A.shape[1]
    bound = (2 * k * U32 + extra) * (np.abs(A) @ np.abs(B)) + 1e-30
    ok = np.abs(C - ref) <= bound
    assert ok.all(), (np.argwhere(~ok)[:5], np.max(np.abs(C - ref) / bound))


class Run:
    def __init__(self, dtype, m, n, k, vb_r, vb_c, seed):
        self.dtype, self.m, self.n, self.k = dtype, m, n, k
        self.A, self.B, self.sc, self.A64, self.B64 = operands(dtype, m, n, k, seed)
        self.desc = abft.make_desc(m, n, k, dtype, vb_r, vb_c)
        self.L = abft.abft_workspace_layout(self.desc)
        self.ws = torch.zeros(self.L.total, dtype=torch.uint8, device="cuda")
        self.C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        abft.abft_encode(self.desc, self.A, self.B, self.ws, **self.sc)
        abft.abft_gemm(self.desc, self.A, self.B, self.C, self.ws)
        torch.cuda.synchronize()

    def region(self, off, shape):
        nb = int(np.prod(shape)) * 8
        return self.ws[off:off + nb].view(torch.float64).reshape(shape).cpu().numpy()


def positions(rep):
    return sorted((e["row"], e["col"], e["kind"]) for e in rep if e["kind"] in (1, 2))


SHAPES = [  # (m, n, k, vb_r, vb_c)
    (256, 512, 256, 128, 128),     # whole pair tiles
    (600, 704, 384, 128, 128),     # last pair tile row 88 rows (no rows for the odd CTA)
    (130, 272, 256, 130, 136),     # one tile row: 128 + 2 rows; 272 = 4 + 1 boxes
    (384, 448, 1024, 128, 64),     # 1.5 pair tile rows, 3-box column tile, longer K
]


@pytest.mark.parametrize("dtype", ["bf16", "bf16x3", "bf16x6", "fp8"])
@pytest.mark.parametrize("shape", SHAPES)
def test_product_checksums_and_verify(dtype, shape, mode):
    m, n, k, vbr, vbc = shape
    r = Run(dtype, m, n, k, vbr, vbc, seed=m + n + k)
    enc = oracle.Encoded(r.A64, r.B64, vbr, vbc, dtype=dtype)
    C = r.C.cpu().numpy().astype(np.float64)
    assert np.isfinite(C).all()
    within(C, r.A64, r.B64, oracle.gemm(r.A64, r.B64), EXTRA[dtype])
    E = r.region(r.L.E, (r.L.R, n))
    F = r.region(r.L.F, (m, r.L.Cc))
    within(E, np.abs(enc.acs), r.B64, enc.E, CS_EXTRA[dtype] + 256 * U32)
    within(F, r.A64, np.abs(enc.bcs), enc.F, CS_EXTRA[dtype] + 256 * U32)
    for reread in (0, 1):
        st, rep, nrep = abft.abft_verify_correct(r.desc, r.C, r.ws, reread_C=reread)
        assert st == abft.OK and nrep == 0, (reread, rep)


@pytest.mark.parametrize("dtype", ["bf16", "bf16x6", "fp8"])
def test_flips_located_like_oracle(dtype, mode):
    """Three graded flips in distinct verify blocks, one of them in the odd CTA's rows of
    a pair tile, armed in the epilogue."""
    m, n, k = 640, 768, 512
    r = Run(dtype, m, n, k, 128, 128, seed=5)
    enc = oracle.Encoded(r.A64, r.B64, 128, 128, dtype=dtype)
    clean = r.C.cpu().numpy().astype(np.float64)
    pos = [(10, 700), (200, 3), (400, 300)]  # rows 200 and 400: a pair tile's second 128 rows
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


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_modes_agree_on_plain_product(dtype, monkeypatch):
    """The checksum-free product of the same operands under the three schedules, each within
    the product bound of the oracle's product (whether they are bit-identical is printed:
    the MMA shapes differ between the modes)."""
    m, n, k = 384, 512, 768
    out = {}
    for name, env in MODES.items():
        for kk, v in env.items():
            monkeypatch.setenv(kk, v)
        A, B, sc, A64, B64 = operands(dtype, m, n, k, 17)
        desc = abft.make_desc(m, n, k, dtype, 128, 128)
        ws = torch.zeros(abft.abft_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
        C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
        abft.abft_encode(desc, A, B, ws, **sc)
        abft.abft_gemm_plain(desc, A, B, C, ws=ws)
        torch.cuda.synchronize()
        out[name] = C.cpu().numpy().astype(np.float64)
    ref = oracle.gemm(A64, B64)
    for C in out.values():
        within(C, A64, B64, ref, 0.0)
    print(dtype, {nm: bool(np.array_equal(out["regular"], C)) for nm, C in out.items()})
