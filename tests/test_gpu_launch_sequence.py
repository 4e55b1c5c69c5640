"""Consecutive products of the same kernel with different operands and outputs, all
buffers alive at once (so no address is reused): every product writes its own C and its
own checksums.  The tensor maps travel with each launch as kernel parameters; this guards
against a launch using an earlier launch's maps, which wrote C into the earlier output."""
import dataclasses

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


def product(w, seed, m, n, k):
    A, B, sa, sb = wl.device_operands(dataclasses.replace(w, m=m, n=n, k=k), seed, "cuda")
    scales = dict(a_scale=sa, b_scale=sb) if sa is not None else {}
    desc = abft.make_desc(m, n, k, w.dtype, 256, 256)
    ws = torch.zeros(abft.abft_workspace_bytes(desc), dtype=torch.uint8, device="cuda")
    C = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    abft.abft_encode(desc, A, B, ws, **scales)
    abft.abft_gemm(desc, A, B, C, ws)
    return dict(A=A, B=B, sa=sa, sb=sb, ws=ws, C=C, desc=desc)


@pytest.mark.parametrize("names", [("bf16x3_16384", "bf16x6_16384", "fp8_16384", "bf16_16384"),
                                   ("fp8_16384", "fp8_16384", "bf16x6_16384", "bf16x6_16384")])
def test_consecutive_products_write_their_own_outputs(names):
    m, n, k = 1024, 1536, 1024
    runs = [product(wl.WORKLOADS[nm], 30 + t, m, n, k) for t, nm in enumerate(names)]
    torch.cuda.synchronize()
    for nm, r in zip(names, runs):
        C = r["C"].cpu().numpy().astype(np.float64)
        assert np.isfinite(C).all(), nm  # every element written
        st, rep, nrep = abft.abft_verify_correct(r["desc"], r["C"], r["ws"], reread_C=1)
        assert st == abft.OK and nrep == 0, (nm, rep)
        # a sample of rows against the binary64 product of the operands' values
        w = wl.WORKLOADS[nm]
        g = wl.rng(7, 3)
        rows = np.sort(g.choice(m, 8, replace=False))
        if w.dtype == "fp8":
            A64 = oracle.dequant_e4m3(r["A"].cpu().numpy(), r["sa"].cpu().numpy())
            B64 = oracle.dequant_e4m3(r["B"].cpu().numpy(), r["sb"].cpu().numpy())
        elif w.dtype == "bf16":
            A64 = oracle.bf16_to_f64(r["A"].cpu().view(torch.int16).numpy().view(np.uint16))
            B64 = oracle.bf16_to_f64(r["B"].cpu().view(torch.int16).numpy().view(np.uint16))
        else:
            A64 = r["A"].cpu().numpy().astype(np.float64)
            B64 = r["B"].cpu().numpy().astype(np.float64)
        ref = A64[rows] @ B64
        mag = np.abs(A64[rows]) @ np.abs(B64)
        extra = {"bf16x3": 2.0 ** -16, "bf16x6": 2.0 ** -25}.get(w.dtype, 0.0)
        assert np.all(np.abs(C[rows] - ref) <= (2 * k * U32 + extra) * mag + 1e-30), nm
