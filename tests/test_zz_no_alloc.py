"""abft_encode_noalloc: the encode for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (code running during CUDA graph capture, real-time or
signal-context threads, plugins that only receive buffers from their host application).
This entry point keeps the encode's partial sums in static device memory inside the
library, so the caller's workspace only has to hold the outputs.  Its outputs must equal
those of abft_encode, on consecutive calls (the static array keeps the previous call's
contents), and a problem too large for the static array must be refused before any work
is launched.  This file is collected last on purpose."""
import ctypes as ct

import numpy as np
import pytest

from paper_0806_3121_gb300 import abft, workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_3121_gb300 import build
    build.build()
    return abft.load()


def outputs(ws, L, m, n, k):
    """acs, bcs and the four norm arrays written by the encode, as numpy arrays."""
    def region(off, count):
        return ws[off:off + 8 * count].view(torch.float64).cpu().numpy()
    return [region(L.acs, L.R * k), region(L.bcs, k * L.Cc), region(L.nArow, m),
            region(L.nAblk, 4 * L.nvr), region(L.nBcol, n), region(L.nBblk, 4 * L.nvc)]


def test_noalloc_encode_matches_encode_on_consecutive_calls():
    m, n, k = 768, 640, 1000  # several verify blocks, ragged chunks along k
    desc = abft.make_desc(m, n, k, "f64", 128, 128, 6, 5)
    L = abft.abft_workspace_layout(desc)
    ws_full = torch.zeros(L.total, dtype=torch.uint8, device="cuda")
    # the no-alloc variant only needs the output part of the workspace; fill it with
    # garbage so that stale contents would show
    ws_out = torch.full((L.scratch,), 0xA5, dtype=torch.uint8, device="cuda")
    for seed in (11, 12):
        A = torch.from_numpy(wl.operand((m, k), "normal", seed, 1)).cuda()
        B = torch.from_numpy(wl.operand((k, n), "uniform", seed, 2)).cuda()
        abft.abft_encode(desc, A, B, ws_full)
        abft.abft_encode_noalloc(desc, A, B, ws_out)
        torch.cuda.synchronize()
        ref = outputs(ws_full, L, m, n, k)
        got = outputs(ws_out, L, m, n, k)
        for r, g in zip(ref, got):
            assert np.allclose(g, r, rtol=1e-12, atol=0.0)
            assert np.array_equal(g, r)  # same kernels, same summation order


def test_noalloc_encode_then_product_and_verify():
    """The outputs feed the rest of the path exactly like abft_encode's."""
    m = n = k = 256
    desc = abft.make_desc(m, n, k, "f64", 64, 64)
    L = abft.abft_workspace_layout(desc)
    ws = torch.zeros(L.total, dtype=torch.uint8, device="cuda")
    A = torch.from_numpy(wl.operand((m, k), "normal", 13, 1)).cuda()
    B = torch.from_numpy(wl.operand((k, n), "normal", 13, 2)).cuda()
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    abft.abft_encode_noalloc(desc, A, B, ws)
    abft.abft_gemm(desc, A, B, C, ws)
    abft.abft_inject_bitflips(desc, C, [(100, 7, 62)])
    st, rep, nrep = abft.abft_verify_correct(desc, C, ws)
    assert st == abft.OK and [(e["row"], e["col"]) for e in rep] == [(100, 7)]


def test_noalloc_encode_refuses_problems_above_the_static_maximum():
    # n = 2^21 columns with k = 256: the column-norm partials alone need 16 MiB
    desc = abft.make_desc(64, 1 << 21, 256, "f64", 64, 1 << 21)
    lib = abft.load()
    st = lib.abft_encode_noalloc(ct.byref(desc), ct.c_void_p(16), ct.c_void_p(16), None, None,
                                 ct.c_void_p(16), None)
    assert st == abft.ERR_INVALID
    assert "static maximum" in lib.abft_last_error().decode()
