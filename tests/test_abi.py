"""The C-ABI library loads, exports every entry point include/abft.h declares, and its
host-side validation and workspace layout behave as documented.  No GPU is touched:
only calls that never launch work run here."""
import ctypes as ct
import os
import re

import pytest

from paper_0806_3121_gb300 import abft, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "abft.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abft.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(abft_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(abft.EXPORTS)


def test_version(lib):
    assert abft.abft_version() >= 100


def test_struct_sizes_match_header(lib):
    assert ct.sizeof(abft.Desc) == 6 * 8 + 6 * 4 + 8 + 2 * 4
    assert ct.sizeof(abft.Fault) == 4 * 4 + 3 * 8 + 2 * 4
    assert ct.sizeof(abft.Problem) == 6 * 8 + 3 * 8
    assert ct.sizeof(abft.GroupTuning) == 2 * 4
    assert ct.sizeof(abft.GroupLayout) == 10 * 8 + 6 * 8


def test_workspace_layout_shapes(lib):
    d = abft.make_desc(11264, 11264, 11264, "f64", 512, 512, 22, 22)
    L = abft.abft_workspace_layout(d)
    assert L.nvr == 22 and L.nvc == 22 and L.bs == 512
    assert L.R == 2 * 22 + 512 and L.Cc == 44
    for off in (L.acs, L.bcs, L.E, L.F, L.nArow, L.nAblk, L.nBcol, L.nBblk, L.car_a, L.car_b,
                L.scratch):
        assert off % 256 == 0
    assert L.car_b >= L.car_a + 2 * 22 * 8 and L.scratch >= L.car_b + 2 * 22 * 8
    assert L.bcs >= L.acs + L.R * 11264 * 8
    assert L.E >= L.bcs + 11264 * L.Cc * 8
    assert L.F >= L.E + L.R * 11264 * 8
    assert L.total >= L.scratch + L.scratch_bytes
    assert abft.abft_workspace_bytes(d) == L.total


def test_ragged_layout(lib):
    d = abft.make_desc(100, 70, 33, "f64", 32, 16)
    L = abft.abft_workspace_layout(d)
    assert L.nvr == 4 and L.nvc == 5 and L.R == 8 and L.Cc == 10 and L.bs == 0


@pytest.mark.parametrize("kw,msg", [
    (dict(m=-1), "negative"),
    (dict(vb_rows=0), "verify block"),
    (dict(vb_rows=65), "verify block"),
    (dict(grid_p=3, grid_q=3), "divide"),
    (dict(grid_p=2, grid_q=0), "both"),
    (dict(lda=10), "leading"),
    (dict(dtype=9), "dtype"),
    (dict(tau_safety=-1.0), "tau_safety"),
])
def test_invalid_descriptors(lib, kw, msg):
    d = abft.make_desc(64, 64, 64, "f64", 32, 32)
    for k, v in kw.items():
        setattr(d, k, v)
    assert lib.abft_workspace_bytes(ct.byref(d)) == 0
    assert msg in lib.abft_last_error().decode()
    with pytest.raises(abft.AbftError) as e:
        abft.abft_workspace_layout(d)
    assert e.value.status == abft.ERR_INVALID


def test_invalid_calls_launch_nothing(lib):
    """Argument errors are caught on the host before any CUDA call (so they are safe
    without a GPU)."""
    d = abft.make_desc(64, 64, 64, "f64", 32, 32, 2, 2)
    st = lib.abft_recover_block(ct.byref(d), None, None, 5, 0, None, None)
    assert st == abft.ERR_INVALID
    st = lib.abft_erase_block(ct.byref(d), None, 0, 9, None)
    assert st == abft.ERR_INVALID
    rows = (ct.c_int64 * 1)(64)
    cols = (ct.c_int64 * 1)(0)
    bits = (ct.c_int32 * 1)(3)
    st = lib.abft_inject_bitflips(ct.byref(d), ct.c_void_p(1), rows, cols, bits, 1, None)
    assert st == abft.ERR_INVALID and "outside" in lib.abft_last_error().decode()
    er = (ct.c_int32 * 2)(0, 7)
    n = ct.c_int32(0)
    st = lib.abft_verify_correct(ct.byref(d), ct.c_void_p(1), ct.c_void_p(1), 1, er, 1, None, 0,
                                 ct.byref(n), None)
    assert st == abft.ERR_INVALID
    d2 = abft.make_desc(64, 64, 64, "f64", 32, 32)
    st = lib.abft_recover_block(ct.byref(d2), ct.c_void_p(1), ct.c_void_p(1), 0, 0, None, None)
    assert st == abft.ERR_INVALID and "grid" in lib.abft_last_error().decode()


@pytest.mark.parametrize("side,kw,status,msg", [
    ("left", dict(m=96), abft.ERR_INVALID, "left chain"),          # earlier product m != m
    ("left", dict(n=40), abft.ERR_INVALID, "left chain"),          # earlier n != this k
    ("left", dict(vb_rows=16), abft.ERR_INVALID, "left chain"),
    ("left", dict(grid_p=0, grid_q=0), abft.ERR_INVALID, "grid"),  # no block checksums to carry
    ("left", dict(dtype=1, lda=64, ldb=80), abft.ERR_INVALID, "binary64 C"),  # bf16 earlier C
    ("right", dict(m=32), abft.ERR_INVALID, "right chain"),        # earlier m != this k
    ("right", dict(vb_cols=8), abft.ERR_INVALID, "right chain"),
    ("right", dict(dtype=1, lda=80), abft.ERR_INVALID, "binary64 C"),
    ("this", dict(dtype=1), abft.ERR_UNSUPPORTED, "ABFT_F64"),     # plain bf16 is not chained
    ("this", dict(dtype=4), abft.ERR_INVALID, "binary32 C"),       # split product, binary64 C
])
def test_chained_encode_validation_launches_nothing(lib, side, kw, status, msg):
    """Shape, grid and dtype mismatches of a chained encode are refused on the host."""
    this = abft.make_desc(64, 48, 80, "f64", 32, 16, 2, 2)       # C' = A' B', A' is 64 x 80
    left = abft.make_desc(64, 80, 20, "f64", 32, 16, 2, 2)       # earlier 64 x 80 product
    right = abft.make_desc(80, 48, 20, "f64", 16, 16)            # earlier 80 x 48 product
    tgt = {"left": left, "right": right, "this": this}[side]
    for k, v in kw.items():
        setattr(tgt, k, v)
    fake = ct.c_void_p(1)
    st = lib.abft_encode_chained(ct.byref(this), fake, fake,
                                 ct.byref(left) if side in ("left", "this") else None,
                                 fake if side in ("left", "this") else None,
                                 ct.byref(right) if side == "right" else None,
                                 fake if side == "right" else None, fake, None)
    assert st == status
    assert msg in lib.abft_last_error().decode()


def test_empty_problem_is_a_no_op(lib):
    d = abft.make_desc(0, 16, 16, "f64", 1, 16)
    assert abft.abft_workspace_bytes(d) > 0
    # nothing to do: returns OK without touching the (NULL) pointers or the GPU
    assert lib.abft_gemm(ct.byref(d), None, None, None, None, ct.c_void_p(1), ct.c_void_p(1), None) == 0


def _fake_problem(m, n, k, **kw):
    # device pointers are only stored by abft_group_create (never dereferenced on the host)
    q = dict(m=m, n=n, k=k, lda=(k + 7) // 8 * 8, ldb=(n + 7) // 8 * 8, ldc=n,
             A=1 << 20, B=2 << 20, C=3 << 20)
    q.update(kw)
    return q


def test_group_layout_host_only(lib):
    """abft_group_create validates and lays out the workspace on the host only."""
    shapes = [(64, 64, 64), (1, 1, 1), (300, 700, 129), (2048, 2048, 2048)]
    g = abft.abft_group_create([_fake_problem(*s) for s in shapes], "bf16")
    try:
        total = abft.abft_group_workspace_bytes(g)
        prev_end = 0
        for p, (m, n, k) in enumerate(shapes):
            L = abft.abft_group_problem_layout(g, p)
            nvr, nvc = -(-m // 128), -(-n // 256)
            assert (L.nvr, L.nvc, L.R16, L.C16) == (nvr, nvc, 4 * nvr, 4 * nvc)
            assert L.acs_ld % 8 == 0 and L.acs_ld >= k and L.bcs_ld % 8 == 0
            offs = [L.acs, L.bcs, L.E16, L.F16, L.obs_col, L.obs_row, L.nArow, L.nAblk, L.nBcol,
                    L.nBblk]
            assert all(o % 256 == 0 for o in offs) and offs == sorted(offs) and offs[0] >= prev_end
            assert L.bcs >= L.acs + L.R16 * L.acs_ld * 2
            assert L.F16 >= L.E16 + L.R16 * n * 4
            prev_end = L.nBblk + 4 * nvc * 8
            assert prev_end <= total
        assert abft.abft_group_get_tuning(g) == dict(boxes_per_tile=4, order=1)
        with pytest.raises(abft.AbftError):
            abft.abft_group_problem_layout(g, len(shapes))
        # calls that need a bound workspace refuse before touching the GPU
        with pytest.raises(abft.AbftError) as e:
            abft.abft_group_encode(g, stream=0)
        assert e.value.status == abft.ERR_INVALID and "bind" in str(e.value)
    finally:
        abft.abft_group_destroy(g)


@pytest.mark.parametrize("kw,msg", [
    (dict(m=0), "sizes"), (dict(k=(1 << 24) + 1), "sizes"), (dict(lda=60), "lda"),
    (dict(ldb=12), "multiples of 8"), (dict(ldc=10), "ldc"), (dict(A=0), "NULL"),
    (dict(B=(2 << 20) + 8), "aligned"),
])
def test_group_invalid_problems(lib, kw, msg):
    with pytest.raises(abft.AbftError) as e:
        q = _fake_problem(64, 64, 64)
        q.update(kw)
        abft.abft_group_create([_fake_problem(64, 64, 64), q])
    assert e.value.status == abft.ERR_INVALID and msg in str(e.value)
    assert "problem 1" in str(e.value)


def test_group_other_dtypes_unsupported(lib):
    with pytest.raises(abft.AbftError) as e:
        abft.abft_group_create([_fake_problem(64, 64, 64)], "f64")
    assert e.value.status == abft.ERR_UNSUPPORTED


def test_misaligned_workspace_is_refused(lib):
    """Every call that takes a workspace checks its 256-byte alignment before launching."""
    d = abft.make_desc(64, 64, 64, "f64", 32, 32)
    ok, bad = ct.c_void_p(1 << 20), ct.c_void_p((1 << 20) + 8)
    st = lib.abft_encode(ct.byref(d), ok, ok, None, None, bad, None)
    assert st == abft.ERR_INVALID and "256-byte" in lib.abft_last_error().decode()
    st = lib.abft_gemm(ct.byref(d), ok, ok, None, None, ok, bad, None)
    assert st == abft.ERR_INVALID and "256-byte" in lib.abft_last_error().decode()
    n = ct.c_int32(0)
    st = lib.abft_verify_correct(ct.byref(d), ok, bad, 1, None, 0, None, 0, ct.byref(n), None)
    assert st == abft.ERR_INVALID and "256-byte" in lib.abft_last_error().decode()
    left = abft.make_desc(64, 64, 16, "f64", 32, 32)
    st = lib.abft_encode_chained(ct.byref(d), ok, ok, ct.byref(left), bad, None, None, ok, None)
    assert st == abft.ERR_INVALID and "256-byte" in lib.abft_last_error().decode()
