"""Thin Python binding of libabft (include/abft.h): argument marshalling only.

Every entry point has the name of the C function it wraps and takes torch tensors (device
memory and streams come from PyTorch) or raw integers for pointers.  All computation runs
in the CUDA kernels of libabft.so; there is no CPU or PyTorch fallback, and a missing
library raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libabft.so")

F64, BF16, BF16X3, FP8_E4M3, BF16X6 = 0, 1, 2, 3, 4
DTYPE_CODES = {"f64": F64, "bf16": BF16, "bf16x3": BF16X3, "fp8": FP8_E4M3, "bf16x6": BF16X6}

OK, ERR_INVALID, ERR_CUDA, ERR_UNSUPPORTED, ERR_UNCORRECTABLE, ERR_TIMEOUT = range(6)
KIND_CORRECTED, KIND_NONFINITE_CORRECTED, KIND_UNCORRECTABLE, KIND_BLOCK_RECOVERED = 1, 2, 3, 4

# Every symbol include/abft.h declares.
EXPORTS = ("abft_workspace_bytes", "abft_workspace_layout", "abft_encode",
           "abft_encode_noalloc", "abft_encode_chained", "abft_gemm", "abft_set_epilogue_faults",
           "abft_gemm_plain", "abft_verify_correct", "abft_recover_block", "abft_recover_blocks",
           "abft_block_partial", "abft_block_restore",
           "abft_inject_bitflips", "abft_erase_block", "abft_kernel_launches",
           "abft_last_error", "abft_version",
           "abft_group_create", "abft_group_workspace_bytes", "abft_group_problem_layout",
           "abft_group_bind",
           "abft_group_set_tuning", "abft_group_get_tuning", "abft_group_autotune",
           "abft_group_encode", "abft_group_gemm", "abft_group_verify_enqueue",
           "abft_group_report", "abft_group_verify_correct", "abft_group_set_epilogue_faults",
           "abft_group_capture", "abft_group_launch", "abft_group_destroy")


class AbftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"abft status {status}: {msg}")
        self.status = status


class Desc(ct.Structure):
    _fields_ = [("m", ct.c_int64), ("n", ct.c_int64), ("k", ct.c_int64),
                ("lda", ct.c_int64), ("ldb", ct.c_int64), ("ldc", ct.c_int64),
                ("dtype", ct.c_int32), ("vb_rows", ct.c_int32), ("vb_cols", ct.c_int32),
                ("grid_p", ct.c_int32), ("grid_q", ct.c_int32), ("flags", ct.c_int32),
                ("tau_safety", ct.c_double), ("grid_f", ct.c_int32), ("reserved", ct.c_int32)]


class Fault(ct.Structure):
    _fields_ = [("row", ct.c_int32), ("col", ct.c_int32), ("kind", ct.c_int32),
                ("side", ct.c_int32), ("delta", ct.c_double), ("r_e", ct.c_double),
                ("r_w", ct.c_double), ("problem", ct.c_int32), ("reserved", ct.c_int32)]

    def as_dict(self):
        return dict(row=self.row, col=self.col, kind=self.kind, side=self.side,
                    delta=self.delta, r_e=self.r_e, r_w=self.r_w, problem=self.problem)


class WsLayout(ct.Structure):
    _fields_ = [("total", ct.c_size_t), ("acs", ct.c_size_t), ("bcs", ct.c_size_t),
                ("E", ct.c_size_t), ("F", ct.c_size_t), ("nArow", ct.c_size_t),
                ("nAblk", ct.c_size_t), ("nBcol", ct.c_size_t), ("nBblk", ct.c_size_t),
                ("scratch", ct.c_size_t), ("scratch_bytes", ct.c_size_t),
                ("R", ct.c_int64), ("Cc", ct.c_int64), ("nvr", ct.c_int64), ("nvc", ct.c_int64),
                ("bs", ct.c_int64), ("acs_ld", ct.c_int64), ("bcs_ld", ct.c_int64),
                ("E16", ct.c_size_t), ("F16", ct.c_size_t), ("acs_rows", ct.c_int64),
                ("bcs_cols", ct.c_int64), ("obs_col", ct.c_size_t), ("obs_row", ct.c_size_t),
                ("inject", ct.c_size_t), ("fused", ct.c_int32), ("planes", ct.c_int32),
                ("acs_plane", ct.c_size_t), ("bcs_plane", ct.c_size_t), ("op_a", ct.c_size_t),
                ("op_b", ct.c_size_t), ("op_a_ld", ct.c_int64), ("op_b_ld", ct.c_int64),
                ("car_a", ct.c_size_t), ("car_b", ct.c_size_t), ("scales", ct.c_size_t),
                ("f8grp", ct.c_size_t), ("f8bt", ct.c_size_t)]


class Problem(ct.Structure):
    _fields_ = [("m", ct.c_int64), ("n", ct.c_int64), ("k", ct.c_int64),
                ("lda", ct.c_int64), ("ldb", ct.c_int64), ("ldc", ct.c_int64),
                ("A", ct.c_void_p), ("B", ct.c_void_p), ("C", ct.c_void_p)]


class GroupLayout(ct.Structure):
    _fields_ = [(f, ct.c_size_t) for f in ("acs", "bcs", "E16", "F16", "obs_col", "obs_row",
                                           "nArow", "nAblk", "nBcol", "nBblk")] + \
               [(f, ct.c_int64) for f in ("nvr", "nvc", "R16", "C16", "acs_ld", "bcs_ld")]


class GroupTuning(ct.Structure):
    _fields_ = [("boxes_per_tile", ct.c_int32), ("order", ct.c_int32)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libabft.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libabft.so not built ({path}); run paper_0806_3121_gb300.build.build()")
        lib = ct.CDLL(path)
        vp, i32, i64 = ct.c_void_p, ct.c_int32, ct.c_int64
        D = ct.POINTER(Desc)
        lib.abft_workspace_bytes.restype = ct.c_size_t
        lib.abft_workspace_bytes.argtypes = [D]
        lib.abft_workspace_layout.argtypes = [D, ct.POINTER(WsLayout)]
        lib.abft_encode.argtypes = [D, vp, vp, vp, vp, vp, vp]
        lib.abft_encode_noalloc.argtypes = [D, vp, vp, vp, vp, vp, vp]
        lib.abft_encode_chained.argtypes = [D, vp, vp, D, vp, D, vp, vp, vp]
        lib.abft_gemm.argtypes = [D, vp, vp, vp, vp, vp, vp, vp]
        lib.abft_gemm_plain.argtypes = [D, vp, vp, vp, vp, vp, vp, vp]
        lib.abft_set_epilogue_faults.argtypes = [D, vp, vp, vp, vp, i32, vp]
        lib.abft_verify_correct.argtypes = [D, vp, vp, i32, vp, i32, vp, i32,
                                            ct.POINTER(ct.c_int32), vp]
        lib.abft_recover_block.argtypes = [D, vp, vp, i32, i32, ct.POINTER(Fault), vp]
        lib.abft_recover_blocks.argtypes = [D, vp, vp, vp, i32, vp, vp]
        lib.abft_block_partial.argtypes = [D, vp, vp, i32, i32, i32, vp, vp]
        lib.abft_block_restore.argtypes = [D, vp, vp, i32, i32, vp, ct.POINTER(Fault), vp]
        lib.abft_inject_bitflips.argtypes = [D, vp, vp, vp, vp, i32, vp]
        lib.abft_erase_block.argtypes = [D, vp, i32, i32, vp]
        lib.abft_last_error.restype = ct.c_char_p
        lib.abft_last_error.argtypes = []
        lib.abft_kernel_launches.restype = ct.c_int64
        lib.abft_kernel_launches.argtypes = []
        lib.abft_version.restype = ct.c_int32
        lib.abft_version.argtypes = []
        G, T = vp, ct.POINTER(GroupTuning)
        lib.abft_group_create.argtypes = [ct.POINTER(Problem), i32, i32, ct.c_double,
                                          ct.POINTER(ct.c_void_p)]
        lib.abft_group_workspace_bytes.restype = ct.c_size_t
        lib.abft_group_workspace_bytes.argtypes = [G]
        lib.abft_group_bind.argtypes = [G, vp, ct.c_size_t, vp]
        lib.abft_group_problem_layout.argtypes = [G, i32, ct.POINTER(GroupLayout)]
        lib.abft_group_set_tuning.argtypes = [G, T, vp]
        lib.abft_group_get_tuning.argtypes = [G, T]
        lib.abft_group_autotune.argtypes = [G, i32, T, ct.POINTER(ct.c_double), vp]
        lib.abft_group_encode.argtypes = [G, vp]
        lib.abft_group_gemm.argtypes = [G, i32, vp]
        lib.abft_group_verify_enqueue.argtypes = [G, vp]
        lib.abft_group_report.argtypes = [G, vp, i32, ct.POINTER(ct.c_int32), vp]
        lib.abft_group_verify_correct.argtypes = [G, vp, i32, ct.POINTER(ct.c_int32), vp]
        lib.abft_group_set_epilogue_faults.argtypes = [G, vp, vp, vp, vp, i32, vp]
        lib.abft_group_capture.argtypes = [G, i32, vp]
        lib.abft_group_launch.argtypes = [G, vp]
        lib.abft_group_destroy.argtypes = [G]
        for name in EXPORTS:  # fail loudly on a library that lacks an entry point
            getattr(lib, name)
        _lib = lib
        return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st: int, allow=(OK,)):
    if st not in allow:
        raise AbftError(st, load().abft_last_error().decode())
    return st


def make_desc(m, n, k, dtype="f64", vb_rows=None, vb_cols=None, grid_p=0, grid_q=0,
              lda=None, ldb=None, ldc=None, tau_safety=0.0, grid_f=0) -> Desc:
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    return Desc(m=m, n=n, k=k, lda=lda or max(k, 1), ldb=ldb or max(n, 1), ldc=ldc or max(n, 1),
                dtype=code, vb_rows=vb_rows or max(m, 1), vb_cols=vb_cols or max(n, 1),
                grid_p=grid_p, grid_q=grid_q, flags=0, tau_safety=tau_safety, grid_f=grid_f,
                reserved=0)


def abft_workspace_bytes(desc: Desc) -> int:
    nb = load().abft_workspace_bytes(ct.byref(desc))
    if nb == 0:
        raise AbftError(ERR_INVALID, load().abft_last_error().decode())
    return nb


def abft_workspace_layout(desc: Desc) -> WsLayout:
    out = WsLayout()
    _check(load().abft_workspace_layout(ct.byref(desc), ct.byref(out)))
    return out


def abft_encode(desc, A, B, ws, a_scale=None, b_scale=None, stream=None):
    _check(load().abft_encode(ct.byref(desc), _ptr(A), _ptr(B), _ptr(a_scale), _ptr(b_scale),
                              _ptr(ws), _stream(stream)))


def abft_encode_noalloc(desc, A, B, ws, a_scale=None, b_scale=None, stream=None):
    """abft_encode without workspace scratch (see include/abft.h); ws needs only the
    bytes below the layout's scratch offset."""
    _check(load().abft_encode_noalloc(ct.byref(desc), _ptr(A), _ptr(B), _ptr(a_scale),
                                      _ptr(b_scale), _ptr(ws), _stream(stream)))


def abft_encode_chained(desc, A, B, ws, left=None, right=None, stream=None):
    """Chained encode (section 3.2): left / right are (desc, ws) of the earlier products
    whose outputs are A / B; their expected checksums are carried, not recomputed."""
    ld, lw = (ct.byref(left[0]), _ptr(left[1])) if left is not None else (None, None)
    rd, rw = (ct.byref(right[0]), _ptr(right[1])) if right is not None else (None, None)
    _check(load().abft_encode_chained(ct.byref(desc), _ptr(A), _ptr(B), ld, lw, rd, rw,
                                      _ptr(ws), _stream(stream)))


def abft_gemm(desc, A, B, C, ws, a_scale=None, b_scale=None, stream=None):
    _check(load().abft_gemm(ct.byref(desc), _ptr(A), _ptr(B), _ptr(a_scale), _ptr(b_scale),
                            _ptr(C), _ptr(ws), _stream(stream)))


def abft_gemm_plain(desc, A, B, C, a_scale=None, b_scale=None, ws=None, stream=None):
    _check(load().abft_gemm_plain(ct.byref(desc), _ptr(A), _ptr(B), _ptr(a_scale),
                                  _ptr(b_scale), _ptr(C), _ptr(ws), _stream(stream)))


def abft_verify_correct(desc, C, ws, erased=(), max_reports=1024, reread_C=1, stream=None):
    """Returns (status, [fault dicts], total report count).  Synchronises the stream."""
    er = (ct.c_int32 * max(1, 2 * len(erased)))(*[v for b in erased for v in b])
    rep = (Fault * max(1, max_reports))()
    nrep = ct.c_int32(0)
    st = load().abft_verify_correct(ct.byref(desc), _ptr(C), _ptr(ws), reread_C,
                                    ct.cast(er, ct.c_void_p), len(erased),
                                    ct.cast(rep, ct.c_void_p), max_reports, ct.byref(nrep),
                                    _stream(stream))
    _check(st, allow=(OK, ERR_UNCORRECTABLE))
    return st, [r.as_dict() for r in rep[:min(nrep.value, max_reports)]], nrep.value


def abft_recover_block(desc, C, ws, bi, bj, stream=None):
    """Returns (status, report entry dict).  Synchronises the stream."""
    f = Fault()
    st = load().abft_recover_block(ct.byref(desc), _ptr(C), _ptr(ws), bi, bj, ct.byref(f),
                                   _stream(stream))
    _check(st, allow=(OK, ERR_UNCORRECTABLE))
    return st, f.as_dict()


def abft_recover_blocks(desc, C, ws, blocks, stream=None):
    """Rebuild several erased blocks [(bi, bj), ...] (up to grid_f per block column).
    Returns (status, [report entry dicts]).  Synchronises the stream."""
    n = len(blocks)
    arr = (ct.c_int32 * max(1, 2 * n))(*[v for b in blocks for v in b])
    rep = (Fault * max(1, n))()
    st = load().abft_recover_blocks(ct.byref(desc), _ptr(C), _ptr(ws), ct.cast(arr, ct.c_void_p),
                                    n, ct.cast(rep, ct.c_void_p), _stream(stream))
    _check(st, allow=(OK, ERR_UNCORRECTABLE))
    return st, [r.as_dict() for r in rep[:n]]


def abft_block_partial(desc, C, ws, bi_skip, bj, with_checksum, out, stream=None):
    """This rank's share of the rebuild of a block of block column bj (block rows spread
    over GPUs): out (bs x bc float64, device) = (with_checksum ? S_bj : 0) minus the local
    blocks of the column other than block row bi_skip (-1: none)."""
    _check(load().abft_block_partial(ct.byref(desc), _ptr(C), _ptr(ws), bi_skip, bj,
                                     1 if with_checksum else 0, _ptr(out), _stream(stream)))


def abft_block_restore(desc, C, ws, bi, bj, total, stream=None):
    """Write the reduced shares `total` (bs x bc float64, device) into block (bi, bj) of C
    and re-check it.  Returns (status, report entry dict).  Synchronises the stream."""
    f = Fault()
    st = load().abft_block_restore(ct.byref(desc), _ptr(C), _ptr(ws), bi, bj, _ptr(total),
                                   ct.byref(f), _stream(stream))
    _check(st, allow=(OK, ERR_UNCORRECTABLE))
    return st, f.as_dict()


def abft_inject_bitflips(desc, C, flips, stream=None):
    n = len(flips)
    rows = (ct.c_int64 * max(1, n))(*[f[0] for f in flips])
    cols = (ct.c_int64 * max(1, n))(*[f[1] for f in flips])
    bits = (ct.c_int32 * max(1, n))(*[f[2] for f in flips])
    _check(load().abft_inject_bitflips(ct.byref(desc), _ptr(C), ct.cast(rows, ct.c_void_p),
                                       ct.cast(cols, ct.c_void_p), ct.cast(bits, ct.c_void_p), n,
                                       _stream(stream)))


def abft_set_epilogue_faults(desc, ws, flips, stream=None):
    """Arm bit flips (row, col, bit) of the product's accumulator outputs; [] disarms."""
    n = len(flips)
    rows = (ct.c_int64 * max(1, n))(*[f[0] for f in flips])
    cols = (ct.c_int64 * max(1, n))(*[f[1] for f in flips])
    bits = (ct.c_int32 * max(1, n))(*[f[2] for f in flips])
    _check(load().abft_set_epilogue_faults(ct.byref(desc), _ptr(ws), ct.cast(rows, ct.c_void_p),
                                           ct.cast(cols, ct.c_void_p), ct.cast(bits, ct.c_void_p),
                                           n, _stream(stream)))


def abft_erase_block(desc, C, bi, bj, stream=None):
    _check(load().abft_erase_block(ct.byref(desc), _ptr(C), bi, bj, _stream(stream)))


def abft_kernel_launches() -> int:
    return load().abft_kernel_launches()


def abft_version() -> int:
    return load().abft_version()


# ---- grouped products (abft_group_*): one handle per group of problems

def abft_group_create(problems, dtype="bf16", tau_safety=0.0):
    """problems: sequence of dicts/tuples (m, n, k, A, B, C[, lda, ldb, ldc]) with A, B, C
    tensors or device pointers.  Returns the opaque handle (an int)."""
    arr = (Problem * max(1, len(problems)))()
    for i, q in enumerate(problems):
        if isinstance(q, dict):
            m, n, k, A, B, C = q["m"], q["n"], q["k"], q["A"], q["B"], q["C"]
            lda, ldb, ldc = q.get("lda", k), q.get("ldb", n), q.get("ldc", n)
        else:
            m, n, k, A, B, C = q[:6]
            lda, ldb, ldc = (q[6:9] if len(q) >= 9 else (k, n, n))
        arr[i] = Problem(m=m, n=n, k=k, lda=lda, ldb=ldb, ldc=ldc, A=_ptr(A), B=_ptr(B),
                         C=_ptr(C))
    h = ct.c_void_p()
    code = DTYPE_CODES[dtype] if isinstance(dtype, str) else int(dtype)
    _check(load().abft_group_create(arr, len(problems), code, tau_safety, ct.byref(h)))
    return h.value


def abft_group_workspace_bytes(g) -> int:
    return load().abft_group_workspace_bytes(g)


def abft_group_problem_layout(g, p) -> GroupLayout:
    out = GroupLayout()
    _check(load().abft_group_problem_layout(g, p, ct.byref(out)))
    return out


def abft_group_bind(g, ws, stream=None):
    _check(load().abft_group_bind(g, _ptr(ws), ws.numel() * ws.element_size()
                                  if hasattr(ws, "numel") else abft_group_workspace_bytes(g),
                                  _stream(stream)))


def abft_group_set_tuning(g, boxes_per_tile=4, order=1, stream=None):
    t = GroupTuning(boxes_per_tile=boxes_per_tile, order=order)
    _check(load().abft_group_set_tuning(g, ct.byref(t), _stream(stream)))


def abft_group_get_tuning(g):
    t = GroupTuning()
    _check(load().abft_group_get_tuning(g, ct.byref(t)))
    return dict(boxes_per_tile=t.boxes_per_tile, order=t.order)


def abft_group_autotune(g, reps=3, stream=None):
    """Returns (tuning dict, best ms or -1 when taken from the cache file)."""
    t = GroupTuning()
    ms = ct.c_double(0.0)
    _check(load().abft_group_autotune(g, reps, ct.byref(t), ct.byref(ms), _stream(stream)))
    return dict(boxes_per_tile=t.boxes_per_tile, order=t.order), ms.value


def abft_group_encode(g, stream=None):
    _check(load().abft_group_encode(g, _stream(stream)))


def abft_group_gemm(g, checksums=True, stream=None):
    _check(load().abft_group_gemm(g, 1 if checksums else 0, _stream(stream)))


def abft_group_verify_enqueue(g, stream=None):
    _check(load().abft_group_verify_enqueue(g, _stream(stream)))


def _group_reports(fn, g, max_reports, stream):
    rep = (Fault * max(1, max_reports))()
    nrep = ct.c_int32(0)
    st = fn(g, ct.cast(rep, ct.c_void_p), max_reports, ct.byref(nrep), _stream(stream))
    _check(st, allow=(OK, ERR_UNCORRECTABLE))
    return st, [r.as_dict() for r in rep[:min(nrep.value, max_reports)]], nrep.value


def abft_group_report(g, max_reports=1024, stream=None):
    """Returns (status, [fault dicts], total count).  Synchronises the stream."""
    return _group_reports(load().abft_group_report, g, max_reports, stream)


def abft_group_verify_correct(g, max_reports=1024, stream=None):
    return _group_reports(load().abft_group_verify_correct, g, max_reports, stream)


def abft_group_set_epilogue_faults(g, flips, stream=None):
    """flips: (problem, row, col, bit) tuples; [] disarms."""
    n = len(flips)
    prob = (ct.c_int32 * max(1, n))(*[f[0] for f in flips])
    rows = (ct.c_int64 * max(1, n))(*[f[1] for f in flips])
    cols = (ct.c_int64 * max(1, n))(*[f[2] for f in flips])
    bits = (ct.c_int32 * max(1, n))(*[f[3] for f in flips])
    _check(load().abft_group_set_epilogue_faults(
        g, ct.cast(prob, ct.c_void_p), ct.cast(rows, ct.c_void_p), ct.cast(cols, ct.c_void_p),
        ct.cast(bits, ct.c_void_p), n, _stream(stream)))


def abft_group_capture(g, checksums=True, stream=None):
    _check(load().abft_group_capture(g, 1 if checksums else 0, _stream(stream)))


def abft_group_launch(g, stream=None):
    _check(load().abft_group_launch(g, _stream(stream)))


def abft_group_destroy(g):
    _check(load().abft_group_destroy(g))
