"""CPU FP64 oracle for Huang-Abraham ABFT matrix multiplication -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The CUDA library never imports, links or calls
it, and it shares no code with the CUDA path.

The arithmetic lives in ``abft_oracle.c`` (plain C, binary64, ``-ffp-contract=off``);
this module compiles it with gcc on first use and wraps it with numpy through ctypes.
Every function cites the part of Bosilca, Delmas, Dongarra and Langou (2008) it
follows; see the C file for the definitions.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abft_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libabft_oracle.so")
_lock = threading.Lock()
_lib = None

KIND_CORRECTED = 1
KIND_NONFINITE = 2
KIND_UNCORRECTABLE = 3
KIND_RECOVERED = 4

ST_OK = 0
ST_INVALID = -1
ST_UNCORRECTABLE = 1

# unit roundoffs
U64 = 2.0 ** -53
U32 = 2.0 ** -24


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libabft_oracle.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OracleCfg(ct.Structure):
    _fields_ = [("m", ct.c_int64), ("n", ct.c_int64), ("k", ct.c_int64),
                ("vb_r", ct.c_int64), ("vb_c", ct.c_int64), ("p", ct.c_int64), ("q", ct.c_int64),
                ("u_acc", ct.c_double), ("u_sum", ct.c_double), ("u_enc", ct.c_double),
                ("u_c", ct.c_double), ("u_cs", ct.c_double), ("s", ct.c_double),
                ("round_f32", ct.c_int32), ("f", ct.c_int32),
                ("car_a", ct.c_void_p), ("car_b", ct.c_void_p)]


class OracleFault(ct.Structure):
    _fields_ = [("row", ct.c_int32), ("col", ct.c_int32), ("kind", ct.c_int32),
                ("side", ct.c_int32), ("delta", ct.c_double), ("r_e", ct.c_double),
                ("r_w", ct.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ct.CDLL(build())
            d, i64, i32 = ct.c_void_p, ct.c_int64, ct.c_int32
            _lib.oracle_weight.restype = ct.c_double
            _lib.oracle_weight.argtypes = [i64, i64]
            _lib.oracle_gemm.argtypes = [i64, i64, i64, d, i64, d, i64, d, i64]
            _lib.oracle_threads.restype = ct.c_int
            _lib.oracle_set_threads.argtypes = [ct.c_int]
            _lib.oracle_encode_A.argtypes = [i64, i64, d, i64, i64, i64, i64, d]
            _lib.oracle_block_coef.restype = ct.c_double
            _lib.oracle_block_coef.argtypes = [i64, i64, i64]
            _lib.oracle_recover_blocks.restype = ct.c_int
            _lib.oracle_recover_blocks.argtypes = [d, d, i64, d, d, d, d, i32, d]
            _lib.oracle_encode_B.argtypes = [i64, i64, d, i64, i64, d]
            _lib.oracle_norms_A.argtypes = [i64, i64, d, i64, i64, d, d]
            _lib.oracle_norms_B.argtypes = [i64, i64, d, i64, i64, d, d]
            _lib.oracle_col_residuals.argtypes = [d, d, i64, d, d, d, d, d, d, d, d]
            _lib.oracle_row_residuals.argtypes = [d, d, i64, d, d, d, d, d, d, d, d]
            _lib.oracle_verify_correct.restype = ct.c_int
            _lib.oracle_verify_correct.argtypes = [d, d, i64, d, d, d, d, d, d, d, i32, d, i32, d]
            _lib.oracle_recover_block.restype = ct.c_int
            _lib.oracle_recover_block.argtypes = [d, d, i64, d, d, d, i32, i32, d]
            _lib.oracle_thresholds_at.argtypes = [d, d, d, d, d, i64, i64, d]
            _lib.oracle_residual_check.restype = ct.c_double
            _lib.oracle_residual_check.argtypes = [i64, i64, i64, d, i64, d, i64, d, i64, d]
            _lib.oracle_bf16_to_f64.argtypes = [d, i64, d]
            _lib.oracle_e4m3_value.restype = ct.c_double
            _lib.oracle_e4m3_value.argtypes = [ct.c_uint8]
            _lib.oracle_dequant_e4m3.argtypes = [i64, i64, d, d, i64, d]
            _lib.oracle_norms_carried_rows.argtypes = [i64, i64, d, i64, d]
            _lib.oracle_norms_carried_cols.argtypes = [i64, i64, d, i64, d]
            _lib.oracle_carry_rows.argtypes = [d, d, d, d]
            _lib.oracle_carry_cols.argtypes = [d, d, d, d]
    return _lib


def threads() -> int:
    """Threads the oracle's GEMM loop runs on (OpenMP)."""
    return int(lib().oracle_threads())


def set_threads(n: int) -> None:
    """Sets the threads of the oracle's GEMM loop (OpenMP)."""
    lib().oracle_set_threads(int(n))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def cdiv(a: int, b: int) -> int:
    return -(-a // b)


# --------------------------------------------------------------------------- numerics
def weight(t: int, vb: int) -> float:
    """Weight of 0-based position t in a verify block of nominal size vb."""
    return lib().oracle_weight(t, vb)


def gemm(A, B) -> np.ndarray:
    """C = A B by the plain triple loop (Eq. (1))."""
    A, B = _f64(A), _f64(B)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    C = np.empty((m, n), np.float64)
    lib().oracle_gemm(m, n, k, _p(A), k, _p(B), n, _p(C), n)
    return C


def block_coef(l: int, I: int, p: int) -> float:
    """Coefficient of block row I in block checksum l (section 2.1, several checksums)."""
    return lib().oracle_block_coef(l, I, p)


def encode_A(A, vb: int, p: int = 0, f: int = 1) -> np.ndarray:
    """Checksum rows of A: [e^T A_I; w^T A_I] per verify block, then the f block checksums
    S^(l) = sum_I c_{l,I} A_I (section 2.1)."""
    A = _f64(A)
    m, k = A.shape
    f = max(1, f)
    rows = 2 * cdiv(m, vb) + (f * (m // p) if p else 0)
    acs = np.empty((rows, k), np.float64)
    lib().oracle_encode_A(m, k, _p(A), k, vb, p, f, _p(acs))
    return acs


def encode_B(B, vb: int) -> np.ndarray:
    """Checksum columns of B: [B_J e, B_J w] per verify block (Eq. (1))."""
    B = _f64(B)
    k, n = B.shape
    bcs = np.empty((k, 2 * cdiv(n, vb)), np.float64)
    lib().oracle_encode_B(k, n, _p(B), n, vb, _p(bcs))
    return bcs


def norms_A(A, vb: int):
    A = _f64(A)
    m, k = A.shape
    nrow = np.empty(m, np.float64)
    nblk = np.empty(4 * cdiv(m, vb), np.float64)
    lib().oracle_norms_A(m, k, _p(A), k, vb, _p(nrow), _p(nblk))
    return nrow, nblk


def norms_B(B, vb: int):
    B = _f64(B)
    k, n = B.shape
    ncol = np.empty(n, np.float64)
    nblk = np.empty(4 * cdiv(n, vb), np.float64)
    lib().oracle_norms_B(k, n, _p(B), n, vb, _p(ncol), _p(nblk))
    return ncol, nblk


def units(dtype: str) -> dict:
    """Rounding units entering the detection threshold for each product dtype.

    f64: everything in binary64.  bf16 / fp8 / bf16x3: the product accumulates in
    binary32 and C is stored in binary32 (no extra storage rounding); the checksum
    operand is fed to the tensor cores as a bf16 hi+lo pair (relative error 2^-17);
    encode sums and the observed block sums of C run in binary32.  bf16x3 (binary32
    inputs split into bf16 hi+lo, product A_hi B_hi + A_hi B_lo + A_lo B_hi) also carries
    the split's deviation from the exact product as u_c.
    """
    if dtype == "f64":
        return dict(u_acc=U64, u_sum=U64, u_enc=U64, u_c=U64, u_cs=U64)
    if dtype == "bf16x6":
        # three bf16 pieces keep 24 bits of each binary32 input: the dropped
        # products and the residual of the pieces are below 2^-25 of a product
        return dict(u_acc=U32, u_sum=U32, u_enc=U32, u_c=2.0 ** -25, u_cs=2.0 ** -26)
    if dtype == "bf16x3":
        # the split product drops A_lo B_lo and carries the hi+lo representation error of
        # the binary32 inputs: C deviates from their exact product by ~2^-17 relative
        return dict(u_acc=U32, u_sum=U32, u_enc=U32, u_c=2.0 ** -17, u_cs=2.0 ** -17)
    return dict(u_acc=U32, u_sum=U32, u_enc=U32, u_c=0.0, u_cs=2.0 ** -17)


def make_cfg(m, n, k, vb_r, vb_c, p=0, q=0, dtype="f64", s=4.0, f=1) -> OracleCfg:
    u = units(dtype)
    return OracleCfg(m=m, n=n, k=k, vb_r=vb_r, vb_c=vb_c, p=p, q=q, s=s,
                     round_f32=0 if dtype == "f64" else 1, f=max(1, f), **u)


def carry_rows(prev: "Encoded") -> np.ndarray:
    """Deviation bound of the column checksum rows carried out of product `prev`
    (2 per row verify block; section 3.2, chained calls)."""
    out = np.empty(2 * cdiv(prev.m, prev.cfg.vb_r), np.float64)
    lib().oracle_carry_rows(ct.byref(prev.cfg), _p(prev.nAblk), _p(prev.nBcol), _p(out))
    return out


def carry_cols(prev: "Encoded") -> np.ndarray:
    """Deviation bound of the row checksum columns carried out of product `prev`
    (2 per column verify block)."""
    out = np.empty(2 * cdiv(prev.n, prev.cfg.vb_c), np.float64)
    lib().oracle_carry_cols(ct.byref(prev.cfg), _p(prev.nBblk), _p(prev.nArow), _p(out))
    return out


class Encoded:
    """Everything the oracle derives from A and B before C is checked.

    left / right (chained calls, section 3.2): an earlier product's Encoded whose
    output C is this product's A (left) or B (right).  Its expected checksums E (rows)
    or F (columns) are carried as this product's encoded rows of A / columns of B
    instead of being computed from A / B, and the thresholds gain the bound of their
    deviation from the stored operand (carry_rows / carry_cols).
    """

    def __init__(self, A, B, vb_r, vb_c, p=0, q=0, dtype="f64", s=4.0, products=True, f=1,
                 left=None, right=None):
        A, B = _f64(A), _f64(B)
        self.A, self.B = A, B
        self.m, self.k = A.shape
        self.n = B.shape[1]
        self.cfg = make_cfg(self.m, self.n, self.k, vb_r, vb_c, p, q, dtype, s, f)
        nvr, nvc = cdiv(self.m, vb_r), cdiv(self.n, vb_c)
        self.nArow, self.nAblk = norms_A(A, vb_r)
        self.nBcol, self.nBblk = norms_B(B, vb_c)
        self.car_a = np.zeros(2 * nvr, np.float64)
        self.car_b = np.zeros(2 * nvc, np.float64)
        if left is not None:
            assert (left.m, left.n, left.cfg.vb_r) == (self.m, self.k, vb_r), "left chain shape"
            rows = 2 * nvr
            if p:
                assert left.cfg.p == p and left.cfg.f >= max(1, f), "left chain erasure grid"
                rows += max(1, f) * (self.m // p)
            self.acs = np.ascontiguousarray(left.E[:rows])
            lib().oracle_norms_carried_rows(nvr, self.k, _p(self.acs), self.k, _p(self.nAblk))
            self.car_a = carry_rows(left)
        else:
            self.acs = encode_A(A, vb_r, p, f)
        if right is not None:
            assert (right.m, right.n, right.cfg.vb_c) == (self.k, self.n, vb_c), "right chain shape"
            self.bcs = np.ascontiguousarray(right.F)
            lib().oracle_norms_carried_cols(self.k, nvc, _p(self.bcs), 2 * nvc, _p(self.nBblk))
            self.car_b = carry_cols(right)
        else:
            self.bcs = encode_B(B, vb_c)
        self.cfg.car_a = self.car_a.ctypes.data
        self.cfg.car_b = self.car_b.ctypes.data
        if products:  # skipped for large shapes, where tests sample E and F instead
            self.E = gemm(self.acs, B)   # expected column checksums (+ block checksum rows)
            self.F = gemm(A, self.bcs)   # expected row checksums

    def col_residuals(self, C):
        C = _f64(C)
        c = self.cfg
        nv = cdiv(c.m, c.vb_r)
        out = [np.empty((nv, c.n), np.float64) for _ in range(4)] + [np.empty((nv, c.n), np.int32)]
        lib().oracle_col_residuals(ct.byref(c), _p(C), c.n, _p(self.E), _p(self.nBcol),
                                   _p(self.nAblk), *[_p(o) for o in out])
        return out  # re, rw, te, tw, nonfinite

    def row_residuals(self, C):
        C = _f64(C)
        c = self.cfg
        nv = cdiv(c.n, c.vb_c)
        out = [np.empty((c.m, nv), np.float64) for _ in range(4)] + [np.empty((c.m, nv), np.int32)]
        lib().oracle_row_residuals(ct.byref(c), _p(C), c.n, _p(self.F), _p(self.nArow),
                                   _p(self.nBblk), *[_p(o) for o in out])
        return out

    def verify_correct(self, C, erased=(), max_reports=4096):
        """Detect / locate / correct on a copy of C; returns (status, report, C_corrected)."""
        C = _f64(C).copy()
        c = self.cfg
        er = np.ascontiguousarray(np.array(erased, np.int32).reshape(-1))
        rep = (OracleFault * max(1, max_reports))()
        nrep = ct.c_int32(0)
        st = lib().oracle_verify_correct(ct.byref(c), _p(C), c.n, _p(self.E), _p(self.F),
                                         _p(self.nArow), _p(self.nAblk), _p(self.nBcol),
                                         _p(self.nBblk), _p(er) if er.size else None,
                                         er.size // 2, ct.cast(rep, ct.c_void_p), max_reports,
                                         ct.byref(nrep))
        report = [dict(row=r.row, col=r.col, kind=r.kind, side=r.side, delta=r.delta,
                       r_e=r.r_e, r_w=r.r_w) for r in rep[:min(nrep.value, max_reports)]]
        return st, report, C, nrep.value

    def thresholds_at(self, i, j):
        """(tau_e, tau_w) of the column line and (tau_e, tau_w) of the row line of (i, j)."""
        out = np.empty(4, np.float64)
        lib().oracle_thresholds_at(ct.byref(self.cfg), _p(self.nArow), _p(self.nAblk),
                                   _p(self.nBcol), _p(self.nBblk), i, j, _p(out))
        return out

    def classify(self, i, j, delta):
        """Class of an error delta at (i, j): 'graded' (non-finite, or both unweighted
        residuals at least 8 thresholds: it must be located), 'benign' (no residual reaches
        half its threshold: it must stay silent) or 'guard' (either is acceptable)."""
        if not np.isfinite(delta):
            return "graded"
        te_c, tw_c, te_r, tw_r = self.thresholds_at(i, j)
        wi = weight(i % self.cfg.vb_r, self.cfg.vb_r)
        wj = weight(j % self.cfg.vb_c, self.cfg.vb_c)
        d = abs(delta)
        if d >= 8 * max(te_c, te_r):
            return "graded"
        if d <= 0.5 * min(te_c, tw_c / wi, te_r, tw_r / wj):
            return "benign"
        return "guard"

    def recover_blocks(self, C, blocks):
        """Rebuild the erased blocks [(bi, bj), ...] on a copy of C (up to f per block
        column); returns (status, C, n_flagged)."""
        C = _f64(C).copy()
        nfl = ct.c_int32(0)
        bl = np.ascontiguousarray(np.array(blocks, np.int32).reshape(-1))
        st = lib().oracle_recover_blocks(ct.byref(self.cfg), _p(C), self.cfg.n, _p(self.E),
                                         _p(self.nBcol), _p(self.nAblk),
                                         _p(bl) if bl.size else None, bl.size // 2,
                                         ct.byref(nfl))
        return st, C, nfl.value

    def recover_block(self, C, bi, bj):
        """Rebuild erased block (bi, bj) on a copy of C; returns (status, C, n_flagged)."""
        C = _f64(C).copy()
        nfl = ct.c_int32(0)
        st = lib().oracle_recover_block(ct.byref(self.cfg), _p(C), self.cfg.n, _p(self.E),
                                        _p(self.nBcol), _p(self.nAblk), bi, bj, ct.byref(nfl))
        return st, C, nfl.value


def residual_check(A, B, C, x) -> float:
    """||Cx - A(Bx)||_inf / (max(m,n,k) eps ||C||_inf ||x||_inf)  (section 4.3)."""
    A, B, C, x = _f64(A), _f64(B), _f64(C), _f64(x)
    m, k = A.shape
    n = B.shape[1]
    return lib().oracle_residual_check(m, n, k, _p(A), k, _p(B), n, _p(C), n, _p(x))


def bf16_to_f64(bits: np.ndarray) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint16)
    out = np.empty(bits.shape, np.float64)
    lib().oracle_bf16_to_f64(_p(bits), bits.size, _p(out))
    return out


def e4m3_value(b: int) -> float:
    return lib().oracle_e4m3_value(b)


def dequant_e4m3(q: np.ndarray, scale: np.ndarray, blk: int = 128) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.uint8)
    scale = np.ascontiguousarray(scale, dtype=np.float32)
    rows, cols = q.shape
    assert scale.shape == (cdiv(rows, blk), cdiv(cols, blk))
    out = np.empty((rows, cols), np.float64)
    lib().oracle_dequant_e4m3(rows, cols, _p(q), _p(scale), blk, _p(out))
    return out
