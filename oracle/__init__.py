"""FP64 CPU oracle for LDPC encoding and sum-product decoding (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``ldpc_oracle.c`` (compiled with gcc by
``oracle.compile``), the brute-force references in ``brute.py`` and the FP64
weighted-BP gradient in ``wbp_ref.py``.

Each wrapper cites the passage of arXiv 2201.04265 it follows; see the C file
for the readings taken where the paper is garbled or silent.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .compile import build, library_path

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            build()
        lib = ctypes.CDLL(path)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_systematic.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p, i32p,
                                          i32p, u8p, ctypes.c_int64]
        lib.oracle_systematic.restype = ctypes.c_int
        lib.oracle_encode.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, u8p, u8p,
                                      ctypes.c_int32, u8p]
        lib.oracle_encode.restype = None
        lib.oracle_syndrome.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, u8p,
                                        ctypes.c_int32, u8p]
        lib.oracle_syndrome.restype = None
        lib.oracle_decode.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, f64p,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_double, f64p, f64p, u8p, i32p, u8p, ctypes.c_int32]
        lib.oracle_decode.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Systematic:
    """Standard-form generator data: G = [I_k : P] up to the column order of H."""
    n: int
    k: int
    rank: int
    info_pos: np.ndarray    # int32 [k], ascending
    parity_pos: np.ndarray  # int32 [rank], ascending
    A: np.ndarray           # uint8 [rank, k]; parity j = XOR_i A[j, i] m_i


def systematic(code) -> Systematic:
    """GF(2) elimination of H (Eq. 2; standard form of Sec. III-B)."""
    lib = _load()
    rp = np.ascontiguousarray(code.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(code.col_idx, dtype=np.int32)
    rank = np.zeros(1, dtype=np.int32)
    info = np.zeros(code.n, dtype=np.int32)
    par = np.zeros(code.n, dtype=np.int32)
    cap = max(1, (code.n * code.n) // 4 + code.n)
    A = np.zeros(cap, dtype=np.uint8)
    rc = lib.oracle_systematic(code.m, code.n, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                               _ptr(rank, ctypes.c_int32), _ptr(info, ctypes.c_int32),
                               _ptr(par, ctypes.c_int32), _ptr(A, ctypes.c_uint8), cap)
    if rc != 0:
        raise ValueError(f"oracle_systematic failed ({rc})")
    r = int(rank[0])
    k = code.n - r
    return Systematic(n=code.n, k=k, rank=r, info_pos=info[:k].copy(), parity_pos=par[:r].copy(),
                      A=A[:r * k].reshape(r, k).copy())


def encode(sysm: Systematic, msg: np.ndarray) -> np.ndarray:
    """Systematic encoding m^T G = p^T (Eq. 3): uint8 [F, k] -> uint8 [F, n]."""
    lib = _load()
    msg = np.ascontiguousarray(msg, dtype=np.uint8)
    F = msg.shape[0]
    cw = np.zeros((F, sysm.n), dtype=np.uint8)
    A = np.ascontiguousarray(sysm.A)
    lib.oracle_encode(sysm.n, sysm.k, _ptr(sysm.info_pos, ctypes.c_int32),
                      _ptr(sysm.parity_pos, ctypes.c_int32), _ptr(A, ctypes.c_uint8),
                      _ptr(msg, ctypes.c_uint8), F, _ptr(cw, ctypes.c_uint8))
    return cw


def syndrome(code, bits: np.ndarray) -> np.ndarray:
    """H z^T over GF(2) (Eq. 1): uint8 [F, n] -> uint8 [F, m]."""
    lib = _load()
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    F = bits.shape[0]
    syn = np.zeros((F, code.m), dtype=np.uint8)
    rp = np.ascontiguousarray(code.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(code.col_idx, dtype=np.int32)
    lib.oracle_syndrome(code.m, code.n, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                        _ptr(bits, ctypes.c_uint8), F, _ptr(syn, ctypes.c_uint8))
    return syn


@dataclass
class DecodeResult:
    post: np.ndarray   # float64 [F, n], total LLR L_v (Eq. 7) of the last iteration
    hard: np.ndarray   # uint8 [F, n], z_v (Eq. 8)
    iters: np.ndarray  # int32 [F]
    ok: np.ndarray     # uint8 [F], H z^T == 0


def decode(code, llr: np.ndarray, iters: int, early_stop: bool = False, clip: float = 20.0,
           weights: np.ndarray | None = None, nthreads: int = 1) -> DecodeResult:
    """Flooding sum-product decoding, FP64 (Sec. II-B, Eqs. 4-8).

    ``weights`` (T x E, CSR edge order) multiplies each check message in
    Eqs. 6 and 7 (weighted BP); None means all ones.
    """
    lib = _load()
    R = np.ascontiguousarray(llr, dtype=np.float64)
    F = R.shape[0]
    post = np.zeros((F, code.n), dtype=np.float64)
    hard = np.zeros((F, code.n), dtype=np.uint8)
    it = np.zeros(F, dtype=np.int32)
    ok = np.zeros(F, dtype=np.uint8)
    rp = np.ascontiguousarray(code.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(code.col_idx, dtype=np.int32)
    wp = None
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if w.shape != (iters, code.nnz):
            raise ValueError("weights must be T x E")
        wp = _ptr(w, ctypes.c_double)
    rc = lib.oracle_decode(code.m, code.n, _ptr(rp, ctypes.c_int32), _ptr(ci, ctypes.c_int32),
                           _ptr(R, ctypes.c_double), F, int(iters), int(bool(early_stop)),
                           float(clip), wp, _ptr(post, ctypes.c_double), _ptr(hard, ctypes.c_uint8),
                           _ptr(it, ctypes.c_int32), _ptr(ok, ctypes.c_uint8), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_decode failed ({rc})")
    return DecodeResult(post=post, hard=hard, iters=it, ok=ok)
