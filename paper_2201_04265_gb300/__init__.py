"""LDPC encoding and sum-product decoding on GB300 (arXiv 2201.04265, Secs. II-III).

Thin Python binding over libldpc.so: every step of encoding and decoding runs
in the library's CUDA kernels; this module only marshals torch tensors
(device memory and streams) into the C ABI of include/ldpc.h.

Packed bit tensors use dtype torch.int32 (the bit pattern of the ABI's
uint32 words, LSB first).
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import DecodeOpts, LdpcError, QcDesc, c_i32, c_i64, c_size, c_vp

SCHED_AUTO, SCHED_PLAIN, SCHED_RESIDENT, SCHED_CLUSTER = 0, 1, 2, 3
_SCHED = {"auto": SCHED_AUTO, "plain": SCHED_PLAIN, "resident": SCHED_RESIDENT, "cluster": SCHED_CLUSTER}

__all__ = ["Code", "encode", "syndrome", "decode", "decode_noalloc", "decode_workspace_size", "DecodeResult",
           "WeightedBP", "weighted_bp", "MixedPlan", "MixedBatch", "HostDecoder",
           "LdpcError", "SCHED_AUTO", "SCHED_PLAIN", "SCHED_RESIDENT", "SCHED_CLUSTER"]


def _stream_handle(stream) -> c_vp:
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_vp(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> c_vp:
    if t is None:
        return c_vp(None)
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return c_vp(t.data_ptr())


class Code:
    """A code object owned by the library (Eq. 2 generator and Tanner-graph layouts).

    ``Code(n, m, row_ptr, col_idx)`` takes H in CSR form (host arrays), or
    ``Code.from_qc(base, z)`` a quasi-cyclic base matrix.  The object lives on
    the CUDA device current at creation unless ``host_only``.
    """

    def __init__(self, n: int, m: int, row_ptr=None, col_idx=None, *, qc=None,
                 host_only: bool = False):
        lib = _lib.load()
        self._lib = lib
        self._h = c_vp(None)
        self._keep = []
        if qc is not None:
            base, z = qc
            base = np.ascontiguousarray(base, dtype=np.int16)
            desc = QcDesc(base.shape[0], base.shape[1], int(z),
                          base.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)))
            self._keep.append(base)
            st = lib.ldpc_code_create(int(n), int(m), None, None, ctypes.byref(desc),
                                      1 if host_only else 0, ctypes.byref(self._h))
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            ci = np.ascontiguousarray(col_idx, dtype=np.int32)
            st = lib.ldpc_code_create(int(n), int(m), c_vp(rp.ctypes.data), c_vp(ci.ctypes.data),
                                      None, 1 if host_only else 0, ctypes.byref(self._h))
        _lib.check(st, "ldpc_code_create")
        n_, m_, k_, r_ = c_i32(), c_i32(), c_i32(), c_i32()
        nnz = c_i64()
        _lib.check(lib.ldpc_code_info(self._h, ctypes.byref(n_), ctypes.byref(m_), ctypes.byref(k_),
                                      ctypes.byref(r_), ctypes.byref(nnz)), "ldpc_code_info")
        self.n, self.m, self.k, self.rank, self.nnz = n_.value, m_.value, k_.value, r_.value, nnz.value
        self.host_only = host_only
        self.device = None if host_only else torch.cuda.current_device()

    @classmethod
    def from_csr_code(cls, code, host_only: bool = False) -> "Code":
        """From any object with n, m, row_ptr, col_idx attributes."""
        return cls(code.n, code.m, code.row_ptr, code.col_idx, host_only=host_only)

    @classmethod
    def from_qc(cls, base, z: int, host_only: bool = False) -> "Code":
        base = np.asarray(base)
        return cls(base.shape[1] * z, base.shape[0] * z, qc=(base, z), host_only=host_only)

    @property
    def handle(self) -> c_vp:
        if not self._h:
            raise ValueError("code is closed")
        return self._h

    @property
    def KW(self) -> int:
        return (self.k + 31) // 32

    @property
    def NW(self) -> int:
        return (self.n + 31) // 32

    def positions(self) -> tuple[np.ndarray, np.ndarray]:
        info = np.zeros(max(self.k, 1), dtype=np.int32)
        par = np.zeros(max(self.rank, 1), dtype=np.int32)
        _lib.check(self._lib.ldpc_code_positions(self.handle, c_vp(info.ctypes.data),
                                                 c_vp(par.ctypes.data)), "ldpc_code_positions")
        return info[:self.k], par[:self.rank]

    def parity_map(self) -> np.ndarray:
        """A = P^T as uint32 [rank, KW]."""
        a = np.zeros((max(self.rank, 1), self.KW), dtype=np.uint32)
        _lib.check(self._lib.ldpc_code_parity_map(self.handle, c_vp(a.ctypes.data)), "ldpc_code_parity_map")
        return a[:self.rank]

    def build_encode_tables(self) -> int:
        """Builds the Four-Russians encoding tables on the device (synchronous);
        `encode` uses them from then on, with the same result bits.  Returns
        the device bytes they hold."""
        nbytes = c_size()
        _lib.check(self._lib.ldpc_encode_tables_build(self.handle, ctypes.byref(nbytes)),
                   "ldpc_encode_tables_build")
        return nbytes.value

    def free_encode_tables(self) -> None:
        _lib.check(self._lib.ldpc_encode_tables_free(self.handle), "ldpc_encode_tables_free")

    def schedule(self) -> tuple[np.ndarray, int]:
        """(evaluation order as CSR edge ids per row, edges not placed conflict-free)."""
        order = np.zeros(max(self.nnz, 1), dtype=np.int32)
        unplaced = c_i64()
        _lib.check(self._lib.ldpc_code_schedule(self.handle, c_vp(order.ctypes.data), ctypes.byref(unplaced)),
                   "ldpc_code_schedule")
        return order[:self.nnz], unplaced.value

    def cluster_shape(self, msg_fp16: bool) -> tuple[int, int]:
        """(CTAs per cluster, frames per group) of the cluster schedule; (0, 0) if none."""
        return self.cluster_layout(msg_fp16)[:2]

    def cluster_layout(self, msg_fp16: bool) -> tuple[int, int, float]:
        """(CTAs per cluster, frames per group, share of base entries kept inside one CTA)."""
        ctas, group, local = c_i32(), c_i32(), ctypes.c_float()
        _lib.check(self._lib.ldpc_code_cluster_shape(self.handle, int(bool(msg_fp16)), ctypes.byref(ctas),
                                                     ctypes.byref(group), ctypes.byref(local)),
                   "ldpc_code_cluster_shape")
        return ctas.value, group.value, float(local.value)

    def close(self) -> None:
        if self._h:
            self._lib.ldpc_code_destroy(self._h)
            self._h = c_vp(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_dev(t: torch.Tensor, name: str, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def encode(code: Code, info_words: torch.Tensor, out: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """Systematic encoding (Eq. 3): int32 [F, KW] packed info -> int32 [F, NW] codewords."""
    F = info_words.shape[0]
    _check_dev(info_words, "info_words", torch.int32, (F, code.KW))
    if out is None:
        out = torch.empty((F, code.NW), dtype=torch.int32, device=info_words.device)
    _check_dev(out, "out", torch.int32, (F, code.NW))
    _lib.check(code._lib.ldpc_encode(code.handle, _ptr(info_words), _ptr(out), F,
                                     _stream_handle(stream)), "ldpc_encode")
    return out


def syndrome(code: Code, bits: torch.Tensor, want_syn: bool = True, stream=None):
    """H z^T (Eq. 1) of packed words [F, NW] -> (int32 [F, ceil(m/32)] or None, uint8 [F])."""
    F = bits.shape[0]
    _check_dev(bits, "bits", torch.int32, (F, code.NW))
    syn = torch.empty((F, (code.m + 31) // 32), dtype=torch.int32, device=bits.device) if want_syn else None
    ok = torch.empty((F,), dtype=torch.uint8, device=bits.device)
    _lib.check(code._lib.ldpc_syndrome(code.handle, _ptr(bits), F, _ptr(syn), _ptr(ok),
                                       _stream_handle(stream)), "ldpc_syndrome")
    return syn, ok


def _opts(max_iters, early_stop, msg_fp16, schedule, clip) -> DecodeOpts:
    sched = _SCHED[schedule] if isinstance(schedule, str) else int(schedule)
    return DecodeOpts(int(max_iters), int(bool(early_stop)), int(bool(msg_fp16)), sched, float(clip))


def decode_workspace_size(code: Code, F: int, max_iters: int = 20, early_stop: bool = False,
                          msg_fp16: bool = False, schedule="auto", clip: float = 20.0) -> int:
    o = _opts(max_iters, early_stop, msg_fp16, schedule, clip)
    nbytes = ctypes.c_size_t()
    _lib.check(code._lib.ldpc_decode_workspace_size(code.handle, int(F), ctypes.byref(o),
                                                    ctypes.byref(nbytes)), "ldpc_decode_workspace_size")
    return nbytes.value


@dataclass
class DecodeResult:
    post: torch.Tensor | None  # float32 [F, n]
    hard: torch.Tensor         # int32 [F, NW]
    iters: torch.Tensor        # int32 [F]
    ok: torch.Tensor           # uint8 [F]


def _workspace(nbytes: int, device, workspace: torch.Tensor | None) -> torch.Tensor:
    if workspace is not None and workspace.numel() >= nbytes:
        ws = workspace
    else:
        ws = torch.empty((max(nbytes, 256),), dtype=torch.uint8, device=device)
    if ws.data_ptr() % 256:
        raise ValueError("workspace must be 256-byte aligned")
    return ws


def decode(code: Code, llr: torch.Tensor, max_iters: int = 20, early_stop: bool = False,
           msg_fp16: bool = False, schedule="auto", clip: float = 20.0, want_post: bool = True,
           workspace: torch.Tensor | None = None, out: DecodeResult | None = None,
           stream=None) -> DecodeResult:
    """Sum-product decoding (Eqs. 4-8) of float32 LLRs [F, n] on the GPU."""
    F = llr.shape[0]
    _check_dev(llr, "llr", torch.float32, (F, code.n))
    dev = llr.device
    o = _opts(max_iters, early_stop, msg_fp16, schedule, clip)
    nbytes = ctypes.c_size_t()
    _lib.check(code._lib.ldpc_decode_workspace_size(code.handle, F, ctypes.byref(o),
                                                    ctypes.byref(nbytes)), "ldpc_decode_workspace_size")
    ws = _workspace(nbytes.value, dev, workspace)
    if out is None:
        out = DecodeResult(
            post=torch.empty((F, code.n), dtype=torch.float32, device=dev) if want_post else None,
            hard=torch.empty((F, code.NW), dtype=torch.int32, device=dev),
            iters=torch.empty((F,), dtype=torch.int32, device=dev),
            ok=torch.empty((F,), dtype=torch.uint8, device=dev))
    _lib.check(code._lib.ldpc_decode(code.handle, _ptr(llr), F, ctypes.byref(o), _ptr(out.post),
                                     _ptr(out.hard), _ptr(out.iters), _ptr(out.ok), _ptr(ws),
                                     ws.numel(), _stream_handle(stream)), "ldpc_decode")
    return out


def decode_noalloc(code: Code, llr: torch.Tensor, max_iters: int = 20, early_stop: bool = False,
                   msg_fp16: bool = False, clip: float = 20.0, out: DecodeResult | None = None,
                   want_post: bool = True, stream=None) -> DecodeResult:
    """Plain-schedule decoding whose scratch is the library's static device array.

    For callers that must not allocate device memory while decoding: the
    library allocates nothing (pass ``out`` to make this wrapper allocate
    nothing either).  Batches whose scratch need exceeds the array's
    NOALLOC_SCRATCH_BYTES are rejected; concurrent calls must be serialised.
    """
    F = llr.shape[0]
    _check_dev(llr, "llr", torch.float32, (F, code.n))
    o = _opts(max_iters, early_stop, msg_fp16, SCHED_PLAIN, clip)
    if out is None:
        dev = llr.device
        out = DecodeResult(
            post=torch.empty((F, code.n), dtype=torch.float32, device=dev) if want_post else None,
            hard=torch.empty((F, code.NW), dtype=torch.int32, device=dev),
            iters=torch.empty((F,), dtype=torch.int32, device=dev),
            ok=torch.empty((F,), dtype=torch.uint8, device=dev))
    _lib.check(code._lib.ldpc_decode_noalloc(code.handle, _ptr(llr), F, ctypes.byref(o), _ptr(out.post),
                                             _ptr(out.hard), _ptr(out.iters), _ptr(out.ok),
                                             _stream_handle(stream)), "ldpc_decode_noalloc")
    return out


def probe_xu_rates() -> tuple[float, float, float]:
    """Results per SM per clock of ex2.approx, rcp.approx and lg2.approx on the
    current device (a measurement aid for the decoder's ALU roofline)."""
    lib = _lib.load()
    rates = (ctypes.c_float * 3)()
    _lib.check(lib.ldpc_probe_xu_rates(rates), "ldpc_probe_xu_rates")
    return float(rates[0]), float(rates[1]), float(rates[2])


class WeightedBP(torch.autograd.Function):
    """Weighted belief propagation with the library's hand-written adjoint.

    ``WeightedBP.apply(llr, w, code, clip)``: llr float32 [F, n], w float32
    [T, nnz] (one weight per edge and iteration, CSR edge order) -> total
    LLRs after T iterations, float32 [F, n].  The forward keeps every
    iteration's messages (checkpoints) for the backward pass, which returns
    the gradients with respect to llr and w.
    """

    @staticmethod
    def forward(ctx, llr, w, code, clip=20.0):
        F = llr.shape[0]
        T = w.shape[0]
        _check_dev(llr, "llr", torch.float32, (F, code.n))
        _check_dev(w, "w", torch.float32, (T, code.nnz))
        nb = ctypes.c_size_t()
        _lib.check(code._lib.ldpc_wbp_checkpoint_size(code.handle, F, T, ctypes.byref(nb)),
                   "ldpc_wbp_checkpoint_size")
        ckpt = _workspace(nb.value, llr.device, None)
        post = torch.empty((F, code.n), dtype=torch.float32, device=llr.device)
        _lib.check(code._lib.ldpc_wbp_forward(code.handle, _ptr(llr), F, T, _ptr(w), float(clip), _ptr(post),
                                              _ptr(ckpt), ckpt.numel(), _stream_handle(None)),
                   "ldpc_wbp_forward")
        ctx.save_for_backward(w)
        ctx.ckpt, ctx.code, ctx.clip, ctx.F = ckpt, code, float(clip), F
        return post

    @staticmethod
    def backward(ctx, grad_post):
        (w,) = ctx.saved_tensors
        code, F, T = ctx.code, ctx.F, w.shape[0]
        grad_post = grad_post.contiguous().to(torch.float32)
        nb = ctypes.c_size_t()
        _lib.check(code._lib.ldpc_decode_backward_workspace_size(code.handle, F, T, ctypes.byref(nb)),
                   "ldpc_decode_backward_workspace_size")
        work = _workspace(nb.value, w.device, None)
        grad_w = torch.empty_like(w)
        grad_llr = torch.empty((F, code.n), dtype=torch.float32, device=w.device) \
            if ctx.needs_input_grad[0] else None
        _lib.check(code._lib.ldpc_decode_backward(code.handle, F, T, _ptr(w), ctx.clip, _ptr(ctx.ckpt),
                                                  ctx.ckpt.numel(), _ptr(grad_post), _ptr(grad_w),
                                                  _ptr(grad_llr), _ptr(work), work.numel(),
                                                  _stream_handle(None)), "ldpc_decode_backward")
        return grad_llr, grad_w, None, None


def weighted_bp(code: Code, llr: torch.Tensor, w: torch.Tensor, clip: float = 20.0) -> torch.Tensor:
    """Total LLRs after ``w.shape[0]`` weighted iterations, differentiable in llr and w."""
    return WeightedBP.apply(llr, w, code, clip)


@dataclass
class MixedBatch:
    """Device-side description of a mixed-code batch (see MixedPlan.batch)."""
    frame_code: torch.Tensor  # int32 [F]
    llr_off: torch.Tensor     # int64 [F], element offset of each frame's LLRs (and posterior)
    hard_off: torch.Tensor    # int64 [F], word offset of each frame's hard decisions
    n_llr: int                # total LLR elements
    n_hard: int               # total hard-decision words


class MixedPlan:
    """Several codes decoded in one persistent launch (ldpc_mixed_* in the C ABI)."""

    def __init__(self, codes, msg_fp16: bool = True):
        self._lib = _lib.load()
        self.codes = list(codes)
        arr = (c_vp * len(self.codes))(*[c.handle.value for c in self.codes])
        self._h = c_vp(None)
        _lib.check(self._lib.ldpc_mixed_create(arr, len(self.codes), int(bool(msg_fp16)), ctypes.byref(self._h)),
                   "ldpc_mixed_create")

    def close(self):
        if self._h:
            self._lib.ldpc_mixed_destroy(self._h)
            self._h = c_vp(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def batch(self, frame_code, device="cuda") -> MixedBatch:
        """Offsets for frames laid out back to back in frame order."""
        fc = np.asarray(frame_code, dtype=np.int32)
        ns = np.array([self.codes[c].n for c in fc], dtype=np.int64)
        nws = (ns + 31) // 32
        llr_off = np.concatenate([[0], np.cumsum(ns)[:-1]]) if len(fc) else np.zeros(0, np.int64)
        hard_off = np.concatenate([[0], np.cumsum(nws)[:-1]]) if len(fc) else np.zeros(0, np.int64)
        return MixedBatch(torch.from_numpy(fc).to(device), torch.from_numpy(llr_off.astype(np.int64)).to(device),
                          torch.from_numpy(hard_off.astype(np.int64)).to(device), int(ns.sum()), int(nws.sum()))

    def config(self) -> dict:
        cfg = _lib.MixedConfig()
        _lib.check(self._lib.ldpc_mixed_get_config(self._h, ctypes.byref(cfg)), "ldpc_mixed_get_config")
        return {"order": cfg.order, "groups_per_item": cfg.groups_per_item, "ctas_per_sm": cfg.ctas_per_sm}

    def set_config(self, order: int = 0, groups_per_item: int = 1, ctas_per_sm: int = 1) -> None:
        cfg = _lib.MixedConfig(order, groups_per_item, ctas_per_sm)
        _lib.check(self._lib.ldpc_mixed_set_config(self._h, ctypes.byref(cfg)), "ldpc_mixed_set_config")

    def workspace(self, F: int, device="cuda") -> torch.Tensor:
        nb = ctypes.c_size_t()
        _lib.check(self._lib.ldpc_mixed_workspace_size(self._h, int(F), ctypes.byref(nb)), "ldpc_mixed_workspace_size")
        return _workspace(nb.value, device, None)

    def outputs(self, b: MixedBatch, want_post: bool = True, device="cuda") -> DecodeResult:
        F = b.frame_code.shape[0]
        return DecodeResult(
            post=torch.empty((b.n_llr,), dtype=torch.float32, device=device) if want_post else None,
            hard=torch.empty((b.n_hard,), dtype=torch.int32, device=device),
            iters=torch.empty((F,), dtype=torch.int32, device=device),
            ok=torch.empty((F,), dtype=torch.uint8, device=device))

    def _args(self, b, llr, max_iters, early_stop, clip, out, ws):
        return (self._h, _ptr(b.frame_code), _ptr(b.llr_off), _ptr(b.hard_off), _ptr(llr), b.frame_code.shape[0],
                int(max_iters), int(bool(early_stop)), float(clip), _ptr(out.post), _ptr(out.hard),
                _ptr(out.iters), _ptr(out.ok), _ptr(ws), ws.numel())

    def decode(self, b: MixedBatch, llr: torch.Tensor, max_iters: int = 50, early_stop: bool = True,
               clip: float = 20.0, out: DecodeResult | None = None, workspace: torch.Tensor | None = None,
               stream=None) -> DecodeResult:
        """Decodes the batch; with ``out`` and ``workspace`` given it queues device
        work only (memsets and kernels), so it can be captured in a CUDA graph."""
        _check_dev(llr, "llr", torch.float32, (b.n_llr,))
        out = out if out is not None else self.outputs(b, device=llr.device)
        ws = workspace if workspace is not None else self.workspace(b.frame_code.shape[0], llr.device)
        _lib.check(self._lib.ldpc_decode_mixed(*self._args(b, llr, max_iters, early_stop, clip, out, ws),
                                               _stream_handle(stream)), "ldpc_decode_mixed")
        return out

    def autotune(self, b: MixedBatch, llr: torch.Tensor, max_iters: int = 50, early_stop: bool = True,
                 clip: float = 20.0, reps: int = 3, stream=None) -> dict:
        out = self.outputs(b, device=llr.device)
        ws = self.workspace(b.frame_code.shape[0], llr.device)
        cfg = _lib.MixedConfig()
        _lib.check(self._lib.ldpc_mixed_autotune(*self._args(b, llr, max_iters, early_stop, clip, out, ws),
                                                 int(reps), _stream_handle(stream), ctypes.byref(cfg)),
                   "ldpc_mixed_autotune")
        return {"order": cfg.order, "groups_per_item": cfg.groups_per_item, "ctas_per_sm": cfg.ctas_per_sm}


class HostDecoder:
    """Decodes batches held in host memory, overlapping the copies with decoding
    (ldpc_decode_host): chunk i is copied in while chunk i-1 is decoded and each
    chunk's results are copied out as soon as they are ready."""

    def __init__(self, code: Code, chunk: int = 8192, max_iters: int = 50, early_stop: bool = False,
                 msg_fp16: bool = True, schedule="auto", clip: float = 20.0, device="cuda"):
        self.code, self.chunk = code, int(chunk)
        self.opts = _opts(max_iters, early_stop, msg_fp16, schedule, clip)
        nb = ctypes.c_size_t()
        _lib.check(code._lib.ldpc_decode_host_workspace_size(code.handle, self.chunk, ctypes.byref(self.opts),
                                                             ctypes.byref(nb)), "ldpc_decode_host_workspace_size")
        self.work = _workspace(nb.value, device, None)

    def outputs(self, F: int, want_post: bool = False, want_hard: bool = True) -> DecodeResult:
        """Page-locked host tensors for the results of F frames."""
        return DecodeResult(
            post=torch.empty((F, self.code.n), dtype=torch.float32, pin_memory=True) if want_post else None,
            hard=torch.empty((F, self.code.NW), dtype=torch.int32, pin_memory=True) if want_hard else None,
            iters=torch.empty((F,), dtype=torch.int32, pin_memory=True),
            ok=torch.empty((F,), dtype=torch.uint8, pin_memory=True))

    def decode(self, llr: torch.Tensor, out: DecodeResult | None = None, stream=None) -> DecodeResult:
        """llr: float32 [F, n] on the host (page-locked for overlap).  The results
        are in ``out`` once the stream has finished (synchronise it first)."""
        if llr.is_cuda or llr.dtype != torch.float32 or not llr.is_contiguous() or llr.shape[1] != self.code.n:
            raise ValueError("llr must be a contiguous float32 host tensor [F, n]")
        F = llr.shape[0]
        out = out if out is not None else self.outputs(F)
        _lib.check(self.code._lib.ldpc_decode_host(self.code.handle, c_vp(llr.data_ptr()), F, ctypes.byref(self.opts),
                                                   _ptr(out.post), _ptr(out.hard), _ptr(out.iters), _ptr(out.ok),
                                                   self.chunk, _ptr(self.work), self.work.numel(),
                                                   _stream_handle(stream)), "ldpc_decode_host")
        return out

    def decode_timeline(self, llr: torch.Tensor, out: DecodeResult | None = None,
                        stream=None) -> tuple[DecodeResult, np.ndarray]:
        """As ``decode``, synchronised, with a record of every chunk: float [chunks, 6]
        of milliseconds from the call's start (upload start/end, decode start/end,
        download start/end)."""
        if llr.is_cuda or llr.dtype != torch.float32 or not llr.is_contiguous() or llr.shape[1] != self.code.n:
            raise ValueError("llr must be a contiguous float32 host tensor [F, n]")
        F = llr.shape[0]
        out = out if out is not None else self.outputs(F)
        ms = np.zeros(((F + self.chunk - 1) // self.chunk, 6), dtype=np.float32)
        _lib.check(self.code._lib.ldpc_decode_host_timeline(
            self.code.handle, c_vp(llr.data_ptr()), F, ctypes.byref(self.opts), _ptr(out.post), _ptr(out.hard),
            _ptr(out.iters), _ptr(out.ok), self.chunk, _ptr(self.work), self.work.numel(), _stream_handle(stream),
            c_vp(ms.ctypes.data)), "ldpc_decode_host_timeline")
        return out, ms
