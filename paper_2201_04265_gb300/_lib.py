"""ctypes loader for libldpc.so (the C ABI declared in include/ldpc.h).

There is no fallback: if the library has not been built the import fails.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libldpc.so")

c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_u32 = ctypes.c_uint32
c_f32 = ctypes.c_float
c_vp = ctypes.c_void_p
c_size = ctypes.c_size_t

NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024  # LDPC_NOALLOC_SCRATCH_BYTES in include/ldpc.h


class LdpcError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {message} (status {status})")
        self.status = status


class QcDesc(ctypes.Structure):
    _fields_ = [("mb", c_i32), ("nb", c_i32), ("z", c_i32), ("shift", ctypes.POINTER(ctypes.c_int16))]


class MixedConfig(ctypes.Structure):
    _fields_ = [("order", c_i32), ("groups_per_item", c_i32), ("ctas_per_sm", c_i32)]


class DecodeOpts(ctypes.Structure):
    _fields_ = [("max_iters", c_i32), ("early_stop", c_i32), ("msg_fp16", c_i32),
                ("schedule", c_i32), ("clip", c_f32)]


# (name, restype, argtypes) of every exported symbol
SIGNATURES = {
    "ldpc_probe_xu_rates": (c_i32, [ctypes.POINTER(ctypes.c_float)]),
    "ldpc_code_create": (c_i32, [c_i32, c_i32, c_vp, c_vp, ctypes.POINTER(QcDesc), c_u32,
                                 ctypes.POINTER(c_vp)]),
    "ldpc_code_info": (c_i32, [c_vp, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32),
                               ctypes.POINTER(c_i32), ctypes.POINTER(c_i32), ctypes.POINTER(c_i64)]),
    "ldpc_code_positions": (c_i32, [c_vp, c_vp, c_vp]),
    "ldpc_code_parity_map": (c_i32, [c_vp, c_vp]),
    "ldpc_code_schedule": (c_i32, [c_vp, c_vp, ctypes.POINTER(c_i64)]),
    "ldpc_test_fail_allocation": (c_i32, [c_i32]),
    "ldpc_code_cluster_shape": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32),
                                        ctypes.POINTER(ctypes.c_float)]),
    "ldpc_code_destroy": (None, [c_vp]),
    "ldpc_encode": (c_i32, [c_vp, c_vp, c_vp, c_i32, c_vp]),
    "ldpc_encode_tables_build": (c_i32, [c_vp, ctypes.POINTER(c_size)]),
    "ldpc_encode_tables_free": (c_i32, [c_vp]),
    "ldpc_syndrome": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp, c_vp]),
    "ldpc_decode_workspace_size": (c_i32, [c_vp, c_i32, ctypes.POINTER(DecodeOpts),
                                           ctypes.POINTER(c_size)]),
    "ldpc_decode": (c_i32, [c_vp, c_vp, c_i32, ctypes.POINTER(DecodeOpts), c_vp, c_vp, c_vp, c_vp,
                            c_vp, c_size, c_vp]),
    "ldpc_decode_noalloc": (c_i32, [c_vp, c_vp, c_i32, ctypes.POINTER(DecodeOpts), c_vp, c_vp, c_vp, c_vp,
                                    c_vp]),
    "ldpc_wbp_checkpoint_size": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_size)]),
    "ldpc_wbp_forward": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_vp, c_f32, c_vp, c_vp, c_size, c_vp]),
    "ldpc_decode_backward_workspace_size": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_size)]),
    "ldpc_decode_backward": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_f32, c_vp, c_size, c_vp, c_vp, c_vp, c_vp,
                                     c_size, c_vp]),
    "ldpc_decode_host_workspace_size": (c_i32, [c_vp, c_i32, ctypes.POINTER(DecodeOpts), ctypes.POINTER(c_size)]),
    "ldpc_decode_host": (c_i32, [c_vp, c_vp, c_i32, ctypes.POINTER(DecodeOpts), c_vp, c_vp, c_vp, c_vp, c_i32,
                                 c_vp, c_size, c_vp]),
    "ldpc_decode_host_timeline": (c_i32, [c_vp, c_vp, c_i32, ctypes.POINTER(DecodeOpts), c_vp, c_vp, c_vp, c_vp,
                                          c_i32, c_vp, c_size, c_vp, c_vp]),
    "ldpc_mixed_create": (c_i32, [ctypes.POINTER(c_vp), c_i32, c_i32, ctypes.POINTER(c_vp)]),
    "ldpc_mixed_destroy": (None, [c_vp]),
    "ldpc_mixed_workspace_size": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_size)]),
    "ldpc_mixed_get_config": (c_i32, [c_vp, ctypes.POINTER(MixedConfig)]),
    "ldpc_mixed_set_config": (c_i32, [c_vp, ctypes.POINTER(MixedConfig)]),
    "ldpc_decode_mixed": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_i32, c_f32, c_vp, c_vp, c_vp,
                                  c_vp, c_vp, c_size, c_vp]),
    "ldpc_mixed_autotune": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_i32, c_f32, c_vp, c_vp, c_vp,
                                    c_vp, c_vp, c_size, c_i32, c_vp, ctypes.POINTER(MixedConfig)]),
    "ldpc_status_string": (ctypes.c_char_p, [c_i32]),
    "ldpc_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run `python -c \"import __graft_entry__ as g; "
                              f"g.build()\"` (needs nvcc)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, where: str) -> None:
    if status != 0:
        lib = load()
        msg = lib.ldpc_last_error().decode(errors="replace") or lib.ldpc_status_string(status).decode()
        raise LdpcError(status, where, msg)
