"""Shared helpers for the GPU-vs-oracle parity tests.

Inputs come from ldpc_synth (seeded) and the oracle's encoder; nothing here
takes a value from the CUDA path.
"""

from __future__ import annotations

import functools
from dataclasses import dataclass

import numpy as np

import ldpc_synth as S
import oracle

CLIP = 20.0
RTOL = 1e-4   # posterior tolerance: 1e-4 relative or 1e-3 absolute,
ATOL = 1e-3   # after clipping both sides to |L| <= 20
HARD_EPS = 1e-3  # hard decisions may differ only where the oracle's |L| < this


@dataclass
class Workload:
    code: S.Code
    sysm: oracle.Systematic
    msgs: np.ndarray  # uint8 [F, k]
    cw: np.ndarray    # uint8 [F, n]
    llr: np.ndarray   # float32 [F, n]


CODES = {
    "c1_gallager_504": lambda: S.gallager_regular(504, 3, 6, seed=1),
    "reg39_1008": lambda: S.random_regular(1008, 3, 9, seed=41),
    "reg312_2016": lambda: S.random_regular(2016, 3, 12, seed=42),
    "reg36_1008": lambda: S.random_regular(1008, 3, 6, seed=5),
    "table1_r025": lambda: S.table1_code(0.25, seed=6),
    "table1_r050": lambda: S.table1_code(0.5, seed=6),
    "table1_r075": lambda: S.table1_code(0.75, seed=6),
    "irregular_37x70": lambda: S.dense_to_code(
        np.random.default_rng(5).integers(0, 2, (37, 70), dtype=np.uint8)),
    "qc_small": lambda: S.qc_expand(S.qc_base_matrix(8, 12, 40, 3, 8, 24, seed=3), 24),
    # irregular (rows of 3..7 ones, columns of 1..4) and small enough to decode on chip
    "qc_irregular_512": lambda: S.qc_expand(S.qc_base_matrix(8, 16, 40, 3, 8, 32, seed=2), 32),
    "c2_random_8064": lambda: S.random_regular(8064, 3, 6, seed=2),
}


@functools.lru_cache(maxsize=None)
def code_and_sys(name: str):
    code = CODES[name]()
    return code, oracle.systematic(code)


def workload(name: str, F: int, ebn0: float, seed: int) -> Workload:
    code, sysm = code_and_sys(name)
    msgs = S.info_bits(F, sysm.k, seed)
    cw = oracle.encode(sysm, msgs)
    llr = S.bpsk_awgn_llr(cw, ebn0, sysm.k / code.n, S.frame_noise(F, code.n, seed + 1))
    return Workload(code, sysm, msgs, cw, llr)


def llr_close(gpu_post: np.ndarray, ora_post: np.ndarray) -> np.ndarray:
    """Elementwise: |g - o| <= max(ATOL, RTOL |o|) after clipping both to +-CLIP."""
    g = np.clip(gpu_post.astype(np.float64), -CLIP, CLIP)
    o = np.clip(ora_post, -CLIP, CLIP)
    return np.abs(g - o) <= np.maximum(ATOL, RTOL * np.abs(o))


def hard_close(gpu_hard: np.ndarray, ora_hard: np.ndarray, ora_post: np.ndarray) -> np.ndarray:
    return (gpu_hard == ora_hard) | (np.abs(ora_post) < HARD_EPS)


def fp32_conditioned_frames(code, llr, iters, early_stop=False, seed=0):
    """Frames whose FP64 decode is stable under an FP32-rounding-sized input
    perturbation (relative 2^-23 per LLR): on those, FP32 arithmetic is expected
    to stay within tolerance; on the others BP itself amplifies rounding beyond
    it, so no single-precision decoder can be held to the FP64 values."""
    rng = np.random.default_rng(seed)
    pert = llr.astype(np.float64) * (1.0 + rng.choice([-1.0, 1.0], size=llr.shape) * 2.0 ** -23)
    a = oracle.decode(code, llr, iters=iters, early_stop=early_stop)
    b = oracle.decode(code, pert, iters=iters, early_stop=early_stop)
    g = np.clip(b.post, -CLIP, CLIP)
    o = np.clip(a.post, -CLIP, CLIP)
    stable = np.all(np.abs(g - o) <= 0.1 * np.maximum(ATOL, RTOL * np.abs(o)), axis=1)
    stable &= (a.iters == b.iters)
    return stable, a
