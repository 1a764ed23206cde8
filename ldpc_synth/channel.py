"""Seeded information bits, Gaussian noise and the BPSK/AWGN channel map.

Every frame draws from its own stream, ``SeedSequence([seed, frame])``, so a
sampled frame of a large batch can be regenerated alone on the host.

The channel follows Sec. III-B (BPSK: bit 0 -> -1, bit 1 -> +1) and Eq. 4
(input LLR 2y/sigma^2, read as ln p(1)/p(0); the printed equation lost its
logarithm).  sigma^2 = 1 / (2 R 10^(EbN0/10)) with R = k/n, the true rate.
"""

from __future__ import annotations

import numpy as np


def _frame_rng(seed: int, frame: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(frame)])))


def _frames(F: int, frames) -> np.ndarray:
    return np.arange(F) if frames is None else np.asarray(frames, dtype=np.int64)


def info_bits(F: int, k: int, seed: int, frames=None) -> np.ndarray:
    """Uniform information bits, uint8 [len(frames) or F, k]."""
    fr = _frames(F, frames)
    out = np.empty((fr.size, k), dtype=np.uint8)
    for i, f in enumerate(fr):
        out[i] = _frame_rng(seed, f).integers(0, 2, size=k, dtype=np.uint8)
    return out


def frame_noise(F: int, n: int, seed: int, frames=None) -> np.ndarray:
    """Standard normal noise, float32 [len(frames) or F, n]."""
    fr = _frames(F, frames)
    out = np.empty((fr.size, n), dtype=np.float32)
    for i, f in enumerate(fr):
        out[i] = _frame_rng(seed, f).standard_normal(n, dtype=np.float32)
    return out


def awgn_sigma2(ebn0_db, rate: float):
    """Noise variance for BPSK at the given Eb/N0 (dB) and code rate."""
    return 1.0 / (2.0 * rate * 10.0 ** (np.asarray(ebn0_db, dtype=np.float64) / 10.0))


def bpsk_awgn_llr(codeword_bits: np.ndarray, ebn0_db, rate: float,
                  noise: np.ndarray) -> np.ndarray:
    """Channel LLRs R_v = 2 y / sigma^2 with y = (2c - 1) + sigma * noise.

    ``ebn0_db`` is a scalar or one value per frame.  Returns float32 [F, n].
    """
    c = np.asarray(codeword_bits, dtype=np.float64)
    s2 = np.asarray(awgn_sigma2(ebn0_db, rate), dtype=np.float64)
    if s2.ndim == 1:
        s2 = s2[:, None]
    y = (2.0 * c - 1.0) + np.sqrt(s2) * noise.astype(np.float64)
    return (2.0 * y / s2).astype(np.float32)


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """Pack bits [F, L] into uint32 words [F, ceil(L/32)], LSB-first; pad bits 0."""
    bits = np.asarray(bits, dtype=np.uint8)
    F, L = bits.shape
    W = (L + 31) // 32
    padded = np.zeros((F, W * 32), dtype=np.uint8)
    padded[:, :L] = bits & 1
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    words = (padded.reshape(F, W, 32).astype(np.uint64) * weights).sum(axis=2)
    return words.astype(np.uint32)


def unpack_bits(words: np.ndarray, L: int) -> np.ndarray:
    """Inverse of ``pack_bits``: uint32 [F, W] -> uint8 [F, L]."""
    words = np.asarray(words, dtype=np.uint32)
    F, W = words.shape
    sh = np.arange(32, dtype=np.uint32)
    bits = ((words[:, :, None] >> sh) & 1).astype(np.uint8).reshape(F, W * 32)
    return bits[:, :L]
