"""Brute-force references on tiny codes (test infrastructure).

These enumerate all 2^n words, so they are only for n <= 20.  They define
what sum-product decoding approximates (Sec. II-B): with channel LLRs
R_u = ln p(y_u|1)/p(y_u|0) (Eq. 4) and equiprobable codewords,
p(c | y) is proportional to exp(sum_u c_u R_u) over the codewords of H
(Eq. 1), which gives the bitwise MAP LLR and the block ML decision below.
"""

from __future__ import annotations

import numpy as np


def all_words(n: int) -> np.ndarray:
    if n > 20:
        raise ValueError("brute force limited to n <= 20")
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> np.arange(n)) & 1).astype(np.uint8)


def codewords(h_dense: np.ndarray) -> np.ndarray:
    """All c with H c^T = 0 over GF(2) (Eq. 1)."""
    h = np.asarray(h_dense, dtype=np.int64)
    words = all_words(h.shape[1])
    syn = (words.astype(np.int64) @ h.T) % 2
    return words[np.all(syn == 0, axis=1)]


def rank_gf2(h_dense: np.ndarray) -> int:
    """GF(2) rank by left-to-right elimination on Python integers (an
    independent second elimination, with the opposite pivot order)."""
    rows = [int("".join(str(int(b)) for b in r[::-1]), 2) for r in np.asarray(h_dense)]
    rank = 0
    n = np.asarray(h_dense).shape[1]
    for col in range(n):
        bit = 1 << col
        piv = next((i for i in range(rank, len(rows)) if rows[i] & bit), None)
        if piv is None:
            continue
        rows[rank], rows[piv] = rows[piv], rows[rank]
        for i in range(len(rows)):
            if i != rank and rows[i] & bit:
                rows[i] ^= rows[rank]
        rank += 1
    return rank


def _logsumexp(a: np.ndarray, axis: int) -> np.ndarray:
    mx = np.max(a, axis=axis, keepdims=True)
    return (mx + np.log(np.sum(np.exp(a - mx), axis=axis, keepdims=True))).squeeze(axis)


def bitwise_map_llr(h_dense: np.ndarray, R: np.ndarray) -> np.ndarray:
    """ln P(c_v = 1 | y) - ln P(c_v = 0 | y) for every bit; R is [F, n]."""
    cws = codewords(h_dense).astype(np.float64)  # [C, n]
    R = np.atleast_2d(np.asarray(R, dtype=np.float64))
    score = R @ cws.T  # [F, C]
    out = np.empty_like(R)
    for v in range(R.shape[1]):
        one = cws[:, v] == 1
        out[:, v] = _logsumexp(score[:, one], 1) - _logsumexp(score[:, ~one], 1)
    return out


def block_ml(h_dense: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Maximum-likelihood codeword argmax_c sum_v c_v R_v, [F, n] uint8."""
    cws = codewords(h_dense)
    R = np.atleast_2d(np.asarray(R, dtype=np.float64))
    return cws[np.argmax(R @ cws.T.astype(np.float64), axis=1)]
