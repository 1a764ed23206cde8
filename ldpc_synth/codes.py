"""Parity-check matrices H built from a seed (inputs to code creation).

Conventions: H is m x n (m checks, n bits; the paper's text prints the shape
garbled as k x (n-k), Sec. II).  Rows are returned in CSR form with the
column indices of each row sorted ascending; the position of an entry in
that CSR order is its *edge index*, the order in which per-edge weights are
given to weighted BP.

Constructions (none of them is spelled out in the paper, which only names
Gallager's construction in Sec. IV; each reading is stated in the function):

* ``gallager_regular`` -- Gallager's banded construction, Sec. IV / Table I.
* ``random_regular``   -- configuration-model (socket) matching with a seeded
  repair of double edges.
* ``qc_base_matrix`` / ``qc_expand`` -- a random quasi-cyclic base matrix
  lifted by circulant shifts.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Code:
    n: int
    m: int
    row_ptr: np.ndarray  # int32 [m+1]
    col_idx: np.ndarray  # int32 [nnz], sorted within each row
    name: str = ""
    qc_shift: np.ndarray | None = None  # int16 [mb, nb], -1 = zero block
    qc_z: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        """H as a dense uint8 m x n matrix (small codes only)."""
        h = np.zeros((self.m, self.n), dtype=np.uint8)
        for c in range(self.m):
            h[c, self.col_idx[self.row_ptr[c]:self.row_ptr[c + 1]]] = 1
        return h

    def row_degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def col_degrees(self) -> np.ndarray:
        return np.bincount(self.col_idx, minlength=self.n)


def _csr_from_rows(rows, n: int) -> tuple[np.ndarray, np.ndarray]:
    row_ptr = np.zeros(len(rows) + 1, dtype=np.int32)
    cols = []
    for i, r in enumerate(rows):
        r = np.unique(np.asarray(r, dtype=np.int64))
        if r.size and (r[0] < 0 or r[-1] >= n):
            raise ValueError("column index out of range")
        row_ptr[i + 1] = row_ptr[i] + r.size
        cols.append(r)
    col_idx = (np.concatenate(cols) if cols else np.zeros(0)).astype(np.int32)
    return row_ptr, col_idx


def dense_to_code(h, name: str = "") -> Code:
    h = np.asarray(h, dtype=np.uint8)
    m, n = h.shape
    rows = [np.nonzero(h[c])[0] for c in range(m)]
    rp, ci = _csr_from_rows(rows, n)
    return Code(n=n, m=m, row_ptr=rp, col_idx=ci, name=name)


def gallager_regular(n: int, dv: int, dc: int, seed: int) -> Code:
    """Gallager's (dv, dc)-regular construction.

    Reading: band 0 has row i covering columns [i*dc, (i+1)*dc); each of the
    bands 1..dv-1 is a column permutation of band 0 drawn from
    ``numpy.random.default_rng(seed)`` (row i of band b covers
    ``perm_b[i*dc:(i+1)*dc]``).  Every column then has weight exactly dv and
    the dv bands sum to the all-ones row, so rank(H) <= m - (dv - 1).
    """
    if n % dc:
        raise ValueError("n must be a multiple of dc")
    rng = np.random.default_rng(seed)
    per_band = n // dc
    rows = [np.arange(i * dc, (i + 1) * dc) for i in range(per_band)]
    for _ in range(1, dv):
        perm = rng.permutation(n)
        rows += [np.sort(perm[i * dc:(i + 1) * dc]) for i in range(per_band)]
    rp, ci = _csr_from_rows(rows, n)
    return Code(n=n, m=len(rows), row_ptr=rp, col_idx=ci,
                name=f"gallager({dv},{dc}) n={n} seed={seed}")


def random_regular(n: int, dv: int, dc: int, seed: int) -> Code:
    """Random (dv, dc)-regular H by socket matching.

    Reading: variable sockets (each bit repeated dv times) are shuffled with
    ``default_rng(seed)`` and matched in order to check sockets (each check
    repeated dc times).  A check that received the same bit twice is repaired
    by swapping that socket with a randomly drawn socket of another check when
    the swap creates no new repeat; this is repeated until H is 0/1 with exact
    degrees.
    """
    if (n * dv) % dc:
        raise ValueError("n*dv must be a multiple of dc")
    m = n * dv // dc
    rng = np.random.default_rng(seed)
    sock = rng.permutation(np.repeat(np.arange(n, dtype=np.int64), dv))
    sock = sock.reshape(m, dc)
    for _ in range(100000):
        bad = [c for c in range(m) if len(set(sock[c].tolist())) < dc]
        if not bad:
            break
        for c in bad:
            row = sock[c].tolist()
            seen = set()
            for j, v in enumerate(row):
                if v not in seen:
                    seen.add(v)
                    continue
                # socket j of check c repeats bit v: swap with another check
                for _try in range(1000):
                    c2 = int(rng.integers(m))
                    j2 = int(rng.integers(dc))
                    v2 = int(sock[c2, j2])
                    if c2 == c or v2 in sock[c] or v in sock[c2]:
                        continue
                    sock[c, j], sock[c2, j2] = v2, v
                    break
                break
    else:  # pragma: no cover
        raise RuntimeError("socket repair did not converge")
    rows = [np.sort(sock[c]) for c in range(m)]
    rp, ci = _csr_from_rows(rows, n)
    code = Code(n=n, m=m, row_ptr=rp, col_idx=ci,
                name=f"random({dv},{dc}) n={n} seed={seed}")
    assert np.all(code.row_degrees() == dc) and np.all(code.col_degrees() == dv)
    return code


def qc_base_matrix(mb: int, nb: int, nnz: int, wmin: int, wmax: int,
                   z: int, seed: int) -> np.ndarray:
    """Random quasi-cyclic base matrix of circulant shifts (-1 = zero block).

    Reading: row weights are wmin plus a seeded multinomial split of the
    ``nnz - mb*wmin`` extra ones, redrawn until every row weight is at most
    wmax; each row draws its columns uniformly without replacement; the whole
    draw is repeated until every column has weight >= 1.  Shifts are uniform in
    [0, z).
    """
    rng = np.random.default_rng(seed)
    extra = nnz - mb * wmin
    if extra < 0 or nnz > mb * wmax:
        raise ValueError("infeasible base-matrix weights")
    for _ in range(10000):
        w = wmin + rng.multinomial(extra, np.full(mb, 1.0 / mb))
        if w.max() > wmax:
            continue
        base = np.full((mb, nb), -1, dtype=np.int16)
        for i in range(mb):
            cols = rng.choice(nb, size=int(w[i]), replace=False)
            base[i, cols] = rng.integers(0, z, size=cols.size)
        if np.all((base >= 0).sum(axis=0) >= 1):
            return base
    raise RuntimeError("could not draw a base matrix")  # pragma: no cover


def qc_expand(base: np.ndarray, z: int, name: str = "") -> Code:
    """Lift a base matrix: entry (i, j, s) connects check i*z + r to bit
    j*z + (r + s) mod z for r in [0, z)."""
    mb, nb = base.shape
    rows = []
    for i in range(mb):
        js = np.nonzero(base[i] >= 0)[0]
        for r in range(z):
            rows.append(js * z + (r + base[i, js].astype(np.int64)) % z)
    rp, ci = _csr_from_rows(rows, nb * z)
    return Code(n=nb * z, m=mb * z, row_ptr=rp, col_idx=ci, name=name,
                qc_shift=base.astype(np.int16), qc_z=z)


# --- small codes printed in the paper -------------------------------------

def fig1_code() -> Code:
    """The (2,4)-regular example H of Fig. 1 (n = 8, 4 checks)."""
    h = [[1, 1, 0, 0, 0, 1, 1, 0],
         [0, 0, 1, 1, 1, 0, 0, 1],
         [1, 1, 0, 0, 0, 1, 0, 1],
         [0, 0, 1, 1, 1, 0, 1, 0]]
    return dense_to_code(h, name="fig1")


def fig2_code() -> Code:
    """H = [P^T | I_4] for the generator G = [I_4 | P] of Fig. 2.

    The columns of P printed in Fig. 2 are (0,1,0,1), (1,0,0,1), (0,0,1,1)
    and (0,0,0,1); row j of H is column j of P followed by e_j.
    """
    p_cols = [(0, 1, 0, 1), (1, 0, 0, 1), (0, 0, 1, 1), (0, 0, 0, 1)]
    h = np.zeros((4, 8), dtype=np.uint8)
    for j, col in enumerate(p_cols):
        h[j, :4] = col
        h[j, 4 + j] = 1
    return dense_to_code(h, name="fig2")


def table1_code(rate: float, seed: int) -> Code:
    """Table I workload: n = 1032, 12 ones per row, 9/6/3 ones per column for
    design rates 1/4, 1/2, 3/4 (Gallager construction)."""
    dv = {0.25: 9, 0.5: 6, 0.75: 3}[rate]
    return gallager_regular(1032, dv, 12, seed)
