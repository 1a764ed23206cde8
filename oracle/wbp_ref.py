"""FP64 reference gradient of weighted belief propagation (test infrastructure).

An independent restatement of the oracle's forward pass in plain PyTorch
float64 CPU ops, differentiated by torch.autograd.  It follows the same
equations as ``ldpc_oracle.c`` (Sec. II-B: Eq. 5 sign-corrected, Eq. 6 written
literally as a sum over the other checks, Eq. 7) with one weight per edge and
iteration multiplying E_cv in Eqs. 6 and 7, and the loss

    loss = mean over frames and bits of BCE(sigmoid(L_v^(T)), c_v)

(sigmoid(L) = P(bit = 1) under the paper's LLR sign, Eq. 4).  Clamping uses
``torch.clamp``, whose gradient passes where min <= x <= max.
"""

from __future__ import annotations

import numpy as np
import torch


class _Graph:
    def __init__(self, code):
        rp = np.asarray(code.row_ptr, dtype=np.int64)
        ci = np.asarray(code.col_idx, dtype=np.int64)
        self.n, self.m, self.E = code.n, code.m, int(rp[-1])
        dmax = int(np.max(np.diff(rp))) if self.m else 0
        rowE = np.full((self.m, dmax), -1, dtype=np.int64)
        for c in range(self.m):
            d = rp[c + 1] - rp[c]
            rowE[c, :d] = np.arange(rp[c], rp[c + 1])
        colcnt = np.bincount(ci, minlength=self.n)
        vmax = int(colcnt.max()) if self.n else 0
        colE = np.full((self.n, vmax), -1, dtype=np.int64)
        fill = np.zeros(self.n, dtype=np.int64)
        for e in range(self.E):
            v = ci[e]
            colE[v, fill[v]] = e
            fill[v] += 1
        self.rowE = torch.from_numpy(rowE)
        self.colE = torch.from_numpy(colE)
        self.var_of_edge = torch.from_numpy(ci)


def _gather_pad(x: torch.Tensor, idx: torch.Tensor, pad: float) -> torch.Tensor:
    """x [F, E], idx [K, D] (-1 = pad) -> [F, K, D]."""
    safe = idx.clamp(min=0)
    g = x[:, safe.reshape(-1)].reshape(x.shape[0], *idx.shape)
    return torch.where(idx.unsqueeze(0) >= 0, g, torch.full_like(g, pad))


def weighted_bp_forward(code, R: torch.Tensor, w: torch.Tensor, clip: float = 20.0,
                        graph: _Graph | None = None) -> torch.Tensor:
    """Total LLR after T = w.shape[0] iterations; R [F, n], w [T, E], float64."""
    g = graph or _Graph(code)
    F = R.shape[0]
    Lvc = R[:, g.var_of_edge]                                   # initial messages, L_vc = R_v
    Lv = R
    for t in range(w.shape[0]):
        M = torch.clamp(Lvc, -clip, clip)
        tn = torch.tanh(-M / 2.0)                               # [F, E]
        T_rows = _gather_pad(tn, g.rowE, 1.0)                   # [F, m, D]
        D = T_rows.shape[2]
        E_rows = []
        for j in range(D):
            others = torch.cat([T_rows[:, :, :j], T_rows[:, :, j + 1:]], dim=2)
            prod = torch.prod(others, dim=2)
            E_rows.append(torch.clamp(-2.0 * torch.atanh(prod), -clip, clip))
        E_rows = torch.stack(E_rows, dim=2)                     # [F, m, D]
        Ecv = torch.zeros(F, g.E, dtype=R.dtype)
        valid = g.rowE >= 0
        Ecv = Ecv.index_put((torch.arange(F)[:, None], g.rowE[valid][None, :]),
                            E_rows[:, valid])
        WE = w[t][None, :] * Ecv                                # weighted messages
        WE_cols = _gather_pad(WE, g.colE, 0.0)                  # [F, n, Dv]
        Lv = R + WE_cols.sum(dim=2)                             # Eq. 7
        Dv = WE_cols.shape[2]
        ext = []
        for j in range(Dv):
            others = torch.cat([WE_cols[:, :, :j], WE_cols[:, :, j + 1:]], dim=2)
            ext.append(R + others.sum(dim=2))                   # Eq. 6
        ext = torch.stack(ext, dim=2)                           # [F, n, Dv]
        validc = g.colE >= 0
        Lvc = torch.zeros(F, g.E, dtype=R.dtype).index_put(
            (torch.arange(F)[:, None], g.colE[validc][None, :]), ext[:, validc])
    return Lv


def bce_loss(Lv: torch.Tensor, bits: torch.Tensor) -> torch.Tensor:
    return torch.nn.functional.binary_cross_entropy_with_logits(Lv, bits, reduction="mean")


def loss_and_grads(code, R: np.ndarray, w: np.ndarray, bits: np.ndarray, clip: float = 20.0):
    """Returns (loss, dloss/dw [T, E], dloss/dR [F, n], L^(T) [F, n]) in float64."""
    Rt = torch.tensor(np.asarray(R, dtype=np.float64), requires_grad=True)
    wt = torch.tensor(np.asarray(w, dtype=np.float64), requires_grad=True)
    bt = torch.tensor(np.asarray(bits, dtype=np.float64))
    Lv = weighted_bp_forward(code, Rt, wt, clip)
    loss = bce_loss(Lv, bt)
    loss.backward()
    return (float(loss.detach()), wt.grad.numpy().copy(), Rt.grad.numpy().copy(),
            Lv.detach().numpy().copy())
