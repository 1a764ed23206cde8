"""Frame sharding over replicas: the batch-processing split of Sec. III-C.

Frames are independent, so a batch of ``l`` frames is cut into ``N``
contiguous blocks, one per process, and decoded with no exchange at all; the
results are then collected on one process, in frame order (the paper gathers
with a variable-count gather).  Process ``q`` takes

    NumElems(q) = floor(l / N) + 1   if q <  l mod N
                  floor(l / N)       if q >= l mod N

frames (Eq. 9, read with ``l`` and ``N`` in the places that make the counts
add up to ``l``: the printed equation divides the process count by the element
count).  Blocks are contiguous and in process order, so concatenating them in
rank order restores the batch.

Communication goes through ``torch.distributed``: ``gloo`` for host tensors,
``nccl`` for device tensors.  Every process knows every count from ``l`` and
``N``, so the gather needs no size exchange: blocks are padded to the largest
count, gathered, and trimmed on the destination.  Weighted-BP training adds one
all-reduce of the weight gradient (``allreduce_mean_``), outside decoding.
"""

from __future__ import annotations

from datetime import timedelta
from typing import Callable

import numpy as np
import torch
import torch.distributed as dist


def num_elems(q: int, N: int, l: int) -> int:
    """Frames given to process q of N when l frames are split (Eq. 9)."""
    if N < 1 or not 0 <= q < N or l < 0:
        raise ValueError(f"bad split: q={q}, N={N}, l={l}")
    return l // N + (1 if q < l % N else 0)


def shard_offsets(N: int, l: int) -> np.ndarray:
    """int64 [N + 1]: process q holds frames [off[q], off[q + 1])."""
    counts = np.array([num_elems(q, N, l) for q in range(N)], dtype=np.int64)
    return np.concatenate([[0], np.cumsum(counts)])


def shard_range(q: int, N: int, l: int) -> tuple[int, int]:
    off = shard_offsets(N, l)
    return int(off[q]), int(off[q + 1])


def _world(group) -> tuple[int, int]:
    if not dist.is_available() or not dist.is_initialized():
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def gatherv(local: torch.Tensor, l: int, group=None, dst: int = 0) -> torch.Tensor | None:
    """Concatenates every process's block (first dimension = its Eq. 9 count
    of the l frames) on process ``dst``; returns None on the others.

    All processes must call it with the same ``l`` and with blocks of the same
    trailing shape and dtype.  Without an initialised process group it returns
    ``local`` (one process holds the whole batch).
    """
    rank, N = _world(group)
    want = num_elems(rank, N, l)
    if local.shape[0] != want:
        raise ValueError(f"process {rank} holds {local.shape[0]} frames, Eq. 9 gives {want}")
    if N == 1:
        return local
    off = shard_offsets(N, l)
    if l == 0:
        return local if rank == dst else None
    cap = int(off[1] - off[0])          # the largest block: process 0's
    padded = local.new_zeros((cap,) + tuple(local.shape[1:]))
    padded[:want] = local
    bufs = [torch.empty_like(padded) for _ in range(N)] if rank == dst else None
    dist.gather(padded, gather_list=bufs, dst=dst, group=group)
    if rank != dst:
        return None
    return torch.cat([bufs[q][:int(off[q + 1] - off[q])] for q in range(N)])


def run_sharded(l: int, work: Callable[[int, int], dict], group=None,
                dst: int = 0) -> dict | None:
    """Runs ``work(f0, f1)`` on this process's block [f0, f1) of the l frames
    and gathers each tensor of the returned dict on ``dst`` (frame order).

    ``work`` returns a dict of tensors whose first dimension is f1 - f0, with
    the same keys on every process; an empty block still calls it (f0 == f1)
    so that every process takes part in every gather.
    """
    rank, N = _world(group)
    f0, f1 = shard_range(rank, N, l)
    out = work(f0, f1)
    res = {}
    for key in sorted(out):
        g = gatherv(out[key], l, group=group, dst=dst)
        res[key] = g
    return res if rank == dst else None


class PeerLost(RuntimeError):
    """A process of the replica group did not reach a step in time."""


def step_barrier(store, step: int, timeout_s: float, group=None) -> None:
    """Host-side liveness check between steps (no counterpart in the paper,
    whose MPI processes are assumed to survive).  Every process announces
    ``step`` in the key-value ``store`` and waits, at most ``timeout_s``
    seconds, for all others to do the same; it raises ``PeerLost`` naming the
    processes that did not arrive.  It runs between steps, when no device work
    or collective of this process is in flight, so a process that exited or
    hung is found before the next gather is started rather than inside it."""
    rank, N = _world(group)
    store.set(f"ldpc-step/{step}/{rank}", "1")
    keys = [f"ldpc-step/{step}/{q}" for q in range(N)]
    try:
        store.wait(keys, timedelta(seconds=timeout_s))
    except Exception as exc:  # the store's own timeout error
        missing = [q for q in range(N) if not store.check([keys[q]])]
        raise PeerLost(f"processes {missing} did not reach step {step} within {timeout_s} s") from exc


def run_sharded_steps(steps: int, l: int, work: Callable[[int, int, int], dict], store, timeout_s: float,
                      group=None, dst: int = 0) -> list:
    """``steps`` rounds of ``run_sharded``, each preceded by ``step_barrier``:
    ``work(step, f0, f1)`` decodes this process's block of step ``step``.
    Returns the gathered results of every step on ``dst`` (None elsewhere);
    raises ``PeerLost`` when a process is missing at a step boundary."""
    out = []
    for step in range(steps):
        step_barrier(store, step, timeout_s, group=group)
        out.append(run_sharded(l, lambda f0, f1, s=step: work(s, f0, f1), group=group, dst=dst))
    return out


def allreduce_mean_(t: torch.Tensor, l: int | None = None, group=None) -> torch.Tensor:
    """Averages a gradient over all processes in place (weighted-BP training
    on replicas).  Each process passes the gradient of the mean loss over its
    own frames; with ``l`` given, each is weighted by its Eq. 9 share of the l
    frames, which gives the gradient of the mean loss over the whole batch,
    otherwise all processes weigh the same."""
    rank, N = _world(group)
    if l is not None:
        if l < 1:
            raise ValueError("l must be positive")
        t.mul_(num_elems(rank, N, l) / l)
    elif N > 1:
        t.div_(N)
    if N > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
