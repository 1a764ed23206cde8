"""Frame sharding over replicas (Sec. III-C batch processing, Eq. 9), on CPU.

The split is pinned by what Eq. 9 must give (counts that add up to the batch,
differ by at most one, the extra frames on the lowest-numbered processes,
contiguous blocks in process order), and the gather by a world-size-2 ``gloo``
run whose collected result must equal one process decoding the whole batch.
"""

import os
import pickle
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2201_04265_gb300 import shard
from parity_util import workload


def test_eq9_split_counts():
    # hand-worked: 10 frames over 4 processes -> 3, 3, 2, 2
    assert [shard.num_elems(q, 4, 10) for q in range(4)] == [3, 3, 2, 2]
    assert [shard.num_elems(q, 3, 2) for q in range(3)] == [1, 1, 0]
    assert list(shard.shard_offsets(4, 10)) == [0, 3, 6, 8, 10]
    for N in range(1, 9):
        for l in range(0, 40):
            c = [shard.num_elems(q, N, l) for q in range(N)]
            assert sum(c) == l
            assert max(c) - min(c) <= 1
            assert c == sorted(c, reverse=True)
            assert sum(x > l // N for x in c) == l % N


def test_eq9_as_printed_does_not_partition():
    # the printed form, floor(N/l) (+1 while q < N mod l), hands out N frames
    # in total whenever l > N: the reason for reading it with l and N exchanged
    N, l = 4, 10
    printed = [N // l + (1 if q < N % l else 0) for q in range(N)]
    assert sum(printed) == 4 != l


def test_bad_split_rejected():
    for args in [(0, 0, 5), (2, 2, 5), (-1, 2, 5), (0, 2, -1)]:
        with pytest.raises(ValueError):
            shard.num_elems(*args)


def test_single_process_is_identity():
    import torch
    t = torch.arange(12).reshape(6, 2)
    assert shard.gatherv(t, 6) is t
    g = torch.ones(3)
    assert shard.allreduce_mean_(g).tolist() == [1.0, 1.0, 1.0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("l", [7, 8, 1])
def test_gloo_two_process_gather_equals_whole_batch(tmp_path, l):
    import shard_worker
    out = str(tmp_path / "r0.pkl")
    mp.start_processes(shard_worker.run, args=(2, _free_port(), l, out), nprocs=2,
                       join=True, start_method="spawn")
    got = pickle.load(open(out, "rb"))
    wl = workload("c1_gallager_504", max(l, 1), 2.0, 9100)
    ref = oracle.decode(wl.code, wl.llr[:l], iters=10, early_stop=True)
    np.testing.assert_array_equal(got["frame"], np.arange(l))
    np.testing.assert_array_equal(got["post"], ref.post)
    np.testing.assert_array_equal(got["hard"], ref.hard)
    np.testing.assert_array_equal(got["iters"], ref.iters)
    np.testing.assert_array_equal(got["ok"], ref.ok)
    # weighted by Eq. 9 shares: (c0 * 1 + c1 * 2) / l; unweighted: (1 + 2) / 2
    c0, c1 = shard.num_elems(0, 2, l), shard.num_elems(1, 2, l)
    np.testing.assert_allclose(got["g"], np.full((3, 5), (c0 + 2 * c1) / l))
    np.testing.assert_allclose(got["h"], np.full(4, 1.5))


def test_lost_peer_is_reported_at_the_next_step(tmp_path):
    """Process 1 leaves after the first step; process 0 finishes that step's
    gather, then reports PeerLost naming process 1 at the second step's
    boundary within its 1 s limit, instead of hanging in a collective."""
    import shard_worker
    out = str(tmp_path / "lost.pkl")
    mp.start_processes(shard_worker.run_with_lost_peer, args=(2, _free_port(), _free_port(), 6, out), nprocs=2,
                       join=True, start_method="spawn")
    got = pickle.load(open(out, "rb"))
    assert got["steps_done"] == 1
    assert got["error"] is not None and "[1]" in got["error"] and "step 1" in got["error"]
    assert got["seconds"] < 20


def test_step_barrier_single_process():
    import datetime
    import torch.distributed as dist
    store = dist.HashStore()
    shard.step_barrier(store, 0, timeout_s=0.1)   # no process group: one process, nothing to wait for
    assert store.check(["ldpc-step/0/0"])
    del datetime
