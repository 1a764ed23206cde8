"""Worker processes for the sharding tests (gloo on CPU, world size 2).

Each process decodes its Eq. 9 block of a small batch with the oracle (the
CPU stand-in for one GPU replica's decoder) and takes part in the gathers;
process 0 writes what it collected to a file for the test to compare.
"""

import os
import pickle

import numpy as np
import torch
import torch.distributed as dist


def run(rank, world, port, l, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2201_04265_gb300 import shard
        from parity_util import workload
        wl = workload("c1_gallager_504", max(l, 1), 2.0, 9100)

        def work(f0, f1):
            r = oracle.decode(wl.code, wl.llr[f0:f1], iters=10, early_stop=True)
            return {"post": torch.from_numpy(r.post), "hard": torch.from_numpy(r.hard),
                    "iters": torch.from_numpy(r.iters), "ok": torch.from_numpy(r.ok),
                    "frame": torch.arange(f0, f1, dtype=torch.int64)}

        got = shard.run_sharded(l, work)
        # gradient averaging: process q contributes (q + 1) * ones
        g = torch.full((3, 5), float(rank + 1), dtype=torch.float64)
        shard.allreduce_mean_(g, l=l if l > 0 else None)
        h = torch.full((4,), float(rank + 1), dtype=torch.float64)
        shard.allreduce_mean_(h)
        if rank == 0:
            with open(out_path, "wb") as f:
                pickle.dump({k: v.numpy() for k, v in got.items()} | {"g": g.numpy(), "h": h.numpy()}, f)
        else:
            assert got is None
    finally:
        dist.destroy_process_group()


def run_with_lost_peer(rank, world, port, store_port, l, out_path):
    """Three sharded steps; process 1 exits after the first (between steps,
    with nothing in flight).  Process 0 must report the lost peer at the next
    step boundary instead of waiting in a gather, and writes what it saw."""
    import datetime
    import time

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    store = dist.TCPStore("127.0.0.1", store_port, world, rank == 0, timeout=datetime.timedelta(seconds=30))
    import oracle
    from paper_2201_04265_gb300 import shard
    from parity_util import workload
    wl = workload("c1_gallager_504", l, 2.0, 9200)

    def work(step, f0, f1):
        r = oracle.decode(wl.code, wl.llr[f0:f1], iters=5)
        return {"post": torch.from_numpy(r.post)}

    if rank == 1:
        shard.run_sharded_steps(1, l, work, store, timeout_s=10.0)
        return  # leaves between steps: never announces step 1
    t0 = time.monotonic()
    result = {"steps_done": 0, "error": None}
    try:
        out = []
        for step in range(3):
            shard.step_barrier(store, step, timeout_s=1.0)
            out.append(shard.run_sharded(l, lambda f0, f1, s=step: work(s, f0, f1)))
            result["steps_done"] = step + 1
        result["posts"] = [o["post"].numpy() for o in out]
    except shard.PeerLost as exc:
        result["error"] = str(exc)
    result["seconds"] = time.monotonic() - t0
    with open(out_path, "wb") as f:
        pickle.dump(result, f)
