"""Host-side logic of the multi-GPU benchmark path (replicas), on CPU with gloo.

Every rank runs its own solves and no collective touches the data path; the
benchmark only needs a barrier, the maximum of the per-rank times and the sum
of the per-rank ray-sample counts.  Two gloo ranks check exactly those.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(False)
    try:
        t = 1.5 if r == 0 else 2.5            # per-rank "device time"
        tmax = bench.dist_max(t, w)
        total = bench.dist_sum(100.0 * (r + 1), w)
        bench.dist_barrier(w)
        q.put((r, w, local, tmax, total))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_summed_samples():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, w, local, tmax, total) in enumerate(got):
        assert rank == r and w == 2 and local == r
        assert tmax == 2.5          # the slowest rank sets the time
        assert total == 300.0       # samples of all ranks add up


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    saved = {k: os.environ.pop(k, None) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    try:
        assert bench.dist_setup(False) == (1, 0, 0)
        assert bench.dist_max(3.0, 1) == 3.0
        assert bench.dist_sum(4.0, 1) == 4.0
    finally:
        for k, v in saved.items():
            if v is not None:
                os.environ[k] = v
