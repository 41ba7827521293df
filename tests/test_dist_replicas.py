"""The benchmark's N > 1 path on CPU: the disk's soft step does not shard, so
N ranks run independent replicas with no data-path collective; the ranks only
meet at barriers and combine their figures (the slowest rank's time, the
units all ranks processed).  Two gloo ranks, set up from the launcher's
environment as torchrun would set it."""
import os
import socket

import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, local, w, dist = bench.dist_setup(None)
    try:
        bench.barrier(dist)
        t_max = bench.allmax(dist, 1.5 + rank)        # elapsed seconds per rank
        units = bench.allsum(dist, 1.0e6 * (rank + 1))  # units each rank processed
        bench.barrier(dist)
        q.put((r, local, w, t_max, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_job_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert got == [(0, 0, 2, 2.5, 3.0e6), (1, 1, 2, 2.5, 3.0e6)]


def test_single_process_needs_no_group():
    import bench
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    r, local, w, dist = bench.dist_setup(None)
    assert (r, local, w, dist) == (0, 0, 1, None)
    bench.barrier(dist)
    assert bench.allmax(dist, 2.0) == 2.0 and bench.allsum(dist, 3.0) == 3.0
