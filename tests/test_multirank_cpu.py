"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): rank and world from the
torchrun environment, a barrier, the max-over-ranks step time, one independent seeded system
per rank (no collective on the data path) and the whole-job value."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    r, w = bench.dist_setup(world, backend="gloo")
    ms = bench.max_over_ranks(1.5 + rank, w)            # rank 1 is the slower one
    bench.barrier(w)
    wl = bench.rank_workload("petn464", r)
    q.put((r, w, ms, len(wl["x"]), wl["x"][:4].copy()))
    dist.destroy_process_group()


def test_two_cpu_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, ms0, n0, x0), (r1, w1, ms1, n1, x1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert ms0 == ms1 == 2.5                              # both ranks see the slowest step time
    assert n0 == n1 == 464                                # same size per rank (weak scaling)
    assert not np.array_equal(x0, x1)                     # independent systems (seeded by rank)
    import bench
    assert bench.job_value(n0, ms0, 2) == 2 * 464 / 2.5e-3
