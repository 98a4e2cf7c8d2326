"""Host-side logic of the multi-rank benchmark path on CPU (gloo, world size 2): every rank
integrates its own replica of the sweep (no data-path collective); the timing reduction takes
the maximum over ranks; the ranks' inputs are distinct."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_1307_3428_gb300 import workloads as wl
    w_, r_, l_ = bench.dist_setup()
    assert (w_, r_) == (world, rank)
    t = bench.max_over_ranks(1.0 + rank, world)
    bench.barrier(world)
    w = wl.sweep512(indices=[0, 1, 2], seed_offset=256 * rank) if rank else \
        wl.sweep512(indices=[0, 1, 2])
    import torch.distributed as dist
    sig = [float(np.abs(i.D0).sum()) for i in w.instances]
    gathered = [None] * world
    dist.all_gather_object(gathered, sig)
    out.put((rank, t, gathered))
    dist.destroy_process_group()


def test_two_rank_gloo_timing_and_shards():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, gathered in res:
        assert t == 2.0                    # max over ranks
        assert gathered[0] != gathered[1]  # independent noise per replica
