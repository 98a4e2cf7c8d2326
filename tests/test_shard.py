"""Instance sharding of one global batch over ranks (paper_1307_3428_gb300/shard.py), on CPU:
the partition's invariants, and a two-rank gloo run of ShardedBatch -- gather of spectra and of
per-instance gradients to rank 0, all-reduce of the batch totals -- against a single-process
run of the same code.  The GPU integrator is replaced by a test-local stand-in with the same
interface (no GPU here); the stand-in computes a per-instance function of the instance only, as
the real integrator does, so any mix-up of instances or ranks shows in the comparison."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1307_3428_gb300 import shard
from paper_1307_3428_gb300 import workloads as wl


def test_partition_covers_every_instance_once_and_balances_cost():
    rng = np.random.default_rng(5)
    for world in (1, 2, 3, 4, 7, 8):
        for n in (0, 1, 3, 16, 257):
            sizes = [int(2 ** k) for k in rng.integers(8, 13, n)]
            costs = [shard.step_cost(N) for N in sizes]
            ranges = [shard.partition(costs, world, r) for r in range(world)]
            assert ranges == shard.shard_sizes(sizes, world)
            owned = [i for a, b in ranges for i in range(a, b)]
            assert owned == list(range(n))            # contiguous, in order, each once
            if n >= 8 * world:
                loads = [sum(costs[a:b]) for a, b in ranges]
                assert max(loads) - min(loads) <= 2 * max(costs)


def test_partition_rejects_bad_arguments():
    with pytest.raises(ValueError):
        shard.partition([1.0, 2.0], 2, 2)
    with pytest.raises(ValueError):
        shard.partition([1.0, -2.0], 2, 0)


class StandInBatch:
    """Test-local stand-in for cme.Batch: 'integrating' multiplies each instance's field by a
    phase that depends on the instance's parameters and the elapsed time; its 'gradients' are
    fixed functions of each instance's parameters and field."""

    def __init__(self, instances, **kw):
        self.insts = list(instances)
        self.tau = 0.0

    def step(self, h, n):
        self.tau += h * n

    def _field(self):
        return [i.D0 * np.exp(1j * (i.sigma + 0.1 * abs(i.A_in)) * self.tau) for i in self.insts]

    def spectrum(self, what=0):
        f = np.concatenate(self._field())
        return np.abs(f) ** 2 if what == 0 else f

    def get_state(self):
        return np.concatenate(self._field())

    def grad(self, h, n, target, eps=1e-20, segment=0):
        T = np.asarray(target).reshape(-1)
        off = np.concatenate([[0], np.cumsum([i.N for i in self.insts])])
        P = self.spectrum(0)
        loss = np.array([np.sum((np.log10(P[a:b] + eps) - T[a:b]) ** 2)
                         for a, b in zip(off[:-1], off[1:])])
        return {"loss": loss,
                "d_sigma": np.array([i.sigma * 2.0 + h * n for i in self.insts]),
                "d_A_in": np.array([complex(i.A_in) * 1j for i in self.insts]),
                "d_D2": np.array([0.5 * i.sigma for i in self.insts]),
                "d_D3": np.array([abs(i.A_in) for i in self.insts]),
                "d_omega": np.concatenate([i.omega * 0.25 for i in self.insts]),
                "d_kappa": np.concatenate([i.kappa + i.sigma for i in self.insts]),
                "d_D0": np.concatenate([np.conj(i.D0) for i in self.insts])}

    def close(self):
        pass


def _global_batch():
    # uneven sizes, in non-decreasing N as a batch requires
    return wl.uneven(per_size=3, nsteps=1, sizes=(64, 128, 256)).instances


def _run(world, rank):
    insts = _global_batch()
    sb = shard.ShardedBatch(insts, make_batch=StandInBatch, world=world, rank=rank)
    sb.step(1e-3, 50)
    T = np.concatenate([np.full(i.N, -3.0) for i in insts])
    out = {"spectrum": sb.spectrum(0), "field": sb.get_state(), "grad": sb.grad(1e-3, 50, T),
           "range": (sb.start, sb.stop)}
    sb.close()
    return out


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, _run(None, None)))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_gather_and_gradient_sums_match_one_process():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _run(1, 0)
    r0, r1 = res[0], res[1]
    # the shards split the batch: rank 0 the cheap start, rank 1 the rest
    assert r0["range"][0] == 0 and r0["range"][1] == r1["range"][0]
    assert r1["range"][1] == len(_global_batch()) and 0 < r0["range"][1] < len(_global_batch())
    # rank 0 holds the global results in global order; rank 1 holds none
    assert np.array_equal(r0["spectrum"], ref["spectrum"])
    assert np.array_equal(r0["field"], ref["field"])
    assert r1["spectrum"] is None and r1["field"] is None
    for k in ("loss", "d_sigma", "d_A_in", "d_D2", "d_D3", "d_omega", "d_kappa", "d_D0"):
        assert np.array_equal(r0["grad"][k], ref["grad"][k]), k
        assert r1["grad"][k] is None
    # batch totals on every rank: sums over all instances
    for r in (r0, r1):
        for k, src in (("loss_total", "loss"), ("d_D2_shared", "d_D2"),
                       ("d_D3_shared", "d_D3"), ("d_sigma_shared", "d_sigma")):
            assert abs(r["grad"][k] - np.sum(ref["grad"][src])) <= 1e-12 * abs(
                np.sum(ref["grad"][src])), k
