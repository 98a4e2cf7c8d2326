"""Instance sharding of one global batch over ranks (one process per GPU).

The instances of a batch are independent problems (the paper's Fig. 1 runs an ensemble of
independent integrations, Sec. 2), so a global batch splits by instance with no exchange while
it steps: each rank integrates a contiguous range of the global instances on its own GPU.  Only
results cross ranks, on the host, after the step loop:

  * spectra and fields are gathered to one rank, in the global instance order;
  * gradients of per-instance parameters (sigma, A_in, the initial field, omega, kappa) are
    gathered the same way;
  * the batch loss and the gradients of parameters shared by every instance (a common D2 or
    D3, or any scalar that all instances take from one value) are sums over instances, and so
    over ranks: an all-reduce of a few scalars.

Argument marshalling and host bookkeeping only: every integration step runs in the CUDA library
through `make_batch` (by default `cme.Batch`).  The collectives are torch.distributed calls on
the default process group (gloo or NCCL); with one process they are skipped.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np


def partition(costs: Sequence[float], world: int, rank: int) -> Tuple[int, int]:
    """Contiguous range [start, stop) of the instances owned by `rank`: the cut points split the
    running sum of per-instance costs (e.g. N log2 N per step) as evenly as contiguous ranges
    allow, so that ranks of an uneven batch finish together.  Every instance is owned by exactly
    one rank; a rank may own none when there are fewer instances than ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    c = np.asarray(costs, dtype=np.float64)
    if np.any(c < 0):
        raise ValueError("instance costs must be non-negative")
    n = len(c)
    if n == 0:
        return 0, 0
    cum = np.concatenate([[0.0], np.cumsum(c)])
    total = cum[-1]

    def cut(r):
        if r <= 0:
            return 0
        if r >= world:
            return n
        if total == 0:
            return (n * r) // world
        # first index whose running cost reaches the share r / world of the total
        return int(np.searchsorted(cum, total * r / world - 1e-12 * total, side="left"))

    return cut(rank), max(cut(rank), cut(rank + 1))


def step_cost(N: int) -> float:
    """Relative cost of one step of an instance of N modes (transforms: N log2 N)."""
    return float(N) * float(np.log2(max(N, 2)))


def _dist():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist
    return None


class ShardedBatch:
    """This rank's share of a global batch.

    instances   the global list (every rank passes the same list, in the same order);
    make_batch  callable(list of instances, **batch_kw) -> an object with step(h, n),
                spectrum(what), get_state(), grad(h, n, target, eps, segment) and close(), as
                cme.Batch; default cme.Batch;
    world, rank default: the torch.distributed default group (1 and 0 without one)."""

    def __init__(self, instances: Sequence, make_batch: Optional[Callable] = None,
                 world: Optional[int] = None, rank: Optional[int] = None, **batch_kw):
        d = _dist()
        self.world = world if world is not None else (d.get_world_size() if d else 1)
        self.rank = rank if rank is not None else (d.get_rank() if d else 0)
        self.instances = list(instances)
        self.sizes = [int(i.N) for i in self.instances]
        self.start, self.stop = partition([step_cost(N) for N in self.sizes], self.world,
                                          self.rank)
        self.local = self.instances[self.start:self.stop]
        if make_batch is None:
            from . import cme
            make_batch = cme.Batch
        self.batch = make_batch(self.local, **batch_kw) if self.local else None
        off = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.offsets = off
        self.mode_range = (int(off[self.start]), int(off[self.stop]))

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None

    def step(self, h: float, nsteps: int):
        if self.batch is not None:
            self.batch.step(h, nsteps)

    # ---- host-side collectives -----------------------------------------------------------
    def _gather_rows(self, local: np.ndarray, dst: int) -> Optional[np.ndarray]:
        """Concatenate every rank's 1-D array on rank `dst`, in rank (= global instance) order;
        other ranks get None."""
        d = _dist()
        if self.world == 1 or d is None:
            return local
        parts = [None] * self.world if self.rank == dst else None
        d.gather_object(local, parts, dst=dst)
        if self.rank != dst:
            return None
        return np.concatenate([np.asarray(p) for p in parts])

    def _allreduce_sum(self, x: np.ndarray) -> np.ndarray:
        d = _dist()
        if self.world == 1 or d is None:
            return x
        import torch
        t = torch.as_tensor(np.asarray(x, dtype=np.float64).copy())
        dev = "cuda" if d.get_backend() == "nccl" else "cpu"
        t = t.to(dev)
        d.all_reduce(t, op=d.ReduceOp.SUM)
        return t.cpu().numpy()

    # ---- results ---------------------------------------------------------------------------
    def spectrum(self, what: int = 0, dst: int = 0) -> Optional[np.ndarray]:
        """The global batch's spectrum (cme_spectrum `what` of every instance, concatenated in
        global order) on rank `dst`; None on the other ranks."""
        if self.batch is not None:
            local = np.asarray(self.batch.spectrum(what))
        else:
            local = np.zeros(0, dtype=np.float64 if what == 0 else np.complex128)
        return self._gather_rows(local, dst)

    def get_state(self, dst: int = 0) -> Optional[np.ndarray]:
        local = (np.asarray(self.batch.get_state()) if self.batch is not None
                 else np.zeros(0, dtype=np.complex128))
        return self._gather_rows(local, dst)

    def grad(self, h: float, nsteps: int, target, eps: float = 1e-20, segment: int = 0,
             dst: int = 0) -> dict:
        """Gradients of the global batch.  `target`: the global target (sum of N values).

        Every rank returns the batch totals, summed over all instances and ranks:
        "loss_total", and "d_D2_shared" / "d_D3_shared" / "d_sigma_shared", the gradients with
        respect to a D2, D3 or sigma that every instance shares.  Rank `dst` also gets the
        per-instance and per-mode arrays of the whole batch in global order ("loss", "d_sigma",
        "d_A_in", "d_D2", "d_D3", "d_omega", "d_kappa", "d_D0"); other ranks get None there."""
        T = np.asarray(target, dtype=np.float64).reshape(-1)
        lo, hi = self.mode_range
        if self.batch is not None:
            g = self.batch.grad(h, nsteps, T[lo:hi], eps, segment)
        else:
            g = {"loss": np.zeros(0), "d_sigma": np.zeros(0), "d_A_in": np.zeros(0, complex),
                 "d_D2": np.zeros(0), "d_D3": np.zeros(0), "d_omega": np.zeros(0),
                 "d_kappa": np.zeros(0), "d_D0": np.zeros(0, complex)}
        sums = self._allreduce_sum(np.array([np.sum(g["loss"]), np.sum(g["d_D2"]),
                                             np.sum(g["d_D3"]), np.sum(g["d_sigma"])]))
        out = {"loss_total": float(sums[0]), "d_D2_shared": float(sums[1]),
               "d_D3_shared": float(sums[2]), "d_sigma_shared": float(sums[3])}
        for k in ("loss", "d_sigma", "d_A_in", "d_D2", "d_D3", "d_omega", "d_kappa", "d_D0"):
            out[k] = self._gather_rows(np.asarray(g[k]), dst)
        return out


def shard_sizes(sizes: Sequence[int], world: int) -> List[Tuple[int, int]]:
    """The (start, stop) instance range of every rank for instances of the given sizes."""
    costs = [step_cost(N) for N in sizes]
    return [partition(costs, world, r) for r in range(world)]
