"""One run's particles split over the ranks of a torch.distributed group.

The only exchange a sparse-grid PIC step needs is the regular-grid charge
density: every rank deposits its own particles, the densities are summed
over the ranks (the paper's Algorithm 2 sums each component grid over the
processes with MPI_Allreduce, Section 4.4; restricting after the sum is the
same by linearity and moves one array instead of one per grid), and every
rank then computes the same fields and pushes its own particles.  The
library's split step (sg_pic_step_deposit / sg_pic_step_fields) brackets
the exchange; this module does the partition and the sum.
"""
from __future__ import annotations

import numpy as np


def partition(n: int, world: int, rank: int) -> tuple:
    """Contiguous index range [lo, hi) of rank's share of n particles; the
    ranges of ranks 0..world-1 tile [0, n) and differ in size by at most one."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need world >= 1 and 0 <= rank < world")
    return n * rank // world, n * (rank + 1) // world


def _dist(group):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist, dist.get_world_size(group), dist.get_rank(group)
    return None, 1, 0


def sum_over_ranks(tensor, group=None):
    """In-place sum of a tensor over the group's ranks (no-op on one rank)."""
    dist, world, _ = _dist(group)
    if dist is not None and world > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor


class ShardedRun:
    """A run whose particles are split over the ranks of `group` (the default
    process group, or a single rank when torch.distributed is not set up).

    Every rank passes the whole particle arrays (host numpy, (N, d)) and
    keeps its partition(N, world, rank) share on its GPU.  Keyword arguments
    are those of Run (adaptive tau is not available).
    """

    def __init__(self, L_box, n, u, v, w, dt, *, group=None, **kw):
        import torch
        from .sgpic import Run
        self.group = group
        dist, self.world, self.rank = _dist(group)
        N = len(w)
        self.lo, self.hi = partition(N, self.world, self.rank)
        sl = slice(self.lo, self.hi)
        self.run = Run(L_box, n, np.asarray(u)[sl], np.asarray(v)[sl], np.asarray(w)[sl], dt, deferred=True, **kw)
        dev = torch.device("cuda", torch.cuda.current_device())
        q = torch.tensor([float(np.sum(np.asarray(w, dtype=np.float64)[sl]))], dtype=torch.float64, device=dev)
        sum_over_ranks(q, group)
        self.charge_total = float(q.item())
        self.run.set_charge_total(self.charge_total)
        tdt = torch.float32 if self.run.dtype == np.float32 else torch.float64
        self.rho = torch.empty((1 << (len(L_box) * n),), dtype=tdt, device=dev)
        self._exchange()
        self.run.start()

    def _exchange(self):
        self.run.density_copy(self.rho, to_run=False)
        sum_over_ranks(self.rho, self.group)
        self.run.density_copy(self.rho, to_run=True)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            self.run.step_deposit()
            self._exchange()
            self.run.step_fields()

    def particles(self):
        """This rank's particles (its partition, original order within it)."""
        return self.run.particles()

    def diagnostics(self):
        """The run's diagnostics with the kinetic energy summed over the ranks
        (the field energy and the charges are the whole run's on every rank)."""
        import torch
        d = self.run.diagnostics()
        ke = torch.tensor([d["kinetic_energy"]], dtype=torch.float64,
                          device=torch.device("cuda", torch.cuda.current_device()))
        sum_over_ranks(ke, self.group)
        d["kinetic_energy"] = float(ke.item())
        return d

    def close(self):
        self.run.close()
