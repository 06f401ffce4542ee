"""One run split by particles across ranks (one process per GPU).

Every rank holds the whole grid and a share of the particles.  A step is
the rank's particle phase, an in-place integer sum of its exchange buffer
over all ranks (torch.distributed all_reduce: NCCL on GPUs), and the field
phase, which every rank computes identically from the summed deposit
(pic_step_particles / pic_exchange_buffer / pic_step_fields of the C ABI).
This module only moves data: the sum of integers is exact and independent
of the order of the ranks, so the split run equals the unsplit one bit for
bit.
"""
from __future__ import annotations

import contextlib

import numpy as np


def shard_bounds(n: int, rank: int, world: int):
    """[lo, hi) of rank's contiguous share of n particles (sizes differ by at most one)."""
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard(p, rank: int, world: int):
    """Rank's share of a synth.Particles set (ids kept)."""
    lo, hi = shard_bounds(len(p), rank, world)
    return p.subset(slice(lo, hi))


def allreduce_sum_int64(t, group=None):
    """In-place integer sum of an int64 tensor over the process group."""
    import torch
    import torch.distributed as dist
    assert t.dtype == torch.int64
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def _device(group=None):
    """Where the group's collectives take their tensors: the GPU for NCCL."""
    import torch.distributed as dist
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


def reduce_counts(walls, live, group=None):
    """Wall tallies [2, 8] and live counts [2] summed over the ranks."""
    import torch
    v = torch.tensor(np.concatenate([np.asarray(walls, np.int64).ravel(),
                                     np.asarray(live, np.int64).ravel()]), dtype=torch.int64,
                     device=_device(group))
    allreduce_sum_int64(v, group)
    v = v.cpu().numpy()
    return v[:16].reshape(2, 8), v[16:]


def reduce_sum_f64(x, group=None):
    """Element-wise FP64 sum over the ranks (kinetic energies, momenta)."""
    import torch
    import torch.distributed as dist
    v = torch.tensor(np.asarray(x, np.float64).ravel(), dtype=torch.float64, device=_device(group))
    dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    return v.cpu().numpy().reshape(np.shape(x))


class DistributedSim:
    """A rank of a particle-decomposed run on this process's GPU.  `sim` is a
    Sim created with decomposed=True; `group` a torch.distributed group whose
    backend reaches the sim's device memory (NCCL)."""

    def __init__(self, sim, group=None):
        self.sim = sim
        self.group = group
        self.buf = sim.exchange_buffer()

    def step(self, n: int = 1):
        import torch
        stream = getattr(self.sim, "torch_stream", None)
        for _ in range(n):
            self.sim.step_particles()
            # the collective runs on the rank's stream, after its particle phase
            with (torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()):
                allreduce_sum_int64(self.buf, self.group)
            self.sim.step_fields()

    def counts(self):
        walls, live = self.sim.counts()
        return reduce_counts(walls, live, self.group)

    def energy(self):
        """[KE_e, KE_i, FE, n] of the whole run (kinetic energies summed over ranks)."""
        e = self.sim.energy().copy()
        e[:2] = reduce_sum_f64(e[:2], self.group)
        return e
