"""Sharded adaptive sampling over several ranks (one GPU per rank).

Samples are independent (arXiv 1910.11039, Section I-A), so the sample
indices of every epoch can be split between ranks; the only exchange is the
epoch aggregate: the ranks' counter deltas are summed (the paper's MPI
reduction of state frames, Algorithms 1-2) and the stopping condition is
checked on the result (the paper checks on rank 0 and broadcasts the flag;
here rank 0 checks and broadcasts too).  The split is deterministic and the
sum is an integer sum, so a sharded run takes exactly the samples, counters
and stop epoch of a single-rank run with the same epoch length.

The driver is written against two small interfaces so that its logic can be
exercised on CPU ranks (gloo) as well as on GPU ranks (NCCL):
  sampler.sample(first, count) -> counter delta of samples [first, first+count)
  state.absorb(delta, samples); state.check() -> bool stop
`LibraryShard` implements both with the C-ABI library on one GPU.
"""
from __future__ import annotations

import math


def epoch_share(tau: int, m: int, world: int, rank: int) -> tuple[int, int]:
    """Rank `rank`'s contiguous share (first, count) of sample indices
    [tau, tau + m): the first m % world ranks take one extra sample."""
    base, extra = divmod(m, world)
    first = tau + rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


class ShardedRun:
    """Epoch loop of the adaptive phase split over the ranks of `group`."""

    def __init__(self, sampler, state, omega_ceil: int, dist, group=None):
        self.sampler = sampler
        self.state = state
        self.omega_ceil = int(omega_ceil)
        self.dist = dist
        self.group = group

    def run(self, epoch_len: int, max_epochs: int = 1 << 40, tau: int = 0):
        """Returns (stopped, tau, epochs)."""
        world = self.dist.get_world_size(self.group)
        rank = self.dist.get_rank(self.group)
        epochs = 0
        stopped = False
        while epochs < max_epochs and not stopped:
            m = max(0, min(epoch_len, self.omega_ceil - tau))
            first, count = epoch_share(tau, m, world, rank)
            delta = self.sampler.sample(first, count)
            self.dist.all_reduce(delta, op=self.dist.ReduceOp.SUM, group=self.group)
            self.state.absorb(delta, m)
            tau += m
            epochs += 1
            flag = self.state.flag_tensor(self.state.check() if rank == 0 else False)
            self.dist.broadcast(flag, src=0, group=self.group)
            stopped = bool(flag.item())
        return stopped, tau, epochs


class LibraryShard:
    """Sampler and epoch state of one rank on its GPU (C-ABI library)."""

    def __init__(self, query, device=None):
        import torch

        self.torch = torch
        self.q = query
        self.n = query.graph.n
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.delta = torch.zeros(self.n, dtype=torch.int32, device=self.device)

    def sample(self, first, count):
        self.delta.zero_()
        if count:
            self.q.sample_range(1, first, count, self.delta.data_ptr())
        return self.delta

    def absorb(self, delta, samples):
        self.q.absorb(delta.data_ptr(), samples)

    def check(self) -> bool:
        stopped, _, _ = self.q.check_stop()
        return stopped

    def flag_tensor(self, value):
        return self.torch.tensor([1 if value else 0], dtype=self.torch.int32, device=self.device)


def epochs_needed(omega_ceil: int, epoch_len: int) -> int:
    return math.ceil(omega_ceil / epoch_len)
