"""Sharded adaptive sampling over several ranks (one GPU per rank).

Samples are independent (arXiv 1910.11039, Section I-A), so the sample
indices of every epoch can be split between ranks; the only exchange is the
epoch aggregate: the ranks' counter deltas are summed (the paper's MPI
reduction of state frames, Algorithms 1-2) and the stopping condition is
checked on the result (the paper checks on rank 0 and broadcasts the flag;
here rank 0 checks and broadcasts too).  The split is deterministic and the
sum is an integer sum, so a sharded run takes exactly the samples, counters
and stop epoch of a single-rank run with the same epoch length.

Two forms of the exchange:
  run()       the ranks' counter deltas (n counters each) are summed with one
              all_reduce per epoch, rank 0 checks and broadcasts the flag;
  run_logs()  the ranks exchange their epoch logs (the interior vertices of
              their sampled paths: at most E * (VD - 2) ids per epoch, against
              n counters), every rank folds all logs in rank order into its
              own copy of the counters and checks the same snapshot, so no
              broadcast is needed; two frames let a rank sample its share of
              epoch e + 1 while the logs of epoch e are exchanged and checked
              (the paper's two state frames per thread, Section IV-B/C).
Both take exactly the samples, counters and stop epoch of a single-rank run
with the same epoch length.

The driver is written against small interfaces so that its logic can be
exercised on CPU ranks (gloo) as well as on GPU ranks (NCCL):
  sampler.sample(first, count) -> counter delta of samples [first, first+count)
  sampler.sample_log(first, count, frame) -> handle; sampler.local_log(handle)
      -> 1-D int32 tensor of the interior vertices of those samples
  state.absorb(delta, samples); state.absorb_log(log, samples);
  state.check() -> bool stop
`LibraryShard` implements them with the C-ABI library on one GPU.
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

    def exchange_logs(self, local):
        """All ranks' logs of one epoch, concatenated in rank order."""
        torch = self._torch()
        world = self.dist.get_world_size(self.group)
        n_local = torch.tensor([int(local.numel())], dtype=torch.int64, device=local.device)
        lens = [torch.zeros_like(n_local) for _ in range(world)]
        self.dist.all_gather(lens, n_local, group=self.group)
        lens = [int(x.item()) for x in lens]
        width = max(lens) if lens else 0
        if width == 0:
            return local[:0]
        padded = torch.zeros(width, dtype=local.dtype, device=local.device)
        padded[:local.numel()] = local
        parts = [torch.zeros_like(padded) for _ in range(world)]
        self.dist.all_gather(parts, padded, group=self.group)
        return torch.cat([p[:k] for p, k in zip(parts, lens)])

    def run_logs(self, epoch_len: int, max_epochs: int = 1 << 40, tau: int = 0):
        """Overlapped epochs with log exchange (see the module docstring).
        Returns (stopped, tau, epochs)."""
        world = self.dist.get_world_size(self.group)
        rank = self.dist.get_rank(self.group)

        def share(t):
            m = max(0, min(epoch_len, self.omega_ceil - t))
            return m, epoch_share(t, m, world, rank)

        m, (first, count) = share(tau)
        pending = [self.sampler.sample_log(first, count, 0), None]
        epochs = 0
        stopped = False
        while epochs < max_epochs:
            k = epochs % 2
            nxt = tau + m
            if epochs + 1 < max_epochs and nxt < self.omega_ceil:
                m1, (f1, c1) = share(nxt)
                pending[1 - k] = self.sampler.sample_log(f1, c1, 1 - k)
            else:
                m1 = 0
            logs = self.exchange_logs(self.sampler.local_log(pending[k]))
            self.state.absorb_log(logs, m)
            tau = nxt
            epochs += 1
            if self.state.check():
                stopped = True
                break
            m = m1
        return stopped, tau, epochs

    @staticmethod
    def _torch():
        import torch
        return torch


class LibraryShard:
    """Sampler and epoch state of one rank on its GPU (C-ABI library)."""

    def __init__(self, query, device=None, log_cap=0):
        import torch

        self.torch = torch
        self.q = query
        self.n = query.graph.n
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.delta = torch.zeros(self.n, dtype=torch.int32, device=self.device)
        # two epoch-log frames, sampled on a side stream so that an epoch's
        # sampling overlaps the previous epoch's exchange
        self.log_cap = int(log_cap)
        if self.log_cap:
            self.logs = [torch.empty(self.log_cap, dtype=torch.int32, device=self.device) for _ in range(2)]
            self.lens = torch.zeros(2, dtype=torch.int32, device=self.device)
            self.stream = torch.cuda.Stream(device=self.device)
            self.ready = [torch.cuda.Event() for _ in range(2)]
            self.free = [torch.cuda.Event() for _ in range(2)]
            for e in self.free:
                e.record(torch.cuda.current_stream(self.device))

    def sample(self, first, count):
        self.delta.zero_()
        if count:
            self.q.sample_range(1, first, count, self.delta.data_ptr())
        return self.delta

    def absorb(self, delta, samples):
        self.q.absorb(delta.data_ptr(), samples)

    def sample_log(self, first, count, k):
        self.stream.wait_event(self.free[k])        # frame k's previous log has been exchanged
        lp = self.lens.data_ptr() + 4 * k
        self.q.sample_range_log(1, first, count, self.logs[k].data_ptr(), self.log_cap, lp, stream=self.stream)
        self.ready[k].record(self.stream)
        return k

    def local_log(self, k):
        cur = self.torch.cuda.current_stream(self.device)
        cur.wait_event(self.ready[k])
        length = int(self.lens[k].item())
        if length > self.log_cap:
            raise RuntimeError(f"epoch log overflow: {length} > {self.log_cap}")
        out = self.logs[k][:length].clone()
        self.free[k].record(cur)
        return out

    def absorb_log(self, log, samples):
        self.q.absorb_log(log.data_ptr(), int(log.numel()), samples)

    def check(self) -> bool:
        stopped, _, _ = self.q.check_stop()
        return stopped

    def flag_tensor(self, value):
        return self.torch.tensor([1 if value else 0], dtype=self.torch.int32, device=self.device)


def epochs_needed(omega_ceil: int, epoch_len: int) -> int:
    return math.ceil(omega_ceil / epoch_len)
