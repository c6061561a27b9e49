"""Sharded adaptive phase over several ranks, on CPU ranks (gloo).

Each rank samples its share of every epoch with the CPU oracle, the deltas
are summed with all_reduce, rank 0 checks the stopping condition and
broadcasts it.  The result must equal the single-process run exactly: same
tau, stop epoch and counters.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_1910_11039_gb300.distributed import ShardedRun, epoch_share


def test_epoch_share_covers_the_epoch_once():
    for m in (0, 1, 7, 100, 1023):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                first, count = epoch_share(50, m, world, r)
                seen.extend(range(first, first + count))
            assert seen == list(range(50, 50 + m))


class OracleShard:
    """CPU stand-in for one rank: oracle sampling and oracle stop check."""

    def __init__(self, g, eps, delta, seed, n_calib):
        import torch
        import oracle
        self.torch, self.orc, self.g, self.seed, self.eps = torch, oracle, g, seed, eps
        vd = oracle.vertex_diameter_bound(g)
        self.omega = oracle.omega(eps, delta, vd)
        cal, _ = oracle.run_samples(g, seed, 0, 0, n_calib)
        self.LL, self.LU, _ = oracle.calibrate_L(cal, n_calib, eps, delta)
        self.counts = np.zeros(g.n, dtype=np.int64)
        self.tau = 0

    def sample(self, first, count):
        c, _ = self.orc.run_samples(self.g, self.seed, 1, first, first + count)
        return self.torch.from_numpy(c.astype(np.int32))

    def absorb(self, delta, samples):
        self.counts += delta.numpy().astype(np.int64)
        self.tau += samples

    def sample_log(self, first, count, frame):
        # the interior vertices of each sampled path, concatenated
        if not hasattr(self, "ws"):
            self.ws = self.orc.Workspace(self.g)
        parts = [self.ws.sample(self.seed, 1, i)[0] for i in range(first, first + count)]
        log = np.concatenate(parts) if parts else np.zeros(0, dtype=np.int32)
        return self.torch.from_numpy(log.astype(np.int32))

    def local_log(self, handle):
        return handle

    def absorb_log(self, log, samples):
        self.counts += np.bincount(log.numpy(), minlength=self.g.n).astype(np.int64)
        self.tau += samples

    def check(self):
        stop, _, _ = self.orc.check_stop(self.counts.astype(np.uint32), self.tau, self.omega, self.eps, self.LL, self.LU)
        return stop

    def flag_tensor(self, value):
        return self.torch.tensor([1 if value else 0], dtype=self.torch.int32)


def _rank_main(rank, world, port, out_dir, E, form="reduce"):
    import torch.distributed as dist
    import oracle
    from paper_1910_11039_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        g = I.config_graph("er2000")
        shard = OracleShard(g, 0.05, 0.1, 1, 1000)
        run = ShardedRun(shard, shard, int(np.ceil(shard.omega)), dist)
        stopped, tau, epochs = run.run(E) if form == "reduce" else run.run_logs(E)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), counts=shard.counts, tau=tau, epochs=epochs,
                 stopped=int(stopped))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("form", ["reduce", "logs"])
@pytest.mark.parametrize("world,E", [(2, 100), (3, 77)])
def test_sharded_run_equals_single_process(orc, world, E, form):
    # reduce: counter deltas summed, rank 0 checks and broadcasts;
    # logs: epoch logs all-gathered, every rank folds them and checks, with the
    # next epoch sampled before the current one is exchanged (two frames)
    import torch.multiprocessing as mp
    from paper_1910_11039_gb300 import inputs as I
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(world, _free_port(), d, E, form), nprocs=world, join=True)
        res = [np.load(os.path.join(d, f"rank{r}.npz")) for r in range(world)]
    g = I.config_graph("er2000")
    counts, cal, LL, LU, R = orc.kadabra(g, 0.05, 0.1, seed=1, epoch_len=E, n_calib=1000)
    for r in res:
        assert int(r["stopped"]) == 1
        assert int(r["tau"]) == R.tau
        assert int(r["epochs"]) == R.stop_epoch + 1
        assert np.array_equal(r["counts"].astype(np.uint32), counts)
