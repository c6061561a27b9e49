"""Host logic of the serving loop, on CPU, against a fake library: admission
by device memory, the priority order handed to the batch, calibration
turning into the adaptive phase, retirement, timings."""
import types

import numpy as np
import pytest

import paper_1910_11039_gb300.server as S
from paper_1910_11039_gb300.autotune import Schedule


class FakeInfo(types.SimpleNamespace):
    pass


class FakeGraph:
    def __init__(self, n):
        self.n = n

    def info(self):
        return dict(n=self.n, nnz=4 * self.n, max_degree=4, offsets_64=0)


def make_fake(steps_needed):
    """A fake kadabra module: every query needs `steps_needed[seed]` adaptive
    steps after one calibration step; device time advances 1 ms per step."""
    clock = {"ns": 0}
    log = {"steps": [], "created": 0, "freed": 0}

    class FakeQuery:
        def __init__(self, graph, calibrate=True, eps=0.1, delta=0.1, seed=1, threads=256, vertex_diameter=0):
            self.g, self.seed, self.phase = graph, seed, 0
            self.left = steps_needed[seed]
            self.cal_left = 1
            self.stop_ns = 0
            self.vd_given = vertex_diameter
            log["created"] += 1

        def info(self):
            return FakeInfo(omega_ceil=1000 * self.g.n, vertex_diameter=7, device_bytes=40 * self.g.n,
                            n_calib=100, cal_done=100 if self.cal_left == 0 else 0, phase=self.phase,
                            stopped=int(self.phase == 2 and self.left == 0), stop_ns=self.stop_ns,
                            tau=10 * steps_needed[self.seed], stop_epoch=steps_needed[self.seed] - 1,
                            samples=11 * steps_needed[self.seed])

        def calibration_begin(self):
            assert self.phase == 0
            self.phase = 1

        def calibration_finish(self):
            assert self.phase == 1 and self.cal_left == 0
            self.phase = 2

        def pipeline_begin(self, E, frames=8):
            assert self.phase == 2

        def result(self, btilde=False):
            return {"counts": np.full(4, self.seed, dtype=np.uint32)}

        def free(self):
            log["freed"] += 1

    class FakeBatch:
        IN_ORDER, ROUND_ROBIN = 1, 0

        def __init__(self, max_n, slots=0, threads=256, offsets_64=False):
            self.last = []

        def set_policy(self, p):
            self.policy = p

        def step(self, qs, sample_budget=0):
            log["steps"].append([q.seed for q in qs])
            clock["ns"] += 1_000_000
            for q in qs:
                if q.phase == 1:
                    q.cal_left = 0
                elif q.left > 0:
                    q.left -= 1
                    if q.left == 0:
                        q.stop_ns = clock["ns"]
            self.last = qs

        def last_ms(self):
            return 1.0

        def poll(self, count):
            out = []
            for q in self.last:
                if q.phase == 1:
                    out.append(1 if q.cal_left == 0 else 0)
                else:
                    out.append(2 if q.left == 0 else 0)
            return np.array(out, dtype=np.int32)

    fake = types.SimpleNamespace(Query=FakeQuery, Batch=FakeBatch, Graph=FakeGraph,
                                 device_clock=lambda stream=None: clock["ns"])
    return fake, log


@pytest.mark.parametrize("policy", ["fifo", "shortest"])
def test_serving_loop_admits_by_memory_and_retires(monkeypatch, policy):
    steps_needed = {1: 5, 2: 1, 3: 3, 4: 2}
    fake, log = make_fake(steps_needed)
    monkeypatch.setattr(S, "K", fake)
    graphs = {"big": FakeGraph(1000), "small": FakeGraph(100)}
    # room for the big query's state plus one small one, not two big ones
    per_big = 40 * 1000 + 4 * 8 * 32 * 5 + 1
    srv = S.Server(graphs, schedule=Schedule(threads=256, divisor=1000, frames=8, min_epoch=32),
                   memory_budget=per_big + 40 * 100 + (1 << 20) + 4 * 8 * 32 * 5, policy=policy)
    reqs = [S.Request(1, "big", 0.1, seed=1), S.Request(2, "small", 0.1, seed=2),
            S.Request(3, "big", 0.1, seed=3), S.Request(4, "small", 0.1, seed=4)]
    done = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in done) == [1, 2, 3, 4]
    assert log["created"] == 4 and log["freed"] == 4
    assert srv.used == 0
    # the two big queries never shared a step (memory budget)
    for step in log["steps"]:
        assert not (1 in step and 3 in step)
    assert srv.stats["admit_waits"] > 0
    for r in done:
        assert r.time_to_stop is not None and r.time_to_stop > 0
        assert r.tau == 10 * steps_needed[r.seed]
        assert np.array_equal(r.counts, np.full(4, r.seed, dtype=np.uint32))
    if policy == "shortest":
        # among queries in their adaptive phase, the smaller graph goes first
        for step in log["steps"]:
            if 2 in step and 1 in step:
                assert step.index(2) < step.index(1)
    else:
        for step in log["steps"]:
            if 2 in step and 1 in step:
                assert step.index(1) < step.index(2)
    s = srv.summary(done)
    assert s["queries"] == 4 and s["tts_p50_s"] > 0


def test_graphs_must_share_offset_width(monkeypatch):
    fake, _ = make_fake({})

    class G64(FakeGraph):
        def info(self):
            return dict(n=self.n, nnz=4, max_degree=1, offsets_64=1)

    monkeypatch.setattr(S, "K", fake)
    with pytest.raises(ValueError):
        S.Server({"a": FakeGraph(10), "b": G64(10)}, memory_budget=1 << 30)


def test_step_budget_floor_grows_with_long_samples(monkeypatch):
    """Steps hand out at least 8 samples per slot, 32 while a query of
    diameter bound above 64 is active (its samples are long)."""
    fake, log = make_fake({1: 3, 2: 3})
    budgets = []

    class BudgetBatch(fake.Batch):
        def info(self):
            return {"slots": 10, "threads": 256, "max_n": 1000}

        def step(self, qs, sample_budget=0):
            budgets.append(sample_budget)
            super().step(qs, sample_budget)

    fake.Batch = BudgetBatch

    class LongQuery(fake.Query):
        def info(self):
            i = super().info()
            i.vertex_diameter = 500 if self.g.n == 1000 else 7
            return i

    fake.Query = LongQuery
    monkeypatch.setattr(S, "K", fake)
    srv = S.Server({"grid": FakeGraph(1000), "rmat": FakeGraph(100)}, memory_budget=1 << 30, step_ms=1e-6)
    assert srv.min_budget == 80 and srv.min_budget_long == 320
    srv.run([S.Request(1, "rmat", 0.1, seed=1)], realtime=False)
    assert min(budgets[1:]) == 80                  # short samples only: the small floor
    budgets.clear()
    srv.run([S.Request(2, "grid", 0.1, seed=2)], realtime=False)
    assert min(budgets[1:]) == 320                 # a long-sample query is active
