"""Many queries in one persistent launch (kadabra_batch_step).

Each query in a batch must end with exactly the tau, counters and stop epoch
it has when run alone, whatever else shares the launch, however the work is
split into steps, and when queries join between steps.
"""
import dataclasses

import numpy as np
import pytest

from paper_1910_11039_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_11039_gb300 import build as B
    B.build()
    from paper_1910_11039_gb300 import kadabra
    kadabra.load()
    torch.cuda.set_device(0)
    return kadabra


SPECS = [  # (graph, eps, seed, epoch length, frames)
    ("er2000", 0.05, 1, 100, 8),
    ("rmat12", 0.03, 2, 300, 4),
    ("rmat14", 0.03, 3, 500, 8),
    ("grid64", 0.05, 4, 250, 2),
    ("rgg5k", 0.05, 5, 300, 16),
    ("er2000", 0.04, 6, 64, 3),      # a second query on the same graph
]


@pytest.fixture(scope="module")
def graphs(K):
    out = {}
    for name, *_ in SPECS:
        if name not in out:
            g = I.config_graph(name)
            out[name] = (g, K.Graph.from_inputs(g))
    return out


def make_queries(K, graphs, specs=SPECS):
    qs = []
    for name, eps, seed, E, F in specs:
        g, G = graphs[name]
        q = K.Query(G, eps=eps, delta=0.1, seed=seed)
        qs.append((q, E, F, g))
    return qs


def expected(orc, g, eps, seed, E):
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=seed, epoch_len=E)
    return counts, R


def check_all(K, orc, qs, specs=SPECS):
    for (q, E, F, g), (name, eps, seed, _, _) in zip(qs, specs):
        res = q.result()
        counts, R = expected(orc, g, eps, seed, E)
        assert q.info().stopped == 1, name
        assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch, name
        assert np.array_equal(res["counts"], counts), name


@pytest.mark.parametrize("policy", [0, 1])
def test_batch_one_launch_matches_alone(K, orc, graphs, policy):
    qs = make_queries(K, graphs)
    b = K.Batch(max(g.n for g, _ in graphs.values()), policy=policy)
    for q, E, F, g in qs:
        q.pipeline_begin(E, frames=F)
    b.step([q for q, *_ in qs])
    assert b.last_ms() > 0
    check_all(K, orc, qs)


@pytest.mark.parametrize("budget,policy", [(1, 0), (97, 0), (1000, 0), (97, 1)])
def test_batch_in_small_steps_matches_alone(K, orc, graphs, budget, policy):
    qs = make_queries(K, graphs)
    b = K.Batch(max(g.n for g, _ in graphs.values()), slots=64, policy=policy)
    for q, E, F, g in qs:
        q.pipeline_begin(E, frames=F)
    for _ in range(100000):
        running = [q for q, *_ in qs if not q.info().stopped]
        if not running:
            break
        b.step(running, sample_budget=budget)
        states = b.poll(len(running))
        assert [int(x) for x in states] == [2 if q.info().stopped else 0 for q in running]
    check_all(K, orc, qs)


def test_queries_join_between_steps(K, orc, graphs):
    qs = make_queries(K, graphs)
    b = K.Batch(max(g.n for g, _ in graphs.values()))
    active = []
    for k, (q, E, F, g) in enumerate(qs):
        q.pipeline_begin(E, frames=F)
        active.append(q)
        b.step(active, sample_budget=500)          # newcomers join the running mix
    for _ in range(100000):
        running = [q for q in active if not q.info().stopped]
        if not running:
            break
        b.step(running, sample_budget=2000)
    check_all(K, orc, qs)


def test_batch_rejects_unbegun_and_oversized(K, graphs):
    g, G = graphs["rmat14"]
    q = K.Query(G, eps=0.05, delta=0.1, seed=1)
    b = K.Batch(1000)
    with pytest.raises(K.KadabraError) as ei:
        b.step([q])
    assert ei.value.status == 7
    q.pipeline_begin(100)
    with pytest.raises(K.KadabraError) as ei:
        b.step([q])
    assert ei.value.status == 1
    with pytest.raises(K.KadabraError) as ei:
        b.set_policy(2)
    assert ei.value.status == 1


def test_autotuned_schedule_matches_oracle(K, orc, graphs):
    """Every trial of the tuner is a full run; the chosen schedule's results
    are those of each query alone with the schedule's epoch length."""
    from paper_1910_11039_gb300 import autotune as AT
    qs = make_queries(K, graphs)
    Q = [q for q, *_ in qs]
    pool = AT.BatchPool(max(g.n for g, _ in graphs.values()))
    best, trials, secs = AT.autotune(Q, pool, threads=(256, 1024), divisors=(16, 64), frames=(4,))
    assert len(trials) == 5 and secs > 0          # base, one thread count, two divisors, one frame count
    assert best.threads in (256, 1024) and best.divisor in (16, 32, 64) and best.frames in (4, 8)
    r = AT.run_mix(pool.get(best.threads), Q, best)
    assert all(r["stopped"])
    for (q, _, _, g), (name, eps, seed, _, _), E in zip(qs, SPECS, r["epoch_lens"]):
        counts, R = expected(orc, g, eps, seed, E)
        res = q.result()
        assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch, name
        assert np.array_equal(res["counts"], counts), name
    # time-to-stop is measured from the launch's submission on the device clock
    assert all(0 < t <= r["ms"] + 5.0 for t in r["tts_ms"])


def test_calibration_inside_batch_matches_calibrate(K, orc, graphs):
    """Queries created without calibration take their calibration samples in
    batch steps beside running queries; budgets and results equal those of
    kadabra_calibrate and of the oracle."""
    qs = make_queries(K, graphs)                       # calibrated the usual way
    fresh = []
    for name, eps, seed, E, F in SPECS:
        g, G = graphs[name]
        fresh.append((K.Query(G, eps=eps, delta=0.1, seed=seed, calibrate=False), E, F, g))
    for (q, *_), (p, *_) in zip(qs, fresh):
        assert p.info().phase == 0 and q.info().phase == 2
        with pytest.raises(K.KadabraError) as ei:
            p.sample_epoch(10)
        assert ei.value.status == 7
    b = K.Batch(max(g.n for g, _ in graphs.values()), slots=96, policy=1)
    for q, E, F, g in qs[:3]:                          # some adaptive queries already running
        q.pipeline_begin(E, frames=F)
    active = [q for q, *_ in qs[:3]]
    for p, *_ in fresh:
        p.calibration_begin()
        active.append(p)
    with pytest.raises(K.KadabraError) as ei:
        fresh[0][0].calibration_finish()               # nothing sampled yet
    assert ei.value.status == 7
    phase = {id(p): 1 for p, *_ in fresh}
    for _ in range(100000):
        b.step(active, sample_budget=257)
        states = b.poll(len(active))
        for q, st in zip(active, states):
            inf = q.info()
            want = (1 if inf.cal_done >= inf.n_calib else 0) if inf.phase == 1 else (2 if inf.stopped else 0)
            assert st == want
        for p, E, F, g in fresh:
            if phase[id(p)] == 1 and p.info().cal_done >= p.info().n_calib:
                p.calibration_finish()
                p.pipeline_begin(E, frames=F)
                phase[id(p)] = 2
        active = [q for q in active if not (q.info().phase == 2 and q.info().stopped)]
        if not active:
            break
    for (q, *_), (p, E, F, g), (name, eps, seed, *_) in zip(qs, fresh, SPECS):
        a, c = q.budgets(), p.budgets()
        for x, y in zip(a, c):
            assert np.array_equal(x, y), name
        counts, R = expected(orc, g, eps, seed, E)
        res = p.result()
        assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch, name
        assert np.array_equal(res["counts"], counts), name


@pytest.mark.parametrize("policy", ["fifo", "shortest"])
def test_server_results_equal_alone_and_in_mix(K, orc, graphs, policy):
    """Requests served together (continuous batching, arrivals while others
    run) give the results each gives alone, and those of the oracle."""
    from paper_1910_11039_gb300.autotune import Schedule
    from paper_1910_11039_gb300.server import Request, Server
    sched = Schedule(threads=256, divisor=32, frames=4)
    reqs = [Request(i, name, eps, 0.1, seed, arrival=0.002 * i) for i, (name, eps, seed, _, _) in enumerate(SPECS)]
    reqs += [Request(10 + i, name, eps, 0.1, seed + 100, arrival=0.001 * i)
             for i, (name, eps, seed, _, _) in enumerate(SPECS[:3])]
    srv = Server({k: v[1] for k, v in graphs.items()}, schedule=sched, step_ms=2.0, policy=policy)
    mixed = {r.rid: r for r in srv.run([dataclasses.replace(r) for r in reqs])}
    assert len(mixed) == len(reqs)
    s = srv.summary(list(mixed.values()))
    assert s["queries"] == len(reqs) and s["tts_p50_s"] > 0 and s["steps"] > 1
    for r in reqs:
        alone = Server({r.graph: graphs[r.graph][1]}, schedule=sched, step_ms=2.0).run([dataclasses.replace(r)])[0]
        m = mixed[r.rid]
        assert (m.tau, m.stop_epoch) == (alone.tau, alone.stop_epoch), r
        assert np.array_equal(m.counts, alone.counts), r
        counts, R = expected(orc, graphs[r.graph][0], r.eps, r.seed, sched.epoch_len(m.omega_ceil))
        assert m.tau == R.tau and m.stop_epoch == R.stop_epoch
        assert np.array_equal(m.counts, counts)


def test_bounded_waits_end_a_step_with_a_timeout(K, orc, graphs):
    """A wait that runs out of polls ends the step with the timeout status,
    without a fault; the query then restarts and runs to the oracle's result."""
    g, G = graphs["er2000"]
    q = K.Query(G, eps=0.05, delta=0.1, seed=1)
    b = K.Batch(g.n)
    b.set_spin_limit(1)               # one frame of 16 samples: every other CTA must wait
    q.pipeline_begin(16, frames=1)
    b.step([q])
    assert b.last_ms() > 0
    assert q.info().device_error & 32
    with pytest.raises(K.KadabraError) as ei:
        q.result()
    assert ei.value.status == 6
    # the context and the query are usable again
    q.reset()
    b.set_spin_limit(1 << 24)
    q.pipeline_begin(16, frames=1)
    b.step([q])
    res = q.result()
    counts, R = expected(orc, g, 0.05, 1, 16)
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
    assert np.array_equal(res["counts"], counts)
    with pytest.raises(K.KadabraError):
        b.set_spin_limit(0)
