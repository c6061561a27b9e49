"""Many queries in one persistent launch (kadabra_batch_step).

Each query in a batch must end with exactly the tau, counters and stop epoch
it has when run alone, whatever else shares the launch, however the work is
split into steps, and when queries join between steps.
"""
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
