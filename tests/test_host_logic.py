"""Host-side logic that needs no GPU: workload specs and schedule rules."""
import math

from paper_1910_11039_gb300 import inputs as I


def test_batched_specs_follow_the_recipe():
    sp = I.batched_specs()
    assert len(sp) == 64
    rmat, rgg = sp[:56], sp[56:]
    assert all(d["kind"] == "rmat" for d in rmat) and all(d["kind"] == "rgg" for d in rgg)
    assert all(12 <= d["scale"] <= 18 and 8 <= d["edge_factor"] <= 32 for d in rmat)
    assert all(50_000 <= d["n"] <= 500_000 and d["avg_degree"] == 10 for d in rgg)
    assert [d["seed"] for d in sp] == list(range(1000, 1064))
    assert sp == I.batched_specs()                     # deterministic
    # the draws cover the ranges (both ends of the scale range appear)
    scales = {d["scale"] for d in rmat}
    assert 12 in scales and 18 in scales


def test_graph_from_spec_matches_config_graph():
    g1 = I.config_graph("rmat12")
    g2 = I.graph_from_spec(I.CONFIGS["rmat12"], "rmat12")
    assert (g1.offsets == g2.offsets).all() and (g1.cols == g2.cols).all()


def test_schedule_epoch_rule():
    from paper_1910_11039_gb300.autotune import Schedule
    s = Schedule(divisor=32, min_epoch=32, max_epoch=4096)
    for omega in (1, 10, 1000, 5000, 17_500, 35_000, 10**6, 10**9):
        E = s.epoch_len(omega)
        assert 32 <= E <= 4096 and E & (E - 1) == 0
        if 32 * 32 <= omega <= 4096 * 32:
            # nearest power of two to omega / divisor (in log scale)
            assert abs(math.log2(E) - math.log2(omega / 32)) <= 0.5 + 1e-12
    assert Schedule(divisor=8).epoch_len(8192) == 1024


def test_serving_stream_recipe():
    reqs = I.serving_requests()
    assert len(reqs) == 2000
    arr = [r["arrival"] for r in reqs]
    assert arr == sorted(arr) and arr[0] > 0
    gaps = [b - a for a, b in zip([0.0] + arr[:-1], arr)]
    mean_gap = sum(gaps) / len(gaps)
    assert abs(mean_gap - 1 / 20.0) < 0.1 / 20.0            # Poisson at 20 per second
    pool = set(I.SERVING_POOL)
    assert {r["graph"] for r in reqs} == pool                # every pool graph is drawn
    eps = [r["eps"] for r in reqs]
    assert set(eps) == {0.01, 0.005} and 0.4 < eps.count(0.01) / len(eps) < 0.6
    assert all(r["delta"] == 0.1 for r in reqs)
    assert len({r["seed"] for r in reqs}) == len(reqs)
    assert reqs == I.serving_requests()                       # deterministic
    assert set(I.SERVING_POOL) >= {f"rmat{s}" for s in range(14, 25)} | {"grid1024", "grid4096"}


def test_checkpoint_file_roundtrip(tmp_path):
    import numpy as np
    from paper_1910_11039_gb300 import kadabra as K
    ck = {"counts": np.arange(10, dtype=np.uint32), "tau": 1234, "epochs": 7, "eps": 0.05, "delta": 0.1,
          "seed": 9, "n_calib": 1000, "delta_rule": 1, "vertex_diameter": 13}
    path = tmp_path / "ck.npz"
    K.save_checkpoint(path, ck)
    back = K.load_checkpoint(path)
    assert set(back) == set(ck)
    assert np.array_equal(back["counts"], ck["counts"]) and back["counts"].dtype == np.uint32
    for k in ("tau", "epochs", "eps", "delta", "seed", "n_calib", "delta_rule", "vertex_diameter"):
        assert back[k] == ck[k] and type(back[k]) is type(ck[k])


def test_autotune_coordinate_descent_on_a_synthetic_cost():
    # The search with a stand-in runner: threads first (at the base divisor and
    # frames), then the divisor at the best threads, then frames; each schedule
    # is tried once, a trial whose queries do not all stop counts as infinite,
    # and the cheapest schedule seen wins.
    from paper_1910_11039_gb300 import autotune as AT

    def cost(s):
        return abs(s.threads - 256) + 3 * abs(math.log2(s.divisor) - 6) + 5 * abs(s.frames - 8)

    calls = []

    def runner(batch, queries, s, stream):
        calls.append(s)
        return {"ms": cost(s), "stopped": [s.frames != 16]}

    class Pool:
        def get(self, threads):
            return None

    best, trials, secs = AT.autotune([object()], Pool(), runner=runner)
    assert (best.threads, best.divisor, best.frames) == (256, 64, 8)
    assert len(calls) == len(set(calls)) == len(trials)
    assert [s.threads for s in calls[:4]] == [1024, 128, 256, 512]     # base first, then the others
    assert all(s.threads == 256 for s in calls[4:])
    assert dict(trials)[AT.Schedule(threads=256, divisor=64, frames=16)] == float("inf")
    assert min(ms for _, ms in trials) == cost(best) and secs >= 0.0
