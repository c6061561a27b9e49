"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Integer results (pairs, distances, path counts, meeting sets, sampled paths,
counters, tau, stop epoch) must match bit for bit; the stop-check maxima
must agree to 1e-12 relative (both sides use the same IEEE operation
sequence, so they are expected to be identical).
"""
import math
import os

import numpy as np
import pytest

from paper_1910_11039_gb300 import inputs as I

pytestmark = pytest.mark.gpu

REL = 1e-12


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


def layered_graph(m, layers=4):
    """Complete bipartite joins between consecutive layers of m vertices:
    pairs two layers apart meet in a whole layer (meeting sets of size m)."""
    src, dst = [], []
    for L in range(layers - 1):
        a = np.arange(L * m, (L + 1) * m)
        b = np.arange((L + 1) * m, (L + 2) * m)
        aa, bb = np.meshgrid(a, b, indexing="ij")
        src.append(aa.ravel())
        dst.append(bb.ravel())
    return I.csr_from_edges(layers * m, np.concatenate(src), np.concatenate(dst), name=f"layered{m}")


GRAPHS = {
    "er2000": lambda: I.config_graph("er2000"),
    "rmat12": lambda: I.config_graph("rmat12"),
    "rmat14": lambda: I.config_graph("rmat14"),
    "grid64": lambda: I.config_graph("grid64"),
    "rgg5k": lambda: I.config_graph("rgg5k"),
    "fullgrid64": lambda: I.full_grid_graph(64, 64),    # path counts beyond 2^K: scaled layers
    "star": lambda: I.star_graph(257),
    "path": lambda: I.path_graph(300),
    "edge": lambda: I.path_graph(2),
    "layered": lambda: layered_graph(700),              # meeting sets larger than shared memory
    "rhg4k": lambda: I.config_graph("rhg4k"),           # random hyperbolic, power-law exponent 3
}


def oracle_trace(orc, g, seed, tag, first, count):
    ws = orc.Workspace(g)
    out = []
    for i in range(first, first + count):
        path, info = ws.sample(seed, tag, i)
        out.append((path, info))
    return out


def compare_trace(recs, paths, ora, cap):
    for k, (r, (path, info)) in enumerate(zip(recs, ora)):
        got = (r.s, r.t, r.d, r.sigma, r.meet_size, r.chosen, r.e_scan, r.n_interior, r.scaled)
        want = (info.s, info.t, info.d, info.sigma, info.meet_size, info.chosen, info.e_scan,
                info.n_interior, info.scaled)
        assert got == want, (k, got, want)
        m = min(len(path), cap)
        assert np.array_equal(paths[k, :m], path[:m]), k


@pytest.mark.parametrize("name", list(GRAPHS))
def test_trace_matches_oracle(K, orc, name):
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.05, delta=0.1, seed=7, n_calib=100)
    count = 300
    cap = 512
    recs, paths = q.sample_trace(1, 1000, count, path_cap=cap)
    compare_trace(recs, paths, oracle_trace(orc, g, 7, 1, 1000, count), cap)
    if name == "layered":
        assert max(r.meet_size for r in recs) > 512
    if name == "fullgrid64":
        assert any(r.scaled for r in recs)


@pytest.mark.parametrize("name", ["er2000", "rmat14", "grid64", "fullgrid64", "layered"])
@pytest.mark.parametrize("rule", [0, 1])
def test_calibration_matches_oracle(K, orc, name, rule):
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.05, delta=0.1, seed=3, n_calib=700, delta_rule=rule)
    LL, LU, cal = q.budgets()
    want_cal, _ = orc.run_samples(g, 3, 0, 0, 700)
    assert np.array_equal(cal, want_cal)
    wLL, wLU, C = orc.calibrate_L(want_cal, 700, 0.05, 0.1, rule=rule, beta=1e-3)
    np.testing.assert_allclose(LL, wLL, rtol=REL, atol=0)
    np.testing.assert_allclose(LU, wLU, rtol=REL, atol=0)
    info = q.info()
    assert info.balance_C == C
    assert info.omega == orc.omega(0.05, 0.1, orc.vertex_diameter_bound(g))


@pytest.mark.parametrize("name,E,epochs", [
    ("er2000", 97, 5), ("rmat12", 500, 3), ("rmat14", 1000, 2), ("grid64", 300, 3),
    ("rgg5k", 256, 2), ("fullgrid64", 200, 2), ("star", 64, 3), ("layered", 400, 2), ("rhg4k", 300, 2),
])
def test_epoch_counters_bit_exact(K, orc, name, E, epochs):
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.01, delta=0.1, seed=11, n_calib=100)
    for e in range(epochs):
        q.sample_epoch(E)
        res = q.result(btilde=False)
        assert res["tau"] == (e + 1) * E
        want, st = orc.run_samples(g, 11, 1, 0, (e + 1) * E)
        assert np.array_equal(res["counts"], want), (name, e)
    info = q.info()
    assert info.samples == epochs * E and info.e_scan == st.e_scan
    assert info.connected == st.connected and info.interior == st.interior
    assert info.scaled == st.scaled


@pytest.mark.parametrize("name,eps,E", [
    ("er2000", 0.05, 100), ("grid64", 0.05, 250), ("rmat14", 0.03, 500), ("rgg5k", 0.05, 300),
    ("star", 0.05, 50), ("path", 0.05, 200), ("rhg4k", 0.03, 256),
])
@pytest.mark.parametrize("rule", [0, 1])
def test_full_run_matches_oracle(K, orc, name, eps, E, rule):
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=eps, delta=0.1, seed=1, delta_rule=rule)
    stopped, epochs = False, 0
    while not stopped:
        q.sample_epoch(E)
        stopped, mf, mg = q.check_stop()
        epochs += 1
        assert epochs < 100000
    res = q.result()
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=1, epoch_len=E, delta_rule=rule)
    assert R.stopped
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch == epochs - 1
    assert np.array_equal(res["counts"], counts)
    assert math.isclose(mf, R.max_f, rel_tol=REL, abs_tol=0) and math.isclose(mg, R.max_g, rel_tol=REL, abs_tol=0)
    np.testing.assert_array_equal(res["btilde"], counts / np.float64(R.tau))
    if g.n <= 5000:
        b = orc.brandes(g)
        assert np.abs(res["btilde"] - b).max() <= eps


def test_run_loop_matches_manual_epochs(K, orc):
    g = GRAPHS["er2000"]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.05, delta=0.1, seed=1)
    assert q.run(100, sync_every=3)
    res = q.result()
    counts, cal, LL, LU, R = orc.kadabra(g, 0.05, 0.1, seed=1, epoch_len=100)
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
    assert np.array_equal(res["counts"], counts)
    # epochs enqueued after the stop take no samples
    q.sample_epoch(100)
    assert q.result(btilde=False)["tau"] == R.tau


@pytest.mark.parametrize("name,eps,E,frames", [
    ("er2000", 0.05, 100, 8), ("er2000", 0.05, 7, 1), ("grid64", 0.05, 250, 2), ("rmat14", 0.03, 500, 8),
    ("rmat14", 0.03, 64, 3), ("rgg5k", 0.05, 300, 16), ("star", 0.05, 50, 4), ("path", 0.05, 200, 8),
    ("fullgrid64", 0.05, 150, 4), ("rhg4k", 0.03, 128, 8),
])
def test_pipelined_run_matches_oracle(K, orc, name, eps, E, frames):
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=eps, delta=0.1, seed=1)
    q.run_pipelined(E, frames=frames)
    res = q.result()
    info = q.info()
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=1, epoch_len=E)
    assert R.stopped and info.stopped == 1
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch == info.epochs - 1
    assert np.array_equal(res["counts"], counts)
    # only samples of checked epochs count: those after the stop are discarded
    assert info.samples == R.tau and info.e_scan == R.e_scan
    assert math.isclose(info.max_f, R.max_f, rel_tol=REL, abs_tol=0)
    assert math.isclose(info.max_g, R.max_g, rel_tol=REL, abs_tol=0)
    # a second pipelined launch on a stopped query takes no samples
    q.run_pipelined(E, frames=frames)
    assert q.result(btilde=False)["tau"] == R.tau


def test_pipelined_run_after_reset_and_until_omega(K, orc):
    g = GRAPHS["er2000"]()
    G = K.Graph.from_inputs(g)
    # eps so small relative to the graph that the run ends at the omega cap
    q = K.Query(G, eps=0.2, delta=0.9, seed=6, n_calib=50, delta_rule=0)
    q.run_pipelined(33, frames=2)
    info = q.info()
    counts, cal, LL, LU, R = orc.kadabra(g, 0.2, 0.9, seed=6, epoch_len=33, n_calib=50, delta_rule=0)
    assert info.tau == R.tau and info.stop_epoch == R.stop_epoch
    assert np.array_equal(q.result()["counts"], counts)
    q.reset()
    q.run_pipelined(33, frames=5)
    assert q.info().tau == R.tau and np.array_equal(q.result()["counts"], counts)


def test_sharded_epochs_on_one_gpu(K, orc):
    """Two ranks' shares of every epoch sampled into separate device arrays,
    summed and absorbed (the sharded epoch aggregate), equal a single run."""
    import torch
    from paper_1910_11039_gb300.distributed import epoch_share
    g = GRAPHS["rmat14"]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.03, delta=0.1, seed=1)
    E, tau, epochs = 500, 0, 0
    omega_ceil = q.info().omega_ceil
    d = [torch.zeros(g.n, dtype=torch.int32, device="cuda") for _ in range(2)]
    while True:
        m = min(E, omega_ceil - tau)
        for r in range(2):
            d[r].zero_()
            first, count = epoch_share(tau, m, 2, r)
            q.sample_range(1, first, count, d[r].data_ptr())
        d[0] += d[1]
        q.absorb(d[0].data_ptr(), m)
        tau += m
        epochs += 1
        stopped, mf, mg = q.check_stop()
        if stopped:
            break
    counts, cal, LL, LU, R = orc.kadabra(g, 0.03, 0.1, seed=1, epoch_len=E)
    res = q.result()
    assert res["tau"] == R.tau == tau and res["stop_epoch"] == R.stop_epoch == epochs - 1
    assert np.array_equal(res["counts"], counts)
    assert math.isclose(mf, R.max_f, rel_tol=REL, abs_tol=0)


def test_sharded_run_driver_single_rank(K, orc):
    import torch
    import torch.distributed as dist
    from paper_1910_11039_gb300.distributed import LibraryShard, ShardedRun
    import os
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        g = GRAPHS["er2000"]()
        G = K.Graph.from_inputs(g)
        q = K.Query(G, eps=0.05, delta=0.1, seed=1)
        shard = LibraryShard(q)
        stopped, tau, epochs = ShardedRun(shard, shard, q.info().omega_ceil, dist).run(100)
        counts, cal, LL, LU, R = orc.kadabra(g, 0.05, 0.1, seed=1, epoch_len=100)
        assert stopped and tau == R.tau and epochs == R.stop_epoch + 1
        assert np.array_equal(q.result()["counts"], counts)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,eps,E", [("rmat14", 0.03, 500), ("grid64", 0.05, 250)])
def test_sharded_log_epochs_on_one_gpu(K, orc, name, eps, E):
    """Three ranks' shares of every epoch sampled into separate epoch logs,
    concatenated and absorbed (the log exchange), equal a single run."""
    import torch
    from paper_1910_11039_gb300.distributed import epoch_share
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=eps, delta=0.1, seed=1)
    info = q.info()
    cap = E * max(1, info.vertex_diameter)
    logs = [torch.empty(cap, dtype=torch.int32, device="cuda") for _ in range(3)]
    lens = torch.zeros(3, dtype=torch.int32, device="cuda")
    tau, epochs = 0, 0
    while True:
        m = min(E, info.omega_ceil - tau)
        for r in range(3):
            first, count = epoch_share(tau, m, 3, r)
            q.sample_range_log(1, first, count, logs[r].data_ptr(), cap, lens.data_ptr() + 4 * r)
        ln = lens.tolist()
        assert max(ln) <= cap
        allv = torch.cat([logs[r][:ln[r]] for r in range(3)])
        q.absorb_log(allv.data_ptr(), allv.numel(), m)
        tau += m
        epochs += 1
        stopped, mf, mg = q.check_stop()
        if stopped:
            break
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=1, epoch_len=E)
    res = q.result()
    assert res["tau"] == R.tau == tau and res["stop_epoch"] == R.stop_epoch == epochs - 1
    assert np.array_equal(res["counts"], counts)


def test_sharded_log_driver_single_rank(K, orc):
    # the overlapped driver (epoch e + 1 sampled on a side stream while epoch
    # e's logs are exchanged over NCCL, folded and checked) on a one-rank group
    import torch.distributed as dist
    from paper_1910_11039_gb300.distributed import LibraryShard, ShardedRun
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    os.environ["MASTER_ADDR"], os.environ["MASTER_PORT"] = "127.0.0.1", str(port)
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        g = GRAPHS["rmat14"]()
        G = K.Graph.from_inputs(g)
        q = K.Query(G, eps=0.03, delta=0.1, seed=1)
        shard = LibraryShard(q, log_cap=256 * max(1, q.info().vertex_diameter))
        stopped, tau, epochs = ShardedRun(shard, shard, q.info().omega_ceil, dist).run_logs(256)
        counts, cal, LL, LU, R = orc.kadabra(g, 0.03, 0.1, seed=1, epoch_len=256)
        assert stopped and tau == R.tau and epochs == R.stop_epoch + 1
        assert np.array_equal(q.result()["counts"], counts)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,eps,E,k", [("er2000", 0.05, 100, 4), ("rmat14", 0.03, 500, 1), ("grid64", 0.05, 250, 7)])
def test_graph_epochs_match_oracle(K, orc, name, eps, E, k):
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=eps, delta=0.1, seed=1)
    assert q.run_graph(E, epochs_per_graph=k)
    res = q.result()
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=1, epoch_len=E)
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
    assert np.array_equal(res["counts"], counts)
    stop_ns = q.info().stop_ns
    assert 0 < stop_ns <= K.device_clock()
    # the instantiated graph is reused after a reset
    q.reset()
    assert q.info().stop_ns == 0
    assert q.run_graph(E, epochs_per_graph=k)
    assert np.array_equal(q.result()["counts"], counts)


def test_reset_reproduces(K):
    g = GRAPHS["rmat12"]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.02, delta=0.1, seed=5)
    q.run(300)
    a = q.result()
    q.reset()
    q.run(300)
    b = q.result()
    assert a["tau"] == b["tau"] and a["stop_epoch"] == b["stop_epoch"]
    assert np.array_equal(a["counts"], b["counts"])


@pytest.mark.parametrize("variant", ["off64", "threads128", "threads512", "one_slot", "device_ptrs", "pinned",
                                     "pinned_off64"])
def test_launch_variants_agree(K, orc, variant):
    import torch
    g = GRAPHS["rmat14"]()
    kw = {}
    if variant == "off64":
        G = K.Graph.from_inputs(g, offsets_64=True)
    elif variant.startswith("pinned"):
        # page-locked host columns are read in place by the adjacency builder
        o64 = variant == "pinned_off64"
        off = torch.from_numpy(g.offsets if o64 else g.offsets32()).pin_memory()
        col = torch.from_numpy(g.cols).pin_memory()
        G = K.Graph(g.n, off.numpy(), col.numpy(), offsets_64=o64)
        assert G.info()["max_degree"] == int(np.diff(g.offsets).max())
    elif variant == "device_ptrs":
        off = torch.from_numpy(g.offsets32()).cuda()
        col = torch.from_numpy(g.cols).cuda()
        G = K.Graph(g.n, off, col, device_ptrs=True)
    else:
        G = K.Graph.from_inputs(g)
        kw = {"threads128": dict(threads=128), "threads512": dict(threads=512), "one_slot": dict(slots=1)}[variant]
    q = K.Query(G, eps=0.02, delta=0.1, seed=2, n_calib=100, **kw)
    q.sample_epoch(1500)
    res = q.result(btilde=False)
    want, _ = orc.run_samples(g, 2, 1, 0, 1500)
    assert np.array_equal(res["counts"], want)


@pytest.mark.parametrize("name,cap", [("er2000", 64), ("rmat14", 96), ("grid64", 200), ("layered", 900),
                                      ("fullgrid64", 1000), ("star", 40)])
def test_small_queue_capacity_spills_and_matches_oracle(K, orc, name, cap):
    # A queue capacity far below what most samples touch: those samples run
    # out of positions, clear their slot and run again on a full-capacity
    # spill slot.  Per-sample records, epoch counters and the pipelined run
    # must still equal the oracle's.
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.03, delta=0.1, seed=5, n_calib=100, queue_cap=cap)
    info = q.info()
    assert info.queue_cap == cap and info.spill_slots == 2
    recs, paths = q.sample_trace(1, 0, 200, path_cap=512)
    compare_trace(recs, paths, oracle_trace(orc, g, 5, 1, 0, 200), 512)
    assert max(r.e_scan for r in recs) > 0
    q.sample_epoch(700)
    want, st = orc.run_samples(g, 5, 1, 0, 700)
    res = q.result(btilde=False)
    assert np.array_equal(res["counts"], want)
    info = q.info()
    assert info.samples == 700 and info.e_scan == st.e_scan and info.device_error == 0
    q.reset()
    q.run_pipelined(128, frames=4)
    counts, cal, LL, LU, R = orc.kadabra(g, 0.03, 0.1, seed=5, n_calib=100, epoch_len=128)
    res = q.result(btilde=False)
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
    assert np.array_equal(res["counts"], counts)


@pytest.mark.parametrize("name,eps,E,cap", [
    ("er2000", 0.05, 100, 0), ("rmat14", 0.03, 256, 0), ("grid64", 0.05, 250, 0), ("layered", 0.05, 200, 0),
    ("fullgrid64", 0.05, 150, 0), ("rhg4k", 0.03, 128, 0), ("rmat14", 0.03, 128, 300), ("grid64", 0.05, 128, 500),
])
def test_cooperative_layers_match_oracle(K, orc, name, eps, E, cap):
    # coop_edges = 1 posts every layer of more than one chunk of frontier
    # vertices for other CTAs to expand together with the sample's own CTA
    # (with a small queue capacity, also on spill slots); the pipelined run
    # must still end exactly as the oracle's.
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    kw = dict(queue_cap=cap) if cap else {}
    q = K.Query(G, eps=eps, delta=0.1, seed=9, coop_edges=1, threads=256, **kw)
    q.run_pipelined(E, frames=8)
    res = q.result(btilde=False)
    info = q.info()
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=9, epoch_len=E)
    assert info.device_error == 0
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
    assert np.array_equal(res["counts"], counts)
    assert info.samples == R.tau and info.e_scan == R.e_scan


@pytest.mark.parametrize("name,eps,E,threads", [
    ("er2000", 0.05, 100, 1024), ("rmat14", 0.03, 256, 1024), ("rmat14", 0.03, 256, 128), ("layered", 0.05, 200, 256),
    ("rhg4k", 0.03, 128, 512), ("fullgrid64", 0.05, 150, 1024),
])
def test_probe_pass_matches_oracle(K, orc, name, eps, E, threads):
    # Small-diameter queries probe a layer against a shared-memory bitmap of
    # the other side's frontier first (probe_edges 1 = every layer, 0 = the
    # default threshold, -1 = never; 128 threads get the smallest map, 2^15
    # bits, which skips frontiers above 2048 vertices).  With the probe, without it,
    # and in the oracle the run ends alike, and the adjacency entries scanned
    # are the same.
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=11, epoch_len=E)
    ora = oracle_trace(orc, g, 11, 1, 0, 64)
    for probe in (1, 0, -1):
        q = K.Query(G, eps=eps, delta=0.1, seed=11, threads=threads, probe_edges=probe)
        q.run_pipelined(E, frames=4)
        res = q.result(btilde=False)
        info = q.info()
        assert info.device_error == 0
        assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
        assert np.array_equal(res["counts"], counts)
        assert info.samples == R.tau and info.e_scan == R.e_scan
        recs, paths = q.sample_trace(1, 0, 64, path_cap=256)
        compare_trace(recs, paths, ora, 256)
        q.free()


@pytest.mark.parametrize("name,eps,E", [("rmat14", 0.03, 128), ("grid64", 0.05, 100), ("er2000", 0.05, 64)])
def test_adaptive_lookahead_matches_full_lookahead(K, orc, name, eps, E):
    # Near the predicted stop a pipelined launch opens fewer epoch frames
    # (the default) than KADABRA_FULL_LOOKAHEAD keeps open; the scheduling
    # differs, the run's end does not.
    g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=13, epoch_len=E)
    launched = {}
    for flags in (0, K.FULL_LOOKAHEAD):
        q = K.Query(G, eps=eps, delta=0.1, seed=13, flags=flags)
        q.run_pipelined(E, frames=16)
        res = q.result(btilde=False)
        info = q.info()
        assert info.device_error == 0
        assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
        assert np.array_equal(res["counts"], counts)
        assert info.samples == R.tau and info.e_scan == R.e_scan
        launched[flags] = q.last_launch().samples
        q.free()
    assert launched[0] >= R.tau and launched[K.FULL_LOOKAHEAD] >= R.tau


def test_omega_clip_and_single_samples(K, orc):
    g = GRAPHS["er2000"]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.2, delta=0.1, seed=4, n_calib=50)
    info = q.info()
    for _ in range(3):
        q.sample_epoch(1)
    assert q.result(btilde=False)["tau"] == 3
    q.sample_epoch(1 << 31)     # clipped at ceil(omega)
    res = q.result(btilde=False)
    assert res["tau"] == info.omega_ceil
    want, _ = orc.run_samples(g, 4, 1, 0, info.omega_ceil)
    assert np.array_equal(res["counts"], want)
    stopped, mf, mg = q.check_stop()
    assert stopped  # tau >= omega


def test_strict_mode_reports_sigma_overflow(K):
    g = GRAPHS["fullgrid64"]()
    G = K.Graph.from_inputs(g)
    # the calibration samples already meet path counts above 2^K
    with pytest.raises(K.KadabraError) as ei:
        K.Query(G, eps=0.05, delta=0.1, seed=7, n_calib=200, flags=K.STRICT_SIGMA)
    assert ei.value.status == 4
    # a query calibrated on few samples reports it from its adaptive epochs
    q = None
    for n_calib in (1, 2, 3, 4, 5):
        try:
            q = K.Query(G, eps=0.05, delta=0.1, seed=7, n_calib=n_calib, flags=K.STRICT_SIGMA)
            break
        except K.KadabraError as e:
            assert e.status == 4
    if q is None:
        pytest.skip("every short calibration already overflowed")
    q.sample_epoch(2000)
    with pytest.raises(K.KadabraError) as ei:
        q.check_stop()
    assert ei.value.status == 4


def test_disconnected_pairs_count_but_add_nothing(K, orc):
    # two disjoint paths: pairs across components are taken and contribute nothing
    src = np.concatenate([np.arange(49), np.arange(50, 99)])
    dst = src + 1
    g = I.csr_from_edges(100, src, dst)
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.02, delta=0.1, seed=9, n_calib=100)
    assert q.info().omega_ceil > 4000
    q.sample_epoch(4000)
    res = q.result(btilde=False)
    want, st = orc.run_samples(g, 9, 1, 0, 4000)
    assert np.array_equal(res["counts"], want)
    assert 0 < st.connected < 4000
    assert q.info().connected == st.connected


@pytest.mark.parametrize("name", ["er2000", "rmat14", "grid64", "grid256", "path", "star", "disjoint", "edgeless",
                                  "rmat12_raw", "rgg5k_raw", "big_second"])
def test_vertex_diameter_bound_matches_oracle(K, orc, name):
    if name == "disjoint":
        src = np.concatenate([np.arange(49), np.arange(50, 70), [80, 81]])
        g = I.csr_from_edges(100, src, src + 1)
    elif name == "edgeless":
        g = I.csr_from_edges(5, np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64))
    elif name == "rmat12_raw":
        g = I.rmat_graph(12, 4, seed=77)        # many components and isolated vertices
    elif name == "rgg5k_raw":
        g = I.rgg_graph(5000, 4, seed=3)        # sparse: many components of all sizes
    elif name == "big_second":
        # a short path on the low ids, a long path (the largest component) after it
        src = np.concatenate([np.arange(0, 9), np.arange(10, 299)])
        g = I.csr_from_edges(300, src, src + 1)
    else:
        g = GRAPHS[name]() if name in GRAPHS else I.config_graph(name)
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.05, delta=0.1, seed=1, n_calib=10)
    assert q.info().vertex_diameter == orc.vertex_diameter_bound(g)
    assert q.info().diameter_ms > 0 and q.info().calibration_ms > 0
    if name == "edgeless":
        q.sample_epoch(50)
        assert q.result(btilde=False)["counts"].sum() == 0 and q.info().connected == 0


def _two_components_star_and_path():
    # a star of 40 vertices (vertex diameter 3) and a separate path of 12
    # (vertex diameter 12): the largest component is the star, and the path's
    # bound 2 * ecc(0) + 1 = 23 exceeds the star's exact value
    pairs = [(0, i) for i in range(1, 40)] + [(40 + i, 41 + i) for i in range(11)]
    p = np.array(pairs)
    return I.csr_from_edges(52, p[:, 0], p[:, 1])


@pytest.mark.parametrize("name", ["er2000", "rmat12", "grid64", "rgg5k", "path", "star", "fullgrid64", "layered",
                                  "rhg4k", "cycle", "disjoint"])
def test_exact_vertex_diameter_matches_oracle(K, orc, name):
    if name == "cycle":
        g = I.cycle_graph(301)
    elif name == "disjoint":
        a, b = I.full_grid_graph(9, 9), I.path_graph(30)
        src = np.concatenate([np.repeat(np.arange(a.n), a.degrees), a.n + np.repeat(np.arange(b.n), b.degrees)])
        dst = np.concatenate([a.cols, a.n + b.cols])
        g = I.csr_from_edges(a.n + b.n, src, dst)
    else:
        g = GRAPHS[name]()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.05, delta=0.1, seed=1, n_calib=100, vertex_diameter=-1)
    info = q.info()
    want = orc.vertex_diameter_exact(g)
    assert info.vd_exact == 1 and info.vertex_diameter == want, (info.vertex_diameter, want)
    assert info.vertex_diameter <= orc.vertex_diameter_bound(g)
    assert info.omega == orc.omega(0.05, 0.1, want)


def test_exact_vertex_diameter_of_a_smaller_component(K, orc):
    # the largest component is a star (vertex diameter 3); a separate path of
    # 12 vertices has the larger vertex diameter (12) and a bound of 23: it is
    # searched too, and the exact value is the path's
    g = _two_components_star_and_path()
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.05, delta=0.1, seed=1, n_calib=100, vertex_diameter=-1)
    info = q.info()
    assert orc.vertex_diameter_exact(g) == 12
    assert info.vd_exact == 1 and info.vertex_diameter == 12


@pytest.mark.parametrize("name", ["er2000", "grid64"])
def test_whole_run_with_exact_diameter_matches_oracle(K, orc, name):
    g = GRAPHS[name]()
    vd = orc.vertex_diameter_exact(g)
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.05, delta=0.1, seed=4, vertex_diameter=-1)
    assert q.info().vertex_diameter == vd
    q.run_pipelined(100, frames=8)
    res = q.result(btilde=False)
    counts, cal, LL, LU, R = orc.kadabra(g, 0.05, 0.1, seed=4, epoch_len=100, vertex_diameter=vd)
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
    assert np.array_equal(res["counts"], counts)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["rmat20", "grid512", "rmat26"])
def test_exact_vertex_diameter_at_size_is_consistent(K, orc, name):
    # Too large for all-pairs; what holds at any size: the eccentricity of any
    # vertex v satisfies ecc(v) + 1 <= VD <= 2 ecc(v) + 1 within its
    # component, and the exact value is at most the bound.
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order, connected_components
    g = I.config_graph(name)
    G = K.Graph.from_inputs(g, offsets_64=g.nnz >= 2**31, skip_validate=True)
    q = K.Query(G, eps=0.01, delta=0.1, seed=1, n_calib=64, vertex_diameter=-1)
    info = q.info()
    # R-MAT graphs end iFUB after a few searches; a mesh's wide fringes may
    # stop it at its effort bound with a proven upper bound instead
    assert info.vd_exact == 1 or name.startswith("grid")
    assert info.vertex_diameter <= orc.vertex_diameter_bound(g)
    if g.nnz >= 2**28:
        return      # the host-side searches below would take minutes
    A = csr_matrix((np.ones(g.nnz, dtype=np.int8), g.cols, g.offsets), shape=(g.n, g.n))
    ncomp, labels = connected_components(A, directed=False)
    big = np.bincount(labels).argmax()
    rng = np.random.default_rng(0)
    cand = np.nonzero(labels == big)[0]
    for v in rng.choice(cand, 4, replace=False):
        order, pred = breadth_first_order(A, int(v), directed=False, return_predecessors=True)
        depth = np.zeros(g.n, dtype=np.int64)
        for x in order[1:]:
            depth[x] = depth[pred[x]] + 1
        ecc = int(depth[order].max())
        assert ecc + 1 <= info.vertex_diameter <= 2 * ecc + 1 or (not info.vd_exact and ecc + 1 <= info.vertex_diameter)


@pytest.mark.slow
def test_rmat20_full_size_epoch_and_trace(K, orc):
    """R-MAT scale 20 (the measured workload) at full size, in the launch
    configuration the benchmark times: one epoch bit-exact, plus per-sample
    records of a sampled index range."""
    g = I.config_graph("rmat20")
    G = K.Graph.from_inputs(g)
    q = K.Query(G, eps=0.01, delta=0.1, seed=1)
    E = 4096
    q.sample_epoch(E)
    res = q.result(btilde=False)
    want, st = orc.run_samples(g, 1, 1, 0, E)
    assert np.array_equal(res["counts"], want)
    info = q.info()
    assert info.e_scan == st.e_scan and info.connected == st.connected
    assert info.vertex_diameter == orc.vertex_diameter_bound(g)
    recs, paths = q.sample_trace(1, 123456, 64, path_cap=64)
    compare_trace(recs, paths, oracle_trace(orc, g, 1, 1, 123456, 64), 64)
    # calibration counts and budgets at full size
    LL, LU, cal = q.budgets()
    want_cal, _ = orc.run_samples(g, 1, 0, 0, info.n_calib)
    assert np.array_equal(cal, want_cal)
    wLL, wLU, _ = orc.calibrate_L(want_cal, info.n_calib, 0.01, 0.1)
    np.testing.assert_allclose(LL, wLL, rtol=REL, atol=0)


@pytest.mark.slow
def test_grid4096_full_size_sampled(K, orc):
    """The 4096 x 4096 grid with 10% of the edges deleted (the high-diameter
    workload) at full size: vertex-diameter bound, and per-sample records of
    sampled indices (paths thousands of layers long, scaled path counts)."""
    g = I.config_graph("grid4096")
    G = K.Graph.from_inputs(g, skip_validate=True)
    q = K.Query(G, eps=0.01, delta=0.1, seed=1, n_calib=64)
    info = q.info()
    assert info.vertex_diameter == orc.vertex_diameter_bound(g)
    assert info.omega == orc.omega(0.01, 0.1, info.vertex_diameter)
    cap = 12000
    recs, paths = q.sample_trace(1, 777, 6, path_cap=cap)
    compare_trace(recs, paths, oracle_trace(orc, g, 1, 1, 777, 6), cap)
    assert all(r.scaled for r in recs)
    assert max(r.d for r in recs) > 1000


@pytest.mark.slow
def test_rmat26_full_size_sampled(K, orc):
    """R-MAT scale 26, edge factor 16 (int64 offsets) at full size: the
    vertex-diameter bound, one epoch of counters bit-exact, and per-sample
    records of a sampled index range."""
    g = I.config_graph("rmat26")
    assert g.n == 1 << 26 and g.nnz > 2_000_000_000
    G = K.Graph.from_inputs(g, offsets_64=True, skip_validate=True)
    q = K.Query(G, eps=0.01, delta=0.1, seed=1, n_calib=256, threads=512)
    info = q.info()
    assert info.offsets_64 == 1
    assert info.vertex_diameter == orc.vertex_diameter_bound(g)
    E = 512
    q.sample_epoch(E)
    res = q.result(btilde=False)
    want, st = orc.run_samples(g, 1, 1, 0, E)
    assert np.array_equal(res["counts"], want)
    assert q.info().e_scan == st.e_scan
    recs, paths = q.sample_trace(1, 5_000_000, 32, path_cap=64)
    compare_trace(recs, paths, oracle_trace(orc, g, 1, 1, 5_000_000, 32), 64)


def _sha(a):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8)).hexdigest()


def _graph_sha(g):
    import hashlib
    h = hashlib.sha256()
    h.update(np.int64(g.n).tobytes())
    h.update(np.ascontiguousarray(g.offsets, dtype=np.int64).view(np.uint8))
    h.update(np.ascontiguousarray(g.cols, dtype=np.int32).view(np.uint8))
    return h.hexdigest()


@pytest.mark.slow
@pytest.mark.parametrize("name,threads", [("rmat26", 1024), ("grid4096", 1024)])
def test_whole_run_at_full_size_matches_oracle_golden(K, name, threads):
    """The two largest single-query workloads, R-MAT scale 26 and the
    4096 x 4096 grid, through the whole method in the benchmarked form
    (diameter bound, calibration, pipelined adaptive phase with E = 1024 and
    8 frames): omega, the diameter bound, the calibration counts, the
    balancing constant, tau, the stop epoch and the counters equal what the
    oracle alone wrote to tests/golden/<name>_run.json (make_config3_runs.py),
    and the f/g maxima agree to 1e-12 relative."""
    import json
    path = os.path.join(os.path.dirname(__file__), "golden", f"{name}_run.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written yet")
    gold = json.load(open(path))
    P = gold["params"]
    g = I.config_graph(name)
    assert g.n == gold["n"] and g.nnz == gold["nnz"]
    assert _graph_sha(g) == gold["graph_sha256"], "the input generator changed since the golden run was written"
    # R-MAT scale 26 is specified with int64 offsets (its 2.10e9 entries would
    # still fit int32 ones)
    G = K.Graph.from_inputs(g, offsets_64=name == "rmat26" or g.nnz >= 2**31, skip_validate=True)
    q = K.Query(G, eps=P["eps"], delta=P["delta"], seed=P["seed"], delta_rule=P["delta_rule"], beta=P["beta"],
                threads=threads)
    assert q.info().offsets_64 == (1 if name == "rmat26" else 0)
    info = q.info()
    assert info.omega == float.fromhex(gold["omega"])
    assert info.vertex_diameter == gold["vertex_diameter"] and info.n_calib == gold["n_calib"]
    assert info.sigma_bits == gold["sigma_bits"]
    assert info.balance_C == float.fromhex(gold["C"])
    LL, LU, cal = q.budgets()
    assert _sha(cal) == gold["cal_sha256"]
    q.run_pipelined(P["epoch_len"], frames=12)     # the benchmarked launch
    res = q.result(btilde=False)
    info = q.info()
    assert info.stopped == 1 and info.device_error == 0
    assert res["tau"] == gold["tau"] and res["stop_epoch"] == gold["stop_epoch"]
    assert int(res["counts"].sum(dtype=np.uint64)) == gold["counts_sum"]
    assert _sha(res["counts"]) == gold["counts_sha256"]
    assert info.samples == gold["tau"] and info.e_scan == gold["e_scan"]
    assert math.isclose(info.max_f, float.fromhex(gold["max_f"]), rel_tol=REL, abs_tol=0)
    assert math.isclose(info.max_g, float.fromhex(gold["max_g"]), rel_tol=REL, abs_tol=0)


@pytest.mark.slow
def test_batched_mix_members_match_oracle(K, orc):
    """Members of the 64-graph mix (R-MAT scale 12 members and the smallest
    random geometric graph) run together in one persistent launch with the
    schedule the autotuner picks for the mix: the R-MAT members bit-exact
    against full oracle runs, the random geometric member by sampled
    per-sample records."""
    from paper_1910_11039_gb300.autotune import Schedule, run_mix
    specs = I.batched_specs()
    idx = [7, 46, 47, 51]
    assert all(specs[i]["kind"] == "rmat" and specs[i]["scale"] == 12 for i in idx)
    gs = [I.graph_from_spec(specs[i], f"mix{i}") for i in idx]
    rgg = I.graph_from_spec(specs[60], "mix60")
    Gs = [K.Graph.from_inputs(g) for g in gs] + [K.Graph.from_inputs(rgg)]
    seeds = [1000 + i for i in idx] + [1060]
    Qs = [K.Query(G, eps=0.02, delta=0.1, seed=s) for G, s in zip(Gs, seeds)]
    sched = Schedule(threads=256, divisor=128, frames=4)
    b = K.Batch(rgg.n, threads=256)
    r = run_mix(b, Qs, sched)
    assert all(r["stopped"])
    for q, g, s, E in zip(Qs[:4], gs, seeds, r["epoch_lens"]):
        counts, cal, LL, LU, R = orc.kadabra(g, 0.02, 0.1, seed=s, epoch_len=E)
        res = q.result()
        assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
        assert np.array_equal(res["counts"], counts)
    recs, paths = Qs[4].sample_trace(1, 12345, 8, path_cap=4000)
    compare_trace(recs, paths, oracle_trace(orc, rgg, 1060, 1, 12345, 8), 4000)


@pytest.mark.slow
def test_rmat20_benchmarked_configuration_matches_oracle(K, orc):
    """R-MAT scale 20 (the benchmarked workload) in exactly the benchmarked
    launch configuration (pipelined, 512 threads per sample, E = 1024, 12
    frames): the whole adaptive phase ends with the oracle's tau, stop epoch
    and counters."""
    g = I.config_graph("rmat20")
    G = K.Graph.from_inputs(g, skip_validate=True)
    q = K.Query(G, eps=0.01, delta=0.1, seed=1, threads=512)
    q.run_pipelined(1024, frames=12)
    res = q.result(btilde=False)
    counts, cal, LL, LU, R = orc.kadabra(g, 0.01, 0.1, seed=1, epoch_len=1024)
    assert R.stopped and q.info().stopped == 1
    assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch
    assert np.array_equal(res["counts"], counts)


def test_checkpoint_resume_is_bit_identical(K, orc, tmp_path):
    """A query restored from a checkpoint (counters, tau, epochs) continues
    exactly as the original: same tau, stop epoch and counters, in the
    stream-ordered and the pipelined form; the checkpoint survives a file."""
    g = GRAPHS["rmat14"]()
    G = K.Graph.from_inputs(g)
    eps, E = 0.03, 200
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=4, epoch_len=E)
    assert R.stop_epoch >= 3
    a = K.Query(G, eps=eps, delta=0.1, seed=4)
    for _ in range(2):
        a.sample_epoch(E)
        stopped, _, _ = a.check_stop()
        assert not stopped
    path = tmp_path / "ck.npz"
    K.save_checkpoint(path, a.checkpoint())
    ck = K.load_checkpoint(path)
    assert ck["tau"] == 2 * E and ck["epochs"] == 2
    for form in ("epochs", "pipelined"):
        b = K.Query(G, eps=eps, delta=0.1, seed=4)
        b.restore(ck)
        if form == "epochs":
            assert b.run(E)
        else:
            b.run_pipelined(E, frames=4)
        res = b.result(btilde=False)
        assert res["tau"] == R.tau and res["stop_epoch"] == R.stop_epoch, form
        assert np.array_equal(res["counts"], counts), form
    with pytest.raises(ValueError):
        K.Query(G, eps=eps, delta=0.1, seed=5).restore(ck)
