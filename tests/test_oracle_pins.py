"""Pins for the CPU oracle, against facts that do not come from the oracle.

Each test ties one oracle function to something fixed independently of it:
numpy's own Philox implementation, networkx's betweenness and shortest-path
enumeration, closed forms (paths, stars, cycles, complete graphs, binomial
path counts in grids), exhaustive enumeration of path distributions, and the
sample counts printed in the paper's Table II.
"""
import itertools
import math
import os

import numpy as np
import pytest

from paper_1910_11039_gb300 import inputs as I

nx = pytest.importorskip("networkx")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def to_nx(g):
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for u in range(g.n):
        for v in g.cols[g.offsets[u]:g.offsets[u + 1]]:
            if u < v:
                G.add_edge(u, int(v))
    return G


def random_small_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    m = rng.random(iu.size) < p
    return I.csr_from_edges(n, iu[m], ju[m])


# --------------------------------------------------------------------------
# Philox-4x64-10 against numpy's independent implementation
# --------------------------------------------------------------------------

@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((1, 0, 0, 0), (5, 0)),
    ((12345, 7, 1, 0), (1, 0)),
    ((2**63 + 11, 2**64 - 1, 3, 9), (0xDEADBEEF, 0x12345678)),
    ((99, 2, 0, 0), (2**64 - 1, 2**64 - 1)),
])
def test_philox_matches_numpy(orc, ctr, key):
    # numpy's Philox advances its counter before producing a block, so a
    # generator started at ctr - 1 yields the block for ctr first.
    start = np.array([ctr[0] - 1, ctr[1], ctr[2], ctr[3]], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
    want = [int(x) for x in bg.random_raw(4)]
    assert orc.philox4x64_10(ctr, key) == want


def test_pair_draw_uniform_over_ordered_pairs(orc):
    n, N = 7, 84000
    hist = np.zeros((n, n), dtype=np.int64)
    for i in range(N):
        s, t = orc.draw_pair(n, 3, 1, i)
        assert 0 <= s < n and 0 <= t < n and s != t
        hist[s, t] += 1
    cells = hist[~np.eye(n, dtype=bool)]
    exp = N / (n * (n - 1))
    chi2 = ((cells - exp) ** 2 / exp).sum()
    # 41 degrees of freedom: mean 41, sd ~9; reject only gross errors
    assert chi2 < 41 + 6 * math.sqrt(2 * 41)


# --------------------------------------------------------------------------
# Exact betweenness: closed forms and networkx
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 8, 9])
def test_brandes_path_closed_form(orc, n):
    b = orc.brandes(I.path_graph(n))
    want = [2 * i * (n - 1 - i) / (n * (n - 1)) for i in range(n)]
    np.testing.assert_allclose(b, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [3, 4, 10])
def test_brandes_star_closed_form(orc, n):
    b = orc.brandes(I.star_graph(n))
    np.testing.assert_allclose(b[0], (n - 2) / n, atol=1e-15)
    np.testing.assert_allclose(b[1:], 0.0, atol=1e-15)


def test_brandes_complete_graph_is_zero(orc):
    np.testing.assert_allclose(orc.brandes(I.complete_graph(7)), 0.0, atol=1e-15)


@pytest.mark.parametrize("n", [5, 6, 9, 12])
def test_brandes_cycle_closed_form(orc, n):
    # sum over ordered pairs of (d(s,t) - 1) split evenly over n vertices
    m = n // 2
    want = m * (m - 1) / (n * (n - 1)) if n % 2 else (m - 1) ** 2 / (n * (n - 1))
    np.testing.assert_allclose(orc.brandes(I.cycle_graph(n)), want, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brandes_matches_networkx(orc, seed):
    g = random_small_graph(25, 0.12, seed)
    G = to_nx(g)
    nxb = nx.betweenness_centrality(G, normalized=True)
    # networkx normalises unordered pairs by 2/((n-1)(n-2)); b(x) uses 1/(n(n-1))
    want = np.array([nxb[v] for v in range(g.n)]) * (g.n - 2) / g.n
    np.testing.assert_allclose(orc.brandes(g), want, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------------
# One sample: distance, path count, validity of the sampled path
# --------------------------------------------------------------------------

def check_path(g, s, t, d, interior, G):
    """interior = the d-1 interior vertices of an s-t path of length d."""
    assert len(interior) == max(d - 1, 0)
    ds = nx.single_source_shortest_path_length(G, s)
    dt = nx.single_source_shortest_path_length(G, t)
    layers = sorted(interior, key=lambda x: ds[x])
    assert [ds[x] for x in layers] == list(range(1, d))
    for x in layers:
        assert ds[x] + dt[x] == d
    full = [s] + layers + [t]
    for a, b in zip(full, full[1:]):
        assert G.has_edge(a, b)


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_sample_pair_distance_sigma_and_path(orc, seed):
    g = random_small_graph(30, 0.1, seed)
    G = to_nx(g)
    ws = orc.Workspace(g)
    for s, t in itertools.permutations(range(g.n), 2):
        interior, info = ws.sample_pair(s, t, seed=9, tag=1, idx=s * 100 + t)
        if not nx.has_path(G, s, t):
            assert info.d == -1 and len(interior) == 0
            continue
        d = nx.shortest_path_length(G, s, t)
        assert info.d == d
        assert info.sigma == sum(1 for _ in nx.all_shortest_paths(G, s, t))
        check_path(g, s, t, d, list(interior), G)


def test_sample_edge_scan_counts_expanded_degrees(orc):
    # star centre 0: pair (1, 2) expands leaf 1 (degree 1), then the tie rule
    # picks s again? no: after layer 1 the s-frontier is {0} with degree n-1,
    # the t-frontier {2} has degree 1, so t expands and meets at 0.
    g = I.star_graph(6)
    ws = orc.Workspace(g)
    interior, info = ws.sample_pair(1, 2, 1, 1, 0)
    assert list(interior) == [0] and info.d == 2 and info.e_scan == 2


@pytest.mark.parametrize("a,b", [(3, 4), (7, 7), (10, 20), (20, 20)])
def test_grid_sigma_is_binomial(orc, a, b):
    g = I.full_grid_graph(24, 24)
    ws = orc.Workspace(g)
    interior, info = ws.sample_pair(0, a * 24 + b, 1, 1, 0)
    assert info.scaled == 0
    assert info.d == a + b
    assert info.sigma == math.comb(a + b, a)


def test_grid_sigma_exact_beyond_64_bits(orc):
    # corner to corner of a 40 x 40 grid: each side's counts stay below 2^K,
    # and the meeting-set sum gives C(78, 39) ~ 2^75 exactly in 128 bits
    g = I.full_grid_graph(40, 40)
    ws = orc.Workspace(g)
    interior, info = ws.sample_pair(0, 40 * 40 - 1, 1, 1, 0)
    assert info.scaled == 0 and info.d == 78
    assert info.sigma == math.comb(78, 39) and info.sigma > 2**64


def test_layered_sigma_matches_enumeration(orc):
    # m**k shortest paths through k complete layers; networkx enumerates them
    g = I.layered_graph(3, 5)
    ws = orc.Workspace(g)
    t = 1 + 5 * 3
    interior, info = ws.sample_pair(0, t, 1, 1, 0)
    assert info.scaled == 0 and info.d == 6
    assert info.sigma == 3**5 == len(enumerate_paths(to_nx(g), 0, t))
    check_path(g, 0, t, 6, list(interior), to_nx(g))


def test_layered_sigma_exact_above_32_bits(orc):
    # 18 complete layers of 8 vertices between s and t: 8**18 = 2**54 paths.
    # Middle layers tie on frontier degree (128), so the s side expands every
    # layer after its second and its deepest scaled layer (16) holds vertices
    # with 8**15 = 2**45 paths each.  A separate star of 16384 leaves sets the
    # maximum degree: K = min(63 - 15, 63 - bitlen(n = 16531)) = 48, so every
    # per-side count stays an exact 64-bit integer and nothing is scaled.
    k = 18
    g = I.layered_graph(8, k, hub_leaves=16384)
    ws = orc.Workspace(g)
    assert ws.K == 48
    t = 1 + k * 8
    for idx in range(3):
        interior, info = ws.sample_pair(0, t, 1, 1, idx)
        assert info.scaled == 0 and info.overflow == 0 and info.d == k + 1
        assert info.sigma == 8**k
        # one interior vertex per layer, in any order
        assert sorted((int(v) - 1) // 8 for v in interior) == list(range(k))
    # counts kept to 48 bits per side (K = 47 - bitlen(max degree) = 32)
    # would have scaled these layers and lost the exact count
    _, narrow = ws.sample_pair(0, t, 1, 1, 0, K=32)
    assert narrow.scaled == 1 and narrow.sigma != 8**k


def test_scaled_sigma_keeps_path_choice_uniform(orc):
    # Corner to corner of a full 64 x 64 grid every side's middle layers hold
    # up to C(63, 31) ~ 2**59.7 paths, above 2**K (K = 50), so layers are
    # scaled.  Rounding a layer's counts up after a shift of sh bits changes
    # each by a relative 2**(1-K) at most, far below what N samples resolve,
    # so the crossing point of every anti-diagonal must still follow the
    # exact law P[path crosses (r, L - r)] = C(L, r) C(D - L, 63 - r) / C(D, 63).
    k = 64
    g = I.full_grid_graph(k, k)
    ws = orc.Workspace(g)
    assert ws.K == 50
    D = 2 * (k - 1)
    t = k * k - 1
    N = 12000
    layers = (9, 40, 63, 100)
    hits = {L: np.zeros(L + 1, dtype=np.int64) for L in layers}
    scaled = 0
    for i in range(N):
        interior, info = ws.sample_pair(0, t, 77, 1, i)
        scaled += info.scaled
        rows, cols = np.divmod(interior.astype(np.int64), k)
        lv = rows + cols
        for L in layers:
            sel = np.nonzero(lv == L)[0]
            assert sel.size == 1
            hits[L][rows[sel[0]]] += 1
    assert scaled == N
    for L in layers:
        r = np.arange(L + 1)
        p = np.array([math.comb(L, int(x)) * math.comb(D - L, k - 1 - int(x)) if 0 <= k - 1 - x <= D - L else 0
                      for x in r], dtype=float) / math.comb(D, k - 1)
        assert abs(p.sum() - 1) < 1e-12
        exp = N * p
        big = exp >= 5
        obs = np.append(hits[L][big], hits[L][~big].sum())
        ex = np.append(exp[big], exp[~big].sum())
        keep = ex > 0
        chi2 = float((((obs - ex) ** 2)[keep] / ex[keep]).sum())
        dof = int(keep.sum()) - 1
        assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (L, chi2, dof)


def test_grid_sigma_beyond_K_scales_or_flags(orc):
    g = I.full_grid_graph(64, 64)
    ws = orc.Workspace(g)
    # a side's layer 63 holds up to C(63, 31) ~ 2^59.7 paths, above 2^K
    assert math.comb(63, 31) > 2**ws.K
    interior, info = ws.sample_pair(0, 64 * 64 - 1, 1, 1, 0)
    assert info.scaled == 1 and info.overflow == 0 and info.d == 126
    assert len(interior) == 125
    G = to_nx(g)
    check_path(g, 0, 64 * 64 - 1, 126, list(interior), G)
    interior, info = ws.sample_pair(0, 64 * 64 - 1, 1, 1, 0, strict=True)
    assert info.overflow == 1 and len(interior) == 0


def enumerate_paths(G, s, t):
    return [tuple(p[1:-1]) for p in nx.all_shortest_paths(G, s, t)]


@pytest.mark.parametrize("graph,s,t", [
    ("grid3x4", 0, 11),       # 10 shortest paths corner to corner
    ("ladder", 0, 9),
    ("er", None, None),
])
def test_path_distribution_is_uniform(orc, graph, s, t):
    if graph == "grid3x4":
        g = I.full_grid_graph(3, 4)
    elif graph == "ladder":
        pairs = [(i, i + 1) for i in range(4)] + [(5 + i, 6 + i) for i in range(4)]
        pairs += [(i, i + 5) for i in range(5)]
        g = I.csr_from_edges(10, np.array(pairs)[:, 0], np.array(pairs)[:, 1])
    else:
        g = random_small_graph(20, 0.2, 11)
    G = to_nx(g)
    if graph == "er":
        # the pair with the most shortest paths
        s, t = max(((a, b) for a, b in itertools.combinations(range(g.n), 2)
                    if nx.has_path(G, a, b)),
                   key=lambda p: (len(enumerate_paths(G, *p)), -p[0], -p[1]))
    paths = enumerate_paths(G, s, t)
    assert len(paths) >= 3
    ws = orc.Workspace(g)
    N = 60000
    hist = {}
    for i in range(N):
        interior, _ = ws.sample_pair(s, t, 21, 1, i)
        ds = nx.single_source_shortest_path_length(G, s) if i == 0 else ds
        key = tuple(sorted(interior, key=lambda x: ds[x]))
        hist[key] = hist.get(key, 0) + 1
    assert set(hist) <= set(paths)
    exp = N / len(paths)
    chi2 = sum((hist.get(p, 0) - exp) ** 2 / exp for p in paths)
    dof = len(paths) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10


def test_sampler_is_unbiased_for_betweenness(orc):
    # E[c~(x)] / tau = b(x): the counters of many samples approach Brandes
    g = random_small_graph(16, 0.2, 13)
    b = orc.brandes(g)
    N = 400000
    counts, st = orc.run_samples(g, 5, 1, 0, N)
    est = counts / N
    sd = np.sqrt(np.maximum(b * (1 - b), 1e-12) / N)
    assert np.all(np.abs(est - b) <= 6 * sd + 1e-6)


# --------------------------------------------------------------------------
# Diameter phase
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_vertex_diameter(orc, seed):
    g = random_small_graph(40, 0.06, seed)
    G = to_nx(g)
    exact = max(max(nx.single_source_shortest_path_length(G, v).values()) for v in G) + 1
    assert orc.vertex_diameter_exact(g) == exact
    assert orc.vertex_diameter_bound(g) >= exact


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_vertex_diameter_bound_by_components(orc, seed):
    # The bound written out with networkx: every component contributes
    # 2 * ecc(its smallest vertex) + 1, the maximum is taken (1 without edges).
    # Sparse graphs: several components, isolated vertices, and components
    # whose smallest vertex is not an end of their longest path.
    g = random_small_graph(60, 0.03, seed)
    G = to_nx(g)
    want = 1
    comps = list(nx.connected_components(G))
    assert len(comps) > 1
    for comp in comps:
        ecc = max(nx.single_source_shortest_path_length(G, min(comp)).values())
        want = max(want, 2 * ecc + 1)
    assert orc.vertex_diameter_bound(g) == want


def test_vertex_diameter_bound_edgeless_and_midpoint_root(orc):
    assert orc.vertex_diameter_bound(I.csr_from_edges(5, np.array([], dtype=np.int64),
                                                      np.array([], dtype=np.int64))) == 1
    # path 3-1-0-2-4: the component's smallest vertex 0 is its midpoint (ecc 2)
    g = I.csr_from_edges(5, np.array([3, 1, 0, 2]), np.array([1, 0, 2, 4]))
    assert orc.vertex_diameter_bound(g) == 5
    assert orc.vertex_diameter_exact(g) == 5


def test_vertex_diameter_path(orc):
    g = I.path_graph(9)
    assert orc.vertex_diameter_exact(g) == 9
    assert orc.vertex_diameter_bound(g) == 17  # from vertex 0: ecc 8 -> 2*8+1


# --------------------------------------------------------------------------
# omega, calibration, stopping functions: weak pins (formulas not printed)
# --------------------------------------------------------------------------

def test_omega_bounds_table2_sample_counts(orc):
    rows = []
    with open(os.path.join(GOLDEN, "table2_samples.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, diam, samples = line.split()
                rows.append((name, int(diam), int(samples)))
    assert len(rows) == 10
    for name, diam, samples in rows:
        assert samples <= orc.omega(0.001, 0.1, diam + 1), name


def test_uniform_rule_closed_form(orc):
    cal = np.array([0, 3, 10, 0, 1], dtype=np.uint32)
    LL, LU, _ = orc.calibrate_L(cal, 20, 0.05, 0.1, rule=0)
    np.testing.assert_allclose(LL, math.log(4 * 5 / 0.1), rtol=1e-15)
    np.testing.assert_allclose(LU, LL, rtol=0)


def test_balanced_rule_respects_budget(orc):
    rng = np.random.default_rng(0)
    n = 5000
    cal = rng.poisson(0.3, n).astype(np.uint32)
    cal[:5] = [400, 200, 90, 50, 20]
    for eps in (0.05, 0.01):
        LL, LU, C = orc.calibrate_L(cal, 1000, eps, 0.1, rule=1, beta=1e-3)
        total = np.exp(-LL).sum() + np.exp(-LU).sum()
        assert total <= 0.1 / 2 * (1 + 1e-9)
        # the floor gives every vertex at least beta*delta/(4n)
        assert np.all(np.exp(-LL) >= 1e-3 * 0.1 / (4 * n) * (1 - 1e-12))
        # more central (by calibration) -> larger failure budget
        order = np.argsort(cal, kind="stable")
        assert np.all(np.diff(LL[order]) <= 1e-12)


def test_stop_functions_limits(orc):
    # b~ = 0 and tau <= 3 omega: the lower deviation f vanishes
    f, g = orc.stop_functions(0, 100, 1000.0, 5.0, 5.0)
    assert f == 0.0 and g > 0
    # both bounds shrink as tau grows at fixed b~, and g >= f
    prev = None
    for tau in (10**3, 10**4, 10**5, 10**6):
        f, g = orc.stop_functions(tau // 10, tau, 5000.0, 4.0, 4.0)
        assert 0 <= f <= g
        if prev:
            assert g < prev[1] and f <= prev[0]
        prev = (f, g)


def _largest_root(h, lo, hi, iters=400):
    """Bisection for the largest root of h on [lo, hi] (h(lo) <= 0 < h(hi))."""
    for _ in range(iters):
        mid = (lo + hi) / 2
        if h(mid) <= 0:
            lo = mid
        else:
            hi = mid
    return lo


def test_stop_functions_solve_the_deviation_bound(orc):
    # f and g are the deviations at which the one-sided tail bound of the
    # adaptive martingale argument, exp(-lam^2 / (2 (omega b + lam / 3))) with
    # lam = tau * deviation, equals delta_L resp. delta_U = exp(-L), taking the
    # unknown b at the far end of the interval: b = b~ - f for the lower
    # deviation, b = b~ + g for the upper one.  So tau f is the largest root
    # of lam^2 = 2 L (omega (b~ - lam / tau) + lam / 3), and tau g that of
    # lam^2 = 2 L (omega (b~ + lam / tau) + lam / 3).  Solved here by 50-digit
    # bisection on that equation, not by the closed form.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(5)
    for _ in range(300):
        tau = int(rng.integers(10, 10**7))
        omega = float(tau * rng.uniform(0.2, 20.0))
        c = int(rng.integers(0, tau + 1)) if rng.random() < 0.8 else int(rng.integers(0, 4))
        LL = float(rng.uniform(2.0, 40.0))
        LU = float(rng.uniform(2.0, 40.0))
        f, g = orc.stop_functions(c, tau, omega, LL, LU)
        T, W, bt = mp.mpf(tau), mp.mpf(omega), mp.mpf(c) / mp.mpf(tau)
        for val, L, sign in ((f, mp.mpf(LL), -1), (g, mp.mpf(LU), +1)):
            h = lambda lam, L=L, sign=sign: lam**2 - 2 * L * (W * (bt + sign * lam / T) + lam / 3)
            hi = mp.mpf(1)
            while h(hi) <= 0:
                hi *= 2
            lam = _largest_root(h, mp.mpf(0), hi)
            exact = lam / T
            # the closed form's evaluation order loses digits to cancellation
            # only relative to the size of its terms
            scale = (L / T) * (abs(mp.mpf(1) / 3 + sign * W / T) + mp.sqrt((mp.mpf(1) / 3 + sign * W / T) ** 2
                                                                             + 2 * bt * W / L))
            assert abs(mp.mpf(val) - exact) <= 1e-14 * scale + mp.mpf(10) ** -300, (c, tau, omega, L, sign)
            # the bound itself: at the computed deviation the tail equals exp(-L)
            if exact > 0:
                tail = lam**2 / (2 * (W * (bt + sign * lam / T) + lam / 3))
                assert abs(tail - L) <= mp.mpf(10) ** -30 * L


@pytest.mark.parametrize("eps,delta,vd,hand", [
    # (0.5 / eps^2) * (floor(log2(VD - 2)) + 1 + ln(2 / delta)), terms by hand:
    # VD - 2 = 8: floor(log2 8) = 3; ln 20 = 2.995732273553991; 50 * 6.995732273553991
    (0.1, 0.1, 10, 349.78661367769955),
    # VD - 2 = 10: floor(log2 10) = 3; 5000 * 6.995732273553991
    (0.01, 0.1, 12, 34978.66136776995),
    # VD - 2 = 1: floor(log2 1) = 0; 200 * 3.995732273553991
    (0.05, 0.1, 3, 799.1464547107982),
    # VD - 2 = 0 is clamped to 1 (a graph with one edge)
    (0.05, 0.1, 2, 799.1464547107982),
    # VD - 2 = 793 (roadNet-PA, D = 794): floor(log2 793) = 9; 500000 * 12.995732273553991
    (0.001, 0.1, 795, 6497866.136776996),
    # VD - 2 = 128: floor(log2 128) = 7; ln 200 = 5.298317366548036; 1250 * 13.298317366548036
    (0.02, 0.01, 130, 16622.896708185045),
])
def test_omega_hand_values(orc, eps, delta, vd, hand):
    # omega with the constant c = 1 instead of 1/2, or ln(1/delta) instead of
    # ln(2/delta), or log2 without the floor, misses these by far more than
    # rounding
    assert orc.omega(eps, delta, vd) == pytest.approx(hand, rel=1e-14)


def test_balanced_rule_single_class_closed_form(orc):
    # one vertex with calibration count 4 of n_cal = 100, nine with none:
    # the budget (1 - beta) delta / 4 is spent on that vertex alone, so the
    # constant solves exp(-C eps^2 n_cal / 4) = (1 - beta) delta / 4, i.e.
    # C* = 4 / (eps^2 n_cal) * ln(4 / ((1 - beta) delta)); bisection returns
    # the upper end of an interval shorter than eps / 10 that holds C*.
    eps, delta, beta, ncal = 0.05, 0.1, 1e-3, 100
    cal = np.zeros(10, dtype=np.uint32)
    cal[0] = 4
    LL, LU, C = orc.calibrate_L(cal, ncal, eps, delta, rule=1, beta=beta)
    Cstar = 4 / (eps**2 * ncal) * math.log(4 / ((1 - beta) * delta))
    assert Cstar <= C <= Cstar + eps / 10
    floor = beta * delta / (4 * 10)
    np.testing.assert_allclose(LL[1:], -math.log(floor), rtol=1e-15)
    assert LL[0] == pytest.approx(-math.log(math.exp(-C * eps**2 / 0.04) + floor), rel=1e-15)
    np.testing.assert_array_equal(LU, LL)


def test_balanced_rule_two_classes_root(orc):
    # two classes: h1 vertices with count c1 and h2 with count c2 of n_cal;
    # C* is the root of h1 exp(-C eps^2 n_cal / c1) + h2 exp(-C eps^2 n_cal / c2)
    # = (1 - beta) delta / 4, found here by 50-digit bisection
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    eps, delta, beta, ncal = 0.02, 0.1, 1e-3, 2000
    cal = np.zeros(5000, dtype=np.uint32)
    cal[:3] = 150
    cal[3:40] = 7
    LL, LU, C = orc.calibrate_L(cal, ncal, eps, delta, rule=1, beta=beta)
    B = (1 - mp.mpf(beta)) * mp.mpf(delta) / 4
    e2n = mp.mpf(eps) ** 2 * ncal
    h = lambda x: B - (3 * mp.exp(-x * e2n / 150) + 37 * mp.exp(-x * e2n / 7))
    Cstar = _largest_root(h, mp.mpf(0), mp.mpf(10) ** 6)
    assert Cstar <= C <= Cstar + eps / 10
    total = float(np.exp(-LL).sum() + np.exp(-LU).sum())
    assert total <= delta / 2


def test_check_stop_at_omega(orc):
    counts = np.zeros(4, dtype=np.uint32)
    L = np.full(4, 50.0)
    stop, mf, mg = orc.check_stop(counts, 1000, 999.5, 1e-9, L, L)
    assert stop
    stop, mf, mg = orc.check_stop(counts, 0, 10.0, 0.5, L, L)
    assert not stop and mf == math.inf


# --------------------------------------------------------------------------
# End to end: the (epsilon, delta) guarantee against exact betweenness
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,eps", [
    ("er2000", 0.05), ("grid64", 0.05), ("star", 0.05), ("path", 0.05), ("rgg5k", 0.05),
])
@pytest.mark.parametrize("rule", [0, 1])
def test_kadabra_within_eps_of_brandes(orc, name, eps, rule):
    if name == "star":
        g = I.star_graph(300)
    elif name == "path":
        g = I.path_graph(300)
    else:
        g = I.config_graph(name)
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=1, epoch_len=200, delta_rule=rule)
    assert R.stopped == 1 and R.tau <= math.ceil(R.omega)
    b = orc.brandes(g)
    err = np.abs(counts / R.tau - b).max()
    assert err <= eps, (name, err)


def test_stop_functions_are_monotone_in_the_counter(orc):
    """f and g, as computed in IEEE double (each step a correctly rounded
    monotone operation), never decrease when the counter grows with the
    budgets fixed.  The pipelined check evaluates one vertex per budget class
    (the class's largest counter) on the strength of this property."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        omega = float(rng.uniform(1e3, 1e6))
        tau = int(rng.integers(1, int(omega)))
        LL = float(rng.uniform(0.5, 60.0))
        LU = float(rng.uniform(0.5, 60.0))
        cs = np.unique(np.concatenate([rng.integers(0, tau + 1, 64), [0, 1, tau]]))
        prev_f = prev_g = -np.inf
        for c in cs:
            f, g = orc.stop_functions(int(c), tau, omega, LL, LU)
            assert f >= prev_f and g >= prev_g, (c, tau, omega, LL, LU)
            prev_f, prev_g = f, g


def test_class_maxima_equal_vertex_maxima(orc):
    """The maxima of f and g over vertices equal the maxima over budget
    classes (vertices with equal (L_L, L_U)) evaluated at each class's largest
    counter: the reduction the pipelined check is built on."""
    rng = np.random.default_rng(5)
    n = 5000
    classes = rng.uniform(1.0, 40.0, size=(12, 2))
    cls = rng.integers(0, len(classes), n)
    LL = classes[cls, 0].copy()
    LU = classes[cls, 1].copy()
    omega, eps = 20000.0, 0.05
    for tau in (50, 700, 9000):
        counts = rng.integers(0, tau + 1, n).astype(np.uint32)
        _, mf, mg = orc.check_stop(counts, tau, omega, eps, LL, LU)
        bf = bg = -np.inf
        for k in range(len(classes)):
            members = cls == k
            if not members.any():
                continue
            f, g = orc.stop_functions(int(counts[members].max()), tau, omega, classes[k, 0], classes[k, 1])
            bf, bg = max(bf, f), max(bg, g)
        assert mf == bf and mg == bg


@pytest.mark.parametrize("name,eps,E,rule", [("er2000", 0.05, 100, 1), ("grid64", 0.05, 64, 0),
                                             ("rmat12", 0.03, 256, 1)])
def test_threaded_driver_equals_the_serial_method(orc, name, eps, E, rule):
    # kadabra_threads splits each phase's sample indices over host threads;
    # the counters are integer sums, so every output equals kadabra()'s
    g = I.config_graph(name)
    counts, cal, LL, LU, R = orc.kadabra(g, eps, 0.1, seed=3, epoch_len=E, delta_rule=rule)
    c2, cal2, LL2, LU2, info = orc.kadabra_threads(g, eps, 0.1, seed=3, epoch_len=E, delta_rule=rule, threads=5)
    assert np.array_equal(counts, c2) and np.array_equal(cal, cal2)
    assert np.array_equal(LL, LL2) and np.array_equal(LU, LU2)
    assert (info["tau"], info["stop_epoch"], info["vd"], info["K"]) == (R.tau, R.stop_epoch, R.vd, R.K)
    assert (info["max_f"], info["max_g"], info["C"]) == (R.max_f, R.max_g, R.C)
