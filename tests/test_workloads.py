"""The seeded input generators follow the stated recipes (sizes, label ranges, densities,
structure, costs and K of every workload) and give the same graphs for the same seed."""
import numpy as np

from paper_2605_00830_gb300 import workloads as W


def _check_graph(g, n_lo, n_hi, n_vlab):
    assert n_lo <= g.n <= n_hi
    assert g.vlabel.shape == (g.n,) and (0 <= g.vlabel).all() and (g.vlabel < n_vlab).all()
    e = np.asarray(g.edges).reshape(-1, 2)
    assert (e[:, 0] < e[:, 1]).all() and (e[:, 1] < g.n).all()          # u < v, in range
    assert len({(int(u), int(v)) for u, v in e}) == len(e)               # no multi-edges


def test_config1_tiny_er():
    w = W.config1()
    assert w.n_pairs == 200 and w.K == 16 and tuple(w.cost) == W.UNIT_COSTS
    for g in w.graphs:
        _check_graph(g, 5, 8, 4)
        assert g.elabel is None


def test_config2_molecule_like():
    w = W.config2(300)
    assert w.K == 100 and tuple(w.cost) == W.SETTING1_COSTS == (2, 4, 4, 1, 2, 2)
    degs = []
    for g in w.graphs:
        _check_graph(g, 10, 40, 10)
        # a spanning tree plus 0-3 extra edges: connected, n - 1 <= m <= n + 2
        assert g.n - 1 <= g.m <= g.n + 2
        adj = {v: set() for v in range(g.n)}
        for u, v in g.edges:
            adj[int(u)].add(int(v))
            adj[int(v)].add(int(u))
        seen, stack = {0}, [0]
        while stack:
            for x in adj[stack.pop()]:
                if x not in seen:
                    seen.add(x)
                    stack.append(x)
        assert len(seen) == g.n
        assert set(np.unique(g.elabel)) <= {0, 1, 2}
        degs.append(2 * g.m / g.n)
    assert 1.9 < np.mean(degs) < 2.2
    # Zipf(1.2) vertex labels: label 0 the most frequent
    lab = np.concatenate([g.vlabel for g in w.graphs])
    assert np.argmax(np.bincount(lab, minlength=10)) == 0


def test_config3_dense_er():
    w = W.config3(40)
    assert w.K == 256 and tuple(w.cost) == W.UNIT_COSTS
    dens = []
    for g in w.graphs:
        _check_graph(g, 50, 200, 8)
        dens.append(2 * g.m / (g.n * (g.n - 1)))
    assert 0.04 < min(dens) and max(dens) < 0.53


def test_config4_perturbed_ba():
    w = W.config4(3, n_range=(500, 560))
    assert w.K == 1024 and tuple(w.cost) == W.UNIT_COSTS
    for p in range(w.n_pairs):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        _check_graph(g1, 500, 560, 16)
        _check_graph(g2, 400, 700, 16)
        assert abs(g1.m - 3 * g1.n) < 20                                 # BA, m = 3
        assert abs(g2.n - g1.n) <= 0.1 * (g1.n + g1.m)                   # 2-10 % of n + m edits


def test_config5_serving_mix():
    w = W.config5(duration_s=0.4, rate=5000.0)
    shape = w.meta["shape"]
    assert len(shape) == w.n_pairs and 1500 < w.n_pairs < 2500            # Poisson, 5,000/s
    assert np.all(np.diff(w.arrival) >= 0) and w.arrival[-1] < 0.4
    frac = np.bincount(shape, minlength=3) / len(shape)
    assert abs(frac[0] - 0.70) < 0.05 and abs(frac[1] - 0.25) < 0.05 and frac[2] < 0.09
    assert set(np.unique(w.k_per_pair)) <= {32, 128, 512}


def test_wide_beam_and_size_sweep():
    w = W.config_wide_beam()
    assert w.n_pairs == 16 and w.K == 100000
    for g in w.graphs:
        _check_graph(g, 18, 22, 10)
    s = W.config_size_sweep(n=300)
    assert s.K == 5000 and tuple(s.cost) == W.SETTING1_COSTS
    for g in s.graphs:
        _check_graph(g, 300, 300, 4)
        assert abs(2 * g.m / (g.n * (g.n - 1)) - 0.4) < 0.02


def test_same_seed_same_graphs():
    for make in (lambda: W.config2(20), lambda: W.config3(3), lambda: W.config5(0.05),
                 lambda: W.config_size_sweep(n=60)):
        a, b = make(), make()
        assert len(a.graphs) == len(b.graphs)
        for x, y in zip(a.graphs, b.graphs):
            assert x.n == y.n and np.array_equal(x.vlabel, y.vlabel)
            assert np.array_equal(x.edges, y.edges)
    assert not np.array_equal(W.config2(5, seed=2).graphs[0].edges,
                              W.config2(5, seed=3).graphs[0].edges)
