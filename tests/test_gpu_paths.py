"""GED matrices (fastged_cross) and edit paths of the K-Best maps on the GPU (Sec. 6: the
nearest-neighbour classification over all test-to-training distances, and the crossover
that applies half of an edit path)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W

from parity_util import gpu_run

pytestmark = pytest.mark.gpu


def _graph_set():
    w = W.config1(8)
    return w.graphs, w.cost, w.K


def test_cross_matrix_equals_oracle():
    graphs, cost, K = _graph_set()
    n = len(graphs)
    rows, cols = np.arange(n), np.arange(n)
    with F.FastGED(cost) as g:
        d = F.fastged_cross(g.h, graphs, rows, cols, K)
        # a rectangular block with repeated and permuted indices
        r2, c2 = np.array([3, 0, 3, 7]), np.array([5, 1])
        d2 = F.fastged_cross(g.h, graphs, r2, c2, K)
    for r in range(n):
        for c in range(n):
            assert d[r, c] == O.kbest(graphs[r], graphs[c], cost, K)[0], (r, c)
    assert np.array_equal(d2, d[np.ix_(r2, c2)])


def test_cross_rejects_bad_indices_and_per_pair_k():
    graphs, cost, K = _graph_set()
    with F.FastGED(cost) as g:
        with pytest.raises(F.FastGEDError):
            F.fastged_cross(g.h, graphs, [0, 99], [1], K)
        with pytest.raises(F.FastGEDError):
            F.fastged_cross(g.h, graphs, [0], [1], K, F.make_options(k_per_pair=[3]))
        assert F.fastged_cross(g.h, graphs, [], [1, 2], K).shape == (0, 2)


def _families(n_each, seed):
    """Two structural families of the same size: molecule-like trees with few rings, and
    dense random graphs."""
    graphs, labels = [], []
    for k in range(n_each):
        st = W.Stream(seed, k)
        graphs.append(W.molecule_like(st, 14))
        labels.append(0)
        graphs.append(W.erdos_renyi(st, 14, 0.5, 10))
        labels.append(1)
    return graphs, np.array(labels)


def test_knn_classification_matches_oracle_distances():
    train, ytr = _families(10, 5)
    test, yte = _families(6, 6)
    K = 32
    pred = F.knn_classify(W.UNIT_COSTS, train, ytr, test, K, k=1)
    # the same 1-NN rule on oracle distances
    ref = []
    for t in test:
        d = [O.kbest(t, g, W.UNIT_COSTS, K)[0] for g in train]
        ref.append(ytr[int(np.argmin(d))])
    assert np.array_equal(pred, np.array(ref))
    assert (pred == yte).mean() >= 0.9


def test_edit_paths_of_gpu_maps_cost_what_the_gpu_reports():
    w = W.config2(120)
    cost, maps, _ = gpu_run(w)
    mm = F.marshal(w)
    for p in range(w.n_pairs):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        mp = maps[mm.map_off[p]:mm.map_off[p + 1]]
        ops, tot = F.fastged_edit_path(w.cost, g1, g2, mp)
        assert tot == int(cost[p])
        assert [tuple(int(x) for x in o) for o in ops] == O.edit_path(g1, g2, w.cost, mp)
        # crossover: half of the path applied to g1 is a valid graph between the two
        half = F.fastged_apply_edit_ops(g1, g2, mp, ops, len(ops) // 2)
        assert half.n <= g1.n + g2.n and (half.edges.size == 0 or half.edges.max() < half.n)
