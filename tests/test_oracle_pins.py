"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: the exact GED is computed by two unrelated
enumerations, the search is checked against hand traces, closed forms and the exhaustive
limit (K >= level width makes Algorithm 1 exhaustive, so it must reach the exact GED;
Sec. 4.5), and the leaf cost is checked against the independent full-path evaluator.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_00830_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_traces.json")


def _graph(d):
    e = np.array(d["edges"], dtype=np.int32).reshape(-1, 2)
    el = None if d.get("elabel") is None else np.array(d["elabel"], dtype=np.int32)
    return W.Graph(n=d["n"], vlabel=np.array(d["vlabel"], dtype=np.int32), edges=e, elabel=el)


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


def _level_width(i, n2):
    """Number of injective partial maps of i g1 vertices into n2 g2 vertices."""
    return sum(math.comb(i, j) * math.perm(n2, j) for j in range(min(i, n2) + 1))


def _exhaustive_evals(n1, n2):
    """n_evals of an exhaustive search: every partial map at level i with j substitutions
    has (n2 - j) + 1 successors, plus one completion per leaf."""
    tot = 0
    for i in range(n1):
        for j in range(min(i, n2) + 1):
            tot += math.comb(i, j) * math.perm(n2, j) * (n2 - j + 1)
    return tot + _level_width(n1, n2)


def _rand_pair(seed, n_lo=0, n_hi=5, p=0.45, nv=3, ne=0):
    st = W.Stream(seed, 99)
    return (W.random_small(st, n_lo, n_hi, p, nv, ne), W.random_small(st, n_lo, n_hi, p, nv, ne))


def _rand_cost(seed):
    st = W.Stream(seed, 98)
    return tuple(int(x) for x in st.randint(1, 6, 6))


# --------------------------------------------------------------------------------------
# golden hand traces and hand-derived exact values
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_golden_exact(case):
    g1, g2 = _graph(case["g1"]), _graph(case["g2"])
    ged, mp, _ = O.brute_ged(g1, g2, case["cost"])
    assert ged == case["exact"]
    assert O.full_cost(g1, g2, case["cost"], mp) == ged
    if g1.n + g2.n <= 10:
        assert O.brute_square(g1, g2, case["cost"]) == case["exact"]


@pytest.mark.parametrize("case", [c for c in _cases() if "kbest" in c], ids=lambda c: c["name"])
def test_golden_kbest_trace(case):
    g1, g2 = _graph(case["g1"]), _graph(case["g2"])
    for exp in case["kbest"]:
        cost, mp, nev = O.kbest(g1, g2, case["cost"], exp["K"])
        assert cost == exp["cost"], exp
        assert list(mp) == exp["map"], exp
        assert nev == exp["n_evals"], exp
        if "leaf_ped" in exp:
            ped, lm = O.kbest_leaves(g1, g2, case["cost"], exp["K"])
            assert list(ped) == exp["leaf_ped"]
            assert lm.tolist() == exp["leaf_map"]
    for exp in case.get("kbest_variant1", []):
        cost, mp, nev = O.kbest(g1, g2, case["cost"], exp["K"], variant=1)
        assert (cost, list(mp), nev) == (exp["cost"], exp["map"], exp["n_evals"])


# --------------------------------------------------------------------------------------
# exact GED: two independent enumerations agree, and closed forms
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(60))
def test_brute_enumerations_agree(seed):
    g1, g2 = _rand_pair(seed, 0, 5, 0.5, 3, ne=2 if seed % 2 else 0)
    while g1.n + g2.n > 9:
        g2 = W.random_small(W.Stream(seed, 97, g2.n), 0, 4, 0.5, 3, 2 if seed % 2 else 0)
    cost = _rand_cost(seed) if seed % 3 else W.UNIT_COSTS
    ged, mp, cnt = O.brute_ged(g1, g2, cost)
    assert ged == O.brute_square(g1, g2, cost)
    assert cnt == _level_width(g1.n, g2.n)


@pytest.mark.parametrize("seed", range(20))
def test_closed_form_empty(seed):
    st = W.Stream(seed, 96)
    g = W.random_small(st, 1, 8, 0.4, 4, 3)
    e = W.empty_graph()
    c = _rand_cost(seed)
    # GED(empty, G) = n*c_vins + m*c_eins ; GED(G, empty) = n*c_vdel + m*c_edel
    for K in (1, 7):
        assert O.kbest(e, g, c, K)[0] == g.n * c[2] + g.m * c[5]
        assert O.kbest(g, e, c, K)[0] == g.n * c[1] + g.m * c[4]
    if g.n <= 8:
        assert O.brute_ged(e, g, W.UNIT_COSTS)[0] == g.n + g.m
        assert O.brute_ged(g, e, W.UNIT_COSTS)[0] == g.n + g.m


@pytest.mark.parametrize("seed", range(20))
def test_closed_form_edgeless(seed):
    """Edgeless graphs with n1 = n2 and 2*c_vsub <= c_vdel + c_vins: the best path
    substitutes everything, paying c_vsub for every vertex outside the label overlap."""
    st = W.Stream(seed, 95)
    n = int(st.randint(1, 6, 1)[0])
    g1 = W.Graph(n, st.randint(0, 3, n).astype(np.int32), np.zeros((0, 2), np.int32))
    g2 = W.Graph(n, st.randint(0, 3, n).astype(np.int32), np.zeros((0, 2), np.int32))
    c = (2, 3, 1, 1, 1, 1) if seed % 2 else (1, 1, 1, 1, 1, 1)
    overlap = sum(min(int(np.sum(g1.vlabel == l)), int(np.sum(g2.vlabel == l))) for l in range(4))
    want = c[0] * (n - overlap)
    assert O.brute_ged(g1, g2, c)[0] == want
    assert O.kbest(g1, g2, c, _level_width(n, n))[0] == want


@pytest.mark.parametrize("seed", range(20))
def test_identity_and_symmetry_exact(seed):
    g1, g2 = _rand_pair(seed, 1, 6, 0.5, 3, ne=2)
    c = _rand_cost(seed)
    sym = (c[0], c[1], c[1], c[3], c[4], c[4])  # c_vdel = c_vins, c_edel = c_eins
    assert O.brute_ged(g1, g1, c)[0] == 0
    assert O.brute_ged(g1, g2, sym)[0] == O.brute_ged(g2, g1, sym)[0]
    # Algorithm 1 with K at least the widest level is exhaustive (Sec. 4.5)
    Kx = max(_level_width(i, g1.n) for i in range(g1.n + 1))
    assert O.kbest(g1, g1, c, Kx)[0] == 0


# --------------------------------------------------------------------------------------
# the K-Best search against the exact GED and the independent evaluator
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(40))
def test_kbest_exhaustive_is_exact(seed):
    g1, g2 = _rand_pair(seed, 0, 6, 0.45, 3, ne=3 if seed % 2 else 0)
    c = _rand_cost(seed) if seed % 3 else W.SETTING1_COSTS
    ged = O.brute_ged(g1, g2, c)[0]
    Kx = max(_level_width(i, g2.n) for i in range(g1.n + 1))
    cost, mp, nev = O.kbest(g1, g2, c, Kx)
    assert cost == ged
    assert O.full_cost(g1, g2, c, mp) == cost
    assert nev == _exhaustive_evals(g1.n, g2.n)
    # variant 1 never does worse than variant 0 (it completes a superset of leaves)
    assert O.kbest(g1, g2, c, max(1, Kx // 7), variant=1)[0] <= O.kbest(g1, g2, c, max(1, Kx // 7))[0]


def test_kbest_exhaustive_n7():
    st = W.Stream(7, 94)
    g1 = W.erdos_renyi(st, 7, 0.4, 3)
    g2 = W.erdos_renyi(st, 7, 0.4, 3)
    Kx = _level_width(7, 7)
    assert Kx == 130922
    cost, mp, nev = O.kbest(g1, g2, W.UNIT_COSTS, Kx)
    assert cost == O.brute_ged(g1, g2, W.UNIT_COSTS)[0]
    assert nev == _exhaustive_evals(7, 7)


def test_kbest_on_config1_is_upper_bound():
    """Every K-Best result is the cost of a complete edit path, hence >= the exact GED
    (Sec. 2.2); the leaf cost equals the independent evaluation of its map."""
    w = W.config1()
    n_opt = 0
    for p in range(0, w.n_pairs, 4):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        ged = O.brute_ged(g1, g2, w.cost)[0]
        cost, mp, nev = O.kbest(g1, g2, w.cost, w.K)
        assert cost >= ged
        assert O.full_cost(g1, g2, w.cost, mp) == cost
        n_opt += cost == ged
    assert n_opt > 0


def test_kbest_result_is_the_best_completed_leaf():
    """The result is the cheapest completion of the final kept list (Algorithm 1, insertions
    at the leaf): min over the leaves of the independent full-path cost. Hence it equals the
    exact GED whenever some leaf's map is optimal (config 1, K = 16)."""
    w = W.config1()
    n_opt = 0
    for p in range(0, w.n_pairs, 2):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        cost, _, _ = O.kbest(g1, g2, w.cost, w.K)
        _, maps = O.kbest_leaves(g1, g2, w.cost, w.K)
        best_leaf = min(O.full_cost(g1, g2, w.cost, m) for m in maps)
        assert cost == best_leaf
        ged = O.brute_ged(g1, g2, w.cost)[0]
        if best_leaf == ged:
            assert cost == ged
            n_opt += 1
    assert n_opt > 0


def prefix_graph(g, k):
    """g restricted to its first k vertices (the edges among them, with their labels)."""
    e = np.asarray(g.edges, dtype=np.int32).reshape(-1, 2)
    keep = (e[:, 0] < k) & (e[:, 1] < k)
    el = None if g.elabel is None else np.asarray(g.elabel, dtype=np.int32)[keep]
    return W.Graph(n=k, vlabel=np.asarray(g.vlabel, dtype=np.int32)[:k], edges=e[keep],
                   elabel=el)


def variant_b_by_definition(g1, g2, cost, K):
    """Variant B completes every successor of the last level: every child (each free g2
    vertex, or the deletion) of the beam kept after the first n1 - 1 levels. That beam is the
    final kept list of the search on g1's first n1 - 1 vertices, which no later vertex of g1
    influences, so it comes from a variant-A run on that prefix; each child is a complete map,
    scored by the independent full-path cost."""
    _, maps = O.kbest_leaves(prefix_graph(g1, g1.n - 1), g2, cost, K)
    best = None
    for m in maps:
        used = set(int(x) for x in m if x >= 0)
        for j in [u for u in range(g2.n) if u not in used] + [-1]:
            c = O.full_cost(g1, g2, cost, list(m) + [j])
            best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("seed", range(40))
def test_variant_b_is_the_best_child_of_the_penultimate_beam(seed):
    g1, g2 = _rand_pair(seed, 1, 6, ne=2 if seed % 2 else 0)
    cost = _rand_cost(seed)
    for K in (1, 2, 3, 5):
        got, mp, _ = O.kbest(g1, g2, cost, K, variant=1)
        assert got == variant_b_by_definition(g1, g2, cost, K)
        assert O.full_cost(g1, g2, cost, mp) == got


def ped_by_definition(g1k, g2, cost, m):
    """Partial edit distance of a map of g1's first k vertices: the full-path cost of the
    prefix map less what the leaf completion adds (every unused g2 vertex and every g2 edge
    with an unused end are insertions)."""
    used = set(int(x) for x in m if x >= 0)
    e2 = np.asarray(g2.edges).reshape(-1, 2)
    pending = cost[2] * (g2.n - len(used)) + cost[5] * sum(
        1 for a, b in e2 if int(a) not in used or int(b) not in used)
    return O.full_cost(g1k, g2, cost, list(m)) - pending


@pytest.mark.parametrize("seed", range(30))
def test_each_level_keeps_the_k_best_children(seed):
    """Algorithm 1 level by level: the list kept after level k is the K smallest children of
    the list kept after level k - 1 (every free target vertex in increasing order, then the
    deletion), ordered by (PED, parent slot, child), each PED recomputed from the definition.
    The kept lists come from runs on g1's first k vertices, which later vertices do not
    influence. The evaluation count is every child scored plus every final leaf completed."""
    g1, g2 = _rand_pair(seed, 1, 6, ne=2 if seed % 3 == 0 else 0)
    cost = _rand_cost(seed)
    for K in (1, 2, 3, 7):
        prev_ped, prev_maps = O.kbest_leaves(prefix_graph(g1, 0), g2, cost, K)
        scored = 0
        for k in range(1, g1.n + 1):
            g1k = prefix_graph(g1, k)
            children = []
            for slot, m in enumerate(prev_maps):
                used = set(int(x) for x in m if x >= 0)
                for j in [u for u in range(g2.n) if u not in used] + [-1]:
                    child = list(m) + [j]
                    key_j = j if j >= 0 else g2.n
                    children.append((ped_by_definition(g1k, g2, cost, child), slot, key_j, child))
            scored += len(children)
            children.sort(key=lambda t: t[:3])
            kept = children[:K]
            ped, maps = O.kbest_leaves(g1k, g2, cost, K)
            assert list(ped) == [c[0] for c in kept]
            assert maps.tolist() == [c[3] for c in kept]
            prev_ped, prev_maps = ped, maps
        # n_evals: every child scored at every level, plus every final leaf completed
        assert O.kbest(g1, g2, cost, K)[2] == scored + len(prev_maps)


def test_kbest_k1_evals_closed_form():
    """With K = 1 the search follows one path: level i scores (n2 - #substitutions so far)
    + 1 successors, and one leaf is completed."""
    w = W.config2(20)
    for p in range(w.n_pairs):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        cost, mp, nev = O.kbest(g1, g2, w.cost, 1)
        subs = 0
        want = 0
        for i in range(g1.n):
            want += g2.n - subs + 1
            subs += int(mp[i] >= 0)
        assert nev == want + 1
        assert O.full_cost(g1, g2, w.cost, mp) == cost


@pytest.mark.parametrize("cfg", ["config2", "config3"])
def test_kbest_leaf_cost_matches_full_cost(cfg):
    w = getattr(W, cfg)(3)
    for p in range(w.n_pairs):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        cost, mp, nev = O.kbest(g1, g2, w.cost, 8)
        assert O.full_cost(g1, g2, w.cost, mp) == cost


def test_kbest_leaves_sorted_and_distinct():
    """The kept list is in key order (non-decreasing PED) and holds distinct partial maps."""
    w = W.config1(30)
    for p in range(w.n_pairs):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        ped, mp = O.kbest_leaves(g1, g2, w.cost, 16)
        assert np.all(np.diff(ped) >= 0)
        assert len({tuple(r) for r in mp.tolist()}) == len(mp)
        for s in range(len(ped)):
            # PED of a leaf = full cost of its map minus the leaf insertions
            ins = [u for u in range(g2.n) if u not in set(mp[s].tolist())]
            e_ins = sum(1 for a, b in g2.edges if a in ins or b in ins)
            assert O.full_cost(g1, g2, w.cost, mp[s]) == ped[s] + len(ins) * w.cost[2] + e_ins * w.cost[5]


# --------------------------------------------------------------------------------------
# optional branching order of the source vertices (descending degree; an extension)
# --------------------------------------------------------------------------------------

def test_degree_order_of_a_known_graph():
    # path 0-1-2 plus a star around 3: degrees 1, 2, 1, 3, 1, 1, 1
    g = W.Graph(7, np.arange(7, dtype=np.int32),
                np.array([[0, 1], [1, 2], [3, 4], [3, 5], [3, 6]], dtype=np.int32))
    assert O.degree_order(g) == [3, 1, 0, 2, 4, 5, 6]
    r = O.relabel(g, O.degree_order(g))
    assert list(r.vlabel) == [3, 1, 0, 2, 4, 5, 6]
    assert sorted(map(tuple, np.sort(r.edges, axis=1).tolist())) == [(0, 4), (0, 5), (0, 6), (1, 2), (1, 3)]


@pytest.mark.parametrize("seed", range(16))
def test_degree_ordered_kbest_exhaustive_is_exact(seed):
    """In the exhaustive limit the branching order cannot matter: the ordered search reaches
    the exact GED, its map (in the original ids) costs exactly what it reports, and the
    number of evaluations is the exhaustive count."""
    g1, g2 = _rand_pair(seed + 100, 0, 6, 0.5, 3, ne=3 if seed % 2 else 0)
    c = _rand_cost(seed) if seed % 3 else W.SETTING2_COSTS
    Kx = max(_level_width(i, g2.n) for i in range(g1.n + 1))
    cost, mp, nev = O.kbest(g1, g2, c, Kx, order=1)
    assert cost == O.brute_ged(g1, g2, c)[0]
    assert O.full_cost(g1, g2, c, mp) == cost
    assert nev == _exhaustive_evals(g1.n, g2.n)


def test_degree_order_equals_index_order_when_already_sorted():
    # a star centred at 0 followed by a path: index order is already descending degree
    g1 = W.Graph(6, np.array([1, 2, 1, 0, 2, 1], dtype=np.int32),
                 np.array([[0, 1], [0, 2], [0, 3], [0, 4], [4, 5]], dtype=np.int32))
    assert O.degree_order(g1) == [0, 4, 1, 2, 3, 5]
    g1 = O.relabel(g1, O.degree_order(g1))
    assert O.degree_order(g1) == list(range(6))
    g2 = W.erdos_renyi(W.Stream(5, 5), 7, 0.4, 3)
    for K in (1, 3, 10):
        a = O.kbest(g1, g2, W.SETTING1_COSTS, K, order=0)
        b = O.kbest(g1, g2, W.SETTING1_COSTS, K, order=1)
        assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1])


def test_degree_ordered_kbest_on_config1_is_a_valid_path():
    w = W.config1(40)
    for p in range(w.n_pairs):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        cost, mp, _ = O.kbest(g1, g2, w.cost, w.K, order=1)
        img = mp[mp >= 0]
        assert len(np.unique(img)) == len(img) and np.all(mp < g2.n)
        assert O.full_cost(g1, g2, w.cost, mp) == cost
        assert cost >= O.brute_ged(g1, g2, w.cost)[0]
