"""GPU parity: the sm_103a path through the C ABI against the CPU oracle, bit-exact on
cost, vertex map and evaluation count (costs are integers, so the tolerance is zero)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W
from parity_util import assert_parity, assert_valid_paths, gpu_run, single

pytestmark = pytest.mark.gpu


def test_config1_full():
    w = W.config1()
    assert_parity(w, gpu_run(w))


def test_config2_prefix():
    w = W.config2(400)
    assert_parity(w, gpu_run(w))


def test_config3_prefix():
    w = W.config3(24)
    assert_parity(w, gpu_run(w))


def test_config4_shaped_small():
    """Large sparse shape at reduced size: BA graphs, perturbed copies, 16-bit vertex maps
    (n2 >= 255) and several 64-bit words per bitset."""
    w = W.config4(6, seed=41, n_range=(150, 320))
    w.K = 48
    assert_parity(w, gpu_run(w))


def test_config4_full_size_sample():
    """One full-size large sparse pair (the smallest of a 64-pair draw) at K = 1024."""
    w = W.config4(64)
    p = int(np.argmin([w.graphs[2 * k].n for k in range(64)]))
    ws = W.subset(w, [p])
    assert_parity(ws, gpu_run(ws))


@pytest.mark.parametrize("hw", [2, 3, 17])
def test_exact_selection_fallback(hw):
    """A tiny histogram window pushes almost every level onto the exact fallback of the
    selection; results must not change."""
    w = W.config2(120)
    assert_parity(w, gpu_run(w, hist_window=hw))
    w1 = W.config1(60)
    assert_parity(w1, gpu_run(w1, hist_window=hw))
    # dense pairs: warps hold thousands of candidates, so the histogram is counted per lane
    w3 = W.subset(W.config3(4), range(4))
    assert_parity(w3, gpu_run(w3, hist_window=hw))


def test_large_costs():
    """Costs spread far beyond the histogram window (fallback on real data)."""
    w = W.config2(80)
    w.cost = (1000, 3001, 2999, 700, 1500, 901)
    assert_parity(w, gpu_run(w))


def test_packed_single_word_entries_at_their_limits():
    """Single-word pairs store each successor as PED << 16 | parent slot << 7 | j when no
    PED can reach 2^16 and K <= 512; other pairs take the two-word kernels. PEDs above 2^15
    set the top bit of the packed entry; K = 512 packs and K = 513 does not."""
    cost = (1000, 1200, 0, 250, 300, 0)   # no insertion costs: a result is a leaf's PED
    pairs = []
    for k in range(12):
        st = W.Stream(31, k)
        big, small = W.molecule_like(st, 39), W.molecule_like(st, 5 + k % 4)
        pairs += [(big, small), (small, big)]
    for a, b in pairs:
        assert a.n * 1200 + a.m * 300 < 65536
    w = single(pairs, cost, 100)
    gpu = gpu_run(w)
    assert_parity(w, gpu)
    assert int(gpu[0].max()) > 32768
    w1 = W.config1(16)
    for K in (512, 513):
        assert_parity(w1, gpu_run(w1, K=K), K=K)


@pytest.mark.parametrize("n2,kmax", [(31, 2048), (64, 512), (100, 512), (128, 256), (200, 256)])
def test_packed_slot_field_at_its_width(n2, kmax):
    """The packed entry gives j the bit length of n2 and the slot the other 16 - jbits bits:
    K = 2^(16 - jbits) fills the slot field (packed), one more takes the unpacked path."""
    st = W.Stream(41, n2)
    g1 = W.erdos_renyi(st, 5, 0.5, 3)
    g2 = W.erdos_renyi(st, n2, 0.08, 3)
    w = single([(g1, g2)], W.UNIT_COSTS, kmax)
    for K in (kmax, kmax + 1):
        assert_parity(w, gpu_run(w, K=K), K=K)


@pytest.mark.parametrize("cfg", ["config1", "config2", "config3"])
def test_degree_vertex_order(cfg):
    """FASTGED_ORDER_DEGREE branches the source vertices by descending degree (ties by
    index) and returns maps in the original ids; the oracle runs Algorithm 1 on the same
    relabelled source graph."""
    w = {"config1": lambda: W.config1(200), "config2": lambda: W.config2(160),
         "config3": lambda: W.subset(W.config3(6), range(6))}[cfg]()
    gpu = gpu_run(w, vertex_order=F.FASTGED_ORDER_DEGREE)
    assert_parity(w, gpu, order=1)
    # a plan returns the same maps (the permutation is undone when reading results)
    mm = F.marshal(w)
    with F.FastGED(w.cost) as g:
        plan = F.fastged_plan_create(g.h, mm, w.K, F.make_options(vertex_order=1))
        F.fastged_plan_run(plan)
        c, m, n = (np.zeros(mm.n_pairs, np.int32), np.zeros(int(mm.map_off[-1]), np.int32),
                   np.zeros(mm.n_pairs, np.int64))
        F.fastged_plan_read(plan, c, m, n)
        F.fastged_plan_destroy(plan)
    for x, y in zip((c, m, n), gpu):
        assert np.array_equal(x, y)


def test_option_combinations():
    """Degree order with per-pair K, degree order with variant B, and variant B solved by a
    cluster team (one large pair, fewer pairs than SMs)."""
    w = W.config2(90, seed=31)
    w.k_per_pair = W.Stream(31, 2).randint(1, 100, w.n_pairs).astype(np.int32)
    assert_parity(w, gpu_run(w, vertex_order=1), order=1)
    w1 = W.config1(80)
    assert_parity(w1, gpu_run(w1, vertex_order=1, variant=1), order=1, variant=1)
    big = W.config4(1, seed=13, n_range=(300, 340))
    assert_parity(big, gpu_run(big, K=64, variant=1), K=64, variant=1)


def test_setting2_costs():
    """The paper's cost setting 2 (expensive insertions and deletions) on molecule-like and
    dense pairs, both branching orders."""
    for w in (W.config2(150), W.subset(W.config3(8), range(8))):
        w.cost = W.SETTING2_COSTS
        assert_parity(w, gpu_run(w))
        assert_parity(w, gpu_run(w, vertex_order=1), order=1)


@pytest.mark.parametrize("case", ["k5000", "k100000", "kmax"])
def test_huge_k(case):
    """The wide-beam regime: K = 5000 on molecule-sized pairs, K = 100,000 on ~14-vertex
    graphs and K = 2^20 on 8-9 vertex graphs, with the default histogram window and with a
    window of 2 (every level then orders its kept beam with the exact selection's sort)."""
    if case == "k5000":
        w = W.config2(6, seed=11)
        K = 5000
    elif case == "k100000":
        st = W.Stream(12, 1)
        pairs = [(W.erdos_renyi(st, 13, 0.3, 4), W.erdos_renyi(st, 14, 0.3, 4)) for _ in range(2)]
        w = single(pairs, W.UNIT_COSTS, 100000)
        K = 100000
    else:
        st = W.Stream(13, 1)
        w = single([(W.erdos_renyi(st, 8, 0.4, 3), W.erdos_renyi(st, 9, 0.4, 3))],
                   W.SETTING1_COSTS, 1 << 20)
        K = 1 << 20
    ref = None
    for hw in (0, 2):
        gpu = gpu_run(w, K=K, hist_window=hw)
        if ref is None:
            assert_parity(w, gpu, K=K)
            ref = gpu
        else:
            for x, y in zip(gpu, ref):
                assert np.array_equal(x, y)


def test_results_do_not_depend_on_pair_order():
    """The same pairs in a permuted order (so other neighbours in the queue, other teams,
    other class positions) give the same per-pair results."""
    w = W.config2(300, seed=41)
    base = gpu_run(w)
    perm = np.random.RandomState(3).permutation(w.n_pairs)
    wp = W.Workload(w.name, w.graphs, w.pairs[perm], w.cost, w.K)
    c, m, n = gpu_run(wp)
    mm, mp = F.marshal(w), F.marshal(wp)
    assert np.array_equal(c, base[0][perm]) and np.array_equal(n, base[2][perm])
    for q, p in enumerate(perm):
        assert np.array_equal(m[mp.map_off[q]:mp.map_off[q + 1]], base[1][mm.map_off[p]:mm.map_off[p + 1]])


def test_concurrent_batches_from_two_host_threads():
    """Two handles used from two host threads at once (the batch flattening shares one host
    thread pool; a call that finds it busy runs serially): results equal serial runs."""
    import threading
    ws = [W.config2(600, seed=21), W.subset(W.config3(12, seed=22), range(12))]
    ref = [gpu_run(w) for w in ws]
    out, errs = [None, None], []

    def work(k):
        try:
            with F.FastGED(ws[k].cost) as g:
                for _ in range(4):
                    out[k] = g.run(ws[k])
                    for x, y in zip(out[k], ref[k]):
                        assert np.array_equal(x, y)
        except Exception as e:   # surfaced in the main thread
            errs.append(e)

    th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs


@pytest.mark.parametrize("bt", [128, 256, 512])
def test_block_sizes(bt):
    w = W.config2(150)
    assert_parity(w, gpu_run(w, block_threads=bt))


def test_plain_form_equals_batched():
    w = W.config2(200)
    a = gpu_run(w)
    b = gpu_run(w, form=F.FASTGED_FORM_PLAIN)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_per_pair_k():
    w = W.config2(90)
    st = W.Stream(77, 1)
    kpp = st.randint(1, 100, w.n_pairs).astype(np.int32)
    w.k_per_pair = kpp
    gpu = gpu_run(w, K=100)
    mm = F.marshal(w)
    cost, maps, nev = gpu
    for p in range(w.n_pairs):
        g1, g2 = w.graphs[2 * p], w.graphs[2 * p + 1]
        rc, rm, rn = O.kbest(g1, g2, w.cost, int(kpp[p]))
        assert (int(cost[p]), int(nev[p])) == (rc, rn)
        assert np.array_equal(maps[mm.map_off[p]:mm.map_off[p + 1]], rm)


def _edge_graphs():
    st = W.Stream(5, 55)
    out = {}
    e = W.empty_graph()
    g = W.random_small(st, 6, 6, 0.5, 3, 2)
    out["empty_source"] = (e, g)
    out["empty_target"] = (g, e)
    out["both_empty"] = (e, e)
    one = W.Graph(1, np.array([2], np.int32), np.zeros((0, 2), np.int32))
    out["single_vertex"] = (one, g)
    for n in (63, 64, 65, 127, 128, 129, 254, 255, 256):
        a = W.erdos_renyi(W.Stream(n, 1), n, 0.08, 5)
        b = W.erdos_renyi(W.Stream(n, 2), n, 0.08, 5)
        out[f"n{n}"] = (a, b)
    # all labels equal: maximal ties
    a = W.erdos_renyi(W.Stream(9, 1), 12, 0.3, 1)
    b = W.erdos_renyi(W.Stream(9, 2), 14, 0.3, 1)
    out["all_equal_labels"] = (a, b)
    # complete graphs
    iu = np.triu_indices(9, 1)
    k9 = W.Graph(9, np.zeros(9, np.int32), np.stack(iu, 1).astype(np.int32))
    iu = np.triu_indices(7, 1)
    k7 = W.Graph(7, np.zeros(7, np.int32), np.stack(iu, 1).astype(np.int32))
    out["complete"] = (k9, k7)
    # n1 > n2 and n1 < n2
    out["n1_gt_n2"] = (W.erdos_renyi(W.Stream(3, 1), 20, 0.2, 3),
                       W.erdos_renyi(W.Stream(3, 2), 7, 0.3, 3))
    out["n1_lt_n2"] = (W.erdos_renyi(W.Stream(4, 1), 7, 0.3, 3),
                       W.erdos_renyi(W.Stream(4, 2), 20, 0.2, 3))
    # many edge labels (8 bit-planes)
    a = W.random_small(W.Stream(6, 1), 15, 15, 0.4, 3, 256)
    b = W.random_small(W.Stream(6, 2), 15, 15, 0.4, 3, 256)
    out["elabels_255"] = (a, b)
    return out


@pytest.mark.parametrize("K", [1, 2, 7, 64, 5000])
@pytest.mark.parametrize("name", sorted(_edge_graphs()))
def test_edge_cases(name, K):
    g1, g2 = _edge_graphs()[name]
    if max(g1.n, g2.n) > 100 and K > 64:
        K = 96
    for cost in (W.UNIT_COSTS, W.SETTING1_COSTS, (3, 1, 2, 5, 1, 4)):
        w = single([(g1, g2), (g2, g1)], cost, K)
        assert_parity(w, gpu_run(w))


def test_batch_mixed_classes():
    """One batch mixing every size class (1..16 words, 8- and 16-bit maps) and labelled /
    unlabelled graphs; each pair must match the oracle as if it ran alone."""
    g = _edge_graphs()
    pairs = [g[k] for k in ("n63", "n129", "n255", "n256", "complete", "elabels_255",
                            "empty_source", "n1_gt_n2")]
    big = W.config4(1, seed=9, n_range=(600, 640))
    pairs.append((big.graphs[0], big.graphs[1]))
    w = single(pairs, W.UNIT_COSTS, 24)
    assert_parity(w, gpu_run(w))


def test_plan_replay_matches_batch_and_is_repeatable():
    w = W.config2(300)
    ref = gpu_run(w)
    mm = F.marshal(w)
    with F.FastGED(w.cost) as g:
        plan = F.fastged_plan_create(g.h, mm, w.K, F.make_options())
        outs = []
        for _ in range(3):
            F.fastged_plan_run(plan)
            c, m, n = (np.zeros(mm.n_pairs, np.int32), np.zeros(int(mm.map_off[-1]), np.int32),
                       np.zeros(mm.n_pairs, np.int64))
            F.fastged_plan_read(plan, c, m, n)
            outs.append((c, m, n))
        info = F.fastged_plan_info(plan)
        F.fastged_plan_destroy(plan)
    assert info["graph_replay"] == 1 and info["launches_per_run"] >= 2
    for o in outs:
        for x, y in zip(o, ref):
            assert np.array_equal(x, y)


def test_config2_full_batch_bench_configuration():
    """The full 20,000-pair molecule-like batch in the launch configuration the benchmark
    times (autotuned plan + CUDA-graph replay): a seeded sample of pairs is checked
    bit-exactly against the oracle, and every pair against the edit-path properties."""
    w = W.config2()
    mm = F.marshal(w)
    with F.FastGED(w.cost) as g:
        plan = F.fastged_plan_create(g.h, mm, w.K, F.make_options(autotune=1))
        F.fastged_plan_run(plan)
        c, m, n = (np.zeros(mm.n_pairs, np.int32), np.zeros(int(mm.map_off[-1]), np.int32),
                   np.zeros(mm.n_pairs, np.int64))
        F.fastged_plan_read(plan, c, m, n)
        F.fastged_plan_destroy(plan)
    idx = sorted(set(W.Stream(2024, 8).randint(0, w.n_pairs - 1, 300).tolist()))
    assert_parity(w, (c, m, n), idx=idx)
    assert_valid_paths(w, (c, m, n))


def test_invalid_inputs():
    g = W.erdos_renyi(W.Stream(1, 1), 6, 0.5, 2)
    h = W.erdos_renyi(W.Stream(1, 2), 5, 0.5, 2)
    dup = W.Graph(g.n, g.vlabel, np.concatenate([g.edges, g.edges[:1]]))
    loop = W.Graph(g.n, g.vlabel, np.concatenate([g.edges, np.array([[2, 2]], np.int32)]))
    outside = W.Graph(g.n, g.vlabel, np.array([[0, 9]], np.int32))
    big = W.Graph(1025, np.zeros(1025, np.int32), np.zeros((0, 2), np.int32))
    badlab = W.Graph(g.n, g.vlabel, g.edges, np.full(g.m, 300, np.int32))
    with F.FastGED(W.UNIT_COSTS) as fg:
        for bad in (dup, loop, outside, big, badlab):
            w = single([(bad, h)], W.UNIT_COSTS, 4)
            with pytest.raises(F.FastGEDError) as ei:
                fg.run(w)
            assert ei.value.code == F.FASTGED_ERR_INVALID_ARG
        w = single([(g, h)], W.UNIT_COSTS, 4)
        for K in (0, -3, (1 << 20) + 1):
            with pytest.raises(F.FastGEDError):
                fg.run(w, K=K)
        # an invalid call leaves the handle usable
        cost, _, _ = fg.run(w)
        assert cost[0] == O.kbest(g, h, W.UNIT_COSTS, 4)[0]
    with pytest.raises(F.FastGEDError):
        F.FastGED((1, -1, 1, 1, 1, 1))
    with pytest.raises(F.FastGEDError):
        big_cost = (1 << 29,) * 6
        with F.FastGED(big_cost) as fg:
            fg.run(single([(g, h)], big_cost, 4))


def test_invalid_entries_across_a_large_batch_report_the_lowest_index():
    """Graphs and pairs are validated in parallel chunks: with several invalid entries spread
    over a 12,000-pair batch, the error names the lowest invalid graph (graph checks come
    first, then pair checks, then edge endpoints), and the handle stays usable."""
    w = W.config2(12000)
    cases = []
    # pairs: graph index out of range at 9000 and 7001, per-pair K out of range at 8000
    pairs = w.pairs.copy()
    pairs[9000, 1] = 10 ** 6
    pairs[7001, 0] = -1
    cases.append((pairs, None, None, "pair 7001: graph index out of range"))
    kpp = np.full(w.n_pairs, 50, np.int32)
    kpp[11000], kpp[8000] = 0, 101
    cases.append((w.pairs, kpp, None, "pair 8000: per-pair K out of range"))
    # edge labels out of range in graphs 18000 and 17000
    mm0 = F.Marshalled(w.graphs, w.pairs)
    el = mm0.el.copy()
    el[int(mm0.m[:18000].sum())] = 99
    el[int(mm0.m[:17000].sum())] = -3
    cases.append((w.pairs, None, ("el", el), "graph 17000: edge label out of range"))
    # a bad endpoint in graph 20001 and a self-loop in graph 15000
    ed = mm0.ed.copy()
    ed[2 * int(mm0.m[:20001].sum()) + 1] = 9999
    e0 = 2 * int(mm0.m[:15000].sum())
    ed[e0] = ed[e0 + 1]
    cases.append((w.pairs, None, ("ed", ed), "graph 15000: bad edge endpoint or self-loop"))
    with F.FastGED(w.cost) as fg:
        for pairs, kpp, patch, msg in cases:
            mm = F.Marshalled(w.graphs, pairs.copy())
            if patch is not None:
                getattr(mm, patch[0])[:] = patch[1]
            cost, maps, nev = F._outputs(mm)
            K = 100
            with pytest.raises(F.FastGEDError) as ei:
                F.fastged_batch_ex(fg.h, mm, K, F.make_options(k_per_pair=kpp), cost, maps, nev)
            assert ei.value.code == F.FASTGED_ERR_INVALID_ARG
            assert msg in str(ei.value)
        ws = W.subset(w, range(200))
        assert_parity(ws, fg.run(ws), idx=list(range(0, 200, 20)))


@pytest.mark.parametrize("cfg", ["config1", "config2", "config3"])
def test_variant_b_complete_every_last_level_successor(cfg):
    n = {"config1": 200, "config2": 150, "config3": 6}[cfg]
    w = getattr(W, cfg)(n)
    b = gpu_run(w, variant=1)
    assert_parity(w, b, variant=1)
    a = gpu_run(w)
    assert np.all(b[0] <= a[0])   # completing a superset of leaves is never worse


def test_golden_hand_traces_on_gpu():
    """The hand-traced cases of Algorithm 1 (tests/golden) through the GPU path."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hand_traces.json")
    for case in json.load(open(path))["cases"]:
        def gr(d):
            e = np.array(d["edges"], dtype=np.int32).reshape(-1, 2)
            el = None if d.get("elabel") is None else np.array(d["elabel"], dtype=np.int32)
            return W.Graph(d["n"], np.array(d["vlabel"], dtype=np.int32), e, el)
        g1, g2 = gr(case["g1"]), gr(case["g2"])
        for variant, key in ((0, "kbest"), (1, "kbest_variant1")):
            for exp in case.get(key, []):
                w = single([(g1, g2)], case["cost"], exp["K"])
                cost, maps, nev = gpu_run(w, variant=variant)
                assert int(cost[0]) == exp["cost"], (case["name"], exp)
                assert maps.tolist() == exp["map"], (case["name"], exp)
                assert int(nev[0]) == exp["n_evals"], (case["name"], exp)


@pytest.mark.parametrize("cl", ["1", "2", "4", "8", "16"])
def test_cluster_teams_match_oracle(cl, monkeypatch):
    """Large pairs (16-bit maps, 4 to 16 words) solved by one CTA or by clusters of 2 to 16
    CTAs sharing the beam through global memory: identical results."""
    monkeypatch.setenv("FASTGED_CLUSTER", cl)
    w = W.config4(3, seed=43, n_range=(260, 700))
    w.K = 40
    assert_parity(w, gpu_run(w))
    w2 = W.config4(2, seed=44, n_range=(255, 300))
    w2.K = 300
    assert_parity(w2, gpu_run(w2, variant=1), variant=1)


def test_autotuned_plans_match_and_fill_the_table(tmp_path, monkeypatch):
    """The autotuner times each size class's team shapes and records the fastest; the plan
    built from the tuned table gives the same results, and the table file is written."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("FASTGED_AUTOTUNE_FILE", str(path))
    F.load().fastged_autotune_clear()
    w = W.concat([W.config2(500), W.config4(2, seed=45, n_range=(300, 400))], "mix")
    w.K = 64
    ref = gpu_run(w, K=64)
    mm = F.marshal(w)
    with F.FastGED(w.cost) as g:
        plan = F.fastged_plan_create(g.h, mm, 64, F.make_options(autotune=1))
        F.fastged_plan_run(plan)
        c, m, n = (np.zeros(mm.n_pairs, np.int32), np.zeros(int(mm.map_off[-1]), np.int32),
                   np.zeros(mm.n_pairs, np.int64))
        F.fastged_plan_read(plan, c, m, n)
        F.fastged_plan_destroy(plan)
    for x, y in zip((c, m, n), ref):
        assert np.array_equal(x, y)
    assert F.load().fastged_autotune_entries() >= 2
    lines = path.read_text().strip().splitlines()
    # key, threads per CTA, CTAs per team, vertex-map placement of one-warp classes, ms
    assert len(lines) >= 2 and all(len(l.split()) == 5 for l in lines)
    F.load().fastged_autotune_clear()
