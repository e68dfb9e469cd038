"""Planted mistakes in the oracle (CPU only): each mutant is a copy of the oracle source
with one plausible error (a dropped term, a swapped cost, a wrong index, a reversed
tie-break), compiled to a temporary library. The pins must reject every mutant."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_00830_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "fastged_oracle.c")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_traces.json")

MUTANTS = {
    "drop_edge_substitution": ("if (e1 != e2) cost += c[C_ESUB]; }", "}"),
    "deleted_neighbour_free": ("if (e1) cost += c[C_EDEL];\n            continue;", "continue;"),
    "edel_eins_swapped": ("else if (e1) cost += c[C_EDEL];                      /* e1 -> eps */",
                          "else if (e1) cost += c[C_EINS];"),
    "deletion_keeps_edges": ("if (ogo_edge(g1, i, k)) cost += c[C_EDEL];   /* its edges go with it */", ";"),
    "wrong_image_index": ("int e2 = ogo_edge(g2, j, map[k]);", "int e2 = ogo_edge(g2, j, k < g2->n ? k : 0);"),
    "child_order_reversed": ("if (a->j != b->j) return a->j < b->j ? -1 : 1;",
                             "if (a->j != b->j) return a->j > b->j ? -1 : 1;"),
    "parent_order_reversed": ("if (a->parent != b->parent) return a->parent < b->parent ? -1 : 1;",
                              "if (a->parent != b->parent) return a->parent > b->parent ? -1 : 1;"),
    "keep_worst": ("if (a->ped != b->ped) return a->ped < b->ped ? -1 : 1;",
                   "if (a->ped != b->ped) return a->ped > b->ped ? -1 : 1;"),
    "leaf_edge_insert_both_ends": ("(!used[a] || !used[b])) total += c[C_EINS];",
                                   "(!used[a] && !used[b])) total += c[C_EINS];"),
    "leaf_tie_last_slot": ("if (total < best) { best = total; best_s = s; }",
                           "if (total <= best) { best = total; best_s = s; }"),
    "keep_one_fewer": ("newL > (size_t)K) newL = (size_t)K;",
                       "newL >= (size_t)K) newL = K > 1 ? (size_t)K - 1 : 1;"),
    "vertex_sub_inverted": ("else if (g1->alpha[a] != g2->alpha[map[a]]) cost += c[C_VSUB];",
                            "else if (g1->alpha[a] == g2->alpha[map[a]]) cost += c[C_VSUB];"),
    "square_edge_sub_always": ("if (e1 && e2) cost += (e1 != e2) ? c[C_ESUB] : 0;",
                               "if (e1 && e2) cost += c[C_ESUB];"),
    "full_cost_ins_del_swapped": ("if (pre[u] < 0) cost += c[C_VINS];", "if (pre[u] < 0) cost += c[C_VDEL];"),
    "variant_b_cuts_to_k": ("if (!(variant == 1 && i == n1 - 1) && newL > (size_t)K)",
                            "if (newL > (size_t)K)"),
}


def _graph(d):
    e = np.array(d["edges"], dtype=np.int32).reshape(-1, 2)
    el = None if d.get("elabel") is None else np.array(d["elabel"], dtype=np.int32)
    return W.Graph(n=d["n"], vlabel=np.array(d["vlabel"], dtype=np.int32), edges=e, elabel=el)


def _pins_pass(lib) -> bool:
    """A compact run of the pins; False as soon as one disagrees."""
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        g1, g2 = _graph(case["g1"]), _graph(case["g2"])
        if O.brute_ged(g1, g2, case["cost"], lib=lib)[0] != case["exact"]:
            return False
        if O.brute_square(g1, g2, case["cost"], lib=lib) != case["exact"]:
            return False
        for exp in case.get("kbest", []):
            cost, mp, nev = O.kbest(g1, g2, case["cost"], exp["K"], lib=lib)
            if (cost, list(mp), nev) != (exp["cost"], exp["map"], exp["n_evals"]):
                return False
            if "leaf_ped" in exp:
                ped, lm = O.kbest_leaves(g1, g2, case["cost"], exp["K"], lib=lib)
                if list(ped) != exp["leaf_ped"] or lm.tolist() != exp["leaf_map"]:
                    return False
        for exp in case.get("kbest_variant1", []):
            cost, mp, nev = O.kbest(g1, g2, case["cost"], exp["K"], variant=1, lib=lib)
            if (cost, list(mp), nev) != (exp["cost"], exp["map"], exp["n_evals"]):
                return False
    for seed in range(12):
        st = W.Stream(seed, 93)
        g1 = W.random_small(st, 1, 5, 0.5, 3, 2)
        g2 = W.random_small(st, 1, 4, 0.5, 3, 2)
        c = tuple(int(x) for x in st.randint(1, 6, 6))
        ged = O.brute_ged(g1, g2, c, lib=lib)[0]
        if ged != O.brute_square(g1, g2, c, lib=lib):
            return False
        Kx = max(sum(math.comb(i, j) * math.perm(g2.n, j) for j in range(min(i, g2.n) + 1))
                 for i in range(g1.n + 1))
        cost, mp, _ = O.kbest(g1, g2, c, Kx, lib=lib)
        if cost != ged or O.full_cost(g1, g2, c, mp, lib=lib) != cost:
            return False
    # variant B: the best child of the beam kept before the last level
    for seed in range(8):
        g1, g2 = _rand_pair_b(seed)
        c = tuple(int(x) for x in W.Stream(seed, 94).randint(1, 6, 6))
        for K in (1, 2):
            got = O.kbest(g1, g2, c, K, variant=1, lib=lib)[0]
            _, maps = O.kbest_leaves(_prefix(g1, g1.n - 1), g2, c, K, lib=lib)
            best = min(O.full_cost(g1, g2, c, list(m) + [j], lib=lib) for m in maps
                       for j in [u for u in range(g2.n) if u not in set(int(x) for x in m)] + [-1])
            if got != best:
                return False
    return True


def _rand_pair_b(seed):
    st = W.Stream(seed, 95)
    return W.random_small(st, 2, 5, 0.5, 3, 2), W.random_small(st, 1, 4, 0.5, 3, 2)


def _prefix(g, k):
    e = np.asarray(g.edges, dtype=np.int32).reshape(-1, 2)
    keep = (e[:, 0] < k) & (e[:, 1] < k)
    el = None if g.elabel is None else np.asarray(g.elabel, dtype=np.int32)[keep]
    return W.Graph(n=k, vlabel=np.asarray(g.vlabel, dtype=np.int32)[:k], edges=e[keep],
                   elabel=el)


def test_unmutated_oracle_passes():
    assert _pins_pass(None)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = O._bind(O.compile_c(str(path), str(tmp_path / "libmutant.so")))
    assert not _pins_pass(lib), f"pins did not catch mutant {name}"


# --------------------------------------------------------------------------------------
# planted mistakes in the Python parts of the oracle (edit paths, branching order)
# --------------------------------------------------------------------------------------
import inspect  # noqa: E402

PY_MUTANTS = {
    "edit_path": {
        "deletion_costed_as_insertion": ("ops.append((OP_EDEL, c_edel, u, v, -1, -1))",
                                         "ops.append((OP_EDEL, c_eins, u, v, -1, -1))"),
        "edge_relabel_always": ("if l2 is not None and l2 != el1[k]:", "if l2 is not None:"),
        "insertions_between_mapped_missed": (
            "if x not in pre or y not in pre or frozenset((pre[x], pre[y])) not in g1_edge:",
            "if x not in pre or y not in pre:"),
        "vertex_relabel_always": ("if phi[v] >= 0 and lab1[v] != lab2[phi[v]]:", "if phi[v] >= 0:"),
        "deleted_vertex_edges_kept": (
            "if phi[u] < 0 or phi[v] < 0 or frozenset((phi[u], phi[v])) not in g2_edge:",
            "if phi[u] >= 0 and phi[v] >= 0 and frozenset((phi[u], phi[v])) not in g2_edge:"),
    },
    "degree_order": {
        "ascending_degree": ("key=lambda v: (-deg[v], v)", "key=lambda v: (deg[v], v)"),
        "ties_by_reverse_index": ("key=lambda v: (-deg[v], v)", "key=lambda v: (-deg[v], -v)"),
    },
}


def _mutant_fn(name, old, new):
    src = inspect.getsource(getattr(O, name))
    assert src.count(old) == 1, (name, old)
    ns = dict(vars(O))
    exec(src.replace(old, new), ns)   # noqa: S102 - a planted mistake in test code
    return ns[name]


def _edit_path_pins_pass(fn) -> bool:
    g1 = W.Graph(3, np.array([0, 1, 2], np.int32), np.array([[0, 1], [1, 2]], np.int32),
                 np.array([0, 1], np.int32))
    g2 = W.Graph(3, np.array([0, 1, 1], np.int32), np.array([[0, 1], [0, 2]], np.int32),
                 np.array([1, 0], np.int32))
    if fn(g1, g2, W.SETTING1_COSTS, [0, 1, -1]) != [
            (O.OP_VINS, 4, -1, -1, 2, -1), (O.OP_EDEL, 2, 1, 2, -1, -1),
            (O.OP_ESUB, 1, 0, 1, 0, 1), (O.OP_EINS, 2, -1, -1, 0, 2),
            (O.OP_VDEL, 4, 2, -1, -1, -1)]:
        return False
    for s in range(40):
        st = W.Stream(s, 71)
        a = W.random_small(st, 0, 7, 0.45, 3, 3 if s % 2 else 0)
        b = W.random_small(st, 0, 7, 0.45, 3, 3 if s % 2 else 0)
        perm = list(np.argsort(st.uniform(b.n))) if b.n else []
        mp = [int(perm.pop()) if perm and st.uniform(1)[0] < 0.75 else -1 for _ in range(a.n)]
        cost = (3, 5, 7, 2, 11, 13)   # distinct, so a swapped cost changes the total
        if sum(o[1] for o in fn(a, b, cost, mp)) != O.full_cost(a, b, cost, mp):
            return False
    return True


def _degree_order_pins_pass(fn) -> bool:
    g = W.Graph(7, np.arange(7, dtype=np.int32),
                np.array([[0, 1], [1, 2], [3, 4], [3, 5], [3, 6]], dtype=np.int32))
    return fn(g) == [3, 1, 0, 2, 4, 5, 6]


def test_python_oracle_pins_pass_on_the_real_functions():
    assert _edit_path_pins_pass(O.edit_path)
    assert _degree_order_pins_pass(O.degree_order)


@pytest.mark.parametrize("fname,mut", [(f, m) for f, ms in PY_MUTANTS.items() for m in ms])
def test_python_oracle_mutant_is_rejected(fname, mut):
    old, new = PY_MUTANTS[fname][mut]
    fn = _mutant_fn(fname, old, new)
    check = _edit_path_pins_pass if fname == "edit_path" else _degree_order_pins_pass
    assert not check(fn), f"the pins accept the mutant {fname}:{mut}"
