"""Edit paths of vertex maps (Sec. 2.3-2.4) and their partial application (the crossover of
Sec. 6): the oracle's edit_path is pinned to a hand-worked example and to the independent
full-path evaluator; the library's host functions must list exactly the oracle's operations.
These run on the CPU: fastged_edit_path and fastged_apply_edit_ops do no GPU work."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W

S1 = W.SETTING1_COSTS   # (vsub 2, vdel 4, vins 4, esub 1, edel 2, eins 2)


def _hand_pair():
    g1 = W.Graph(3, np.array([0, 1, 2], np.int32), np.array([[0, 1], [1, 2]], np.int32),
                 np.array([0, 1], np.int32))
    g2 = W.Graph(3, np.array([0, 1, 1], np.int32), np.array([[0, 1], [0, 2]], np.int32),
                 np.array([1, 0], np.int32))
    return g1, g2


def test_oracle_edit_path_hand_example():
    """v0 -> u0 and v1 -> u1 keep their labels, v2 is deleted, u2 inserted; edge (v0, v1)
    becomes the g2 edge (u0, u1) with another label, (v1, v2) goes with v2, and (u0, u2)
    comes with u2: 4 + 1 + 2 + 2 + 4 = 13 under setting 1."""
    g1, g2 = _hand_pair()
    ops = O.edit_path(g1, g2, S1, [0, 1, -1])
    assert ops == [(O.OP_VINS, 4, -1, -1, 2, -1), (O.OP_EDEL, 2, 1, 2, -1, -1),
                   (O.OP_ESUB, 1, 0, 1, 0, 1), (O.OP_EINS, 2, -1, -1, 0, 2),
                   (O.OP_VDEL, 4, 2, -1, -1, -1)]
    assert sum(o[1] for o in ops) == 13 == O.full_cost(g1, g2, S1, [0, 1, -1])


def _random_map(st, n1, n2):
    perm = list(np.argsort(st.uniform(n2))) if n2 else []
    out = []
    for v in range(n1):
        if perm and st.uniform(1)[0] < 0.75:
            out.append(int(perm.pop()))
        else:
            out.append(-1)
    return np.array(out, dtype=np.int32)


def _cases(n):
    for s in range(n):
        st = W.Stream(s, 61)
        ne = 3 if s % 2 else 0
        g1 = W.random_small(st, 0, 8, 0.4, 3, ne)
        g2 = W.random_small(st, 0, 8, 0.4, 3, ne)
        yield s, g1, g2, _random_map(st, g1.n, g2.n)


@pytest.mark.parametrize("s,g1,g2,mp", list(_cases(60)))
def test_oracle_edit_path_costs_match_full_cost(s, g1, g2, mp):
    cost = tuple(int(x) for x in W.Stream(s, 62).randint(0, 7, 6))
    ops = O.edit_path(g1, g2, cost, mp)
    assert sum(o[1] for o in ops) == O.full_cost(g1, g2, cost, mp)
    # each changed element is edited once: vertex ops cover every g2 vertex outside the image
    # and every deleted g1 vertex
    assert sum(o[0] == O.OP_VINS for o in ops) == g2.n - int((mp >= 0).sum())
    assert sum(o[0] == O.OP_VDEL for o in ops) == int((mp < 0).sum())


@pytest.mark.parametrize("s,g1,g2,mp", list(_cases(60)))
def test_library_edit_path_equals_oracle(s, g1, g2, mp):
    cost = tuple(int(x) for x in W.Stream(s, 63).randint(0, 7, 6))
    ops, tot = F.fastged_edit_path(cost, g1, g2, mp)
    ref = O.edit_path(g1, g2, cost, mp)
    assert [tuple(int(x) for x in o) for o in ops] == ref
    assert tot == O.full_cost(g1, g2, cost, mp)


def _as_g2(g1, g2, mp, res):
    """Map the vertices of an applied result back to g2 ids (surviving g1 vertices in order,
    then inserted g2 vertices in insertion order) and return (labels, edge dict) over g2."""
    ids = [int(mp[v]) for v in range(g1.n) if mp[v] >= 0]
    ids += [x for x in range(g2.n) if x not in set(int(y) for y in mp)]
    lab = {ids[r]: int(res.vlabel[r]) for r in range(res.n)}
    el = np.zeros(res.edges.shape[0], np.int32) if res.elabel is None else res.elabel
    edges = {frozenset((ids[int(a)], ids[int(b)])): int(l) for (a, b), l in zip(res.edges, el)}
    return lab, edges


@pytest.mark.parametrize("s,g1,g2,mp", list(_cases(40)))
def test_applying_the_whole_path_gives_g2_and_prefixes_are_valid(s, g1, g2, mp):
    ops, _ = F.fastged_edit_path(S1, g1, g2, mp)
    full = F.fastged_apply_edit_ops(g1, g2, mp, ops, len(ops))
    lab, edges = _as_g2(g1, g2, mp, full)
    assert lab == {x: int(g2.vlabel[x]) for x in range(g2.n)}
    el2 = np.zeros(g2.edges.shape[0], np.int32) if g2.elabel is None else g2.elabel
    assert edges == {frozenset((int(a), int(b))): int(l) for (a, b), l in zip(g2.edges, el2)}
    for k in range(len(ops) + 1):   # every prefix is a valid graph (the crossover applies half)
        r = F.fastged_apply_edit_ops(g1, g2, mp, ops, k)
        assert r.edges.size == 0 or (r.edges.min() >= 0 and r.edges.max() < r.n)
        assert len({frozenset(map(int, e)) for e in r.edges}) == r.edges.shape[0]


def test_hand_example_applied_half():
    g1, g2 = _hand_pair()
    mp = np.array([0, 1, -1], np.int32)
    ops, tot = F.fastged_edit_path(S1, g1, g2, mp)
    assert tot == 13 and len(ops) == 5
    half = F.fastged_apply_edit_ops(g1, g2, mp, ops, 2)   # insert u2, delete (v1, v2)
    assert half.n == 4 and list(half.vlabel) == [0, 1, 2, 1]
    assert half.edges.tolist() == [[0, 1]] and half.elabel.tolist() == [0]


def test_edit_path_rejects_bad_maps_and_small_arrays():
    g1, g2 = _hand_pair()
    for bad in ([0, 0, -1], [0, 3, -1], [0, -2, 1]):
        with pytest.raises(F.FastGEDError):
            F.fastged_edit_path(S1, g1, g2, bad)
    lib = F.load()
    a, b = F._OneGraph(g1), F._OneGraph(g2)
    mp = np.array([0, 1, -1], np.int32)
    ops = np.zeros(2, F.EDIT_OP_DTYPE)
    n = F.ctypes.c_int32(0)
    cm = F._cost_model(S1)
    rc = lib.fastged_edit_path(F.ctypes.byref(cm), F.ctypes.byref(a.st), F.ctypes.byref(b.st),
                               mp.ctypes.data, ops.ctypes.data, 2, F.ctypes.byref(n), None)
    assert rc == F.FASTGED_ERR_INVALID_ARG and n.value == 5
    # an operation list out of order (edge insertion before its vertex exists) is refused
    ops, _ = F.fastged_edit_path(S1, g1, g2, mp)
    with pytest.raises(F.FastGEDError):
        F.fastged_apply_edit_ops(g1, g2, mp, ops[[3, 0, 1, 2, 4]], 5)
