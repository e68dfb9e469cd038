"""The stored K-Best results (tests/golden/kbest_*.txt): one line per pair of the workload
their header names, and the oracle gives the stored values again for a few of each file's
cheap pairs (the expensive targets are checked for structure only)."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location(
    "make_kbest_golden", os.path.join(HERE, "golden", "make_kbest_golden.py"))
G = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(G)

# pairs recomputed on the CPU per target (cheap ones only)
RECHECK = {"config2": [0, 1, 7, 19999], "config3": [0, 4095], "config5_2000": [0, 1, 2, 3],
           "widebeam": [0]}


def stored():
    return sorted(n for n in G.TARGETS if os.path.exists(G.golden_path(n)))


@pytest.mark.parametrize("name", stored())
def test_golden_file_matches_its_workload(name):
    w = G.TARGETS[name][0]()
    idx, cost, nev, dig = G.load(name)
    assert idx.tolist() == list(range(w.n_pairs))
    assert all(len(d) == 16 and int(d, 16) >= 0 for d in dig)
    assert (cost >= 0).all() and (nev > 0).all()
    with open(G.golden_path(name)) as f:
        head = f.readline()
    assert head.startswith("# ") and G.TARGETS[name][1] in head
    for p in RECHECK.get(name, []):
        a, b = (int(x) for x in w.pairs[p])
        k = int(w.k_per_pair[p]) if w.k_per_pair is not None else w.K
        c, m, n = O.kbest(w.graphs[a], w.graphs[b], w.cost, k)
        assert (c, n, G.map_digest(m)) == (cost[p], nev[p], dig[p]), p


def test_map_digest_is_the_blake2b_of_the_int32_map():
    import hashlib
    m = np.array([3, -1, 0, 7], dtype=np.int32)
    assert G.map_digest(m) == hashlib.blake2b(m.astype("<i4").tobytes(), digest_size=8).hexdigest()
    assert G.map_digest([3, -1, 0, 7]) == G.map_digest(m)
    assert G.map_digest([3, -1, 0, 8]) != G.map_digest(m)
