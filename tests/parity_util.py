"""Helpers shared by the GPU parity tests: run a workload through the C ABI and through
the CPU oracle on the same seeded inputs, and compare element by element."""
import os

import numpy as np

from oracle import oracle as O
from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W

THREADS = max(1, min(16, os.cpu_count() or 1))


def gpu_run(w, K=None, **opts):
    with F.FastGED(w.cost) as g:
        return g.run(w, K, **opts)


def oracle_run(w, idx, K=None, variant=0, order=0):
    return O.kbest_workload(w, idx, K=K, variant=variant, threads=THREADS, order=order)


def assert_parity(w, gpu, idx=None, K=None, variant=0, order=0):
    """Bit-exact cost, vertex map and evaluation count on the pairs idx (all by default)."""
    cost, maps, nev = gpu
    mm = F.marshal(w)
    if idx is None:
        idx = range(w.n_pairs)
    idx = list(idx)
    ref = oracle_run(w, idx, K=K, variant=variant, order=order)
    bad = []
    for p, (rc, rm, rn) in zip(idx, ref):
        gm = maps[mm.map_off[p]:mm.map_off[p + 1]]
        if int(cost[p]) != rc or not np.array_equal(gm, rm) or int(nev[p]) != rn:
            bad.append((p, int(cost[p]), rc, int(nev[p]), rn, gm.tolist()[:12], rm.tolist()[:12]))
    assert not bad, f"{len(bad)} of {len(idx)} pairs differ; first: {bad[:3]}"


def assert_valid_paths(w, gpu, idx=None):
    """Properties that hold at any size: each map is an injective partial map into g2, and
    the returned cost is the cost of the edit path that map induces."""
    cost, maps, _ = gpu
    mm = F.marshal(w)
    if idx is None:
        idx = range(w.n_pairs)
    for p in idx:
        g1, g2 = w.graphs[w.pairs[p][0]], w.graphs[w.pairs[p][1]]
        gm = maps[mm.map_off[p]:mm.map_off[p + 1]]
        img = gm[gm >= 0]
        assert np.all(gm >= -1) and np.all(gm < g2.n) and len(np.unique(img)) == len(img)
        assert O.full_cost(g1, g2, w.cost, gm) == int(cost[p]), p


def single(pairs, cost, K, name="custom"):
    """A Workload from an explicit list of (g1, g2) graph pairs."""
    graphs = []
    for a, b in pairs:
        graphs += [a, b]
    return W.Workload(name, graphs, np.arange(len(graphs), dtype=np.int32).reshape(-1, 2),
                      tuple(cost), K)
