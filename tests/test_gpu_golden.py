"""Whole-batch GPU parity against stored oracle results.

tests/golden/kbest_<target>.txt hold, for every pair of a seeded workload, the CPU oracle's
cost, evaluation count and a 64-bit digest of its vertex map; tests/golden/make_kbest_golden.py
wrote them and calls only the oracle. Each test runs the whole batch on the GPU through the C
ABI and compares every pair: cost and evaluation count bit-exact, the map identical (equal
digests). The batches are the full configurations: the 20,000 molecule-like pairs (config 2),
the 4,096 dense ER pairs (config 3), the 64 BA pairs at K = 1024 (config 4), the first 2,000
queries of the serving stream at their drawn K (config 5, as a batch and through the server),
the wide beam (16 molecule-sized pairs at K = 100,000) and the graph-size sweep (G(n, 0.4)
pairs at K = 5,000).
"""
import importlib.util
import os
import time

import numpy as np
import pytest

from paper_2605_00830_gb300 import fastged as F

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
_spec = importlib.util.spec_from_file_location(
    "make_kbest_golden", os.path.join(HERE, "golden", "make_kbest_golden.py"))
G = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(G)

TARGETS = ["config2", "config3", "config4", "config5_2000", "widebeam", "sizesweep_200",
           "sizesweep_300", "sizesweep_500", "sizesweep_950"]


def compare(name, w, cost, maps, nev):
    idx, gc, gn, gd = G.load(name)
    assert idx.tolist() == list(range(w.n_pairs))
    mm = F.marshal(w)
    bad = []
    for p in range(w.n_pairs):
        m = maps[mm.map_off[p]:mm.map_off[p + 1]]
        if int(cost[p]) != gc[p] or int(nev[p]) != gn[p] or G.map_digest(m) != gd[p]:
            bad.append((p, int(cost[p]), int(gc[p]), int(nev[p]), int(gn[p])))
    assert not bad, (f"{len(bad)} of {w.n_pairs} pairs differ from the oracle "
                     f"(pair, cost, oracle cost, n_evals, oracle n_evals): {bad[:5]}")


@pytest.mark.parametrize("name", TARGETS)
def test_batch_matches_stored_oracle(name):
    w = G.TARGETS[name][0]()
    with F.FastGED(w.cost) as g:
        c, m, n = g.run(w)
    compare(name, w, c, m, n)


@pytest.mark.parametrize("name", ["config2", "config5_2000"])
def test_cta_teams_match_stored_oracle(name):
    """The same batches with every pair solved by a CTA team (no one-warp classes)."""
    w = G.TARGETS[name][0]()
    with F.FastGED(w.cost) as g:
        c, m, n = g.run(w, team=F.FASTGED_TEAM_CTA)
    compare(name, w, c, m, n)


def test_config2_bench_configuration_matches_stored_oracle():
    """The 20,000-pair molecule-like batch in the launch configuration the benchmark times:
    an autotuned device-resident plan, replayed as a CUDA graph (twice)."""
    w = G.TARGETS["config2"][0]()
    mm = F.marshal(w)
    with F.FastGED(w.cost) as g:
        plan = F.fastged_plan_create(g.h, mm, w.K, F.make_options(autotune=1))
        for _ in range(2):
            F.fastged_plan_run(plan)
            c, m, n = (np.zeros(mm.n_pairs, np.int32), np.zeros(int(mm.map_off[-1]), np.int32),
                       np.zeros(mm.n_pairs, np.int64))
            F.fastged_plan_read(plan, c, m, n)
            compare("config2", w, c, m, n)
        F.fastged_plan_destroy(plan)


def test_served_config5_matches_stored_oracle():
    """The first 2,000 queries of the serving stream submitted to the continuous-batching
    server (each at its drawn K): every served result equals the oracle's."""
    w = G.TARGETS["config5_2000"][0]()
    idx, gc, gn, gd = G.load("config5_2000")
    mm = F.marshal(w)
    srv = F.Server(w.cost)
    try:
        for p in range(w.n_pairs):
            a, b = (int(x) for x in w.pairs[p])
            while True:
                rc = srv.submit(mm, a, b, int(w.k_per_pair[p]), p)
                if rc != F.FASTGED_ERR_BUSY:
                    assert rc == F.FASTGED_OK, F.fastged_last_error()
                    break
                time.sleep(0.001)
        got = {}
        deadline = time.time() + 600
        while len(got) < w.n_pairs and time.time() < deadline:
            for tag, status, cost, mp, nev, _, _ in srv.poll(timeout_ms=50):
                assert status == F.FASTGED_OK, (tag, status)
                got[tag] = (cost, mp, nev)
    finally:
        srv.stop()
        srv.close()
    assert len(got) == w.n_pairs
    bad = [p for p in range(w.n_pairs)
           if got[p][0] != gc[p] or got[p][2] != gn[p] or G.map_digest(got[p][1]) != gd[p]]
    assert not bad, f"{len(bad)} served results differ from the oracle; first {bad[:5]}"
