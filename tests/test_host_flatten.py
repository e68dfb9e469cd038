"""Host logic of the batch flattening, on the CPU.

The host runtime (paper_2605_00830_gb300/csrc/fastged_runtime.cu) holds no device code; here it
is built with g++ against fakes of the CUDA calls it makes (tests/host_probe.py), and what
its flattening produces for a batch -- validation errors, size classes, the heaviest-first
pair order, the graph table, the map offsets, the staging bytes, the cap on resident teams --
is checked against plain Python restatements of the same rules. The batches span many of the
chunks the flattening works in, so the parallel passes and their combination are exercised.
"""
import ctypes
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W

from host_probe import load

META_DTYPE = np.dtype([("n", "<i4"), ("m", "<i4"), ("W", "<i4"), ("pad", "<i4"),
                       ("adj_off", "<i8"), ("plane_off", "<i8"), ("lab_off", "<i8"),
                       ("edge_off", "<i8")])
BATCH_FIELDS = ("n_graphs n_pairs K B labelled has_kpp n_vlab n_edges adj_words plane_words "
                "map_total off_meta off_vlab off_edges off_elab off_pairs off_order off_mapoff "
                "off_kpp in_bytes woff_err woff_cost woff_nev woff_map out_bytes woff_queue "
                "woff_pool woff_scratch work_bytes n_classes perm_size").split()
CLASS_FIELDS = ("W wide w32 pk cluster n1max n2max m1max kmax n_order order_off block grid "
                "slice_bytes scratch_off smem_bytes warp").split()


@pytest.fixture(scope="module")
def lib():
    L = load()
    yield L
    L.fake_set_free_bytes(250 << 30)


class Flat:
    """What one flatten call produced."""

    def __init__(self, L, w, K=None, cost=None, pairs=None, mm=None, **opts):
        self.w = w
        self.mm = mm if mm is not None else F.Marshalled(w.graphs, w.pairs if pairs is None
                                                          else pairs)
        self.K = K if K is not None else w.K
        self.cost = tuple(cost if cost is not None else w.cost)
        self.opts = F.make_options(**opts)
        c = (ctypes.c_int32 * 6)(*self.cost)
        self.rc = L.probe_flatten(ctypes.addressof(self.mm.pl), self.K,
                                  ctypes.addressof(self.opts), c)
        self.err = L.probe_error().decode()
        if self.rc != 0:
            return
        v = (ctypes.c_int64 * len(BATCH_FIELDS))()
        L.probe_batch(v)
        self.b = dict(zip(BATCH_FIELDS, v))
        self.classes, self.orders = [], []
        for k in range(self.b["n_classes"]):
            x = (ctypes.c_int64 * len(CLASS_FIELDS))()
            L.probe_class(k, x)
            cl = dict(zip(CLASS_FIELDS, x))
            o = np.zeros(max(cl["n_order"], 1), np.int32)
            L.probe_class_order(k, o.ctypes.data)
            self.classes.append(cl)
            self.orders.append(o[:cl["n_order"]])
        self.meta = np.zeros(max(self.b["n_graphs"], 1), META_DTYPE)
        L.probe_meta(self.meta.ctypes.data)
        self.meta = self.meta[:self.b["n_graphs"]]
        self.map_off = np.zeros(max(self.b["n_pairs"], 1), np.int64)
        L.probe_map_off(self.map_off.ctypes.data)
        self.map_off = self.map_off[:self.b["n_pairs"]]
        self.perm = np.zeros(max(self.b["perm_size"], 1), np.int32)
        L.probe_perm(self.perm.ctypes.data)
        self.perm = self.perm[:self.b["perm_size"]]
        self.staging = ctypes.string_at(L.probe_staging(), self.b["in_bytes"])

    def region(self, off, dtype, count):
        a = np.frombuffer(self.staging, dtype=dtype, count=count, offset=self.b[off])
        return a.copy()


# ---- plain restatements of the runtime's rules -------------------------------------------

def words_class(n2):
    w = (n2 + 63) // 64
    return 1 if w <= 1 else 2 if w <= 2 else 4 if w <= 4 else 8 if w <= 8 else 16


def class_key(g1, g2, kp, cost):
    """(W, wide, w32, pk, warp): bitset words of g2 (a single-word pair that cannot pack its
    successors into 32 bits moves to two words), 16-bit map entries, 32-bit words, packed,
    and one warp per pair (single-word pairs whose source has at most 64 vertices, whose
    target has at most 63 (the deletion is the bit after the last vertex) and whose K is at
    most 128, under the default team option and variant A; their 32-bit word instance takes
    targets of at most 31 vertices)."""
    vsub, vdel, vins, esub, edel, eins = cost
    ped_bound = g1.n * max(vsub, vdel) + g1.m * max(esub, edel) + g2.m * eins
    jb = int(g2.n).bit_length()
    pk = ped_bound < 65536 and jb <= 16 and kp <= (1 << (16 - jb))
    W = words_class(g2.n)
    if W == 1 and not pk:
        W = 2
    warp = W == 1 and g1.n <= 64 and g2.n <= 63 and kp <= 128
    return (W, g2.n >= 255, W == 1 and g2.n <= (31 if warp else 32), pk, warp)


def work_bucket(g1, g2, kp):
    """Heaviest first: 1023 - floor(16 log2(n1 * min(K, n1 n2 + 1) * (n2 + 1)))."""
    wt = float(g1.n) * float(min(kp, 1 + g2.n * g1.n)) * float(g2.n + 1)
    q = 0 if wt < 1.0 else int(math.log2(wt) * 16.0)
    return 1023 - min(max(q, 0), 1023)


def _mix():
    w2 = W.config2(6000)
    w3 = W.config3(60)
    w4 = W.config4(3, n_range=(240, 300))
    return W.concat([W.subset(w2, range(3000)), w3, W.config1(), w4,
                     W.subset(w2, range(3000, 6000))])


# ---- tests ---------------------------------------------------------------------------

@pytest.mark.parametrize("per_pair_k", [False, True])
def test_classes_and_heaviest_first_order(lib, per_pair_k):
    w = _mix()
    kpp = (np.arange(w.n_pairs) * 7919 % 500 + 1).astype(np.int32) if per_pair_k else None
    K = 500 if per_pair_k else 64
    f = Flat(lib, w, K=K, cost=(2, 4, 4, 1, 2, 2), k_per_pair=kpp)
    assert f.rc == 0, f.err
    g = w.graphs
    keys, first = {}, []
    for p in range(w.n_pairs):
        a, d = (int(x) for x in w.pairs[p])
        kp = int(kpp[p]) if per_pair_k else K
        key = class_key(g[a], g[d], kp, f.cost)
        if key not in keys:
            keys[key] = []
            first.append(key)
        keys[key].append((work_bucket(g[a], g[d], kp), p, a, d, kp))
    assert len(f.classes) == len(first) >= 4
    off = 0
    for cl, order, key in zip(f.classes, f.orders, first):
        Wk, wide, w32, pk, warp = key
        assert (cl["W"], cl["wide"], cl["w32"], cl["pk"], cl["warp"]) == (
            Wk, int(wide or Wk >= 8), int(w32), int(pk), int(warp))
        items = keys[key]
        expect = [p for _, p, _, _, _ in sorted(items)]
        assert order.tolist() == expect
        assert cl["n1max"] == max(g[a].n for _, _, a, _, _ in items)
        assert cl["m1max"] == max(g[a].m for _, _, a, _, _ in items)
        assert cl["n2max"] == max(g[d].n for _, _, _, d, _ in items)
        assert cl["kmax"] == max(kp for *_, kp in items)
        assert cl["order_off"] == off
        off += len(order)
    # the staged order is the classes' orders one after another
    staged = f.region("off_order", np.int32, w.n_pairs)
    assert staged.tolist() == np.concatenate(f.orders).tolist()
    if per_pair_k:
        assert f.region("off_kpp", np.int32, w.n_pairs).tolist() == kpp.tolist()


def test_graph_table_and_staging_bytes(lib):
    w = _mix()
    f = Flat(lib, w, K=32, cost=(2, 4, 4, 1, 2, 2))
    assert f.rc == 0, f.err
    g = w.graphs
    n = np.array([x.n for x in g])
    m = np.array([x.m for x in g])
    Wd = np.maximum(1, (n + 63) // 64)
    maxlab = max([int(np.max(x.elabel)) for x in g if x.elabel is not None and x.m > 0] + [0])
    B = 0
    while (1 << B) <= maxlab:
        B += 1
    B = 2 if B == 1 else B
    assert f.b["B"] == B and f.b["labelled"] == int(B > 0)
    excl = lambda a: np.concatenate([[0], np.cumsum(a)[:-1]]).astype(np.int64)
    assert f.meta["n"].tolist() == n.tolist() and f.meta["m"].tolist() == m.tolist()
    assert f.meta["W"].tolist() == Wd.tolist()
    assert f.meta["lab_off"].tolist() == excl(n).tolist()
    assert f.meta["edge_off"].tolist() == excl(m).tolist()
    assert f.meta["adj_off"].tolist() == excl(n * Wd).tolist()
    assert f.meta["plane_off"].tolist() == (excl(n * Wd) * B).tolist()
    assert (f.b["n_vlab"], f.b["n_edges"], f.b["adj_words"]) == (n.sum(), m.sum(), (n * Wd).sum())
    # staged copies
    staged_meta = np.frombuffer(f.staging, META_DTYPE, count=len(g), offset=f.b["off_meta"])
    assert staged_meta.tobytes() == f.meta.tobytes()
    assert np.array_equal(f.region("off_vlab", np.int32, n.sum()),
                          np.concatenate([np.asarray(x.vlabel, np.int32) for x in g]))
    assert np.array_equal(f.region("off_edges", np.int32, 2 * m.sum()),
                          np.concatenate([np.asarray(x.edges, np.int32).reshape(-1) for x in g]))
    el = np.concatenate([np.asarray(x.elabel, np.int32) if x.elabel is not None
                         else np.zeros(x.m, np.int32) for x in g])
    assert np.array_equal(f.region("off_elab", np.int32, m.sum()), el)
    assert np.array_equal(f.region("off_pairs", np.int32, 2 * w.n_pairs).reshape(-1, 2), w.pairs)
    n1 = n[w.pairs[:, 0]]
    assert f.map_off.tolist() == excl(n1).tolist()
    assert f.region("off_mapoff", np.int64, w.n_pairs).tolist() == f.map_off.tolist()
    assert f.b["map_total"] == n1.sum()
    # regions in order, 256-byte aligned, inside the staging buffer
    offs = [f.b[k] for k in ("off_meta", "off_vlab", "off_edges", "off_elab", "off_pairs",
                             "off_order", "off_mapoff", "off_kpp", "in_bytes")]
    assert offs == sorted(offs) and all(o % 256 == 0 for o in offs)
    # device work region: results first (one copy back), then queues, pools, scratch
    assert f.b["woff_err"] == 0 < f.b["woff_cost"] < f.b["woff_nev"] < f.b["woff_map"]
    assert f.b["out_bytes"] <= f.b["woff_queue"] < f.b["woff_pool"] < f.b["woff_scratch"]
    scratch = sum(-(-cl["slice_bytes"] * (cl["grid"] // cl["cluster"]) // 256) * 256
                  for cl in f.classes)
    assert f.b["work_bytes"] == f.b["woff_scratch"] + max(scratch, 256)
    assert f.b["woff_pool"] + 8 * (f.b["adj_words"] + f.b["plane_words"]) <= f.b["woff_scratch"]


def test_degree_order_permutation(lib):
    w = W.subset(W.config2(3000), range(3000))
    f = Flat(lib, w, K=16, cost=w.cost, vertex_order=1)
    assert f.rc == 0, f.err
    assert f.b["perm_size"] == f.b["map_total"]
    for p in range(0, w.n_pairs, 7):
        g1 = w.graphs[int(w.pairs[p][0])]
        o = int(f.map_off[p])
        assert f.perm[o:o + g1.n].tolist() == O.degree_order(g1)
    # the relabelled copies are appended after the caller's graphs and the pairs point at them
    assert f.b["n_graphs"] == len(w.graphs) + len(set(int(a) for a in w.pairs[:, 0]))
    staged_pairs = f.region("off_pairs", np.int32, 2 * w.n_pairs).reshape(-1, 2)
    assert (staged_pairs[:, 0] >= len(w.graphs)).all()
    assert np.array_equal(staged_pairs[:, 1], w.pairs[:, 1])


def _bad_batches():
    """(name, make(w) -> (Marshalled, options), expected message). Several invalid entries,
    far apart: the lowest index is reported, graph checks before pair checks before edge
    endpoints."""
    out = []

    def pairs_bad(w):
        pr = w.pairs.copy()
        pr[9000, 1] = 10 ** 6
        pr[7001, 0] = -1
        return F.Marshalled(w.graphs, pr), {}
    out.append(("pair index", pairs_bad, "pair 7001: graph index out of range"))

    def kpp_bad(w):
        kpp = np.full(w.n_pairs, 50, np.int32)
        kpp[11000], kpp[8000] = 0, 101
        return F.Marshalled(w.graphs, w.pairs.copy()), {"k_per_pair": kpp}
    out.append(("per-pair K", kpp_bad, "pair 8000: per-pair K out of range"))

    def elabel_bad(w):
        mm = F.Marshalled(w.graphs, w.pairs.copy())
        mm.el[int(mm.m[:18000].sum())] = 99
        mm.el[int(mm.m[:17000].sum())] = -3
        return mm, {}
    out.append(("edge label", elabel_bad, "graph 17000: edge label out of range"))

    def edge_bad(w):
        mm = F.Marshalled(w.graphs, w.pairs.copy())
        mm.ed[2 * int(mm.m[:20001].sum()) + 1] = 9999
        e0 = 2 * int(mm.m[:15000].sum())
        mm.ed[e0] = mm.ed[e0 + 1]
        return mm, {}
    out.append(("endpoint", edge_bad, "graph 15000: bad edge endpoint or self-loop"))

    def size_bad(w):
        mm = F.Marshalled(w.graphs, w.pairs.copy())
        mm.gs["n"][19000] = 5000
        mm.gs["m"][16000] = -1
        return mm, {}
    out.append(("sizes", size_bad, "graph 16000: m out of range"))

    def pair_and_edge(w):
        mm = F.Marshalled(w.graphs, w.pairs.copy())
        mm.pairs[100, 1] = 10 ** 6
        mm.ed[2 * int(mm.m[:50].sum()) + 1] = 9999
        return mm, {}
    out.append(("pair before endpoint", pair_and_edge, "pair 100: graph index out of range"))
    return out


@pytest.fixture(scope="module")
def big():
    return W.config2(12000)


@pytest.mark.parametrize("case", _bad_batches(), ids=lambda c: c[0])
def test_lowest_index_error(lib, big, case):
    _, make, msg = case
    mm, opts = make(big)
    f = Flat(lib, big, K=100, mm=mm, **opts)
    assert f.rc == F.FASTGED_ERR_INVALID_ARG
    assert f.err == msg
    # the next valid batch goes through
    ok = Flat(lib, W.subset(big, range(100)), K=100)
    assert ok.rc == 0, ok.err


def test_argument_errors(lib):
    w = W.subset(W.config2(50), range(50))
    cases = [({"K": 0}, "K out of range"), ({"K": (1 << 20) + 1}, "K out of range"),
             ({"variant": 2}, "variant must be 0 or 1"),
             ({"hist_window": 1}, "hist_window out of range"),
             ({"block_threads": 64}, "block_threads must be 128, 256 or 512"),
             ({"vertex_order": 3}, "vertex_order must be 0 or 1")]
    for kw, msg in cases:
        K = kw.pop("K", 16)
        f = Flat(lib, w, K=K, **kw)
        assert f.rc == F.FASTGED_ERR_INVALID_ARG and f.err == msg
    f = Flat(lib, w, K=16, cost=(1 << 28, 4, 4, 1, 2, 2))
    assert f.rc == F.FASTGED_ERR_INVALID_ARG and f.err == "pair 0: costs can overflow int32"


def test_empty_batches_and_empty_graphs(lib):
    w = W.config2(10)
    f = Flat(lib, W.Workload("e", w.graphs, np.zeros((0, 2), np.int32), w.cost, 8))
    assert f.rc == 0 and f.b["n_pairs"] == 0 and f.b["n_classes"] == 0
    f = Flat(lib, W.Workload("e", [], np.zeros((0, 2), np.int32), w.cost, 8))
    assert f.rc == 0 and f.b["n_graphs"] == 0
    eg = W.empty_graph()
    ws = W.Workload("e", [eg, eg, w.graphs[0]], np.array([[0, 1], [2, 0], [0, 2]], np.int32),
                    w.cost, 7)
    f = Flat(lib, ws)
    assert f.rc == 0, f.err
    assert f.map_off.tolist() == [0, 0, w.graphs[0].n]
    assert sorted(np.concatenate(f.orders).tolist()) == [0, 1, 2]


def test_resident_teams_capped_by_free_memory(lib):
    w = W.config_wide_beam()
    full = Flat(lib, w, K=100000)
    assert full.rc == 0, full.err
    teams = [cl["grid"] // cl["cluster"] for cl in full.classes]
    need = sum(cl["slice_bytes"] * t for cl, t in zip(full.classes, teams))
    assert need > 0
    lib.fake_set_free_bytes(need // 2)        # half of it may be used: a quarter of the need
    try:
        capped = Flat(lib, w, K=100000)
    finally:
        lib.fake_set_free_bytes(250 << 30)
    assert capped.rc == 0, capped.err
    used = 0
    for cl, t0 in zip(capped.classes, teams):
        t = cl["grid"] // cl["cluster"]
        assert 1 <= t < t0 and cl["grid"] % cl["cluster"] == 0
        used += cl["slice_bytes"] * t
    assert used <= need // 4
    # same pairs, same order: only the number of resident teams changes
    for a, b in zip(full.orders, capped.orders):
        assert np.array_equal(a, b)


def test_pinned_allocation_failure(lib):
    w = W.subset(W.config2(200), range(200))
    # the staging buffer asks for headroom first and falls back to the exact size: one
    # failed allocation is absorbed, two are reported
    lib.probe_reset()
    lib.fake_fail_pinned_alloc(1)
    assert Flat(lib, w, K=16).rc == 0
    lib.probe_reset()
    lib.fake_fail_pinned_alloc(2)
    f = Flat(lib, w, K=16)
    assert f.rc == F.FASTGED_ERR_OOM and "cudaMallocHost" in f.err
    lib.probe_reset()
    lib.fastged_inject_fault(F.FASTGED_INJECT_ALLOC, 1)
    f = Flat(lib, w, K=16)
    assert f.rc == F.FASTGED_ERR_OOM and "injected" in f.err
    f = Flat(lib, w, K=16)
    assert f.rc == 0, f.err


_DIGEST = r"""
import hashlib, sys
sys.path[:0] = [{root!r}, {tests!r}]
from host_probe import load
import test_host_flatten as T
L = load()
f = T.Flat(L, T._mix(), K=64, cost=(2, 4, 4, 1, 2, 2), vertex_order=1)
assert f.rc == 0, f.err
h = hashlib.sha256(f.staging)
for o in f.orders:
    h.update(o.tobytes())
for a in (f.meta, f.map_off, f.perm):
    h.update(a.tobytes())
print(h.hexdigest())
"""


def test_staged_bytes_do_not_depend_on_the_thread_count(lib):
    """The flattening's chunks are sized by the number of host threads; what it stages, its
    classes, their orders, the graph table, the map offsets and the branching permutation
    must be the same for any number (FASTGED_HOST_THREADS; one process per count, since the
    pool is sized once)."""
    here = os.path.dirname(os.path.abspath(__file__))
    code = _DIGEST.format(root=os.path.dirname(here), tests=here)
    digests = set()
    for t in ("1", "3", "16"):
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           timeout=600, env=dict(os.environ, FASTGED_HOST_THREADS=t))
        assert r.returncode == 0, r.stderr[-2000:]
        digests.add(r.stdout.strip().splitlines()[-1])
    assert len(digests) == 1

