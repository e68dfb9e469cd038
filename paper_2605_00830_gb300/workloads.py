"""Seeded synthetic workloads for the K-Best graph edit distance path.

This module only *generates inputs*: graphs, pair lists, cost models and beam widths K.
It holds none of the method's arithmetic, so both the CPU oracle (``oracle/``) and the CUDA
path's tests and bench draw their inputs from here without sharing any GED code.

Randomness is a counter-based splitmix64 stream (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): value(key, i) = mix64(key + (i+1)*phi),
phi = 0x9E3779B97F4A7C15. It is reimplemented here in numpy uint64 arithmetic so the same
seed gives the same graphs on every machine and numpy version.

Workload shapes follow the paper's experimental inputs (Sec. 5): small random graphs
(Table 1, n = 10), molecule-like graphs standing in for MUTA / Mutagenicity, dense random
graphs, and large sparse graphs like those of Fig. 4d. No dataset record is reproduced;
every graph is drawn from the generators below. Cost settings: unit costs, and the paper's
"setting 1" (vertex sub 2, vertex ins/del 4, edge sub 1, edge ins/del 2; Sec. 5).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

_PHI = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# cost model order used throughout: (v_sub, v_del, v_ins, e_sub, e_del, e_ins)
UNIT_COSTS = (1, 1, 1, 1, 1, 1)
SETTING1_COSTS = (2, 4, 4, 1, 2, 2)   # the paper's default costs (Sec. 5, "Setting 1")
SETTING2_COSTS = (4, 12, 12, 1, 10, 10)  # the paper's "Setting 2" (Sec. 5)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _fold(*parts: int) -> np.uint64:
    key = np.array([0x6A09E667F3BCC908], dtype=np.uint64)
    with np.errstate(over="ignore"):
        for p in parts:
            key = _mix64(key + np.array([p & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) * _PHI
                         + _PHI)
    return key[0]


class Stream:
    """A counter-based random stream identified by a tuple of integers."""

    def __init__(self, *key_parts: int):
        self.key = _fold(*key_parts)
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.ctr + 1, self.ctr + n + 1, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return _mix64(self.key + idx * _PHI)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def randint(self, lo: int, hi: int, n: int) -> np.ndarray:
        """n integers uniform on [lo, hi] (inclusive)."""
        return lo + np.floor(self.uniform(n) * (hi - lo + 1)).astype(np.int64)


@dataclass
class Graph:
    """Simple undirected labelled graph (no loops, no multi-edges).

    edges is an (m, 2) int32 array with edges[k, 0] < edges[k, 1]; elabel is an int32
    array of length m, or None for unlabelled edges.
    """
    n: int
    vlabel: np.ndarray
    edges: np.ndarray
    elabel: Optional[np.ndarray] = None

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])


@dataclass
class Workload:
    name: str
    graphs: List[Graph]
    pairs: np.ndarray              # (n_pairs, 2) int32: (source g1, target g2) graph indices
    cost: Tuple[int, int, int, int, int, int]
    K: int
    # serving only: arrival time (s) and K per request
    arrival: Optional[np.ndarray] = None
    k_per_pair: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def n_pairs(self) -> int:
        return int(self.pairs.shape[0])


def _make_graph(n: int, vlabel, edge_set, elabel_of=None) -> Graph:
    if edge_set:
        e = np.array(sorted(edge_set), dtype=np.int32).reshape(-1, 2)
    else:
        e = np.zeros((0, 2), dtype=np.int32)
    el = None
    if elabel_of is not None:
        el = np.array([elabel_of[(int(a), int(b))] for a, b in e], dtype=np.int32)
    return Graph(n=int(n), vlabel=np.asarray(vlabel, dtype=np.int32), edges=e, elabel=el)


def erdos_renyi(st: Stream, n: int, p: float, n_labels: int) -> Graph:
    """G(n, p): every unordered pair is an edge with probability p."""
    lab = st.randint(0, n_labels - 1, n)
    iu = np.triu_indices(n, 1)
    coin = st.uniform(len(iu[0])) < p
    e = np.stack([iu[0][coin], iu[1][coin]], axis=1).astype(np.int32)
    return Graph(n=n, vlabel=lab.astype(np.int32), edges=e, elabel=None)


_ZIPF10 = np.array([k ** -1.2 for k in range(1, 11)], dtype=np.float64)
_ZIPF10_CDF = np.cumsum(_ZIPF10 / _ZIPF10.sum())
_ELAB_CDF = np.array([0.70, 0.95, 1.0])


def molecule_like(st: Stream, n: int) -> Graph:
    """Random recursive spanning tree plus 0-3 extra ring-closing edges.

    Vertex t >= 1 attaches to a uniformly chosen earlier vertex; then U{0..3} extra edges
    join random non-adjacent pairs. Vertex labels are Zipf(1.2) over 10 values, edge labels
    0/1/2 with probabilities 70/25/5 %.
    """
    lab = np.searchsorted(_ZIPF10_CDF, st.uniform(n), side="right")
    lab = np.minimum(lab, 9)
    edges = set()
    if n > 1:
        par = np.floor(st.uniform(n - 1) * np.arange(1, n)).astype(np.int64)
        for t in range(1, n):
            a, b = int(par[t - 1]), t
            edges.add((min(a, b), max(a, b)))
    n_extra = int(st.randint(0, 3, 1)[0])
    tries = st.randint(0, max(n - 1, 0), 2 * 32 * max(n_extra, 1))
    added, k = 0, 0
    while added < n_extra and k + 1 < len(tries):
        a, b = int(tries[k]), int(tries[k + 1])
        k += 2
        if a == b:
            continue
        e = (min(a, b), max(a, b))
        if e in edges:
            continue
        edges.add(e)
        added += 1
    e_sorted = sorted(edges)
    el_draw = np.searchsorted(_ELAB_CDF, st.uniform(len(e_sorted)), side="right")
    el_draw = np.minimum(el_draw, 2)
    elabel_of = {e: int(l) for e, l in zip(e_sorted, el_draw)}
    return _make_graph(n, lab, e_sorted, elabel_of)


def barabasi_albert(st: Stream, n: int, m: int, n_labels: int) -> Graph:
    """Preferential attachment: start from a clique on m+1 vertices; every later vertex
    joins m distinct earlier vertices drawn with probability proportional to degree."""
    lab = st.randint(0, n_labels - 1, n)
    edges = set()
    targets: List[int] = []
    m0 = min(n, m + 1)
    for a in range(m0):
        for b in range(a + 1, m0):
            edges.add((a, b))
            targets += [a, b]
    draws = st.uniform(max(1, (n - m0) * m * 8))
    d = 0
    for t in range(m0, n):
        chosen = set()
        while len(chosen) < m and d < len(draws):
            chosen.add(targets[int(draws[d] * len(targets))])
            d += 1
        for c in chosen:
            edges.add((c, t))
            targets += [c, t]
    return _make_graph(n, lab, edges)


def perturb(st: Stream, g: Graph, rate: float, n_labels: int) -> Graph:
    """Apply round(rate*(n+m)) random edits (vertex insert / delete / relabel, edge
    insert / delete, chosen uniformly), then shuffle the vertex ids."""
    lab = list(int(x) for x in g.vlabel)
    alive = list(range(g.n))
    adj = {v: set() for v in range(g.n)}
    for a, b in g.edges:
        adj[int(a)].add(int(b))
        adj[int(b)].add(int(a))
    nxt = g.n
    n_ops = int(round(rate * (g.n + g.m)))
    ops = st.randint(0, 4, n_ops)
    pool = st.uniform(max(1, n_ops * 16))
    q = 0

    def draw(k: int) -> int:
        nonlocal q
        v = int(pool[q % len(pool)] * k)
        q += 1
        return min(v, k - 1)

    for op in ops:
        op = int(op)
        if op == 0:  # vertex insertion, wired to 3 random existing vertices
            v = nxt
            nxt += 1
            lab.append(draw(n_labels))
            adj[v] = set()
            for _ in range(3):
                if alive:
                    u = alive[draw(len(alive))]
                    adj[v].add(u)
                    adj[u].add(v)
            alive.append(v)
        elif op == 1 and len(alive) > 2:  # vertex deletion with its edges
            v = alive.pop(draw(len(alive)))
            for u in adj[v]:
                adj[u].discard(v)
            adj[v] = set()
        elif op == 2 and alive:  # relabel
            v = alive[draw(len(alive))]
            lab[v] = draw(n_labels)
        elif op == 3 and len(alive) > 1:  # edge insertion
            for _ in range(8):
                a, b = alive[draw(len(alive))], alive[draw(len(alive))]
                if a != b and b not in adj[a]:
                    adj[a].add(b)
                    adj[b].add(a)
                    break
        elif op == 4:  # edge deletion
            cand = [v for v in alive if adj[v]]
            if cand:
                a = cand[draw(len(cand))]
                nb = sorted(adj[a])
                b = nb[draw(len(nb))]
                adj[a].discard(b)
                adj[b].discard(a)
    n2 = len(alive)
    perm = np.argsort(st.uniform(n2), kind="stable")   # new id of alive[k] is perm[k]
    new_id = {alive[k]: int(perm[k]) for k in range(n2)}
    vl = np.zeros(n2, dtype=np.int32)
    for old, new in new_id.items():
        vl[new] = lab[old]
    edges = set()
    for a in alive:
        for b in adj[a]:
            x, y = new_id[a], new_id[b]
            if x < y:
                edges.add((x, y))
    return _make_graph(n2, vl, edges)


# ----------------------------------------------------------------------------------------
# The five workload configurations
# ----------------------------------------------------------------------------------------

def config1(n_pairs: int = 200, seed: int = 1) -> Workload:
    """Tiny plain method: ER graphs with 5-8 vertices, p = 0.35, 4 vertex labels,
    unlabelled edges, unit costs, K = 16."""
    graphs = []
    for p in range(n_pairs):
        for role in (0, 1):
            st = Stream(seed, 1, p, role)
            n = int(st.randint(5, 8, 1)[0])
            graphs.append(erdos_renyi(st, n, 0.35, 4))
    pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
    return Workload("er_n5-8_p0.35_K16", graphs, pairs, UNIT_COSTS, 16)


def config2(n_pairs: int = 20000, seed: int = 2) -> Workload:
    """Batched molecule-like: 10-40 vertices, tree + 0-3 ring edges, Zipf labels,
    3 edge labels, the paper's setting-1 costs, K = 100."""
    graphs = []
    for p in range(n_pairs):
        for role in (0, 1):
            st = Stream(seed, 2, p, role)
            n = int(st.randint(10, 40, 1)[0])
            graphs.append(molecule_like(st, n))
    pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
    return Workload("molecule_n10-40_K100", graphs, pairs, SETTING1_COSTS, 100)


def config3(n_pairs: int = 4096, seed: int = 3) -> Workload:
    """Batched dense mix: ER with 50-200 vertices, density U[0.05, 0.5] per graph,
    8 vertex labels, unlabelled edges, unit costs, K = 256."""
    graphs = []
    for p in range(n_pairs):
        for role in (0, 1):
            st = Stream(seed, 3, p, role)
            n = int(st.randint(50, 200, 1)[0])
            dens = 0.05 + 0.45 * float(st.uniform(1)[0])
            graphs.append(erdos_renyi(st, n, dens, 8))
    pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
    return Workload("er_n50-200_d0.05-0.5_K256", graphs, pairs, UNIT_COSTS, 256)


def config4(n_pairs: int = 64, seed: int = 4, n_range=(500, 1000)) -> Workload:
    """Large sparse: BA (m = 3) with 500-1000 vertices, 16 vertex labels; g2 = g1 after
    2-10 % random vertex/edge edits and an id shuffle; unit costs, K = 1024."""
    graphs = []
    for p in range(n_pairs):
        st = Stream(seed, 4, p)
        n = int(st.randint(n_range[0], n_range[1], 1)[0])
        g1 = barabasi_albert(st, n, 3, 16)
        rate = 0.02 + 0.08 * float(st.uniform(1)[0])
        g2 = perturb(st, g1, rate, 16)
        graphs += [g1, g2]
    pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
    return Workload("ba_m3_n500-1000_K1024", graphs, pairs, UNIT_COSTS, 1024)


def config_wide_beam(n_pairs: int = 16, seed: int = 6, K: int = 100000) -> Workload:
    """Wide-beam regime (the paper's K sweep up to 10^5-10^6 on ~20-vertex graphs):
    molecule-like graphs with 18-22 vertices, the paper's setting-1 costs, K = 100,000."""
    graphs = []
    for p in range(n_pairs):
        for role in (0, 1):
            st = Stream(seed, 6, p, role)
            graphs.append(molecule_like(st, int(st.randint(18, 22, 1)[0])))
    pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
    return Workload(f"molecule_n18-22_K{K}", graphs, pairs, SETTING1_COSTS, K)


def config_size_sweep(n_pairs: int = 1, seed: int = 7, n: int = 950, K: int = 5000,
                      density: float = 0.4) -> Workload:
    """Scaling with graph size (the paper's Fig. 4d setting): pairs of random G(n, 0.4)
    graphs with n vertices each, 4 uniform vertex labels, unlabelled edges, the paper's
    setting-1 costs, K = 5,000."""
    graphs = []
    for p in range(n_pairs):
        for role in (0, 1):
            st = Stream(seed, 7, n, p, role)
            graphs.append(erdos_renyi(st, n, density, 4))
    pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
    return Workload(f"er_n{n}_d{density}_K{K}", graphs, pairs, SETTING1_COSTS, K)


def config5(duration_s: float = 60.0, rate: float = 5000.0, seed: int = 5,
            max_requests: Optional[int] = None) -> Workload:
    """Serving stream: Poisson arrivals at `rate` req/s for `duration_s`; 70 % molecule-like
    (10-40), 25 % dense ER (50-200), 5 % BA (500-1000) pairs; K uniform in {32, 128, 512}.
    One cost model serves the whole stream: the paper's setting 1."""
    st = Stream(seed, 5)
    n_est = int(duration_s * rate * 1.2 + 100)
    gaps = -np.log1p(-st.uniform(n_est)) / rate
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    if max_requests is not None:
        t = t[:max_requests]
    n = len(t)
    kind = st.uniform(n)
    kchoice = st.randint(0, 2, n)
    ks = np.array([32, 128, 512], dtype=np.int32)[kchoice]
    graphs = []
    shape = []
    for r in range(n):
        s = Stream(seed, 5, 1, r)
        if kind[r] < 0.70:
            shape.append(0)
            for _ in (0, 1):
                graphs.append(molecule_like(s, int(s.randint(10, 40, 1)[0])))
        elif kind[r] < 0.95:
            shape.append(1)
            for _ in (0, 1):
                nn = int(s.randint(50, 200, 1)[0])
                graphs.append(erdos_renyi(s, nn, 0.05 + 0.45 * float(s.uniform(1)[0]), 8))
        else:
            shape.append(2)
            g1 = barabasi_albert(s, int(s.randint(500, 1000, 1)[0]), 3, 16)
            graphs += [g1, perturb(s, g1, 0.02 + 0.08 * float(s.uniform(1)[0]), 16)]
    pairs = np.arange(2 * n, dtype=np.int32).reshape(-1, 2)
    return Workload("serve_mix_poisson", graphs, pairs, SETTING1_COSTS, 512, arrival=t,
                    k_per_pair=ks, meta={"shape": np.array(shape, dtype=np.int32)})


def random_small(st: Stream, n_lo: int, n_hi: int, p: float, n_vlab: int,
                 n_elab: int = 0) -> Graph:
    """Small ER graph with optional edge labels, for pins and edge cases."""
    n = int(st.randint(n_lo, n_hi, 1)[0])
    g = erdos_renyi(st, n, p, n_vlab)
    if n_elab > 0:
        g.elabel = st.randint(0, n_elab - 1, g.m).astype(np.int32)
    return g


def empty_graph() -> Graph:
    return Graph(n=0, vlabel=np.zeros(0, dtype=np.int32), edges=np.zeros((0, 2), np.int32))


def concat(workloads: List[Workload], name: str = "concat") -> Workload:
    """Join several workloads that share one cost model and K into one pair list."""
    graphs: List[Graph] = []
    pairs = []
    for w in workloads:
        base = len(graphs)
        graphs += w.graphs
        pairs.append(w.pairs + base)
    return Workload(name, graphs, np.concatenate(pairs).astype(np.int32), workloads[0].cost,
                    workloads[0].K)


def subset(w: Workload, idx) -> Workload:
    """The pairs idx of w, with only the graphs they reference."""
    idx = np.asarray(idx, dtype=np.int64)
    graphs, pairs, remap = [], [], {}
    for p in idx:
        row = []
        for g in w.pairs[p]:
            g = int(g)
            if g not in remap:
                remap[g] = len(graphs)
                graphs.append(w.graphs[g])
            row.append(remap[g])
        pairs.append(row)
    pairs = np.array(pairs, dtype=np.int32).reshape(-1, 2)
    return Workload(w.name + "_subset", graphs, pairs, w.cost, w.K,
                    k_per_pair=None if w.k_per_pair is None else w.k_per_pair[idx])
