"""ctypes front end for the plain C oracle (fastged_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check, the benchmark's CPU baseline and the
oracle's own accuracy report (accuracy_report.py) are the only callers. Nothing on the product
path imports this module. The oracle shares no
code with the CUDA path; its only common input is the graph description produced by the
seeded workload generators (which hold none of the method's arithmetic).

Functions follow the paper (Dabah & Herten):
  full_cost     cost of the edit path a complete vertex map induces (Sec. 2.2-2.4)
  brute_ged     exact GED by enumerating every injective partial vertex map (Sec. 2.2)
  brute_square  exact GED by enumerating bijections of the (n1+n2)-square extended sets
  kbest         the K-Best search (Algorithm 1, Sec. 4.1-4.2, insertions at the leaf)
  edit_path     the edit operations a complete vertex map induces (Sec. 2.3: vertex
                substitution / deletion / insertion, and the implied edge substitution /
                deletion / insertion, incident edges of deleted or inserted vertices included)
  degree_order  an optional branching order of the source vertices (descending degree, ties
                by index); the paper branches v_0..v_{n1-1} in index order, so this is an
                extension: kbest(order=1) runs Algorithm 1 on the source graph relabelled in
                that order and returns the map in the original vertex ids
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from types import SimpleNamespace
from typing import List, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fastged_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIB = None


class _OgoGraph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("alpha", ctypes.POINTER(ctypes.c_int)),
                ("adj", ctypes.POINTER(ctypes.c_ubyte))]


def lib_path() -> str:
    return os.path.join(_BUILD, f"liboracle_{platform.machine()}.so")


def compile_c(src: str, out: str) -> str:
    """Compile one C file to a shared library (plain C99, -O2, no target-specific flags)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-shared", "-fPIC",
                           src, "-o", tmp])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle (once; again only when the source is newer)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    return compile_c(_SRC, out)


def _bind(path: str):
    lib = ctypes.CDLL(path)
    G = ctypes.POINTER(_OgoGraph)
    ip = ctypes.POINTER(ctypes.c_int)
    llp = ctypes.POINTER(ctypes.c_longlong)
    lib.ogo_full_cost.argtypes = [G, G, ip, ip]
    lib.ogo_full_cost.restype = ctypes.c_longlong
    lib.ogo_brute_ged.argtypes = [G, G, ip, ip, llp]
    lib.ogo_brute_ged.restype = ctypes.c_longlong
    lib.ogo_brute_square.argtypes = [G, G, ip]
    lib.ogo_brute_square.restype = ctypes.c_longlong
    lib.ogo_kbest.argtypes = [G, G, ip, ctypes.c_int, ctypes.c_int, llp, ip, llp]
    lib.ogo_kbest.restype = ctypes.c_int
    lib.ogo_kbest_leaves.argtypes = [G, G, ip, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip,
                                     llp, ip]
    lib.ogo_kbest_leaves.restype = ctypes.c_int
    return lib


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = _bind(build())
    return _LIB


class _Dense:
    """Dense byte-matrix form of one graph, kept alive while the C call runs."""

    def __init__(self, g):
        n = int(g.n)
        self.alpha = np.ascontiguousarray(np.asarray(g.vlabel, dtype=np.int32).reshape(n))
        adj = np.zeros((n, n), dtype=np.uint8)
        e = np.asarray(g.edges, dtype=np.int64).reshape(-1, 2)
        if e.shape[0]:
            lab = (np.zeros(e.shape[0], dtype=np.int64) if g.elabel is None
                   else np.asarray(g.elabel, dtype=np.int64))
            if lab.max(initial=0) > 254 or lab.min(initial=0) < 0:
                raise ValueError("oracle stores edge labels 0..254")
            adj[e[:, 0], e[:, 1]] = lab + 1
            adj[e[:, 1], e[:, 0]] = lab + 1
        self.adj = np.ascontiguousarray(adj.reshape(-1))
        self.st = _OgoGraph(n, self.alpha.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            self.adj.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))


def _cost(cost: Sequence[int]):
    arr = (ctypes.c_int * 6)(*[int(x) for x in cost])
    return arr


def full_cost(g1, g2, cost, mapping, lib=None) -> int:
    d1, d2 = _Dense(g1), _Dense(g2)
    m = np.ascontiguousarray(np.asarray(mapping, dtype=np.int32).reshape(-1))
    if m.shape[0] != g1.n:
        raise ValueError("mapping length must equal n1")
    v = (lib or _lib()).ogo_full_cost(ctypes.byref(d1.st), ctypes.byref(d2.st), _cost(cost),
                             m.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if v < 0:
        raise ValueError("not an injective partial map")
    return int(v)


def brute_ged(g1, g2, cost, lib=None) -> Tuple[int, np.ndarray, int]:
    """Exact GED over all injective partial maps; returns (ged, one optimal map, #maps)."""
    d1, d2 = _Dense(g1), _Dense(g2)
    out = np.zeros(max(g1.n, 1), dtype=np.int32)
    cnt = ctypes.c_longlong(0)
    v = (lib or _lib()).ogo_brute_ged(ctypes.byref(d1.st), ctypes.byref(d2.st), _cost(cost),
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             ctypes.byref(cnt))
    if v < 0:
        raise ValueError("brute_ged supports n <= 10")
    return int(v), out[:g1.n].copy(), int(cnt.value)


def brute_square(g1, g2, cost, lib=None) -> int:
    """Exact GED over bijections of the padded (n1+n2) square form."""
    d1, d2 = _Dense(g1), _Dense(g2)
    v = (lib or _lib()).ogo_brute_square(ctypes.byref(d1.st), ctypes.byref(d2.st), _cost(cost))
    if v < 0:
        raise ValueError("brute_square supports n1 + n2 <= 10")
    return int(v)


def degree_order(g) -> List[int]:
    """Vertices of g by descending degree (number of incident edges), ties by index."""
    deg = [0] * int(g.n)
    for u, v in np.asarray(g.edges, dtype=np.int64).reshape(-1, 2):
        deg[int(u)] += 1
        deg[int(v)] += 1
    return sorted(range(int(g.n)), key=lambda v: (-deg[v], v))


def relabel(g, perm: Sequence[int]):
    """g with vertex k renamed so that new vertex k is old vertex perm[k]."""
    inv = {int(old): new for new, old in enumerate(perm)}
    e = np.asarray(g.edges, dtype=np.int64).reshape(-1, 2)
    edges = np.array([[inv[int(u)], inv[int(v)]] for u, v in e], dtype=np.int32).reshape(-1, 2)
    lab = np.asarray(g.vlabel, dtype=np.int32)
    vlabel = np.array([int(lab[old]) for old in perm], dtype=np.int32)
    return SimpleNamespace(n=int(g.n), vlabel=vlabel, edges=edges,
                           elabel=None if g.elabel is None else np.asarray(g.elabel))


def kbest(g1, g2, cost, K: int, variant: int = 0, lib=None, order: int = 0
          ) -> Tuple[int, np.ndarray, int]:
    """K-Best search (Algorithm 1). Returns (cost, map with -1 = deleted, n_evals).
    order = 1 branches the source vertices in degree_order (the map still uses g1's ids)."""
    if order == 1:
        perm = degree_order(g1)
        c, m, nev = kbest(relabel(g1, perm), g2, cost, K, variant, lib)
        out = np.zeros(int(g1.n), dtype=np.int32)
        for k, old in enumerate(perm):
            out[old] = m[k]
        return c, out, nev
    d1, d2 = _Dense(g1), _Dense(g2)
    out_cost = ctypes.c_longlong(0)
    out_map = np.zeros(max(g1.n, 1), dtype=np.int32)
    nev = ctypes.c_longlong(0)
    rc = (lib or _lib()).ogo_kbest(ctypes.byref(d1.st), ctypes.byref(d2.st), _cost(cost), int(K),
                          int(variant), ctypes.byref(out_cost),
                          out_map.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          ctypes.byref(nev))
    if rc != 0:
        raise RuntimeError("oracle kbest failed")
    return int(out_cost.value), out_map[:g1.n].copy(), int(nev.value)


def kbest_leaves(g1, g2, cost, K: int, variant: int = 0, lib=None
                 ) -> Tuple[np.ndarray, np.ndarray]:
    """The final kept List (before the leaf insertions) in slot order: (PED[L], map[L, n1])."""
    d1, d2 = _Dense(g1), _Dense(g2)
    cap = K * (g2.n + 1) if variant == 1 else K
    ped = np.zeros(max(cap, 1), dtype=np.int64)
    mp = np.zeros(max(cap * g1.n, 1), dtype=np.int32)
    L = ctypes.c_int(0)
    rc = (lib or _lib()).ogo_kbest_leaves(ctypes.byref(d1.st), ctypes.byref(d2.st),
                                          _cost(cost), int(K), int(variant), int(cap),
                                          ctypes.byref(L),
                                          ped.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                          mp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise RuntimeError("oracle kbest_leaves failed")
    n = min(L.value, cap)
    return ped[:n].copy(), mp[:n * g1.n].reshape(n, g1.n).copy()


def kbest_workload(w, idx=None, K=None, variant: int = 0, threads: int = 1, order: int = 0
                   ) -> List[Tuple[int, np.ndarray, int]]:
    """Run kbest on pairs idx of a Workload (all pairs by default). With threads > 1 the
    pairs run concurrently on host threads (ctypes releases the GIL during the call)."""
    if idx is None:
        idx = range(w.n_pairs)
    idx = list(idx)

    def one(p):
        a, b = int(w.pairs[p][0]), int(w.pairs[p][1])
        k = K if K is not None else (int(w.k_per_pair[p]) if w.k_per_pair is not None
                                     else w.K)
        return kbest(w.graphs[a], w.graphs[b], w.cost, k, variant, order=order)

    if threads <= 1:
        return [one(p) for p in idx]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, idx))


# operation kinds of edit_path, in the order the path lists its groups
OP_VINS, OP_VSUB, OP_EDEL, OP_ESUB, OP_EINS, OP_VDEL = range(6)


def edit_path(g1, g2, cost, mapping) -> List[Tuple[int, int, int, int, int, int]]:
    """Edit operations from g1 to g2 under the complete vertex map `mapping` (g2 image of each
    g1 vertex, -1 = deleted), as tuples (kind, cost, g1_u, g1_v, g2_u, g2_v) with -1 for an
    unused field. Only operations that change something are listed: a substitution that
    keeps the vertex (or edge) label costs nothing and is no edit. Groups, each by
    increasing index (edges in input order): vertex insertions, vertex substitutions, edge
    deletions, edge substitutions, edge insertions, vertex deletions.

    Sec. 2.3: v -> u substitutes, v -> eps deletes, eps -> u inserts; for two edited g1
    vertices the edge between them is substituted when both graphs have it, deleted when only
    g1 has it, inserted when only g2 has it; a deleted vertex takes its edges with it and an
    inserted vertex brings its edges. Costs per operation as in Sec. 2.4 (six constants)."""
    c_vsub, c_vdel, c_vins, c_esub, c_edel, c_eins = (int(x) for x in cost)
    phi = [int(x) for x in mapping]
    n1, n2 = int(g1.n), int(g2.n)
    lab1 = [int(x) for x in g1.vlabel]
    lab2 = [int(x) for x in g2.vlabel]
    e1 = [tuple(int(a) for a in e) for e in np.asarray(g1.edges).reshape(-1, 2)]
    e2 = [tuple(int(a) for a in e) for e in np.asarray(g2.edges).reshape(-1, 2)]
    el1 = [0] * len(e1) if g1.elabel is None else [int(x) for x in g1.elabel]
    el2 = [0] * len(e2) if g2.elabel is None else [int(x) for x in g2.elabel]
    g2_edge = {frozenset(e): el2[k] for k, e in enumerate(e2)}
    g1_edge = {frozenset(e) for e in e1}
    pre = {x: v for v, x in enumerate(phi) if x >= 0}     # g2 vertex -> its g1 preimage
    ops = []
    for x in range(n2):                                  # eps -> u
        if x not in pre:
            ops.append((OP_VINS, c_vins, -1, -1, x, -1))
    for v in range(n1):                                  # v -> u with a label change
        if phi[v] >= 0 and lab1[v] != lab2[phi[v]]:
            ops.append((OP_VSUB, c_vsub, v, -1, phi[v], -1))
    for (u, v) in e1:                                    # e1 -> eps
        if phi[u] < 0 or phi[v] < 0 or frozenset((phi[u], phi[v])) not in g2_edge:
            ops.append((OP_EDEL, c_edel, u, v, -1, -1))
    for k, (u, v) in enumerate(e1):                      # e1 -> e2 with a label change
        if phi[u] >= 0 and phi[v] >= 0:
            l2 = g2_edge.get(frozenset((phi[u], phi[v])))
            if l2 is not None and l2 != el1[k]:
                ops.append((OP_ESUB, c_esub, u, v, phi[u], phi[v]))
    for (x, y) in e2:                                    # eps -> e2
        if x not in pre or y not in pre or frozenset((pre[x], pre[y])) not in g1_edge:
            ops.append((OP_EINS, c_eins, -1, -1, x, y))
    for v in range(n1):                                  # v -> eps
        if phi[v] < 0:
            ops.append((OP_VDEL, c_vdel, v, -1, -1, -1))
    return ops
