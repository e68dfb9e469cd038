"""ctypes front end for the plain C oracle (fastged_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU baseline are
the only callers. Nothing on the product path imports this module. The oracle shares no
code with the CUDA path; its only common input is the graph description produced by the
seeded workload generators (which hold none of the method's arithmetic).

Functions follow the paper (Dabah & Herten):
  full_cost     cost of the edit path a complete vertex map induces (Sec. 2.2-2.4)
  brute_ged     exact GED by enumerating every injective partial vertex map (Sec. 2.2)
  brute_square  exact GED by enumerating bijections of the (n1+n2)-square extended sets
  kbest         the K-Best search (Algorithm 1, Sec. 4.1-4.2, insertions at the leaf)
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
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


def kbest(g1, g2, cost, K: int, variant: int = 0, lib=None) -> Tuple[int, np.ndarray, int]:
    """K-Best search (Algorithm 1). Returns (cost, map with -1 = deleted, n_evals)."""
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


def kbest_workload(w, idx=None, K=None, variant: int = 0, threads: int = 1
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
        return kbest(w.graphs[a], w.graphs[b], w.cost, k, variant)

    if threads <= 1:
        return [one(p) for p in idx]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, idx))
