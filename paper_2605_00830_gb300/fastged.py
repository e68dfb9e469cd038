"""Thin Python binding of the libfastged C ABI (include/fastged.h).

Only argument marshalling lives here: every step of the K-Best path runs in the library's
sm_103a kernels. The binding loads the in-tree library and fails loudly when it is missing;
there is no CPU fallback. Names follow the C ABI (fastged_create, fastged_batch, ...).

Graph batches are marshalled without Python loops: the graphs of a workload are
concatenated into three flat arrays and the array of fastged_graph structs is filled with
numpy from base addresses and offsets.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

FASTGED_OK = 0
FASTGED_ERR_INVALID_ARG = -1
FASTGED_ERR_OOM = -2
FASTGED_ERR_CUDA = -3
FASTGED_ERR_TIMEOUT = -4
FASTGED_ERR_BUSY = -5
FASTGED_ERR_STOPPED = -6
FASTGED_ERR_CANCELLED = -7
FASTGED_FORM_BATCHED = 0
FASTGED_FORM_PLAIN = 1
FASTGED_INJECT_ALLOC = 0
FASTGED_INJECT_LAUNCH = 1
FASTGED_INJECT_ADMISSION = 2
FASTGED_ORDER_INDEX = 0
FASTGED_ORDER_DEGREE = 1
FASTGED_TEAM_AUTO = 0
FASTGED_TEAM_CTA = 1

EXPORTED = ["fastged_version", "fastged_last_error", "fastged_create", "fastged_destroy",
            "fastged_batch", "fastged_batch_ex", "fastged_plan_create", "fastged_plan_run",
            "fastged_plan_read", "fastged_plan_info", "fastged_plan_kernel_ms",
            "fastged_plan_destroy", "fastged_measure_int_peak", "fastged_batch_noalloc",
            "fastged_serve_start", "fastged_serve_submit", "fastged_serve_poll",
            "fastged_serve_get_stats", "fastged_serve_cancel", "fastged_serve_stop",
            "fastged_serve_destroy",
            "fastged_autotune_entries", "fastged_autotune_clear", "fastged_edit_path",
            "fastged_apply_edit_ops", "fastged_cross", "fastged_set_timeout",
            "fastged_inject_fault"]


class FastGEDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fastged error {code}: {msg}")
        self.code = code


class CostModel(ctypes.Structure):
    _fields_ = [("v_sub", ctypes.c_int32), ("v_del", ctypes.c_int32), ("v_ins", ctypes.c_int32),
                ("e_sub", ctypes.c_int32), ("e_del", ctypes.c_int32), ("e_ins", ctypes.c_int32)]


class GraphC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("vlabel", ctypes.c_void_p), ("m", ctypes.c_int32),
                ("edges", ctypes.c_void_p), ("elabel", ctypes.c_void_p)]


class PairList(ctypes.Structure):
    _fields_ = [("n_graphs", ctypes.c_int32), ("graphs", ctypes.c_void_p),
                ("n_pairs", ctypes.c_int32), ("pairs", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("k_per_pair", ctypes.c_void_p), ("hist_window", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("use_cuda_graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("vertex_order", ctypes.c_int32),
                ("team", ctypes.c_int32), ("max_sms", ctypes.c_int32),
                ("cluster", ctypes.c_int32)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int32), ("n_classes", ctypes.c_int32),
                ("launches_per_run", ctypes.c_int32), ("graph_replay", ctypes.c_int32),
                ("input_bytes", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("output_bytes", ctypes.c_int64), ("block_threads", ctypes.c_int32 * 8),
                ("grid", ctypes.c_int32 * 8), ("words", ctypes.c_int32 * 8),
                ("smem_bytes", ctypes.c_int32 * 8)]


class DeviceBatch(ctypes.Structure):
    """fastged_device_batch: device arrays of a flattened batch plus host bounds."""
    _fields_ = [("n_graphs", ctypes.c_int32), ("n_pairs", ctypes.c_int32),
                ("max_n", ctypes.c_int32), ("max_m", ctypes.c_int32),
                ("max_elabel", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("total_vertices", ctypes.c_int64), ("total_edges", ctypes.c_int64),
                ("map_len", ctypes.c_int64),
                ("graph_n", ctypes.c_void_p), ("graph_m", ctypes.c_void_p),
                ("vlabel_off", ctypes.c_void_p), ("edge_off", ctypes.c_void_p),
                ("vlabel", ctypes.c_void_p), ("edges", ctypes.c_void_p),
                ("elabel", ctypes.c_void_p), ("pairs", ctypes.c_void_p),
                ("map_off", ctypes.c_void_p)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("max_batch_pairs", ctypes.c_int32),
                ("min_batch_pairs", ctypes.c_int32), ("max_pending", ctypes.c_int32),
                ("max_wait_us", ctypes.c_int32), ("max_retries", ctypes.c_int32),
                ("hbm_reserve_bytes", ctypes.c_int64)]


class ServeResult(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("cost", ctypes.c_int32),
                ("n1", ctypes.c_int32), ("pad", ctypes.c_int32), ("map_offset", ctypes.c_int64),
                ("n_evals", ctypes.c_int64), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "batches",
                                              "batched_pairs", "rejected_busy",
                                              "admission_waits", "pending", "lanes_busy")]


_GRAPH_DTYPE = np.dtype({"names": ["n", "vlabel", "m", "edges", "elabel"],
                         "formats": ["<i4", "<u8", "<i4", "<u8", "<u8"],
                         "offsets": [0, 8, 16, 24, 32], "itemsize": 40})
assert ctypes.sizeof(GraphC) == 40 and ctypes.sizeof(Options) == 48

_LIB = None


def load(path: Optional[str] = None, build_if_missing: bool = True):
    """Load libfastged (building it in-tree first when asked). Raises when it is absent."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    # FASTGED_LIBRARY names another build of the library (the bounds-checked one, say)
    p = path or os.environ.get("FASTGED_LIBRARY") or _build.lib_path()
    if not os.path.exists(p):
        if not build_if_missing:
            raise RuntimeError(f"libfastged not built ({p}); run __graft_entry__.build()")
        p = _build.build()
    lib = ctypes.CDLL(p)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.fastged_version.restype = ctypes.c_int
    lib.fastged_last_error.argtypes = [vp]
    lib.fastged_last_error.restype = ctypes.c_char_p
    lib.fastged_create.argtypes = [ctypes.POINTER(CostModel), ctypes.POINTER(vp)]
    lib.fastged_destroy.argtypes = [vp]
    lib.fastged_destroy.restype = None
    lib.fastged_batch.argtypes = [vp, ctypes.POINTER(PairList), i32, vp, vp]
    lib.fastged_batch_ex.argtypes = [vp, ctypes.POINTER(PairList), i32, ctypes.POINTER(Options),
                                     vp, vp, vp]
    lib.fastged_plan_create.argtypes = [vp, ctypes.POINTER(PairList), i32,
                                        ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.fastged_plan_run.argtypes = [vp, vp]
    lib.fastged_plan_read.argtypes = [vp, vp, vp, vp]
    lib.fastged_plan_info.argtypes = [vp, ctypes.POINTER(PlanStats)]
    lib.fastged_plan_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.fastged_plan_destroy.argtypes = [vp]
    lib.fastged_plan_destroy.restype = None
    dp = ctypes.POINTER(ctypes.c_double)
    lib.fastged_measure_int_peak.argtypes = [dp, dp, dp]
    lib.fastged_batch_noalloc.argtypes = [ctypes.POINTER(CostModel), ctypes.POINTER(DeviceBatch),
                                          i32, vp, vp, vp, vp]
    lib.fastged_serve_start.argtypes = [ctypes.POINTER(CostModel), ctypes.POINTER(ServeConfig),
                                        ctypes.POINTER(vp)]
    lib.fastged_serve_submit.argtypes = [vp, vp, vp, i32, ctypes.c_uint64]
    lib.fastged_serve_poll.argtypes = [vp, ctypes.POINTER(ServeResult), i32, vp, i64, i32]
    lib.fastged_serve_get_stats.argtypes = [vp, ctypes.POINTER(ServeStats)]
    lib.fastged_serve_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.fastged_serve_stop.argtypes = [vp]
    lib.fastged_serve_stop.restype = None
    lib.fastged_serve_destroy.argtypes = [vp]
    lib.fastged_serve_destroy.restype = None
    lib.fastged_edit_path.argtypes = [ctypes.POINTER(CostModel), ctypes.POINTER(GraphC),
                                      ctypes.POINTER(GraphC), vp, vp, i32, vp, vp]
    lib.fastged_apply_edit_ops.argtypes = [ctypes.POINTER(GraphC), ctypes.POINTER(GraphC), vp,
                                           vp, i32, vp, vp, vp, vp, vp]
    lib.fastged_cross.argtypes = [vp, vp, i32, vp, i32, vp, i32, i32, ctypes.POINTER(Options),
                                  vp]
    lib.fastged_set_timeout.argtypes = [vp, i32]
    lib.fastged_inject_fault.argtypes = [i32, i32]
    lib.fastged_autotune_entries.restype = ctypes.c_int
    lib.fastged_autotune_clear.restype = None
    for name in EXPORTED:
        if name in ("fastged_destroy", "fastged_plan_destroy", "fastged_last_error",
                    "fastged_version", "fastged_serve_stop", "fastged_serve_destroy",
                    "fastged_autotune_clear"):
            continue
        getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _LIB = lib
    return lib


def _check(lib, rc: int):
    if rc != FASTGED_OK:
        msg = lib.fastged_last_error(None)
        raise FastGEDError(rc, msg.decode() if msg else "")


class Marshalled:
    """A workload's graphs and pairs in the C layout, kept alive for the duration of calls."""

    def __init__(self, graphs, pairs):
        ng = len(graphs)
        self.n = np.fromiter((g.n for g in graphs), dtype=np.int32, count=ng)
        self.m = np.fromiter((g.edges.shape[0] for g in graphs), dtype=np.int32, count=ng)
        self.vl = (np.concatenate([np.asarray(g.vlabel, dtype=np.int32) for g in graphs])
                   if ng else np.zeros(0, np.int32))
        self.ed = (np.concatenate([np.asarray(g.edges, dtype=np.int32).reshape(-1) for g in graphs])
                   if ng else np.zeros(0, np.int32))
        labelled = [g.elabel is not None for g in graphs]
        self.el = None
        if any(labelled):
            self.el = np.concatenate([np.asarray(g.elabel, dtype=np.int32) if g.elabel is not None
                                      else np.zeros(g.edges.shape[0], np.int32) for g in graphs])
        self.vl = np.ascontiguousarray(self.vl)
        self.ed = np.ascontiguousarray(self.ed)
        voff = np.zeros(ng, dtype=np.uint64)
        eoff = np.zeros(ng, dtype=np.uint64)
        if ng:
            voff[1:] = np.cumsum(self.n[:-1], dtype=np.uint64)
            eoff[1:] = np.cumsum(self.m[:-1], dtype=np.uint64)
        self.gs = np.zeros(ng, dtype=_GRAPH_DTYPE)
        self.gs["n"] = self.n
        self.gs["m"] = self.m
        vbase = self.vl.ctypes.data if self.vl.size else 0
        ebase = self.ed.ctypes.data if self.ed.size else 0
        self.gs["vlabel"] = np.where(self.n > 0, vbase + voff * 4, 0)
        self.gs["edges"] = np.where(self.m > 0, ebase + eoff * 8, 0)
        if self.el is not None and self.el.size:
            self.gs["elabel"] = np.where(self.m > 0, self.el.ctypes.data + eoff * 4, 0)
        self.pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        self.pl = PairList(ng, self.gs.ctypes.data if ng else None, self.pairs.shape[0],
                           self.pairs.ctypes.data if self.pairs.size else None)
        self.n1 = self.n[self.pairs[:, 0]] if self.pairs.size else np.zeros(0, np.int32)
        self.map_off = np.zeros(self.pairs.shape[0] + 1, dtype=np.int64)
        if self.pairs.size:
            self.map_off[1:] = np.cumsum(self.n1, dtype=np.int64)

    @property
    def n_pairs(self) -> int:
        return int(self.pairs.shape[0])


def marshal(w) -> Marshalled:
    """Marshal a Workload (cached on the object)."""
    mm = getattr(w, "_marshalled", None)
    if mm is None:
        mm = Marshalled(w.graphs, w.pairs)
        try:
            w._marshalled = mm
        except AttributeError:
            pass
    return mm


def make_options(form: int = FASTGED_FORM_BATCHED, variant: int = 0, k_per_pair=None,
                 hist_window: int = 0, block_threads: int = 0, use_cuda_graph: int = 1,
                 autotune: int = 0, vertex_order: int = FASTGED_ORDER_INDEX,
                 team: int = FASTGED_TEAM_AUTO, max_sms: int = 0, cluster: int = 0):
    kpp = None
    if k_per_pair is not None:
        kpp = np.ascontiguousarray(np.asarray(k_per_pair, dtype=np.int32))
    o = Options(form, variant, kpp.ctypes.data if kpp is not None else None, hist_window,
                block_threads, use_cuda_graph, autotune, vertex_order, team, max_sms, cluster)
    o._keep = kpp
    return o


def fastged_version() -> int:
    return int(load().fastged_version())


def fastged_last_error() -> str:
    return load().fastged_last_error(None).decode()


def fastged_create(cost: Sequence[int]) -> int:
    lib = load()
    h = ctypes.c_void_p()
    _check(lib, lib.fastged_create(ctypes.byref(CostModel(*[int(x) for x in cost])),
                                   ctypes.byref(h)))
    return h.value


def fastged_destroy(h: int) -> None:
    load().fastged_destroy(h)


def _outputs(mm: Marshalled):
    return (np.zeros(mm.n_pairs, np.int32), np.zeros(int(mm.map_off[-1]), np.int32),
            np.zeros(mm.n_pairs, np.int64))


def fastged_batch(h: int, mm: Marshalled, K: int, out_cost: np.ndarray, out_mapping: np.ndarray):
    lib = load()
    _check(lib, lib.fastged_batch(h, ctypes.byref(mm.pl), int(K), out_cost.ctypes.data,
                                  out_mapping.ctypes.data if out_mapping.size else None))


def fastged_batch_ex(h: int, mm: Marshalled, K: int, opt: Optional[Options],
                     out_cost: np.ndarray, out_mapping: np.ndarray,
                     out_nevals: Optional[np.ndarray]):
    lib = load()
    _check(lib, lib.fastged_batch_ex(h, ctypes.byref(mm.pl), int(K),
                                     ctypes.byref(opt) if opt is not None else None,
                                     out_cost.ctypes.data,
                                     out_mapping.ctypes.data if out_mapping.size else None,
                                     out_nevals.ctypes.data if out_nevals is not None else None))


def fastged_plan_create(h: int, mm: Marshalled, K: int, opt: Optional[Options] = None) -> int:
    lib = load()
    p = ctypes.c_void_p()
    _check(lib, lib.fastged_plan_create(h, ctypes.byref(mm.pl), int(K),
                                        ctypes.byref(opt) if opt is not None else None,
                                        ctypes.byref(p)))
    return p.value


def fastged_plan_run(plan: int, stream: int = 0) -> None:
    lib = load()
    _check(lib, lib.fastged_plan_run(plan, stream or None))


def fastged_plan_read(plan: int, out_cost, out_mapping, out_nevals) -> None:
    lib = load()
    _check(lib, lib.fastged_plan_read(
        plan, out_cost.ctypes.data if out_cost is not None else None,
        out_mapping.ctypes.data if out_mapping is not None and out_mapping.size else None,
        out_nevals.ctypes.data if out_nevals is not None else None))


def fastged_plan_info(plan: int) -> dict:
    lib = load()
    st = PlanStats()
    _check(lib, lib.fastged_plan_info(plan, ctypes.byref(st)))
    nc = st.n_classes
    return {"n_pairs": st.n_pairs, "n_classes": nc, "launches_per_run": st.launches_per_run,
            "graph_replay": st.graph_replay, "input_bytes": st.input_bytes,
            "device_bytes": st.device_bytes, "output_bytes": st.output_bytes,
            "block_threads": list(st.block_threads[:nc]), "grid": list(st.grid[:nc]),
            "words": list(st.words[:nc]), "smem_bytes": list(st.smem_bytes[:nc])}


def fastged_plan_kernel_ms(plan: int) -> float:
    lib = load()
    ms = ctypes.c_float(0.0)
    _check(lib, lib.fastged_plan_kernel_ms(plan, ctypes.byref(ms)))
    return float(ms.value)


def fastged_plan_destroy(plan: int) -> None:
    load().fastged_plan_destroy(plan)


def fastged_measure_int_peak() -> dict:
    """Device-wide 32-bit LOP3 / IADD / POPC rates (ops per second)."""
    lib = load()
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib, lib.fastged_measure_int_peak(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"lop3": a.value, "iadd": b.value, "popc": c.value}


def fastged_batch_noalloc(cost: Sequence[int], batch: DeviceBatch, K: int, d_out_cost: int,
                          d_out_mapping: int, d_out_nevals: int = 0, stream: int = 0) -> None:
    """Allocation-free batch on device inputs and outputs (device addresses as ints)."""
    lib = load()
    _check(lib, lib.fastged_batch_noalloc(ctypes.byref(CostModel(*[int(x) for x in cost])),
                                          ctypes.byref(batch), int(K), d_out_cost,
                                          d_out_mapping, d_out_nevals or None, stream or None))


def split_maps(mm: Marshalled, flat: np.ndarray):
    return [flat[mm.map_off[p]:mm.map_off[p + 1]] for p in range(mm.n_pairs)]


class FastGED:
    """Convenience wrapper: one handle (cost model) on the current device."""

    def __init__(self, cost: Sequence[int]):
        self.cost = tuple(int(x) for x in cost)
        self.h = fastged_create(self.cost)

    def close(self):
        if self.h:
            fastged_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, w, K: Optional[int] = None, **opts) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(costs[n_pairs], flat maps, nevals[n_pairs]) for a Workload."""
        mm = marshal(w)
        if K is None:
            K = w.K
        if "k_per_pair" not in opts and w.k_per_pair is not None:
            opts["k_per_pair"] = w.k_per_pair
            K = max(K, int(np.max(w.k_per_pair)))
        cost, maps, nev = _outputs(mm)
        fastged_batch_ex(self.h, mm, K, make_options(**opts), cost, maps, nev)
        return cost, maps, nev


def serve_config(lanes=16, max_batch_pairs=4096, min_batch_pairs=64, max_pending=1 << 20,
                 max_wait_us=200, hbm_reserve_bytes=1 << 30, max_retries=0) -> ServeConfig:
    return ServeConfig(lanes, max_batch_pairs, min_batch_pairs, max_pending, max_wait_us,
                       max_retries, hbm_reserve_bytes)


class Server:
    """Continuous-batching server (fastged_serve_*). Queries reference graphs of a marshalled
    workload; results come back through poll()."""

    def __init__(self, cost: Sequence[int], cfg: Optional[ServeConfig] = None):
        self.lib = load()
        s = ctypes.c_void_p()
        _check(self.lib, self.lib.fastged_serve_start(
            ctypes.byref(CostModel(*[int(x) for x in cost])),
            ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(s)))
        self.s = s.value

    def submit(self, mm: "Marshalled", g1: int, g2: int, K: int, tag: int) -> int:
        """Queue (graph g1, graph g2) of a marshalled workload; returns the status code."""
        base = mm.gs.ctypes.data
        return self.lib.fastged_serve_submit(self.s, base + 40 * int(g1), base + 40 * int(g2),
                                             int(K), int(tag))

    def poll(self, max_results: int = 4096, map_cap: int = 1 << 20, timeout_ms: int = 10):
        """[(tag, status, cost, map, n_evals, latency_ms, queue_ms)] of finished queries (the
        map is empty for a query that failed)."""
        out = (ServeResult * max_results)()
        buf = np.zeros(map_cap, np.int32)
        n = self.lib.fastged_serve_poll(self.s, out, max_results, buf.ctypes.data, map_cap,
                                        timeout_ms)
        if n < 0:
            _check(self.lib, n)
        res = []
        for r in out[:n]:
            # a failed query has no map in the buffer
            mp = (buf[r.map_offset:r.map_offset + r.n1].copy() if r.status == FASTGED_OK
                  else np.zeros(0, np.int32))
            res.append((r.tag, r.status, r.cost, mp, r.n_evals, r.latency_ms, r.queue_ms))
        return res

    def cancel(self, tag: int) -> int:
        """Cancel the still-queued queries with this tag; returns how many were cancelled."""
        n = self.lib.fastged_serve_cancel(self.s, int(tag))
        if n < 0:
            _check(self.lib, n)
        return n

    def stats(self) -> dict:
        st = ServeStats()
        _check(self.lib, self.lib.fastged_serve_get_stats(self.s, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def stop(self):
        if self.s:
            self.lib.fastged_serve_stop(self.s)

    def close(self):
        if self.s:
            self.lib.fastged_serve_destroy(self.s)
            self.s = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



# ------------------------------------------------------------------------------------------
# edit paths and GED matrices
# ------------------------------------------------------------------------------------------
FASTGED_OP_VINS, FASTGED_OP_VSUB, FASTGED_OP_EDEL = 0, 1, 2
FASTGED_OP_ESUB, FASTGED_OP_EINS, FASTGED_OP_VDEL = 3, 4, 5
EDIT_OP_DTYPE = np.dtype([("kind", "<i4"), ("cost", "<i4"), ("g1_u", "<i4"), ("g1_v", "<i4"),
                          ("g2_u", "<i4"), ("g2_v", "<i4")])


class _OneGraph:
    """One graph as a fastged_graph struct (its arrays kept alive with it)."""

    def __init__(self, g):
        self.vl = np.ascontiguousarray(np.asarray(g.vlabel, dtype=np.int32).reshape(-1))
        self.ed = np.ascontiguousarray(np.asarray(g.edges, dtype=np.int32).reshape(-1))
        self.el = (None if g.elabel is None else
                   np.ascontiguousarray(np.asarray(g.elabel, dtype=np.int32).reshape(-1)))
        self.st = GraphC(int(g.n), self.vl.ctypes.data if self.vl.size else None,
                         int(self.ed.size // 2), self.ed.ctypes.data if self.ed.size else None,
                         self.el.ctypes.data if self.el is not None and self.el.size else None)


def _cost_model(cost: Sequence[int]) -> CostModel:
    return CostModel(*[int(x) for x in cost])


def fastged_edit_path(cost: Sequence[int], g1, g2, mapping) -> Tuple[np.ndarray, int]:
    """(operations as an EDIT_OP_DTYPE array, their total cost) of the edit path the vertex
    map induces from g1 to g2."""
    lib = load()
    a, b = _OneGraph(g1), _OneGraph(g2)
    mp = np.ascontiguousarray(np.asarray(mapping, dtype=np.int32).reshape(-1))
    cm = _cost_model(cost)
    n = ctypes.c_int32(0)
    tot = ctypes.c_int64(0)
    _check(lib, lib.fastged_edit_path(ctypes.byref(cm), ctypes.byref(a.st), ctypes.byref(b.st),
                                      mp.ctypes.data if mp.size else None, None, 0,
                                      ctypes.byref(n), None))
    ops = np.zeros(n.value, dtype=EDIT_OP_DTYPE)
    _check(lib, lib.fastged_edit_path(ctypes.byref(cm), ctypes.byref(a.st), ctypes.byref(b.st),
                                      mp.ctypes.data if mp.size else None,
                                      ops.ctypes.data if ops.size else None, int(ops.size),
                                      ctypes.byref(n), ctypes.byref(tot)))
    return ops, int(tot.value)


def fastged_apply_edit_ops(g1, g2, mapping, ops: np.ndarray, n_apply: int):
    """The graph obtained from g1 by applying the first n_apply operations of its edit path
    to g2 (vertex ids: surviving g1 vertices in order, then inserted g2 vertices)."""
    from .workloads import Graph
    lib = load()
    a, b = _OneGraph(g1), _OneGraph(g2)
    mp = np.ascontiguousarray(np.asarray(mapping, dtype=np.int32).reshape(-1))
    ops = np.ascontiguousarray(ops, dtype=EDIT_OP_DTYPE)
    nmax = int(g1.n) + int(g2.n)
    mmax = a.ed.size // 2 + b.ed.size // 2
    vl = np.zeros(max(nmax, 1), np.int32)
    ed = np.zeros(max(2 * mmax, 1), np.int32)
    labelled = a.el is not None or b.el is not None
    el = np.zeros(max(mmax, 1), np.int32) if labelled else None
    on, om = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib, lib.fastged_apply_edit_ops(ctypes.byref(a.st), ctypes.byref(b.st),
                                           mp.ctypes.data if mp.size else None,
                                           ops.ctypes.data if ops.size else None, int(n_apply),
                                           ctypes.byref(on), vl.ctypes.data, ctypes.byref(om),
                                           ed.ctypes.data,
                                           el.ctypes.data if el is not None else None))
    return Graph(on.value, vl[:on.value].copy(), ed[:2 * om.value].reshape(-1, 2).copy(),
                 el[:om.value].copy() if el is not None else None)


def fastged_cross(h: int, graphs, rows, cols, K: int, opt: Optional[Options] = None
                  ) -> np.ndarray:
    """GED matrix [len(rows), len(cols)] from graphs[rows[r]] to graphs[cols[c]]."""
    lib = load()
    mm = Marshalled(graphs, np.zeros((0, 2), np.int32))
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32).reshape(-1))
    c = np.ascontiguousarray(np.asarray(cols, dtype=np.int32).reshape(-1))
    out = np.zeros((r.size, c.size), np.int32)
    _check(lib, lib.fastged_cross(h, mm.gs.ctypes.data if len(graphs) else None, len(graphs),
                                  r.ctypes.data if r.size else None, int(r.size),
                                  c.ctypes.data if c.size else None, int(c.size), int(K),
                                  ctypes.byref(opt) if opt is not None else None,
                                  out.ctypes.data if out.size else None))
    return out


def knn_classify(cost: Sequence[int], train, train_labels, test, K: int, k: int = 1
                 ) -> np.ndarray:
    """Label of each test graph by majority among its k nearest training graphs under the
    K-Best GED (ties: the smaller label); one GED matrix batch computes every distance."""
    graphs = list(train) + list(test)
    rows = np.arange(len(train), len(graphs))
    cols = np.arange(len(train))
    with FastGED(cost) as g:
        d = fastged_cross(g.h, graphs, rows, cols, K)
    lab = np.asarray(train_labels)
    out = np.zeros(len(test), dtype=lab.dtype)
    for t in range(len(test)):
        near = np.argsort(d[t], kind="stable")[:k]
        vals, cnt = np.unique(lab[near], return_counts=True)
        out[t] = vals[np.argmax(cnt)]
    return out


def fastged_set_timeout(h: int, ms: int) -> None:
    lib = load()
    _check(lib, lib.fastged_set_timeout(h, int(ms)))


def fastged_inject_fault(kind: int, countdown: int) -> None:
    lib = load()
    _check(lib, lib.fastged_inject_fault(int(kind), int(countdown)))
