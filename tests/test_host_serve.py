"""The serving dispatcher's host logic, on the CPU.

serve.cu is host code: it is built with g++ against fakes of the CUDA calls (see
tests/host_probe.py). Batches do no device work there: a batch's completion callback runs on a
fake stream after a set delay and its results are zeros, so what is checked is the dispatcher:
every submitted query comes back exactly once with its tag and its map length, batches respect
their size limit, the queue pushes back when full, admission waits for memory while other
batches run, a failed launch is reported for every query of that batch (or the batch is
retried, up to max_retries times), a cancelled query
comes back cancelled while the others run, and stop drains the queue and then refuses new
queries.
"""
import ctypes
import threading
import time

import numpy as np
import pytest

from host_probe import load
from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    L = load()
    yield L
    L.fake_set_free_bytes(250 << 30)
    L.fake_set_host_fn_delay_us(0)


class HostServer(F.Server):
    """F.Server on the test library."""

    def __init__(self, L, cost, cfg=None):
        self.lib = L
        s = ctypes.c_void_p()
        F._check(L, L.fastged_serve_start(ctypes.byref(F.CostModel(*cost)),
                                          ctypes.byref(cfg) if cfg is not None else None,
                                          ctypes.byref(s)))
        self.s = s.value


def _mix(n, seed=3):
    """Molecule-like, dense and large (300-400 vertex) pairs, K from {32, 128, 512}."""
    a = W.config2(n, seed=seed)
    b = W.config3(max(n // 8, 2), seed=seed)
    c = W.config4(3, seed=seed, n_range=(300, 400))
    w = W.concat([a, b, c])
    k = np.array([32, 128, 512])[np.arange(w.n_pairs) % 3].astype(np.int32)
    return w, k


def _submit_all(srv, mm, w, kk, idx, retry=True):
    busy = 0
    for p in idx:
        while True:
            rc = srv.submit(mm, w.pairs[p][0], w.pairs[p][1], int(kk[p]), int(p))
            if rc == F.FASTGED_ERR_BUSY and retry:
                busy += 1
                time.sleep(0.0005)
                continue
            assert rc == F.FASTGED_OK, rc
            break
    return busy


def _collect(srv, n, timeout_s=60.0):
    got = {}
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        for r in srv.poll(timeout_ms=20):
            assert r[0] not in got, "a query came back twice"
            got[r[0]] = r
    return got


def test_every_query_completes_once(lib):
    lib.fake_set_host_fn_delay_us(300)
    w, kk = _mix(400)
    mm = F.Marshalled(w.graphs, w.pairs)
    cfg = F.serve_config(lanes=4, max_batch_pairs=48, min_batch_pairs=8, max_wait_us=300)
    srv = HostServer(lib, w.cost, cfg)
    lib.fake_max_pack_graphs(1)
    chunks = np.array_split(np.random.RandomState(1).permutation(w.n_pairs), 3)
    ts = [threading.Thread(target=_submit_all, args=(srv, mm, w, kk, c)) for c in chunks]
    for t in ts:
        t.start()
    got = _collect(srv, w.n_pairs)
    for t in ts:
        t.join()
    st = srv.stats()
    srv.close()
    assert sorted(got) == list(range(w.n_pairs))
    for p, (tag, status, cost, mp, nev, lat, qms) in got.items():
        assert status == F.FASTGED_OK and cost == 0 and nev == 0
        assert len(mp) == w.graphs[int(w.pairs[p][0])].n
        assert lat >= qms >= 0.0
    assert st["submitted"] == st["completed"] == st["batched_pairs"] == w.n_pairs
    assert st["failed"] == 0 and st["pending"] == 0 and st["lanes_busy"] == 0
    assert st["batches"] >= -(-w.n_pairs // 48)
    assert lib.fake_max_pack_graphs(0) <= 2 * 48   # two graphs per query


def test_batches_stop_at_the_size_limit(lib):
    # one lane whose batches take 100 ms: while the first runs, the rest of 300 queries of one
    # size bucket queue up, so every later batch is cut at max_batch_pairs
    lib.fake_set_host_fn_delay_us(100000)
    w = W.config2(1200, seed=8)
    keep = [p for p in range(w.n_pairs) if w.graphs[int(w.pairs[p][1])].n <= 32][:300]
    w = W.subset(w, keep)
    kk = np.full(w.n_pairs, 32, np.int32)
    mm = F.Marshalled(w.graphs, w.pairs)
    cfg = F.serve_config(lanes=1, max_batch_pairs=40, min_batch_pairs=1, max_wait_us=0)
    srv = HostServer(lib, w.cost, cfg)
    lib.fake_max_pack_graphs(1)
    _submit_all(srv, mm, w, kk, range(w.n_pairs))
    got = _collect(srv, w.n_pairs)
    st = srv.stats()
    srv.close()
    assert sorted(got) == list(range(w.n_pairs))
    assert lib.fake_max_pack_graphs(0) == 2 * 40
    assert st["batches"] >= -(-w.n_pairs // 40)


def test_full_queue_pushes_back(lib):
    lib.fake_set_host_fn_delay_us(3000)
    w, kk = _mix(120, seed=4)
    mm = F.Marshalled(w.graphs, w.pairs)
    cfg = F.serve_config(lanes=2, max_batch_pairs=8, min_batch_pairs=4, max_pending=6,
                         max_wait_us=100)
    srv = HostServer(lib, w.cost, cfg)
    busy = _submit_all(srv, mm, w, kk, range(w.n_pairs))
    got = _collect(srv, w.n_pairs)
    st = srv.stats()
    srv.close()
    assert busy > 0 and st["rejected_busy"] == busy
    assert sorted(got) == list(range(w.n_pairs))
    assert st["completed"] == w.n_pairs and st["failed"] == 0


def test_admission_waits_for_memory(lib):
    lib.fake_set_host_fn_delay_us(1000)
    lib.fake_set_free_bytes(0)   # a batch is admitted only when nothing else runs
    try:
        w, kk = _mix(80, seed=5)
        mm = F.Marshalled(w.graphs, w.pairs)
        cfg = F.serve_config(lanes=3, max_batch_pairs=8, min_batch_pairs=1, max_wait_us=50)
        srv = HostServer(lib, w.cost, cfg)
        _submit_all(srv, mm, w, kk, range(w.n_pairs))
        got = _collect(srv, w.n_pairs)
        st = srv.stats()
        srv.close()
    finally:
        lib.fake_set_free_bytes(250 << 30)
    assert sorted(got) == list(range(w.n_pairs))
    assert st["admission_waits"] > 0 and st["failed"] == 0


def test_failed_launch_is_reported_for_its_queries(lib):
    lib.fake_set_host_fn_delay_us(200)
    w, kk = _mix(60, seed=6)
    mm = F.Marshalled(w.graphs, w.pairs)
    cfg = F.serve_config(lanes=2, max_batch_pairs=16, min_batch_pairs=16, max_wait_us=100000)
    srv = HostServer(lib, w.cost, cfg)
    lib.fastged_inject_fault(F.FASTGED_INJECT_LAUNCH, 1)   # the next batch fails to launch
    _submit_all(srv, mm, w, kk, range(w.n_pairs))
    srv.stop()                                              # flush the partial batches
    # the raw C results: a failed query reports no map entries (n1 = 0)
    out = (F.ServeResult * w.n_pairs)()
    buf = np.zeros(1 << 16, np.int32)
    n = lib.fastged_serve_poll(srv.s, out, w.n_pairs, buf.ctypes.data, buf.size, 100)
    assert n == w.n_pairs
    got = {}
    for r in out[:n]:
        a = int(w.pairs[r.tag][0])
        assert r.n1 == (w.graphs[a].n if r.status == F.FASTGED_OK else 0)
        got[r.tag] = (r.tag, r.status, r.cost, buf[r.map_offset:r.map_offset + r.n1])
    st = srv.stats()
    srv.close()
    assert sorted(got) == list(range(w.n_pairs))
    failed = [p for p, r in got.items() if r[1] != F.FASTGED_OK]
    assert all(got[p][1] == F.FASTGED_ERR_CUDA and len(got[p][3]) == 0 for p in failed)
    assert 1 <= len(failed) <= 16 and st["failed"] == len(failed)
    assert st["completed"] == w.n_pairs


def test_stop_drains_then_refuses(lib):
    lib.fake_set_host_fn_delay_us(2000)
    w, kk = _mix(40, seed=7)
    mm = F.Marshalled(w.graphs, w.pairs)
    cfg = F.serve_config(lanes=2, max_batch_pairs=4, min_batch_pairs=4, max_wait_us=1000000)
    srv = HostServer(lib, w.cost, cfg)
    _submit_all(srv, mm, w, kk, range(w.n_pairs))
    srv.stop()                       # returns once every queued query has run
    st = srv.stats()
    assert st["pending"] == 0 and st["lanes_busy"] == 0 and st["completed"] == w.n_pairs
    assert srv.submit(mm, w.pairs[0][0], w.pairs[0][1], 8, 999) == F.FASTGED_ERR_STOPPED
    got = _collect(srv, w.n_pairs)
    srv.close()
    assert sorted(got) == list(range(w.n_pairs))


@pytest.mark.parametrize("fails,retries,ok", [(1, 1, True), (2, 1, False), (1, 0, False),
                                               (3, 3, True)])
def test_failed_batch_is_retried(lib, fails, retries, ok):
    """A query whose batch fails goes back to the queue up to max_retries times; only then is
    its failure reported."""
    lib.fake_set_host_fn_delay_us(0)
    w, kk = _mix(4, seed=10)
    mm = F.Marshalled(w.graphs, w.pairs)
    srv = HostServer(lib, w.cost, F.serve_config(lanes=1, max_retries=retries))
    lib.fake_fail_launches(fails)
    try:
        _submit_all(srv, mm, w, kk, [0])
        got = _collect(srv, 1, timeout_s=30)
        st = srv.stats()
    finally:
        lib.fake_fail_launches(0)
        srv.close()
    assert list(got) == [0]
    assert got[0][1] == (F.FASTGED_OK if ok else F.FASTGED_ERR_CUDA)
    assert st["failed"] == (0 if ok else 1) and st["completed"] == 1
    assert st["batches"] == min(fails, retries + 1) + (1 if ok else 0)


def test_retries_recover_a_failed_batch_in_a_stream(lib):
    lib.fake_set_host_fn_delay_us(200)
    w, kk = _mix(60, seed=11)
    mm = F.Marshalled(w.graphs, w.pairs)
    cfg = F.serve_config(lanes=2, max_batch_pairs=16, min_batch_pairs=8, max_wait_us=500,
                         max_retries=1)
    srv = HostServer(lib, w.cost, cfg)
    lib.fastged_inject_fault(F.FASTGED_INJECT_LAUNCH, 2)   # the second batch fails once
    _submit_all(srv, mm, w, kk, range(w.n_pairs))
    got = _collect(srv, w.n_pairs)
    st = srv.stats()
    srv.close()
    assert sorted(got) == list(range(w.n_pairs))
    assert all(r[1] == F.FASTGED_OK for r in got.values())
    assert st["failed"] == 0 and st["completed"] == w.n_pairs
    assert st["batched_pairs"] > w.n_pairs          # the failed batch's queries ran twice


def test_cancel_queued_queries(lib):
    # one lane whose batch takes 200 ms: the first query occupies it, the rest stay queued
    lib.fake_set_host_fn_delay_us(200000)
    w, kk = _mix(40, seed=9)
    w = W.subset(w, range(21))
    kk = kk[:21]
    mm = F.Marshalled(w.graphs, w.pairs)
    cfg = F.serve_config(lanes=1, max_batch_pairs=64, min_batch_pairs=1000,
                         max_wait_us=10000000)
    srv = HostServer(lib, w.cost, cfg)
    _submit_all(srv, mm, w, kk, [0])
    t0 = time.time()                           # the dispatcher launches it on the idle lane
    while srv.stats()["batches"] < 1 and time.time() - t0 < 10:
        time.sleep(0.001)
    _submit_all(srv, mm, w, kk, range(1, 21))
    # a tag used twice: both queued copies go
    assert srv.submit(mm, w.pairs[5][0], w.pairs[5][1], int(kk[5]), 5) == F.FASTGED_OK
    assert srv.cancel(3) == 1 and srv.cancel(5) == 2 and srv.cancel(7) == 1
    assert srv.cancel(0) == 0                  # already running
    assert srv.cancel(999) == 0                # never submitted
    assert lib.fastged_serve_cancel(None, 1) == F.FASTGED_ERR_INVALID_ARG
    srv.stop()
    out = (F.ServeResult * 64)()
    buf = np.zeros(1 << 16, np.int32)
    n = lib.fastged_serve_poll(srv.s, out, 64, buf.ctypes.data, buf.size, 100)
    st = srv.stats()
    srv.close()
    status = {}
    for r in out[:n]:
        status.setdefault(int(r.tag), []).append(r.status)
        if r.status == F.FASTGED_ERR_CANCELLED:
            assert r.n1 == 0
    assert n == 22
    assert status[3] == status[7] == [F.FASTGED_ERR_CANCELLED]
    assert status[5] == [F.FASTGED_ERR_CANCELLED] * 2
    assert all(v == [F.FASTGED_OK] for t, v in status.items() if t not in (3, 5, 7))
    assert st["submitted"] == st["completed"] == 22 and st["failed"] == 0
    assert st["batched_pairs"] == 22 - 4


def test_invalid_submissions(lib):
    w = W.config2(4)
    g = w.graphs[0]
    dup = W.Graph(g.n, g.vlabel, np.concatenate([g.edges, g.edges[:1]]), None)
    loop = W.Graph(g.n, g.vlabel, np.concatenate([g.edges, np.array([[1, 1]], np.int32)]), None)
    badlab = W.Graph(g.n, g.vlabel, g.edges, np.full(g.m, 300, np.int32))
    ws = W.Workload("bad", [g, w.graphs[1], dup, loop, badlab],
                    np.zeros((0, 2), np.int32), w.cost, 8)
    mm = F.Marshalled(ws.graphs, ws.pairs)
    srv = HostServer(lib, w.cost)
    assert srv.submit(mm, 0, 1, 0, 1) == F.FASTGED_ERR_INVALID_ARG
    assert srv.submit(mm, 0, 1, (1 << 20) + 1, 1) == F.FASTGED_ERR_INVALID_ARG
    for bad in (2, 3, 4):
        assert srv.submit(mm, bad, 1, 8, 1) == F.FASTGED_ERR_INVALID_ARG
        assert srv.submit(mm, 0, bad, 8, 1) == F.FASTGED_ERR_INVALID_ARG
    assert srv.submit(mm, 0, 1, 8, 7) == F.FASTGED_OK
    srv.stop()
    got = srv.poll(timeout_ms=100)
    srv.close()
    assert [r[0] for r in got] == [7]
    big = (1 << 29,) * 6
    srv = HostServer(lib, big)
    assert srv.submit(mm, 0, 1, 8, 1) == F.FASTGED_ERR_INVALID_ARG
    srv.close()
