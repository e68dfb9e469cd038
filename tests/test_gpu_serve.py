"""Serving: queries submitted over time from several host threads, batched continuously
while earlier batches run, must each give exactly the result of the same query alone."""
import threading
import time

import numpy as np
import pytest

from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W
from parity_util import assert_parity, gpu_run

pytestmark = pytest.mark.gpu


def _mix(n=300, seed=5):
    """Serving-shaped mix at reduced size: molecule-like, dense ER and BA pairs, K drawn
    from {32, 128, 512} (large pairs capped at K = 64 to keep the test short)."""
    w = W.config5(duration_s=10.0, rate=1000.0, seed=seed, max_requests=n)
    shape = w.meta["shape"]
    keep = [p for p in range(w.n_pairs) if shape[p] != 2][: n - 6]
    keep += [p for p in range(w.n_pairs) if shape[p] == 2][:6]
    ws = W.subset(w, sorted(keep))
    k = ws.k_per_pair.copy()
    big = np.array([ws.graphs[int(ws.pairs[p][1])].n > 300 for p in range(ws.n_pairs)])
    k[big] = np.minimum(k[big], 64)
    ws.k_per_pair = k
    return ws


def _serve(w, cfg, threads=3, jitter_s=0.0005):
    mm = F.marshal(w)
    srv = F.Server(w.cost, cfg)
    order = np.random.RandomState(0).permutation(w.n_pairs)
    chunks = np.array_split(order, threads)

    def submitter(idx):
        for p in idx:
            while True:
                rc = srv.submit(mm, w.pairs[p][0], w.pairs[p][1], int(w.k_per_pair[p]), int(p))
                if rc != F.FASTGED_ERR_BUSY:
                    assert rc == F.FASTGED_OK, F.fastged_last_error()
                    break
                time.sleep(0.001)
            time.sleep(jitter_s)

    ts = [threading.Thread(target=submitter, args=(c,)) for c in chunks]
    for t in ts:
        t.start()
    got = {}
    deadline = time.time() + 600
    while len(got) < w.n_pairs and time.time() < deadline:
        for r in srv.poll(timeout_ms=50):
            got[int(r[0])] = r
    for t in ts:
        t.join()
    stats = srv.stats()
    srv.close()
    return got, stats


def test_served_results_equal_results_alone():
    w = _mix()
    cfg = F.serve_config(lanes=4, max_batch_pairs=64, min_batch_pairs=8, max_wait_us=300)
    got, stats = _serve(w, cfg)
    assert len(got) == w.n_pairs
    assert stats["batches"] > 1 and stats["failed"] == 0
    cost = np.array([got[p][2] for p in range(w.n_pairs)], np.int32)
    maps = np.concatenate([got[p][3] for p in range(w.n_pairs)]).astype(np.int32)
    nev = np.array([got[p][4] for p in range(w.n_pairs)], np.int64)
    assert all(got[p][1] == F.FASTGED_OK for p in range(w.n_pairs))
    # the same queries alone, one per batch call, and in one big batch
    alone = gpu_run(w, K=int(w.k_per_pair.max()))
    for x, y in zip((cost, maps, nev), alone):
        assert np.array_equal(x, y)
    # and the oracle on a sample
    assert_parity(w, (cost, maps, nev), idx=list(range(0, w.n_pairs, 10)))


def test_admission_and_backpressure():
    w = _mix(80, seed=6)
    # a reserve larger than the device: batches only launch when nothing else runs
    cfg = F.serve_config(lanes=3, max_batch_pairs=16, min_batch_pairs=4, max_pending=8,
                         hbm_reserve_bytes=1 << 60)
    got, stats = _serve(w, cfg, threads=2, jitter_s=0.0)
    assert len(got) == w.n_pairs and stats["failed"] == 0
    assert stats["rejected_busy"] > 0          # max_pending pushed back on submitters
    alone = gpu_run(w, K=int(w.k_per_pair.max()))
    cost = np.array([got[p][2] for p in range(w.n_pairs)], np.int32)
    assert np.array_equal(cost, alone[0])


def test_invalid_submissions_and_stop():
    w = W.config2(4)
    mm = F.marshal(w)
    srv = F.Server(w.cost)
    assert srv.submit(mm, 0, 1, 0, 1) == F.FASTGED_ERR_INVALID_ARG
    assert srv.submit(mm, 0, 1, (1 << 20) + 1, 1) == F.FASTGED_ERR_INVALID_ARG
    for p in range(4):
        assert srv.submit(mm, w.pairs[p][0], w.pairs[p][1], 100, p) == F.FASTGED_OK
    srv.stop()                                   # drains every queued query
    assert srv.submit(mm, 0, 1, 8, 9) == F.FASTGED_ERR_STOPPED
    res = srv.poll(timeout_ms=1000)
    assert sorted(r[0] for r in res) == [0, 1, 2, 3]
    srv.close()
