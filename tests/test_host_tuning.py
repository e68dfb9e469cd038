"""The autotuner's choice and the handle's wait bound, on the CPU.

The host runtime is built against fakes of the CUDA calls (tests/host_probe.py). The fakes
report a set elapsed time for each team shape (threads per CTA, CTAs per cluster), so the
autotuner must pick the fastest shape of every size class, time each shape twice, and record
the choice once; and events that stay "not ready" longer than a handle's timeout make
fastged_batch_ex return FASTGED_ERR_TIMEOUT without waiting, after which the handle drains
and serves the next batch.
"""
import ctypes
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
    L.fake_set_shape_ms(0, 0, 0.0)
    L.fake_events_busy_for_ms(0)
    L.fastged_autotune_clear()


def _handle(L, cost):
    h = ctypes.c_void_p()
    assert L.fastged_create(ctypes.byref(F.CostModel(*cost)), ctypes.byref(h)) == F.FASTGED_OK
    return h.value


def _plan(L, h, mm, K, **opts):
    p = ctypes.c_void_p()
    o = F.make_options(**opts)
    rc = L.fastged_plan_create(h, ctypes.byref(mm.pl), K, ctypes.byref(o), ctypes.byref(p))
    assert rc == F.FASTGED_OK, L.fastged_last_error(None)
    st = F.PlanStats()
    assert L.fastged_plan_info(p, ctypes.byref(st)) == F.FASTGED_OK
    return p.value, st


def _probe_classes(L, w, K):
    """(block, cluster) of every size class when the batch is planned now."""
    c = (ctypes.c_int32 * 6)(*w.cost)
    mm = F.Marshalled(w.graphs, w.pairs)
    o = F.make_options()
    assert L.probe_flatten(ctypes.addressof(mm.pl), K, ctypes.addressof(o), c) == 0
    v = (ctypes.c_int64 * 31)()
    L.probe_batch(v)
    out = []
    for k in range(v[29]):
        x = (ctypes.c_int64 * 16)()
        L.probe_class(k, x)
        out.append((x[11], x[4]))   # block, cluster
    return out


def test_autotuner_picks_the_fastest_block_size(lib):
    lib.fastged_autotune_clear()
    lib.fake_set_shape_ms(0, 0, 0.0)
    for block, ms in ((128, 3.0), (256, 2.0), (512, 1.0)):
        lib.fake_set_shape_ms(block, 1, ms)
    w = W.config2(3000)                       # two size classes (n2 <= 32, 33-40)
    mm = F.Marshalled(w.graphs, w.pairs)
    h = _handle(lib, w.cost)
    n0 = lib.fake_kbest_launches()
    p, st = _plan(lib, h, mm, w.K, autotune=1)
    assert st.n_classes == 2
    # three shapes per class, each timed twice, one launch per timing run
    assert lib.fake_kbest_launches() - n0 == 2 * 3 * 2
    assert [st.block_threads[k] for k in range(2)] == [512, 512]
    assert lib.fastged_autotune_entries() == 2
    # the table now answers for these classes: no more timing runs, even when the timings
    # change, and a batch planned without autotuning uses the recorded shapes
    lib.fake_set_shape_ms(512, 1, 9.0)
    n1 = lib.fake_kbest_launches()
    p2, st2 = _plan(lib, h, mm, w.K, autotune=1)
    assert lib.fake_kbest_launches() == n1
    assert [st2.block_threads[k] for k in range(2)] == [512, 512]
    assert _probe_classes(lib, w, w.K) == [(512, 1), (512, 1)]
    # a fixed block size skips the table
    p3, st3 = _plan(lib, h, mm, w.K, autotune=1, block_threads=128)
    assert [st3.block_threads[k] for k in range(2)] == [128, 128]
    for q in (p, p2, p3):
        lib.fastged_plan_destroy(q)
    lib.fastged_destroy(h)
    # without entries, a class gets the default shape again (256 threads for K > 32,
    # 128 for K <= 32)
    lib.fastged_autotune_clear()
    assert lib.fastged_autotune_entries() == 0
    assert _probe_classes(lib, w, w.K) == [(256, 1), (256, 1)]
    assert _probe_classes(lib, w, 32) == [(128, 1), (128, 1)]


def test_autotuner_picks_the_fastest_cluster_size(lib):
    lib.fastged_autotune_clear()
    lib.fake_set_shape_ms(0, 0, 0.0)
    for (block, cl), ms in (((256, 1), 5.0), ((512, 4), 1.0), ((512, 8), 2.0),
                            ((512, 16), 3.0)):
        lib.fake_set_shape_ms(block, cl, ms)
    w = W.config4(4, n_range=(600, 700))      # a few large pairs: cluster teams are eligible
    mm = F.Marshalled(w.graphs, w.pairs)
    h = _handle(lib, w.cost)
    n0 = lib.fake_kbest_launches()
    p, st = _plan(lib, h, mm, 64, autotune=1)
    ncls = st.n_classes
    assert lib.fake_kbest_launches() - n0 == ncls * 4 * 2
    assert all(b == (512, 4) for b in _probe_classes(lib, w, 64))
    lib.fastged_plan_destroy(p)
    lib.fastged_destroy(h)
    lib.fastged_autotune_clear()


def test_timeout_returns_early_and_the_handle_recovers(lib):
    w = W.config2(300)
    mm = F.Marshalled(w.graphs, w.pairs)
    h = _handle(lib, w.cost)
    cost, maps, nev = F._outputs(mm)
    o = F.make_options()

    def run():
        return lib.fastged_batch_ex(h, ctypes.byref(mm.pl), w.K, ctypes.byref(o),
                                    cost.ctypes.data, maps.ctypes.data, nev.ctypes.data)

    assert lib.fastged_set_timeout(h, -1) == F.FASTGED_ERR_INVALID_ARG
    assert lib.fastged_set_timeout(h, 30) == F.FASTGED_OK
    lib.fake_events_busy_for_ms(3000)          # the batch "runs" for 3 s
    cost[:] = -7
    t0 = time.time()
    assert run() == F.FASTGED_ERR_TIMEOUT
    assert time.time() - t0 < 1.0
    assert b"timeout" in lib.fastged_last_error(None)
    assert (cost == -7).all()                  # no outputs on failure
    lib.fake_events_busy_for_ms(0)
    assert run() == F.FASTGED_OK               # drains the timed-out batch first
    assert (cost == 0).all() and (nev == 0).all()
    # without a bound the call waits for the stream instead of polling the event
    assert lib.fastged_set_timeout(h, 0) == F.FASTGED_OK
    lib.fake_events_busy_for_ms(3000)
    t0 = time.time()
    assert run() == F.FASTGED_OK
    assert time.time() - t0 < 1.0
    lib.fake_events_busy_for_ms(0)
    lib.fastged_destroy(h)


def test_failed_device_allocation_leaves_the_handle_usable(lib):
    """A batch that needs more device memory than the handle holds, when cudaMalloc fails:
    FASTGED_ERR_OOM, no outputs written, and the next call allocates afresh and succeeds."""
    small, big = W.config2(50), W.config2(3000)
    h = _handle(lib, small.cost)
    o = F.make_options()

    def run(w):
        mm = F.Marshalled(w.graphs, w.pairs)
        cost, maps, nev = F._outputs(mm)
        cost[:] = -5
        rc = lib.fastged_batch_ex(h, ctypes.byref(mm.pl), w.K, ctypes.byref(o),
                                  cost.ctypes.data, maps.ctypes.data, nev.ctypes.data)
        return rc, cost

    assert run(small)[0] == F.FASTGED_OK
    lib.fake_fail_device_alloc(1)
    rc, cost = run(big)
    assert rc == F.FASTGED_ERR_OOM and b"cudaMalloc" in lib.fastged_last_error(None)
    assert (cost == -5).all()
    rc, cost = run(big)
    assert rc == F.FASTGED_OK and (cost == 0).all()
    assert run(small)[0] == F.FASTGED_OK
    lib.fastged_destroy(h)

