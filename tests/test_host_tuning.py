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


def _probe_classes(L, w, K, team=F.FASTGED_TEAM_CTA, full=False, **opts):
    """(block, cluster) of every size class when the batch is planned now (with full=True,
    a dict of the class's fields)."""
    c = (ctypes.c_int32 * 6)(*w.cost)
    mm = F.Marshalled(w.graphs, w.pairs)
    o = F.make_options(team=team, **opts)
    assert L.probe_flatten(ctypes.addressof(mm.pl), K, ctypes.addressof(o), c) == 0
    v = (ctypes.c_int64 * 31)()
    L.probe_batch(v)
    out = []
    names = ("W wide w32 pk cluster n1max n2max m1max kmax n_order order_off block grid "
             "slice_bytes scratch_off smem_bytes warp").split()
    for k in range(v[29]):
        x = (ctypes.c_int64 * 17)()
        L.probe_class(k, x)
        out.append(dict(zip(names, x)) if full else (x[11], x[4]))   # block, cluster
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
    p, st = _plan(lib, h, mm, w.K, autotune=1, team=F.FASTGED_TEAM_CTA)
    assert st.n_classes == 2
    # three shapes per class, each timed twice, one launch per timing run
    assert lib.fake_kbest_launches() - n0 == 2 * 3 * 2
    assert [st.block_threads[k] for k in range(2)] == [512, 512]
    assert lib.fastged_autotune_entries() == 2
    # the table now answers for these classes: no more timing runs, even when the timings
    # change, and a batch planned without autotuning uses the recorded shapes
    lib.fake_set_shape_ms(512, 1, 9.0)
    n1 = lib.fake_kbest_launches()
    p2, st2 = _plan(lib, h, mm, w.K, autotune=1, team=F.FASTGED_TEAM_CTA)
    assert lib.fake_kbest_launches() == n1
    assert [st2.block_threads[k] for k in range(2)] == [512, 512]
    assert _probe_classes(lib, w, w.K) == [(512, 1), (512, 1)]
    # a fixed block size skips the table
    p3, st3 = _plan(lib, h, mm, w.K, autotune=1, block_threads=128, team=F.FASTGED_TEAM_CTA)
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


def _warp_bytes(n1, n2, m1, K, B, w32, gmap):
    """Shared memory of one warp of a one-warp class: g2 records (16-byte padded: adjacency
    word, B label planes, cost entry; one per target vertex, the deletion and the stand-in
    of finished walks), labels, neighbour offsets and lists, two beams of
    Img / PED / inner-edge counts, the 16-bit entries, node offsets, kept list, selection,
    and the two map buffers unless they are in global scratch."""
    a = lambda x: (x + 15) // 16 * 16
    wb = 4 if w32 else 8
    rec = a(wb * (1 + B) + 4)
    mrow = a(max(n1, 1))
    parts = [(n2 + 2) * rec, max(n2, 1) * 4, (n1 + 1) * 4, max(m1, 1) * 4, K * wb, K * wb,
             K * 4, K * 4, K * 2, K * 2, K * (n2 + 1) * 2, (K + 1) * 2, K * 4, K * 4,
             K * 4]
    if not gmap:
        parts += [K * mrow, K * mrow]
    return sum(a(x) for x in parts)


def test_one_warp_classes_and_their_tuning(lib):
    """Molecule-like pairs (K <= 128) go to one-warp classes: CTAs of 4 warps by default,
    vertex maps in shared memory while 16 warps still fit an SM, grid capped by the pairs.
    The autotuner times 64/128 threads with the maps in shared or global memory (the
    fake reports the placement as cluster 100 + gmap) and keeps the fastest; the maps then
    move to a per-warp block of global scratch."""
    lib.fastged_autotune_clear()
    lib.fake_set_shape_ms(0, 0, 0.0)
    times = {(64, 100): 3.0, (128, 100): 5.0, (64, 101): 7.0, (128, 101): 2.0}
    for (block, cl), ms in times.items():
        lib.fake_set_shape_ms(block, cl, ms)
    w = W.config2(3000)
    cls = _probe_classes(lib, w, w.K, team=F.FASTGED_TEAM_AUTO, full=True)
    assert len(cls) == 2 and all(c["warp"] == 1 for c in cls)
    assert sorted(c["w32"] for c in cls) == [0, 1]
    for c in cls:
        args = (c["n1max"], c["n2max"], c["m1max"], c["kmax"], 2, bool(c["w32"]))
        gmap = 233472 // _warp_bytes(*args, False) < 16
        assert c["block"] == 128 and c["smem_bytes"] == 4 * _warp_bytes(*args, gmap)
        mrow = (c["n1max"] + 15) // 16 * 16
        assert c["slice_bytes"] == (4 * ((2 * c["kmax"] * mrow + 255) // 256 * 256) if gmap
                                    else 0)
        assert 1 <= c["grid"] <= min(152 * (2048 // 128), (c["n_order"] + 3) // 4)
    mm = F.Marshalled(w.graphs, w.pairs)
    h = _handle(lib, w.cost)
    n0 = lib.fake_kbest_launches()
    p, st = _plan(lib, h, mm, w.K, autotune=1)
    assert lib.fake_kbest_launches() - n0 == 2 * 4 * 2
    assert [st.block_threads[k] for k in range(2)] == [128, 128]
    for c in _probe_classes(lib, w, w.K, team=F.FASTGED_TEAM_AUTO, full=True):
        assert c["block"] == 128 and c["warp"] == 1
        assert c["slice_bytes"] > 0 and c["slice_bytes"] % (4 * 256) == 0
    # K past the one-warp limit: CTA teams again
    assert all(c["warp"] == 0 for c in _probe_classes(lib, w, 129, team=F.FASTGED_TEAM_AUTO,
                                                       full=True))
    lib.fastged_plan_destroy(p)
    lib.fastged_destroy(h)
    lib.fastged_autotune_clear()


def test_autotuner_picks_the_fastest_cluster_size(lib):
    lib.fastged_autotune_clear()
    lib.fake_set_shape_ms(0, 0, 0.0)
    for (block, cl), ms in (((256, 1), 5.0), ((512, 2), 4.0), ((512, 4), 1.0), ((512, 8), 2.0),
                            ((512, 16), 3.0)):
        lib.fake_set_shape_ms(block, cl, ms)
    w = W.config4(4, n_range=(600, 700))      # a few large pairs: cluster teams are eligible
    mm = F.Marshalled(w.graphs, w.pairs)
    h = _handle(lib, w.cost)
    n0 = lib.fake_kbest_launches()
    p, st = _plan(lib, h, mm, 64, autotune=1)
    ncls = st.n_classes
    assert lib.fake_kbest_launches() - n0 == ncls * 5 * 2
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
    lib.fake_fail_device_alloc(2)   # the allocation with headroom, then the exact size
    rc, cost = run(big)
    assert rc == F.FASTGED_ERR_OOM and b"cudaMalloc" in lib.fastged_last_error(None)
    assert (cost == -5).all()
    rc, cost = run(big)
    assert rc == F.FASTGED_OK and (cost == 0).all()
    assert run(small)[0] == F.FASTGED_OK
    lib.fastged_destroy(h)



def _cluster_rule(kmax, n2max, npairs, sms=152):
    """CTAs per cluster team without a tuning entry: about 20,000 successors of a level per
    CTA (2 to 8; 16 for a handful of very wide pairs), halved while the teams would take
    more than two waves of the GPU."""
    succ = kmax * (n2max + 1)
    cl = 2 if succ <= 40000 else 4 if succ <= 160000 else 8
    if succ >= 2000000 and npairs * 16 <= sms:
        cl = 16
    while cl > 2 and npairs * cl > 2 * sms:
        cl //= 2
    return cl


def test_cluster_size_follows_the_beam_and_the_pair_count(lib):
    lib.fastged_autotune_clear()
    lib.fake_set_shape_ms(0, 0, 0.0)
    seen = {}
    for K, npairs in ((32, 3), (128, 3), (512, 3), (1024, 60), (5000, 2)):
        w = W.config4(npairs, n_range=(600, 700))
        cls = _probe_classes(lib, w, K, full=True)
        assert cls and all(c["cluster"] > 1 for c in cls)
        for c in cls:
            assert c["cluster"] == _cluster_rule(c["kmax"], c["n2max"], c["n_order"])
            assert c["grid"] == min(152 // c["cluster"], c["n_order"]) * c["cluster"]
        seen[(K, npairs)] = cls[0]["cluster"]
    # hand-checked cases: 600-700 target vertices
    assert seen == {(32, 3): 2, (128, 3): 4, (512, 3): 8, (1024, 60): 4, (5000, 2): 16}


def test_max_sms_caps_the_resident_teams(lib):
    lib.fastged_autotune_clear()
    w = W.config4(20, n_range=(600, 700))
    base = _probe_classes(lib, w, 512, full=True)
    for cap in (1, 24, 100):
        capped = _probe_classes(lib, w, 512, full=True, max_sms=cap)
        for b, c in zip(base, capped):
            cl = b["cluster"]
            assert c["cluster"] == cl and c["grid"] % cl == 0
            assert c["grid"] == min(b["grid"] // cl, max(1, cap // cl)) * cl
    # one-CTA teams (two per SM in the fake) and one-warp teams (CTAs per SM by their
    # shared memory)
    w2 = W.config2(3000)
    for team in (F.FASTGED_TEAM_AUTO, F.FASTGED_TEAM_CTA):
        base = _probe_classes(lib, w2, 100, team=team, full=True)
        capped = _probe_classes(lib, w2, 100, team=team, full=True, max_sms=10)
        for b, c in zip(base, capped):
            if c["warp"]:
                occ = min((233472 - 1024) // (c["smem_bytes"] + 1024), 2048 // c["block"])
            else:
                occ = 2
            assert c["grid"] == min(b["grid"], 10 * occ) < b["grid"]
    c = (ctypes.c_int32 * 6)(*w2.cost)
    mm = F.Marshalled(w2.graphs, w2.pairs)
    o = F.make_options(max_sms=-1)
    assert lib.probe_flatten(ctypes.addressof(mm.pl), 100, ctypes.addressof(o), c) == F.FASTGED_ERR_INVALID_ARG


def test_cluster_option_forces_the_team_size(lib):
    lib.fastged_autotune_clear()
    w = W.config4(3, n_range=(600, 700))
    for cl in (1, 2, 4, 16):
        cls = _probe_classes(lib, w, 512, full=True, cluster=cl)
        assert cls and all(c["cluster"] == cl for c in cls)
    # classes that cannot use clusters ignore it: the molecule batch keeps one-CTA teams
    w2 = W.config2(500)
    assert all(c[1] == 1 for c in _probe_classes(lib, w2, 100, cluster=8))
    c = (ctypes.c_int32 * 6)(*w.cost)
    mm = F.Marshalled(w.graphs, w.pairs)
    for bad in (3, -1, 32):
        o = F.make_options(cluster=bad)
        assert lib.probe_flatten(ctypes.addressof(mm.pl), 64, ctypes.addressof(o), c) == F.FASTGED_ERR_INVALID_ARG
