"""Failure handling without faulting the GPU: host-side injected faults (a failed allocation,
a skipped launch, a refused admission) and a bounded wait. Every failing call must report its
error and leave the handle or server usable, with later results still exact."""
import time

import numpy as np
import pytest

from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W
from parity_util import assert_parity, gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _disarm():
    yield
    for kind in (F.FASTGED_INJECT_ALLOC, F.FASTGED_INJECT_LAUNCH, F.FASTGED_INJECT_ADMISSION):
        F.fastged_inject_fault(kind, 0)


def test_injected_allocation_failure_leaves_the_handle_usable():
    w = W.config2(60)
    with F.FastGED(w.cost) as g:
        F.fastged_inject_fault(F.FASTGED_INJECT_ALLOC, 1)
        with pytest.raises(F.FastGEDError) as ei:
            g.run(w)
        assert ei.value.code == F.FASTGED_ERR_OOM
        assert_parity(w, g.run(w))


def test_injected_launch_failure_in_a_batch_and_a_plan():
    w = W.config2(60)
    ref = gpu_run(w)
    with F.FastGED(w.cost) as g:
        F.fastged_inject_fault(F.FASTGED_INJECT_LAUNCH, 1)
        with pytest.raises(F.FastGEDError) as ei:
            g.run(w)
        assert ei.value.code == F.FASTGED_ERR_CUDA
        for x, y in zip(g.run(w), ref):
            assert np.array_equal(x, y)
        mm = F.marshal(w)
        plan = F.fastged_plan_create(g.h, mm, w.K, F.make_options())
        F.fastged_inject_fault(F.FASTGED_INJECT_LAUNCH, 1)
        with pytest.raises(F.FastGEDError):
            F.fastged_plan_run(plan)      # fails while the run is being captured
        F.fastged_plan_run(plan)          # captured again, now complete
        c, m, n = F._outputs(mm)
        F.fastged_plan_read(plan, c, m, n)
        F.fastged_plan_destroy(plan)
        for x, y in zip((c, m, n), ref):
            assert np.array_equal(x, y)


def test_timeout_returns_early_and_the_handle_recovers():
    big = W.config4(2, seed=9, n_range=(600, 640))
    small = W.config1(30)
    ref_big = gpu_run(big)
    with F.FastGED(big.cost) as g:
        F.fastged_set_timeout(g.h, 1)
        t = time.perf_counter()
        with pytest.raises(F.FastGEDError) as ei:
            g.run(big)
        assert ei.value.code == F.FASTGED_ERR_TIMEOUT
        assert time.perf_counter() - t < 5.0
        # the next call waits for the background batch, then runs normally
        assert_parity(small, g.run(small))
        F.fastged_set_timeout(g.h, 0)
        for x, y in zip(g.run(big), ref_big):
            assert np.array_equal(x, y)
        with pytest.raises(F.FastGEDError):
            F.fastged_set_timeout(g.h, -1)


def test_injected_admission_refusal_is_retried():
    w = W.config2(40)
    ref = gpu_run(w)
    mm = F.marshal(w)
    F.fastged_inject_fault(F.FASTGED_INJECT_ADMISSION, 1)
    srv = F.Server(w.cost, F.serve_config(lanes=2, min_batch_pairs=8))
    for p in range(w.n_pairs):
        assert srv.submit(mm, w.pairs[p][0], w.pairs[p][1], w.K, p) == F.FASTGED_OK
    got = {}
    deadline = time.time() + 120
    while len(got) < w.n_pairs and time.time() < deadline:
        for r in srv.poll(timeout_ms=50):
            got[int(r[0])] = r
    st = srv.stats()
    srv.close()
    assert len(got) == w.n_pairs and st["admission_waits"] >= 1 and st["failed"] == 0
    assert np.array_equal(np.array([got[p][2] for p in range(w.n_pairs)], np.int32), ref[0])


def test_fault_arguments_are_checked():
    for kind, cd in ((3, 1), (-1, 1), (0, -2)):
        with pytest.raises(F.FastGEDError):
            F.fastged_inject_fault(kind, cd)


def test_injected_launch_failure_while_serving():
    """A served batch whose launch fails reports the error for each of its queries; the
    server keeps serving, and the failed queries succeed when submitted again."""
    w = W.config2(40)
    ref = gpu_run(w)
    mm = F.marshal(w)
    srv = F.Server(w.cost, F.serve_config(lanes=2, min_batch_pairs=8))
    F.fastged_inject_fault(F.FASTGED_INJECT_LAUNCH, 1)

    def serve(tags):
        for t in tags:
            p = t % 1000
            assert srv.submit(mm, w.pairs[p][0], w.pairs[p][1], w.K, t) == F.FASTGED_OK
        got, deadline = {}, time.time() + 120
        while len(got) < len(tags) and time.time() < deadline:
            for r in srv.poll(timeout_ms=50):
                got[int(r[0])] = r
        assert len(got) == len(tags)
        return got

    got = serve(list(range(w.n_pairs)))
    failed = [t for t, r in got.items() if r[1] != F.FASTGED_OK]
    assert failed and all(got[t][1] == F.FASTGED_ERR_CUDA for t in failed)
    for t, r in got.items():
        if r[1] == F.FASTGED_OK:
            assert r[2] == ref[0][t]
    again = serve([1000 + t for t in failed])
    for t, r in again.items():
        assert r[1] == F.FASTGED_OK and r[2] == ref[0][t - 1000]
    st = srv.stats()
    srv.close()
    assert st["failed"] == len(failed)
