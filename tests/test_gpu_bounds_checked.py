"""The bounds-checked build (-DFASTGED_BOUNDS_CHECK) on the GPU.

Every index of the K-Best kernels is checked there against the array it addresses; a
violation sets a bit of the batch's status word and sends the access to the array's first
element instead, so nothing leaves a buffer, and the call then fails with FASTGED_ERR_CUDA.
Here the checked library solves a mix of batches that reaches every kernel family (one-warp
teams, one-CTA teams with shared and global regions, cluster teams, the exact-selection
fallbacks, variant B, label planes, the allocation-free entry point) and must report no
violation and agree with the oracle; and with the selection list declared shorter than the
kernels use (its buffer keeps its real size), each family must report the violation.
"""
import os

import numpy as np
import pytest

from paper_2605_00830_gb300 import build as B
from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W
from parity_util import assert_parity, gpu_run, single

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def checked_library():
    """The checked build, loaded in place of the normal one for this module's tests."""
    path = B.build(checked=True)
    saved = F._LIB
    F._LIB = F.load(path)
    yield F._LIB
    F._LIB = saved


def _labelled(n_pairs, seed, max_label):
    w = W.config2(n_pairs, seed=seed)
    st = W.Stream(seed, 99)
    for g in w.graphs:
        g.elabel = st.randint(0, max_label, g.m).astype(np.int32)
    return w


CASES = {
    "tiny_warp": lambda: (W.config1(), {}),
    "molecule_warp": lambda: (W.config2(300), {}),
    "molecule_cta": lambda: (W.config2(300), {"team": F.FASTGED_TEAM_CTA}),
    "molecule_fallback": lambda: (W.config2(60), {"hist_window": 2}),
    "molecule_fallback_cta": lambda: (W.config2(60), {"hist_window": 2,
                                                       "team": F.FASTGED_TEAM_CTA}),
    "eight_planes": lambda: (_labelled(40, 17, 6), {}),
    "dense": lambda: (W.subset(W.config3(6), range(6)), {}),
    "variant_b": lambda: (W.config1(80), {"variant": 1}),
    "degree_order": lambda: (W.config2(80), {"vertex_order": F.FASTGED_ORDER_DEGREE}),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_checked_build_matches_oracle(name):
    w, opts = CASES[name]()
    gpu = gpu_run(w, **opts)
    assert_parity(w, gpu, variant=opts.get("variant", 0),
                  order=1 if opts.get("vertex_order") else 0)


def test_checked_build_large_and_cluster_pairs(monkeypatch):
    """16-bit maps with 4 to 16 words on one-CTA and cluster teams, and a wide beam."""
    w = W.config4(3, seed=41, n_range=(150, 320))
    w.K = 48
    assert_parity(w, gpu_run(w))
    monkeypatch.setenv("FASTGED_CLUSTER", "8")
    w2 = W.config4(2, seed=43, n_range=(260, 700))
    w2.K = 40
    assert_parity(w2, gpu_run(w2))
    st = W.Stream(12, 1)
    wb = single([(W.erdos_renyi(st, 12, 0.3, 4), W.erdos_renyi(st, 13, 0.3, 4))],
                W.UNIT_COSTS, 100000)
    assert_parity(wb, gpu_run(wb, K=100000), K=100000)


@pytest.mark.parametrize("team", [F.FASTGED_TEAM_AUTO, F.FASTGED_TEAM_CTA])
def test_checked_build_reports_an_index_past_its_array(monkeypatch, team):
    """The selection list declared four entries long: the placement's writes past it are
    reported (and redirected), the call fails, and the next call is exact again."""
    w = W.config2(40)
    monkeypatch.setenv("FASTGED_CHECK_SHRINK_SEL", "1")
    with pytest.raises(F.FastGEDError) as ei:
        gpu_run(w, team=team)
    assert ei.value.code == F.FASTGED_ERR_CUDA and "bounds check" in str(ei.value)
    monkeypatch.delenv("FASTGED_CHECK_SHRINK_SEL")
    assert_parity(w, gpu_run(w, team=team))


def test_checked_build_allocation_free_entry_point():
    torch = pytest.importorskip("torch")
    from test_zz_no_alloc import _device_batch, _run_noalloc
    w = W.config2(50)
    with F.FastGED(w.cost) as g:
        ref = g.run(w)
    b, keep, mm = _device_batch(w, torch)
    rc, c, m, n = _run_noalloc(w, b, mm, torch)
    assert rc == F.FASTGED_OK
    for x, y in zip((c, m, n), ref):
        assert np.array_equal(x, y)
