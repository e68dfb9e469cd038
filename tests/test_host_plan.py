"""Device-resident plans and the binding's loading rule, on the CPU.

The host runtime is built against fakes of the CUDA calls (tests/host_probe.py); the fakes count
the K-Best launches and report a set elapsed time per team shape. A plan must count its
launches the way the benchmark reports them (one packing launch, then one K-Best launch per
size class, or per pair in the plain form), keep that count across replays, read back the
kernel time of its last run, and refuse null arguments. The Python binding must refuse to run
when the library is missing instead of falling back to anything else.
"""
import ctypes
import os

import numpy as np
import pytest

from host_probe import load
from paper_2605_00830_gb300 import fastged as F
from paper_2605_00830_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    L = load()
    L.fastged_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.fastged_plan_read.argtypes = [ctypes.c_void_p] * 4
    L.fastged_plan_kernel_ms.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]
    yield L
    L.fake_set_shape_ms(0, 0, 0.0)


def _handle(L, cost):
    h = ctypes.c_void_p()
    assert L.fastged_create(ctypes.byref(F.CostModel(*cost)), ctypes.byref(h)) == F.FASTGED_OK
    return h.value


@pytest.mark.parametrize("form,graph", [(F.FASTGED_FORM_BATCHED, 1), (F.FASTGED_FORM_BATCHED, 0),
                                        (F.FASTGED_FORM_PLAIN, 1)])
def test_plan_launch_count_and_replay(lib, form, graph):
    w = W.config2(500)
    mm = F.Marshalled(w.graphs, w.pairs)
    h = _handle(lib, w.cost)
    p = ctypes.c_void_p()
    o = F.make_options(form=form, use_cuda_graph=graph, block_threads=128)
    assert lib.fastged_plan_create(h, ctypes.byref(mm.pl), w.K, ctypes.byref(o),
                                   ctypes.byref(p)) == F.FASTGED_OK
    lib.fake_set_shape_ms(0, 0, 0.0)
    lib.fake_set_shape_ms(128, 1, 2.5)
    n_classes = None
    for run in range(3):
        n0 = lib.fake_kbest_launches()
        assert lib.fastged_plan_run(p, None) == F.FASTGED_OK
        launched = lib.fake_kbest_launches() - n0
        st = F.PlanStats()
        assert lib.fastged_plan_info(p, ctypes.byref(st)) == F.FASTGED_OK
        n_classes = st.n_classes
        per_run = w.n_pairs if form == F.FASTGED_FORM_PLAIN else n_classes
        # graph replay: the launches happen once, at capture; after that the graph runs
        replayed = form != F.FASTGED_FORM_PLAIN and graph == 1
        assert launched == (per_run if (run == 0 or not replayed) else 0)
        assert st.launches_per_run == 1 + per_run
        assert st.graph_replay == int(replayed)
        assert st.n_pairs == w.n_pairs
        ms = ctypes.c_float()
        assert lib.fastged_plan_kernel_ms(p, ctypes.byref(ms)) == F.FASTGED_OK
    assert n_classes == 2
    cost, maps, nev = F._outputs(mm)
    cost[:] = -1
    assert lib.fastged_plan_read(p, cost.ctypes.data, maps.ctypes.data,
                                 nev.ctypes.data) == F.FASTGED_OK
    assert (cost == 0).all()          # the fakes deliver zeros
    lib.fastged_plan_destroy(p)
    lib.fastged_destroy(h)


def test_plan_null_arguments(lib):
    assert lib.fastged_plan_run(None, None) == F.FASTGED_ERR_INVALID_ARG
    assert lib.fastged_plan_read(None, None, None, None) == F.FASTGED_ERR_INVALID_ARG
    ms = ctypes.c_float()
    assert lib.fastged_plan_kernel_ms(None, ctypes.byref(ms)) == F.FASTGED_ERR_INVALID_ARG
    assert lib.fastged_plan_info(None, None) == F.FASTGED_ERR_INVALID_ARG
    lib.fastged_plan_destroy(None)
    w = W.config2(4)
    mm = F.Marshalled(w.graphs, w.pairs)
    p = ctypes.c_void_p()
    assert lib.fastged_plan_create(None, ctypes.byref(mm.pl), 8, None,
                                   ctypes.byref(p)) == F.FASTGED_ERR_INVALID_ARG


def test_binding_refuses_to_run_without_the_library():
    missing = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host", "_build",
                           "no_such_dir", "libfastged_missing.so")
    with pytest.raises(RuntimeError, match="not built"):
        F.load(missing, build_if_missing=False)
