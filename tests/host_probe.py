"""Builds the host runtime (fastged_runtime.cu, serve.cu: no device code) with g++ against
the fakes in tests/host/ into one test library, for the CPU tests of the host logic."""
import ctypes
import os
import subprocess

import pytest

from paper_2605_00830_gb300 import fastged as F

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HOST = os.path.join(HERE, "host")
CSRC = os.path.join(ROOT, "paper_2605_00830_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
RUNTIME = [os.path.join(CSRC, "fastged_runtime.cu"), os.path.join(CSRC, "serve.cu")]
SOURCES = [os.path.join(HOST, "fake_cuda.cpp"), os.path.join(HOST, "flatten_probe.cpp")]
LIB = os.path.join(HOST, "_build", "libhost_probe.so")


def build() -> str:
    deps = RUNTIME + SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC)
                                if f.endswith((".h", ".cuh"))]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    if os.path.exists(LIB) and all(os.path.getmtime(d) <= os.path.getmtime(LIB) for d in deps):
        return LIB
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    # -Bsymbolic: the runtime's calls bind to the fakes in this library even when a real
    # CUDA runtime is loaded globally in the process (torch)
    cmd = (["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-Wl,-Bsymbolic",
            "-I", cuda_inc, "-I", INCLUDE, "-I", CSRC, "-x", "c++"] + RUNTIME + ["-x", "c++"]
           + SOURCES + ["-o", tmp, "-lpthread", "-ldl"])
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    os.replace(tmp, LIB)
    return LIB


def load():
    """The test library, with argument types for every entry point the CPU tests call."""
    L = ctypes.CDLL(build())
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    L.probe_flatten.argtypes = [vp, i32, vp, vp]
    L.probe_error.restype = ctypes.c_char_p
    L.probe_staging.restype = vp
    L.probe_batch.argtypes = [vp]
    L.probe_class.argtypes = [ctypes.c_int, vp]
    L.probe_class_order.argtypes = [ctypes.c_int, vp]
    for name in ("probe_meta", "probe_map_off", "probe_perm"):
        getattr(L, name).argtypes = [vp]
    L.fake_set_free_bytes.argtypes = [ctypes.c_ulonglong]
    L.fake_fail_pinned_alloc.argtypes = [ctypes.c_int]
    L.fake_fail_device_alloc.argtypes = [ctypes.c_int]
    L.fake_set_host_fn_delay_us.argtypes = [ctypes.c_int]
    L.fake_max_pack_graphs.argtypes = [ctypes.c_int]
    L.fake_fail_launches.argtypes = [ctypes.c_int]
    L.fake_set_shape_ms.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_float]
    L.fake_kbest_launches.restype = ctypes.c_longlong
    L.fake_events_busy_for_ms.argtypes = [ctypes.c_int]
    L.fastged_create.argtypes = [ctypes.POINTER(F.CostModel), ctypes.POINTER(vp)]
    L.fastged_destroy.argtypes = [vp]
    L.fastged_destroy.restype = None
    L.fastged_batch_ex.argtypes = [vp, ctypes.POINTER(F.PairList), i32, ctypes.POINTER(F.Options),
                                   vp, vp, vp]
    L.fastged_set_timeout.argtypes = [vp, i32]
    L.fastged_plan_create.argtypes = [vp, ctypes.POINTER(F.PairList), i32,
                                      ctypes.POINTER(F.Options), ctypes.POINTER(vp)]
    L.fastged_plan_info.argtypes = [vp, ctypes.POINTER(F.PlanStats)]
    L.fastged_plan_destroy.argtypes = [vp]
    L.fastged_plan_destroy.restype = None
    L.fastged_autotune_clear.restype = None
    L.fastged_inject_fault.argtypes = [i32, i32]
    L.fastged_last_error.argtypes = [vp]
    L.fastged_last_error.restype = ctypes.c_char_p
    L.fastged_serve_start.argtypes = [ctypes.POINTER(F.CostModel), ctypes.POINTER(F.ServeConfig),
                                      ctypes.POINTER(vp)]
    L.fastged_serve_submit.argtypes = [vp, vp, vp, i32, ctypes.c_uint64]
    L.fastged_serve_poll.argtypes = [vp, ctypes.POINTER(F.ServeResult), i32, vp, ctypes.c_int64,
                                     i32]
    L.fastged_serve_get_stats.argtypes = [vp, ctypes.POINTER(F.ServeStats)]
    L.fastged_serve_cancel.argtypes = [vp, ctypes.c_uint64]
    for name in ("fastged_serve_stop", "fastged_serve_destroy"):
        getattr(L, name).argtypes = [vp]
        getattr(L, name).restype = None
    return L
