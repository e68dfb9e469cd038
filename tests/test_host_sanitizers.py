"""The host runtime under ThreadSanitizer and AddressSanitizer + UndefinedBehaviorSanitizer.

tests/host/sanitize_driver.cpp drives the runtime's host code (fastged_runtime.cu, serve.cu)
through the public C API against the fakes of tests/host/fake_cuda.cpp: batches from two
handles on two threads at once (the shared host thread pool and its polling workers), invalid
batches, the degree order, an autotuned plan, and the server fed by three submitting threads
while the main thread polls. Built with each sanitizer, it must exit 0 with no report; a
sanitizer report stops it at once. The only suppression is NVTX's own lazy initialisation
(tests/host/tsan.supp), which is toolkit header code.
"""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HOST = os.path.join(HERE, "host")
CSRC = os.path.join(ROOT, "paper_2605_00830_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = [os.path.join(CSRC, "fastged_runtime.cu"), os.path.join(CSRC, "serve.cu")]
DRIVER = [os.path.join(HOST, "fake_cuda.cpp"), os.path.join(HOST, "sanitize_driver.cpp")]
BUILD = os.path.join(HOST, "_build")

VARIANTS = {
    "tsan": (["-fsanitize=thread"],
             {"TSAN_OPTIONS": f"halt_on_error=1 suppressions={os.path.join(HOST, 'tsan.supp')}"}),
    "asan": (["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
              "-fno-omit-frame-pointer"],
             {"ASAN_OPTIONS": "detect_leaks=1:halt_on_error=1",
              "UBSAN_OPTIONS": "print_stacktrace=1:halt_on_error=1"}),
}


def _build(name, flags):
    exe = os.path.join(BUILD, f"sanitize_driver_{name}")
    deps = SOURCES + DRIVER + [os.path.join(CSRC, f) for f in os.listdir(CSRC)
                               if f.endswith((".h", ".cuh"))]
    deps += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    if os.path.exists(exe) and all(os.path.getmtime(d) <= os.path.getmtime(exe) for d in deps):
        return exe
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    os.makedirs(BUILD, exist_ok=True)
    tmp = exe + f".tmp{os.getpid()}"
    cmd = (["g++", "-std=c++17", "-O1", "-g"] + flags +
           ["-I", cuda_inc, "-I", INCLUDE, "-I", CSRC, "-x", "c++"] + SOURCES + ["-x", "c++"] +
           DRIVER + ["-o", tmp, "-lpthread", "-ldl"])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and "unrecognized" in r.stderr:
        pytest.skip(f"{name} not supported by this compiler")
    assert r.returncode == 0, r.stderr
    os.replace(tmp, exe)
    return exe


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_host_runtime_is_clean_under_sanitizer(name):
    flags, env = VARIANTS[name]
    exe = _build(name, flags)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600, cwd=BUILD,
                       env=dict(os.environ, **env))
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "host runtime driver: 300 served, 0 failures" in r.stdout
    for marker in ("WARNING: ThreadSanitizer", "ERROR: AddressSanitizer", "runtime error:",
                   "ERROR: LeakSanitizer"):
        assert marker not in out, out[-4000:]
