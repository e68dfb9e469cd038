"""bench.py's output contract, on the CPU.

The benchmark's own logic (timing bookkeeping, the roofline, the e2e, plain-form, serving and
CPU-baseline legs, the clock sampling) runs with torch's CUDA calls and the binding's device
calls replaced by stand-ins that return fixed values, and a stand-in nvidia-smi; the test
checks that one JSON line comes out with every key of the contract and that the numbers
follow from the stand-ins' values. The reference arm (the oracle) runs as it is, on a small
sample. Nothing here measures anything.
"""
import json
import os
import stat
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMI_ROW = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Active"


@pytest.fixture()
def fake_smi(monkeypatch):
    d = os.path.join(ROOT, "tests", "_build", "fake_smi")
    os.makedirs(d, exist_ok=True)
    exe = os.path.join(d, "nvidia-smi")
    with open(exe, "w") as f:
        f.write(f"#!/bin/sh\nwhile true; do echo '{SMI_ROW}'; sleep 0.05; done\n")
    os.chmod(exe, os.stat(exe).st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])


def _stand_ins(monkeypatch):
    import torch
    from paper_2605_00830_gb300 import fastged as F

    class Event:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 4.0                         # ms per step

    class Stream:
        cuda_stream = 1234

    real_empty = torch.empty
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "Stream", Stream)
    monkeypatch.setattr(torch.cuda, "set_stream", lambda s: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: real_empty(16, dtype=torch.uint8))

    class Handle:
        def __init__(self, cost):
            self.h = 1

        def close(self):
            pass

    def plan_read(p, c, m, n):
        c[:] = 7
        n[:] = 5000

    def batch_ex(h, mm, K, o, c, m, n):
        c[:] = 7

    class Server:
        def __init__(self, cost, cfg=None):
            self.q = []

        def submit(self, mm, a, b, K, tag):
            self.q.append(tag)
            return 0

        def poll(self, timeout_ms=10):
            out = [(t, 0, 1, np.zeros(1, np.int32), 1, 3.0, 1.0) for t in self.q]
            self.q = []
            return out

        def stats(self):
            return {"batches": 2, "batched_pairs": 20}

        def close(self):
            pass

    info = {"n_pairs": 0, "n_classes": 2, "launches_per_run": 3, "graph_replay": 1,
            "input_bytes": 1000, "device_bytes": 3000, "output_bytes": 200,
            "block_threads": [128, 128], "grid": [912, 1064], "words": [1, 1],
            "smem_bytes": [1, 1]}
    for name, fn in (("load", lambda *a, **k: None), ("FastGED", Handle),
                     ("fastged_plan_create", lambda h, mm, K, o: "plan"),
                     ("fastged_plan_run", lambda p, s=None: None),
                     ("fastged_plan_kernel_ms", lambda p: 3.0),
                     ("fastged_plan_read", plan_read),
                     ("fastged_plan_info", lambda p: dict(info)),
                     ("fastged_plan_destroy", lambda p: None),
                     ("fastged_measure_int_peak",
                      lambda: {"lop3": 2.0e13, "iadd": 2.0e13, "popc": 5.0e12}),
                     ("fastged_batch_ex", batch_ex), ("Server", Server)):
        monkeypatch.setattr(F, name, fn)


def _run_bench(monkeypatch, capsys, argv):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    assert bench.main() == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_bench_line_has_every_contract_key(monkeypatch, capsys, fake_smi):
    _stand_ins(monkeypatch)
    d = _run_bench(monkeypatch, capsys, ["--steps", "3", "--warmup", "3", "--pairs", "400",
                                          "--cpu-sample", "64", "--plain-sample", "40",
                                          "--serve-window", "0.1", "--suite-cpu-seconds", "0.3"])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] >= 3
    assert d["unit"] == "pairs/s" and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["ms_per_step"] == pytest.approx(4.0)
    assert d["value"] == pytest.approx(400 / 4e-3)
    assert d["gpu_launches"] == 3 * 3 and d["dtype"] == "int32"
    assert "workload" in d["config"] and "l2" in d["config"]
    r = d["roofline"]
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(20.0)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert "traffic" in r                      # null away from the captured full-size batch
    e = d["e2e"]
    assert e["h2d_bytes_per_step"] == 1000 and e["d2h_bytes_per_step"] == 200
    assert e["unit"] == "pairs/s" and e["value"] > 0
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and "64" in c["sample"]
    assert d["cpu_baseline_1core"]["cores"] == 1
    assert d["clocks"]["sm_mhz"] == 2070.0 and d["clocks"]["reasons"] == ["sw_power_cap"]
    assert d["plain_form"]["sample_pairs"] == 40
    for leg in ("serve", "serve_sustained"):
        assert {"p50_ms", "p99_ms", "completed", "offered_rps", "by_shape"} <= set(d[leg])
        shapes = d[leg]["by_shape"]
        assert sum(v["n"] for v in shapes.values()) == d[leg]["completed"]
        assert "molecule" in shapes and shapes["molecule"]["p50_ms"] == pytest.approx(3.0)
    # the other workloads: configs 1, 3, 4, the wide beam and the size sweep, each with its
    # throughput, evaluation rate, ALU roofline, HBM roofline where the beam spills, and a
    # bounded (or skipped) oracle sample
    suite = d["suite"]
    assert {"config1", "dense", "large", "widebeam", "sizesweep_n50", "sizesweep_n950"} <= set(suite)
    for key, rec in suite.items():
        for k in ("workload", "value", "evals_per_s", "kernel_ms", "roofline", "cpu_baseline"):
            assert k in rec, (key, k)
        assert rec["roofline"]["bound"] == "alu" and rec["roofline"]["peak"] == pytest.approx(20.0)
        cb = rec["cpu_baseline"]
        assert cb["kind"] == "oracle" and (cb["value"] is None) == cb["sample"].startswith("skipped")
    assert "roofline_hbm" in suite["large"] and "roofline_hbm" in suite["widebeam"]
    assert suite["large"]["cpu_baseline"]["value"] is None
    assert "roofline_hbm" not in suite["config1"]


class _SetAttr:
    """monkeypatch's setattr, for the spawned ranks below (nothing is undone there)."""

    def setattr(self, obj, name, value):
        setattr(obj, name, value)


def _write_fake_smi():
    d = os.path.join(ROOT, "tests", "_build", "fake_smi")
    os.makedirs(d, exist_ok=True)
    exe = os.path.join(d, "nvidia-smi")
    with open(exe, "w") as f:
        f.write(f"#!/bin/sh\nwhile true; do echo '{SMI_ROW}'; sleep 0.05; done\n")
    os.chmod(exe, os.stat(exe).st_mode | stat.S_IXUSR)
    return d


def _bench_rank(rank, world, port, out_dir):
    import contextlib
    import io
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    os.environ["PATH"] = _write_fake_smi() + os.pathsep + os.environ["PATH"]
    sys.path.insert(0, ROOT)
    _stand_ins(_SetAttr())
    import bench
    sys.argv = ["bench.py", "--gpus", str(world), "--steps", "3", "--warmup", "3",
                "--pairs", "200", "--plain-sample", "20", "--serve-window", "0.1", "--no-suite"]
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"rc={rc}\n" + buf.getvalue())


def test_bench_under_two_ranks(tmp_path):
    """The torchrun path with two gloo ranks: rank 0 alone prints, value and e2e are the whole
    job's (both ranks' pairs over the slowest rank's time), and the oracle legs are left out."""
    mp = pytest.importorskip("torch.multiprocessing")
    port = 31500 + (os.getpid() % 2000)
    mp.spawn(_bench_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    out0 = open(tmp_path / "r0.txt").read().splitlines()
    out1 = open(tmp_path / "r1.txt").read().splitlines()
    assert out0[0] == "rc=0" and out1[0] == "rc=0"
    assert not [l for l in out1 if l.startswith("{")]
    lines = [l for l in out0 if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["scaling"] == "weak"
    assert d["value"] == pytest.approx(2 * 200 / 4e-3)
    assert d["ms_per_step"] == pytest.approx(4.0)
    assert d["e2e"]["value"] > 0 and "serve" in d and "plain_form" in d
    assert "cpu_baseline" not in d and "cpu_baseline_1core" not in d
    assert d["config"]["parallelism"] == "replicas2"


@pytest.mark.parametrize("workload,pairs", [("dense", 6), ("large", 2), ("sizesweep", 1)])
def test_other_workloads_keep_the_oracle_legs_bounded(monkeypatch, capsys, fake_smi,
                                                      workload, pairs):
    """On the slower batches the oracle legs stop at their time bound, or are skipped (with
    the reason) when one pair alone would take far longer."""
    _stand_ins(monkeypatch)
    d = _run_bench(monkeypatch, capsys, ["--workload", workload, "--pairs", str(pairs),
                                          "--steps", "3", "--warmup", "3", "--plain-sample", "2",
                                          "--serve-window", "0.05", "--cpu-seconds", "1",
                                          "--no-suite"])
    for key in ("cpu_baseline", "cpu_baseline_1core"):
        leg = d[key]
        if workload in ("large", "sizesweep"):
            assert leg["value"] is None and leg["sample"].startswith("skipped")
        else:
            assert leg["value"] > 0 and leg["sample"].startswith("first ")
    r = _run_bench(monkeypatch, capsys, ["--impl", "reference", "--workload", workload,
                                          "--pairs", str(pairs), "--steps", "1", "--warmup", "0",
                                          "--cpu-seconds", "1"])
    if workload in ("large", "sizesweep"):
        assert r == {"impl": "reference", "unavailable": r["unavailable"]}
        assert "skipped" in r["unavailable"]
    else:
        assert r["value"] > 0


def test_reference_arm_line(monkeypatch, capsys):
    d = _run_bench(monkeypatch, capsys, ["--impl", "reference", "--steps", "1", "--warmup", "0",
                                          "--pairs", "200", "--cpu-sample", "40"])
    assert d["impl"] == "reference" and d["unit"] == "pairs/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
