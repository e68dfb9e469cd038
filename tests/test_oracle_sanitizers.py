"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a driver runs every
oracle entry point on seeded small graphs (including empty ones); the sanitized build must
run clean and print exactly what the plain build prints."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(ROOT, "oracle", "fastged_oracle.c"), os.path.join(HERE, "oracle_driver.c")]


def _build_and_run(tmp_path, name, flags, env=None):
    exe = str(tmp_path / name)
    subprocess.check_call(["gcc", "-std=c99", "-O1", "-g", *flags, *SRC, "-o", exe])
    return subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)


def test_oracle_runs_clean_under_asan_and_ubsan(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    plain = _build_and_run(tmp_path, "plain", [])
    assert plain.returncode == 0, plain.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1")
    try:
        san = _build_and_run(tmp_path, "san", ["-fsanitize=address,undefined",
                                               "-fno-sanitize-recover=all",
                                               "-fno-omit-frame-pointer"], env=env)
    except subprocess.CalledProcessError:
        pytest.skip("the sanitizer runtimes are not available")
    assert san.returncode == 0, san.stderr[-4000:]
    assert "runtime error" not in san.stderr and "ERROR: AddressSanitizer" not in san.stderr
    assert san.stdout == plain.stdout
    assert plain.stdout.count("case ") == 80
