"""The bounds-checked variant of the K-Best kernels compiles (sm_103a, no GPU needed): the
instances for unlabelled edges of every kernel family, with -DFASTGED_BOUNDS_CHECK. The
GPU side of the checked build is tests/test_gpu_bounds_checked.py."""
import os
import shutil
import subprocess

import pytest

from paper_2605_00830_gb300 import build as B


def test_checked_kernels_compile(tmp_path):
    nvcc = shutil.which(B.NVCC) or (B.NVCC if os.path.exists(B.NVCC) else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path / "kbest_b0_checked.o")
    # ptxas without optimisation: this only proves that the checked instances compile
    cmd = [nvcc] + B.ARCH + ["-O1", "-Xptxas", "-O0", "-std=c++17", "-Xcompiler", "-fPIC",
                             "-I", B.INCLUDE, "-I", B.CSRC, "-DFASTGED_BOUNDS_CHECK", "-c",
                             os.path.join(B.CSRC, "kbest_b0.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert os.path.getsize(out) > 0
