"""The FP32-bulk pair formula refines the hardware reciprocal square root
with one Newton-Raphson step (a textbook method).  Checked on the GPU
against 1/sqrt computed in FP64 and rounded: at most 1 ulp over 2^24
log-spaced arguments, and no worse than the unrefined seed."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_refined_rsqrt_within_one_ulp(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    assert os.path.exists(nvcc), "the GPU tests need the CUDA toolkit"
    exe = str(tmp_path / "rsqrt_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    os.path.join(HERE, "rsqrt_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    refined, seed = (float(v) for v in out.stdout.split())
    assert refined <= 1.0, (refined, seed)
    assert refined <= seed, (refined, seed)
