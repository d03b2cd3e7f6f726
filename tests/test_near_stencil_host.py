"""The lattice kernel's exact near pairs at theta = 0.5 run over a stencil
fixed at compile time (16 pairs (d, -d), constant coefficients).  Compiled
for the host, it must be exactly the plan's near set for every parity class,
with 1/|d| and 1/|d|^3 to an ulp."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2412_15518_gb300", "csrc")


def cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_near_stencil_matches_the_plan(tmp_path):
    inc = cuda_include()
    if inc is None:
        pytest.skip("needs the CUDA headers")
    exe = str(tmp_path / "near_stencil_check")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", inc, "-x", "c++",
                    os.path.join(HERE, "near_stencil_check.cpp"),
                    os.path.join(CSRC, "tree_host.cpp"), os.path.join(CSRC, "flops.cpp"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip().splitlines()[-1] == "0"
