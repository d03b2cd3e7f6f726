"""The FP32-bulk form widens its FP32 partial sums to FP64 with integer
operations instead of the hardware conversion (which issues on the FP64
pipe).  The same header function, compiled for the host, must agree with
the compiler's float -> double conversion bit for bit on every binary32
value."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_widen_is_exact_for_every_float(tmp_path):
    inc = cuda_include()
    if inc is None:
        pytest.skip("needs the CUDA headers")
    exe = str(tmp_path / "widen_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-x", "c++", "-I", inc,
                    os.path.join(HERE, "widen_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip().splitlines()[-1] == "0"
