"""The persistent launch's work items, built on the host (tree_host.cpp):
the grouped items that the FP64 and FP32-bulk forms run (a node's cells
regrouped by their numbers of pairs, every lane walking its own parity list)
cover exactly the pairs of the parity-class items that the other kernels
run, once each, and the adjoint's items of its two passes the partners
each pass reverses, every interior target in exactly one item that starts
its pass-2 range (where its octupole adjoint is formed), with every index in
bounds (items_check.cpp)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2412_15518_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "paper_2412_15518_gb300", "csrc")


def cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def items_check(tmp_path_factory):
    inc = cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("items") / "items_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wno-unknown-pragmas", "-I", inc,
                    "-I", os.path.join(HERE, "..", "include"),
                    os.path.join(HERE, "items_check.cpp"), os.path.join(SRC, "tree_host.cpp"),
                    os.path.join(SRC, "flops.cpp"), "-o", exe], check=True)
    return exe


TREES = {
    "amr_l3_seams": lambda: I.amr_leaves(3, 2e-4, I.BINARY),
    "amr_l2_ragged": lambda: I.amr_leaves(2, 5e-4, I.BINARY, lmin=1),
    "root_leaf": lambda: np.array([[0, 0, 0, 0]], np.int32),
    "uniform_l2": lambda: I.uniform_leaves(2, seed=1),
}


@pytest.mark.parametrize("tree", sorted(TREES))
@pytest.mark.parametrize("theta,chunk", [(0.5, 263), (0.5, 7), (0.35, 64), (0.7, 1000)])
def test_grouped_items_cover_the_same_pairs(items_check, tmp_path, tree, theta, chunk):
    path = tmp_path / "leaves.bin"
    np.asarray(TREES[tree](), np.int32).tofile(path)
    r = subprocess.run([items_check, str(path), str(theta), str(chunk)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    n_pairs = int(r.stdout.split()[1])
    assert n_pairs > 0
