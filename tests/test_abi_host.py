"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/octofmm.h declares, validates trees and counts interactions on the
host (device -1, no CUDA call) exactly as the oracle does."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2412_15518_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fmm():
    from paper_2412_15518_gb300 import fmm as F
    return F


def declared_functions():
    src = open(os.path.join(ROOT, "include", "octofmm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(ot_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(fmm):
    names = declared_functions()
    assert "ot_solve_gravity" in names and "ot_gravity_backward" in names
    lib = ctypes.CDLL(fmm.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(fmm.EXPORTS) == names


def test_error_strings(fmm):
    assert fmm.ot_error_string(0) == "ok"
    for code in range(-1, -11, -1):
        assert fmm.ot_error_string(code) != "unknown error"


@pytest.mark.parametrize("name", ["sphere_l1", "binary_l3"])
def test_uniform_counts(fmm, name):
    lv, _ = I.workload(name)
    c = fmm.host_only_counts(lv)
    want = {"sphere_l1": (959280, 114744), "binary_l3": (64121280, 8120568)}[name]
    assert (c["n_m2l"], c["n_p2p"], c["n_seam"]) == (*want, 0)


def test_amr_counts_match_oracle(fmm):
    lv = I.amr_leaves(3, 2e-4, I.BINARY)
    rho = I.density(lv, I.BINARY, seed=5)
    c = fmm.host_only_counts(lv)
    _, _, oc = O.solve(lv, rho, return_counts=True)
    assert (c["n_m2l"], c["n_p2p"], c["n_seam"]) == (oc["m2l"], oc["p2p"], oc["seam"])
    assert c["n_leaf_nodes"] == list(np.bincount(lv[:, 0], minlength=c["n_levels"]))


def test_invalid_trees(fmm):
    good = I.uniform_leaves(1)
    with pytest.raises(fmm.OTError) as e:
        fmm.host_only_counts(good[1:])
    assert e.value.code == -2
    with pytest.raises(fmm.OTError) as e:
        fmm.host_only_counts(np.concatenate([good, good[:1]]))
    assert e.value.code == -2
    with pytest.raises(fmm.OTError) as e:
        fmm.host_only_counts(np.array([[1, 2, 0, 0]], np.int32))
    assert e.value.code == -2
    with pytest.raises(fmm.OTError) as e:
        fmm.host_only_counts(np.zeros((0, 4), np.int32))
    assert e.value.code == -1


def test_unbalanced_tree_rejected(fmm):
    # level-1 octants, one refined twice in its corner next to the others
    lv = [[1, x, y, z] for z in range(2) for y in range(2) for x in range(2)][1:]
    lv += [[2, x, y, z] for z in range(2) for y in range(2) for x in range(2)][:-1]
    lv += [[3, x, y, z] for z in range(2, 4) for y in range(2, 4) for x in range(2, 4)]
    lv = np.array(lv, np.int32)
    assert O.check_tree(lv) == 0          # complete, so the oracle accepts it
    assert not I.is_balanced(lv)
    with pytest.raises(fmm.OTError) as e:
        fmm.host_only_counts(lv)
    assert e.value.code == -3
    fmm.host_only_counts(I.balance(lv))


def test_solves_refused_without_device(fmm):
    h = fmm.ot_build_tree(I.uniform_leaves(1), -1)
    try:
        with pytest.raises(fmm.OTError) as e:
            fmm._check(fmm._lib.ot_solve_gravity(fmm._P(h), None, None, None, None, None), "x")
        assert e.value.code == -1
    finally:
        fmm.ot_destroy_tree(h)
