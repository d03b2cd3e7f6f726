"""The GPU library's pair formulas, compiled for the host, against the
oracle's unpacked formulation.

`pair_check.cpp` evaluates, in FP64, the forward cell-to-cell interaction
exactly as the general kernel assembles it (the compact contractions of
`pair_formula.cuh`, the Kronecker parts of L2 and L3 restored from the
traces, the correction's target term from the quartic pair sum and the
target's octupole per unit mass) and its reverse (`adjoint_pair.cuh`: both
roles and the R-gradient; in the kernel's cell units the target's quartic
sum is the forward pair's own, as the adjoint kernel takes it from the
forward pass).  The oracle forms every D tensor unpacked
(3^n entries) and sums plain index contractions.  Symmetric tensors travel
packed; an adjoint's packed entry is the value at each of its positions.
"""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
P2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
P3 = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2), (1, 1, 1), (1, 1, 2),
      (1, 2, 2), (2, 2, 2)]


def cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def full(p, ranks):
    f = np.zeros((3,) * ranks)
    for v, idx in zip(p, P2 if ranks == 2 else P3):
        for t in set(itertools.permutations(idx)):
            f[t] = v
    return f


@pytest.fixture(scope="module")
def pair_check(tmp_path_factory):
    inc = cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("pair") / "pair_check")
    subprocess.run(["g++", "-O1", "-std=c++17", "-Wno-unknown-pragmas", "-I", inc, "-x", "c++",
                    os.path.join(HERE, "pair_check.cpp"), "-o", exe], check=True)
    return exe


def random_cases(n, seed):
    rng = np.random.default_rng(seed)
    cases = []
    for t in range(n):
        XA = rng.uniform(0, 1, 3)
        XB = XA + rng.uniform(1.5, 3.0, 3) * rng.choice([-1, 1], 3)
        cases.append(dict(
            am=t % 2, G=rng.uniform(0.5, 2.0), XA=XA, XB=XB,
            mA=0.0 if t % 5 == 4 else rng.uniform(0.5, 1.5),   # zero-mass targets too
            M3A=0.1 * rng.standard_normal(10), mB=rng.uniform(0.5, 1.5),
            M2B=0.1 * rng.standard_normal(6), M3B=0.1 * rng.standard_normal(10),
            E0=rng.standard_normal(), E1=rng.standard_normal(3), E2=rng.standard_normal(6),
            E3=rng.standard_normal(10), a=rng.standard_normal(3)))
    return cases


def run(exe, cases):
    keys = ["XA", "XB", "mA", "M3A", "mB", "M2B", "M3B", "E0", "E1", "E2", "E3", "a"]
    lines = []
    for c in cases:
        vals = [c["G"]] + [float(v) for k in keys for v in np.atleast_1d(c[k])]
        lines.append(str(c["am"]) + " " + " ".join(repr(v) for v in vals))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         timeout=60, check=True).stdout.split("\n")
    return [np.array([float(x) for x in ln.split()]) for ln in out[:len(cases)]]


def moments(c):
    momA = np.concatenate([[c["mA"]], c["XA"], np.zeros(9), full(c["M3A"], 3).reshape(-1)])
    momB = np.concatenate([[c["mB"]], c["XB"], full(c["M2B"], 2).reshape(-1),
                           full(c["M3B"], 3).reshape(-1)])
    return momA, momB


def test_forward_pair_matches_the_oracle(pair_check):
    cases = random_cases(40, 3)
    worst = 0.0
    for c, h in zip(cases, run(pair_check, cases)):
        momA, momB = moments(c)
        o = O.m2l(momA, momB, G=c["G"], am_correction=bool(c["am"]))
        oL2, oL3 = o[4:13].reshape(3, 3), o[13:40].reshape(3, 3, 3)
        want = np.concatenate([o[0:4], [oL2[i] for i in P2], [oL3[i] for i in P3], o[40:43]])
        worst = max(worst, np.abs(h[:23] - want).max() / np.abs(want).max())
    assert worst < 1e-13, worst


def test_split_pair_matches_the_oracle(pair_check):
    """The FP32-bulk form's split pair (monopole part in FP64, the source's
    quadrupole and octupole contractions in FP32): with both parts in double
    it is the same expansion as the oracle's to rounding (1e-13), so the
    split loses no term; with the FP32 part in float every component stays
    within 1e-6 of the expansion's largest entry, and the monopole-only
    components (L2, L3: no source multipole enters them at total order 3)
    stay FP64-exact (1e-13)."""
    cases = random_cases(40, 5)
    worst64 = worst32 = worst_mono = 0.0
    for c, h in zip(cases, run(pair_check, cases)):
        momA, momB = moments(c)
        o = O.m2l(momA, momB, G=c["G"], am_correction=bool(c["am"]))
        oL2, oL3 = o[4:13].reshape(3, 3), o[13:40].reshape(3, 3, 3)
        want = np.concatenate([o[0:4], [oL2[i] for i in P2], [oL3[i] for i in P3], o[40:43]])
        s64, s32 = h[54:77], h[77:100]
        scale = np.abs(want).max()
        worst64 = max(worst64, np.abs(s64 - want).max() / scale)
        worst32 = max(worst32, np.abs(s32 - want).max() / scale)
        worst_mono = max(worst_mono, np.abs(s32[4:20] - want[4:20]).max() / np.abs(want[4:20]).max())
    assert worst64 < 1e-13, worst64
    assert worst32 < 1e-6, worst32
    assert worst_mono < 1e-13, worst_mono


def test_reverse_pair_matches_the_oracle(pair_check):
    cases = random_cases(40, 4)
    worst = 0.0
    for c, h in zip(cases, run(pair_check, cases)):
        momA, momB = moments(c)
        Eb = np.concatenate([[c["E0"]], c["E1"], full(c["E2"], 2).reshape(-1),
                             full(c["E3"], 3).reshape(-1), c["a"]])
        oa, ob = O.m2l_reverse(momA, momB, Eb, G=c["G"], am_correction=bool(c["am"]))
        obM2, obM3 = ob[4:13].reshape(3, 3), ob[13:40].reshape(3, 3, 3)
        oaM3 = oa[13:40].reshape(3, 3, 3)
        # dJ/dmB, dJ/dM2B, dJ/dM3B, dJ/dmA, dJ/dM3A, dJ/dR (R = XA - XB)
        want = np.concatenate([[ob[0]], [obM2[i] for i in P2], [obM3[i] for i in P3], [oa[0]],
                               [oaM3[i] for i in P3], oa[1:4]])
        scale = max(np.abs(oa).max(), np.abs(ob).max())
        worst = max(worst, np.abs(h[23:54] - want).max() / scale)
        # the kernel's cell units (R, M2, M3 over h, h^2, h^3; adjoints pre-scaled)
        worst = max(worst, np.abs(h[100:131] - want).max() / scale)
        assert np.abs(oa[1:4] + ob[1:4]).max() <= 1e-12 * np.abs(oa[1:4]).max()  # R-gradient only
    assert worst < 1e-13, worst


def test_leaf_target_reverse_pair_matches_the_oracle(pair_check):
    """The reverse pair for a leaf target (the adjoint kernel's pass 1, which
    skips the target's E2, E3 and octupole): against the oracle's reverse with
    those set to zero."""
    cases = random_cases(40, 6)
    worst = 0.0
    for c, h in zip(cases, run(pair_check, cases)):
        c0 = dict(c, M3A=np.zeros(10), E2=np.zeros(6), E3=np.zeros(10))
        momA, momB = moments(c0)
        Eb = np.concatenate([[c0["E0"]], c0["E1"], np.zeros(9 + 27), c0["a"]])
        oa, ob = O.m2l_reverse(momA, momB, Eb, G=c["G"], am_correction=bool(c["am"]))
        obM2, obM3 = ob[4:13].reshape(3, 3), ob[13:40].reshape(3, 3, 3)
        want = np.concatenate([[ob[0]], [obM2[i] for i in P2], [obM3[i] for i in P3], oa[1:4]])
        worst = max(worst, np.abs(h[131:151] - want).max() / max(np.abs(oa).max(), np.abs(ob).max()))
    assert worst < 1e-13, worst
