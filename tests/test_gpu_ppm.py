"""GPU PPM reconstruction of the 26 directional cell values
(ot_ppm_reconstruct) against the oracle (oracle/ppm.py), element by element.

Both sides evaluate the same formulas operation by operation in FP64
without fused multiply-adds, so the limiter takes the same branch on both
and the values agree bit for bit: the comparison is exact equality.
"""
import numpy as np
import pytest
import torch

from oracle import ppm as P
from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fmm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_15518_gb300 import fmm as F
    return F


CASES = {
    # uniform level 1, shuffled leaf order, random fields (every limiter branch)
    "l1_random": lambda: (lambda lv: (lv, np.random.default_rng(3).standard_normal((lv.shape[0], 3, 512))))(
        I.uniform_leaves(1, seed=2)),
    # uniform level 2, the hydro fields of the binary
    "l2_hydro": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=1)))(I.uniform_leaves(2)),
    # uniform level 3 (the level-3 binary's tree), hydro fields
    "l3_hydro": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=2)))(I.uniform_leaves(3, seed=5)),
    # a lone root leaf: every ghost cell is clamped
    "root": lambda: (np.array([[0, 0, 0, 0]], np.int32),
                     np.random.default_rng(9).standard_normal((1, 2, 512))),
    # smooth data with plateaus: equal neighbours exercise the extremum test's ties
    "l1_plateaus": lambda: (lambda lv: (lv, np.round(I.hydro_fields(lv, seed=4), 2)))(I.uniform_leaves(1)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_ppm_matches_oracle_bit_for_bit(fmm, case):
    lv, u = CASES[case]()
    tree = fmm.Tree(lv)
    out = tree.ppm(torch.from_numpy(np.ascontiguousarray(u)).cuda())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = P.reconstruct(lv, u)
    diff = int((got != want).sum())
    print(f"ppm {case}: {got.size} values, {diff} differ, max |diff| {np.abs(got - want).max():.2e}")
    assert diff == 0
    tree.close()


def test_ppm_rejects_mixed_levels_and_bad_sizes(fmm):
    lv = I.amr_leaves(3, 2e-4, I.BINARY)
    tree = fmm.Tree(lv)
    u = torch.zeros((lv.shape[0], 1, 512), dtype=torch.float64, device="cuda")
    out = torch.empty((lv.shape[0], 1, 26, 512), dtype=torch.float64, device="cuda")
    with pytest.raises(fmm.OTError) as e:
        fmm.ot_ppm_reconstruct(tree.handle, u, out)
    assert e.value.code == -1
    tree.close()
    lv = I.uniform_leaves(1)
    tree = fmm.Tree(lv)
    with pytest.raises(fmm.OTError) as e:
        fmm._check(fmm._lib.ot_ppm_reconstruct(fmm._P(tree.handle), fmm._ptr(u), 0, fmm._ptr(out), None), "x")
    assert e.value.code == -1
    tree.close()
