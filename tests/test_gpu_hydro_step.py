"""GPU coupled time step (ot_hydro_rk3_step) against the oracle
(oracle/hydro_step.py).

Without gravity both sides evaluate the same operations in the same order
(the hydro right-hand side and the Runge-Kutta combinations, FP64, no fused
multiply-adds): the step agrees bit for bit.  With gravity each stage's g
comes from the GPU's FMM on one side and the oracle's on the other, which
agree to about 1e-15; the step then agrees to a tolerance of 1e-9 of each
field's magnitude (a PPM limiter decision can in principle turn on such a
difference; none does on these inputs).
"""
import numpy as np
import pytest
import torch

from oracle import hydro_step as S
from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def fmm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_15518_gb300 import fmm as F
    return F


def gpu_step(fmm, lv, u, dt, gravity):
    tree = fmm.Tree(lv)
    ug = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    tree.hydro_step(ug, dt, GAMMA, gravity=gravity)
    torch.cuda.synchronize()
    status = tree.info()["device_status"]
    tree.close()
    return ug.cpu().numpy(), status


CASES = {
    "uniform_l2": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=21)))(I.uniform_leaves(2, seed=4)),
    "binary_l1_l2": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=22)))(
        I.amr_leaves(2, 5e-4, I.BINARY, lmin=1)),
    "binary_l1_l3": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=23)))(I.amr_leaves(3, 2e-4, I.BINARY)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_step_without_gravity_matches_oracle_bit_for_bit(fmm, case):
    lv, u = CASES[case]()
    got, status = gpu_step(fmm, lv, u, 1e-3, False)
    want = S.rk3_step(lv, u, 1e-3, GAMMA, gravity=False)
    assert status == 0
    diff = int((got != want).sum())
    print(f"step {case}: {got.size} values, {diff} differ")
    assert diff == 0
    assert np.abs(got - u).max() > 0.0


@pytest.mark.parametrize("case", ["uniform_l2", "binary_l1_l3"])
def test_step_with_gravity_matches_oracle(fmm, case):
    lv, u = CASES[case]()
    got, status = gpu_step(fmm, lv, u, 1e-3, True)
    want = S.rk3_step(lv, u, 1e-3, GAMMA, gravity=True)
    assert status == 0
    scale = np.abs(want).max(axis=(0, 2))
    err = np.abs(got - want).max(axis=(0, 2)) / scale
    print(f"step with gravity {case}: relative error per field {err}")
    assert np.all(err < 1e-9)
    # gravity does act on the step
    nograv = S.rk3_step(lv, u, 1e-3, GAMMA, gravity=False)
    assert np.abs(want - nograv).max() > 1e-9 * np.abs(want).max()


def test_step_rejects_bad_arguments(fmm):
    lv = I.uniform_leaves(1)
    tree = fmm.Tree(lv)
    u = torch.ones((lv.shape[0], 5, 512), dtype=torch.float64, device="cuda")
    for dt, gamma, grav in ((float("nan"), GAMMA, 1), (1e-3, 1.0, 1), (1e-3, GAMMA, 2)):
        with pytest.raises(fmm.OTError) as e:
            fmm.ot_hydro_rk3_step(tree.handle, u, dt, gamma, grav)
        assert e.value.code == -1
    with pytest.raises(fmm.OTError):
        fmm.ot_hydro_rk3_step(tree.handle, u, 1e-3, GAMMA, 1, fmm.make_opts(theta=0.1))
    tree.close()
