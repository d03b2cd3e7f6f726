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
    try:
        status = tree.info()["device_status"]
    except fmm.OTError as e:
        status = e.info["device_status"]
    tree.close()
    return ug.cpu().numpy(), status


def only_density_bit(fmm, status):
    """The binary's 1e-10 atmosphere next to the stars drives some stage
    densities below zero (this scheme has no positivity fix): the density
    bit may be set, nothing else."""
    return status & ~fmm.OT_STATUS_BAD_DENSITY == 0


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
    assert only_density_bit(fmm, status)
    diff = int((got != want).sum())
    print(f"step {case}: {got.size} values, {diff} differ")
    assert diff == 0
    assert np.abs(got - u).max() > 0.0


@pytest.mark.parametrize("case", ["uniform_l2", "binary_l1_l3"])
def test_step_with_gravity_matches_oracle(fmm, case):
    lv, u = CASES[case]()
    got, status = gpu_step(fmm, lv, u, 1e-3, True)
    want = S.rk3_step(lv, u, 1e-3, GAMMA, gravity=True)
    assert only_density_bit(fmm, status)
    scale = np.abs(want).max(axis=(0, 2))
    err = np.abs(got - want).max(axis=(0, 2)) / scale
    print(f"step with gravity {case}: relative error per field {err}")
    assert np.all(err < 1e-9)
    # gravity does act on the step
    nograv = S.rk3_step(lv, u, 1e-3, GAMMA, gravity=False)
    assert np.abs(want - nograv).max() > 1e-9 * np.abs(want).max()


def test_positive_state_keeps_the_status_word_clear(fmm):
    """A blob in a uniform gas (no near vacuum): every stage state stays
    physical and the status word stays clear."""
    lv = I.amr_leaves(2, 5e-4, I.BINARY, lmin=1)
    x = I.cell_centres(lv)
    r2 = ((x[..., 0] - 0.45) ** 2 + (x[..., 1] - 0.5) ** 2 + (x[..., 2] - 0.52) ** 2) / 0.0625
    b = np.maximum(1.0 - r2, 0.0) ** 4
    u = np.stack([1.0 + 0.5 * b, 0.3 * b, -0.2 * b, 0.1 * b, 1.5 + 0.8 * b], axis=1)
    got, status = gpu_step(fmm, lv, u, 1e-3, True)
    assert status == 0
    assert np.abs(got - S.rk3_step(lv, u, 1e-3, GAMMA, gravity=True)).max() < 1e-9 * np.abs(u).max()


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
