"""GPU tests of the C-ABI calls beside the solve itself.

* ot_compute_moments + ot_get_moments: the moments of every level against
  the oracle's level moments (the upward pass of Sec. 4.3.2), element by
  element.  Both sides are FP64 moment shifts of the same point masses,
  summed in different orders (the oracle's upward pass is itself pinned
  against moments taken directly from the points), so they agree to
  rounding relative to each group's natural scale: max m for m, the domain size for X, max m h^2 for
  M2 and max m h^3 for M3 (h = the level's cell side; |M2| <= 3/4 m h^2 and
  |M3| <= (3/4)^(3/2) m h^3 for points inside the cell): 1e-14.
* ot_set_launch_shape: a fixed shape keeps parity in every form, with items
  of up to 1000 stencil entries; the device status word latches a
  non-physical hydro state (made on the host: nothing faults), which
  ot_tree_info reports once.
* ot_alu_peaks: the measured CUDA-core peaks are positive and ordered.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P2 = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
P3 = [(0, 0, 0), (0, 0, 1), (0, 0, 2), (0, 1, 1), (0, 1, 2), (0, 2, 2), (1, 1, 1), (1, 1, 2),
      (1, 2, 2), (2, 2, 2)]


@pytest.fixture(scope="module")
def fmm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_15518_gb300 import fmm as F
    return F


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def packed_from_oracle(mom):
    """[n, 512, 40] oracle moments -> [n, 20, 512] packed (m, X, M2, M3)."""
    m2 = mom[..., 4:13].reshape(mom.shape[:2] + (3, 3))
    m3 = mom[..., 13:40].reshape(mom.shape[:2] + (3, 3, 3))
    cols = [mom[..., 0]] + [mom[..., 1 + a] for a in range(3)]
    cols += [m2[..., i, j] for i, j in P2] + [m3[..., i, j, k] for i, j, k in P3]
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("case", ["binary_l3", "amr"])
def test_moments_of_every_level_match_the_oracle(fmm, case):
    if case == "amr":
        lv = I.amr_leaves(4, 5e-5, I.BINARY)
        rho = I.density(lv, I.BINARY, seed=7)
        origin, size = (0.25, -0.5, 1.0), 2.0
    else:
        lv, rho = I.workload("binary_l3")
        origin, size = (0.0, 0.0, 0.0), 1.0
    tree = fmm.Tree(lv, origin=origin, size=size)
    r = torch.from_numpy(rho).cuda()
    # a solve of the wide FP32 form first: its upward pass differs, and
    # ot_compute_moments must replace its result by the FP64 moments
    tree.solve(r, precision=fmm.OT_PRECISION_FP32_WIDE)
    tree.compute_moments(r)
    nl = tree.info()["n_levels"]
    for L in range(nl):
        xyz, mom = tree.moments(L)
        torch.cuda.synchronize()
        oxyz, omom = O.level_moments(lv, rho, L, origin=origin, size=size)
        want = packed_from_oracle(omom)
        order = {tuple(v): i for i, v in enumerate(oxyz)}
        idx = np.array([order[tuple(v)] for v in xyz])
        got = mom.cpu().numpy()
        want = want[idx]
        h = size / (8 * 2 ** L)
        mmax = np.abs(want[:, 0]).max()
        for name, sl, scale in (("m", slice(0, 1), mmax), ("X", slice(1, 4), size),
                                ("M2", slice(4, 10), mmax * h * h),
                                ("M3", slice(10, 20), mmax * h ** 3)):
            e = float(np.abs(got[:, sl] - want[:, sl]).max() / scale)
            print(f"{case} level {L} {name}: {e:.2e}")
            assert e < 1e-14, (case, L, name, e)
    with pytest.raises(fmm.OTError) as e:
        out = torch.empty((1, 20, 512), dtype=torch.float64, device="cuda")
        fmm.ot_get_moments(tree.handle, nl, out)
    assert e.value.code == -1
    tree.close()


def test_fixed_launch_shape_keeps_parity(fmm):
    lv = I.amr_leaves(3, 2e-4, I.BINARY)
    rho = I.density(lv, I.BINARY, seed=5)
    phi_o, g_o = O.solve(lv, rho)
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    for chunk, cps in ((17, 1), (263, 8), (1000, 2)):
        tree.set_launch_shape(chunk, cps)
        info = tree.info()
        assert info["tuned_chunk"] == chunk and info["tuned_ctas_per_sm"] == cps
        for prec, tol in ((fmm.OT_PRECISION_FP64, 1e-12), (fmm.OT_PRECISION_FP32_BULK, 1e-6),
                          (fmm.OT_PRECISION_FP32_WIDE, 1e-6)):
            phi, g = tree.solve(r, precision=prec)
            torch.cuda.synchronize()
            assert rel(phi.cpu().numpy(), phi_o) < tol, (chunk, prec)
            assert rel(g.cpu().numpy(), g_o) < tol, (chunk, prec)
    with pytest.raises(fmm.OTError):
        tree.set_launch_shape(0, 4)
    with pytest.raises(fmm.OTError):
        tree.set_launch_shape(64, 0)
    tree.close()


def test_items_of_any_length_in_every_form(fmm):
    """Items of up to 1000 stencil entries at theta = 0.35 (lists of about 700
    entries at levels >= 1): the general kernels of all three forms take them
    (the wide FP32 form adds a lane's FP32 partial sums to the FP64 expansion
    every 64 pairs, so its error does not grow with the item length), and the
    device status word stays clear."""
    lv = I.uniform_leaves(2)
    rho = I.density(lv, I.BINARY, seed=2)
    theta = 0.35
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    phi_o, g_o = O.solve(lv, rho, theta=theta)
    for chunk in (1000, 64):
        tree.set_launch_shape(chunk, 4)
        for prec, tol in ((fmm.OT_PRECISION_FP64, 1e-12), (fmm.OT_PRECISION_FP32_BULK, 1e-8),
                          (fmm.OT_PRECISION_FP32_WIDE, 1e-6)):
            phi, g = tree.solve(r, theta=theta, precision=prec)
            torch.cuda.synchronize()
            assert rel(phi.cpu().numpy(), phi_o) < tol, (chunk, prec)
            assert rel(g.cpu().numpy(), g_o) < tol, (chunk, prec)
            assert tree.info()["device_status"] == 0
    tree.close()


def test_device_status_latch_reports_a_non_physical_state_once(fmm):
    """A hydro state with a zero density in one cell: the faces kernel
    latches bit 4 of the status word; ot_tree_info reports it once as
    OT_ERR_DEVICE_STATUS and clears it; a physical state then leaves it
    clear."""
    lv = I.uniform_leaves(1)
    u = torch.from_numpy(I.hydro_fields(lv, seed=3)).cuda()
    tree = fmm.Tree(lv)
    bad = u.clone()
    bad[2, 0, 100] = 0.0
    tree.hydro_rhs(bad)
    torch.cuda.synchronize()
    with pytest.raises(fmm.OTError) as e:
        tree.info()
    assert e.value.code == -8                       # OT_ERR_DEVICE_STATUS
    assert tree.info()["device_status"] == 0        # reported once, then cleared
    d = tree.hydro_rhs(u)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(d).all())
    assert tree.info()["device_status"] == 0
    tree.close()


def test_alu_peaks_are_measured(fmm):
    p = fmm.ot_alu_peaks(0, reps=2)
    print("measured peaks", p)
    assert p["fp64_tflops"] > 0.1
    assert p["fp32_tflops"] > 10 * p["fp64_tflops"]
    assert p["fp32x2_tflops"] > 0.5 * p["fp32_tflops"]
