"""GPU parity: the C-ABI solve against the CPU oracle, element by element.

Tolerances (max |gpu - oracle| / max |oracle| per field):
  FP64 form       1e-12  (both sides FP64; they differ only in summation
                          order, FMA contraction and the reciprocal square
                          root, each ~1e-16 per operation)
  FP32-bulk form  1e-6   (per-pair multipole terms in FP32, unit roundoff
                          6e-8, accumulated in FP64; stated target 1e-6)
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6


@pytest.fixture(scope="module")
def fmm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_15518_gb300 import fmm as F
    return F


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def gpu_solve(fmm, lv, rho, **opts):
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    phi, g = tree.solve(r, **opts)
    torch.cuda.synchronize()
    out = phi.cpu().numpy(), g.cpu().numpy()
    tree.close()
    return out


def small_amr():
    lv = I.amr_leaves(3, 2e-4, I.BINARY)
    return lv, I.density(lv, I.BINARY, seed=5)


CASES = {
    "sphere_l1_shuffled": lambda: (lambda lv: (lv, I.density(lv, I.SPHERE, 0)))(
        I.uniform_leaves(1, seed=3)),
    "amr_l3_seams": small_amr,
    # empty space outside the stars: cells and whole interior cells of zero mass
    "sphere_l1_empty": lambda: (lambda lv: (lv, I.density(lv, I.SPHERE, 0, atmosphere=0.0)))(
        I.uniform_leaves(1, seed=3)),
    "amr_l3_empty": lambda: (lambda lv: (lv, I.density(lv, I.BINARY, 5, atmosphere=0.0)))(
        I.amr_leaves(3, 2e-4, I.BINARY)),
    "root_leaf": lambda: (np.array([[0, 0, 0, 0]], np.int32),
                          I.density(np.array([[0, 0, 0, 0]], np.int32), I.SPHERE, 2)),
    "amr_l2_ragged": lambda: (lambda lv: (lv, I.density(lv, I.BINARY, 4)))(
        I.amr_leaves(2, 5e-4, I.BINARY, lmin=1)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("am", [True, False])
def test_fp64_matches_oracle(fmm, case, am):
    lv, rho = CASES[case]()
    phi, g = gpu_solve(fmm, lv, rho, am_correction=am)
    phi_o, g_o = O.solve(lv, rho, am_correction=am)
    assert rel(phi, phi_o) < TOL64
    assert rel(g, g_o) < TOL64


@pytest.mark.parametrize("theta", [0.4, 1.0 / 3.0, 0.75])
def test_fp64_other_theta(fmm, theta):
    lv, rho = CASES["amr_l3_seams"]()
    phi, g = gpu_solve(fmm, lv, rho, theta=theta)
    phi_o, g_o = O.solve(lv, rho, theta=theta)
    assert rel(phi, phi_o) < TOL64
    assert rel(g, g_o) < TOL64


@pytest.mark.parametrize("theta", [0.4, 1.0 / 3.0, 0.75])
def test_fp32_bulk_other_theta(fmm, theta):
    # near sets other than theta = 0.5's run the lattice kernel's generic near
    # loop; theta = 1/3 also takes the widest far halo
    lv, rho = CASES["amr_l3_seams"]()
    phi, g = gpu_solve(fmm, lv, rho, theta=theta, precision=fmm.OT_PRECISION_FP32_BULK)
    phi_o, g_o = O.solve(lv, rho, theta=theta)
    assert rel(phi, phi_o) < TOL32
    assert rel(g, g_o) < TOL32


def test_fp64_self_term_and_G(fmm):
    lv, rho = CASES["sphere_l1_shuffled"]()
    phi, g = gpu_solve(fmm, lv, rho, self_term=True, G=6.674e-8)
    phi_o, g_o = O.solve(lv, rho, self_term=True, G=6.674e-8)
    assert rel(phi, phi_o) < TOL64
    assert rel(g, g_o) < TOL64


@pytest.fixture(scope="module")
def binary_l3():
    lv, rho = I.workload("binary_l3")
    phi_o, g_o = O.solve(lv, rho)
    return lv, rho, phi_o, g_o


def test_fp64_binary_l3_full(fmm, binary_l3):
    lv, rho, phi_o, g_o = binary_l3
    phi, g = gpu_solve(fmm, lv, rho)
    assert rel(phi, phi_o) < TOL64
    assert rel(g, g_o) < TOL64
    # conservation of the GPU result (Sec. 4.3.1)
    x = I.cell_centres(lv)
    m = rho * (1.0 / 64) ** 3
    f = m[:, :, None] * np.moveaxis(g, 1, 2)
    assert np.abs(f.sum((0, 1))).max() / np.abs(f).sum() < 1e-14
    tq = np.cross(x - 0.5, f)
    assert np.abs(tq.sum((0, 1))).max() / np.abs(tq).sum() < 1e-12


def test_fp32_bulk_binary_l3(fmm, binary_l3):
    lv, rho, phi_o, g_o = binary_l3
    phi, g = gpu_solve(fmm, lv, rho, precision=fmm.OT_PRECISION_FP32_BULK)
    assert rel(phi, phi_o) < TOL32
    assert rel(g, g_o) < TOL32


@pytest.mark.parametrize("case", ["sphere_l1_shuffled", "amr_l3_seams", "amr_l2_ragged",
                                  "amr_l3_empty"])
def test_fp32_bulk_matches_oracle(fmm, case):
    lv, rho = CASES[case]()
    phi, g = gpu_solve(fmm, lv, rho, precision=fmm.OT_PRECISION_FP32_BULK)
    phi_o, g_o = O.solve(lv, rho)
    assert rel(phi, phi_o) < TOL32
    assert rel(g, g_o) < TOL32


def test_amr6_sampled(fmm):
    """The ~4,900-leaf level-6 AMR tree: GPU everywhere, oracle on a seeded
    sample of 3,000 leaf cells (their ancestors' expansions in full)."""
    lv, rho = I.workload("binary_amr6")
    rng = np.random.default_rng(11)
    sample = rng.choice(lv.shape[0] * 512, size=3000, replace=False)
    phi_s, g_s = O.solve_sample(lv, rho, sample)
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    for prec, tol in ((fmm.OT_PRECISION_FP64, TOL64), (fmm.OT_PRECISION_FP32_BULK, TOL32)):
        phi, g = tree.solve(r, precision=prec)
        torch.cuda.synchronize()
        phi = phi.cpu().numpy().reshape(-1)[sample]
        g = np.moveaxis(g.cpu().numpy(), 1, 2).reshape(-1, 3)[sample]
        assert rel(phi, phi_s) < tol, prec
        assert rel(g, g_s) < tol, prec
    tree.close()


def test_fp32_bulk_error_bounded_for_any_item_length(fmm):
    """The FP32 partial sums are flushed every 64 pairs whatever the plan's
    item length (their rounding error grows with the summation length: on
    this tree 8.6e-7 in g with 263-pair sums, 3.1e-7 with 64).  The tree is
    tuned for the FP64 form first, which may choose the longest items; the
    FP32-bulk solve is then compared with the FP64 GPU solve (itself within
    1e-12 of the oracle)."""
    lv, rho = I.workload("binary_amr6")
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    tree.autotune(r)
    p64, g64 = tree.solve(r)
    p32, g32 = tree.solve(r, precision=fmm.OT_PRECISION_FP32_BULK)
    torch.cuda.synchronize()
    assert rel(p32.cpu().numpy(), p64.cpu().numpy()) < 5e-7
    assert rel(g32.cpu().numpy(), g64.cpu().numpy()) < 5e-7
    tree.close()


def test_graph_replay_and_host_buffers(fmm):
    lv, rho = CASES["amr_l3_seams"]()
    rho2 = I.density(lv, I.BINARY, seed=9)
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    phi, g = tree.empty_outputs()
    tree.solve(r, phi, g)
    r.copy_(torch.from_numpy(rho2))
    tree.solve(r, phi, g)          # replays the captured graph on new densities
    torch.cuda.synchronize()
    phi_o, g_o = O.solve(lv, rho2)
    assert rel(phi.cpu().numpy(), phi_o) < TOL64
    assert rel(g.cpu().numpy(), g_o) < TOL64
    hr = torch.from_numpy(rho2).pin_memory()
    hp = torch.empty((lv.shape[0], 512), dtype=torch.float64).pin_memory()
    hg = torch.empty((lv.shape[0], 3, 512), dtype=torch.float64).pin_memory()
    tree.solve_host(hr, hp, hg)
    torch.cuda.synchronize()
    assert rel(hp.numpy(), phi_o) < TOL64
    assert rel(hg.numpy(), g_o) < TOL64
    tree.close()


def test_autotune_keeps_parity(fmm):
    lv, rho = CASES["amr_l3_seams"]()
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    tree.autotune(r)
    info = tree.info()
    assert info["tuned_chunk"] in (32, 64, 128, 263)
    phi, g = tree.solve(r)
    torch.cuda.synchronize()
    phi_o, g_o = O.solve(lv, rho)
    assert rel(phi.cpu().numpy(), phi_o) < TOL64
    assert rel(g.cpu().numpy(), g_o) < TOL64
    assert info["device_status"] == 0
    tree.close()


def test_error_codes(fmm):
    lv, rho = CASES["sphere_l1_shuffled"]()
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    phi, g = tree.empty_outputs()
    with pytest.raises(fmm.OTError) as e:          # host memory where device is required
        fmm.ot_solve_gravity(tree.handle, torch.from_numpy(rho), phi, g)
    assert e.value.code == -4
    big = torch.zeros(rho.size + 1, dtype=torch.float64, device="cuda")
    mis = big.view(torch.uint8)[4:4 + 8 * rho.size]  # 4-byte offset
    with pytest.raises(fmm.OTError) as e:
        fmm._check(fmm._lib.ot_solve_gravity(fmm._P(tree.handle), fmm._ptr(mis), fmm._ptr(phi),
                                             fmm._ptr(g), None, None), "x")
    assert e.value.code == -5
    with pytest.raises(fmm.OTError) as e:
        tree.solve(r, phi, g, theta=0.2)
    assert e.value.code == -1
    with pytest.raises(fmm.OTError) as e:
        tree.solve(r, phi, g, precision=7)
    assert e.value.code == -1
    tree.solve(r, phi, g)                           # still usable afterwards
    torch.cuda.synchronize()
    assert tree.info()["device_status"] == 0
    tree.close()


def test_amr8_full_size_sampled(fmm):
    """The level-8 AMR binary (43,240 leaves, 22.1M cells) at full size, in the
    launch configuration the benchmark times: both forms on the GPU, the
    oracle on 2,000 seeded leaf cells (and the expansions of their
    ancestors); momentum and torque residuals over every cell."""
    lv, rho = I.workload("binary_amr8")
    rng = np.random.default_rng(12)
    sample = rng.choice(lv.shape[0] * 512, size=2000, replace=False)
    phi_s, g_s = O.solve_sample(lv, rho, sample)
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    for prec, tol in ((fmm.OT_PRECISION_FP64, TOL64), (fmm.OT_PRECISION_FP32_BULK, TOL32)):
        tree.autotune(r, precision=prec)
        phi, g = tree.solve(r, precision=prec)
        torch.cuda.synchronize()
        assert rel(phi.view(-1)[torch.from_numpy(sample).cuda()].cpu().numpy(), phi_s) < tol, prec
        gs = g.permute(0, 2, 1).reshape(-1, 3)[torch.from_numpy(sample).cuda()].cpu().numpy()
        assert rel(gs, g_s) < tol, prec
        if prec == fmm.OT_PRECISION_FP64:
            h = torch.from_numpy(1.0 / (8.0 * 2.0 ** lv[:, 0])).cuda()
            m = r * (h ** 3)[:, None]
            f = m[:, None, :] * g                                   # [n, 3, 512]
            x = torch.from_numpy(I.cell_centres(lv) - 0.5).cuda()   # [n, 512, 3]
            mom = (f.sum((0, 2)).abs().max() / f.abs().sum()).item()
            fx = f.permute(0, 2, 1)
            tq = torch.cross(x, fx, dim=2)
            ang = (tq.sum((0, 1)).abs().max() / tq.abs().sum()).item()
            print(f"amr8 residuals: momentum {mom:.2e}, torque {ang:.2e}")
            assert mom < 1e-13 and ang < 1e-11
    tree.close()
