"""GPU parity: the C-ABI solve against the CPU oracle, element by element.

Tolerances (max |gpu - oracle| / max |oracle| per field):
  FP64 form       1e-12  (both sides FP64; they differ only in summation
                          order, FMA contraction and the reciprocal square
                          root, each ~1e-16 per operation)
  FP32-bulk and   1e-6   (per-pair terms in FP32, unit roundoff 6e-8,
  wide FP32 forms         accumulated in FP64; stated target 1e-6)

Conservation (Sec. 4.3.1): with F_c = m_c g_c over every leaf cell,
  momentum  |sum F| / sum |F|              and
  torque    |sum (x - x0) x F| / sum |(x - x0) x F|
are zero up to rounding.  Bounds: FP64 1e-14 / 1e-12 (level-3 binary) and
1e-13 / 1e-11 (level-8 AMR binary, 22.1M cells); the FP32-bulk form keeps
every monopole term, the correction's sums and every sum in FP64, so only
the FP32 rounding of the source quadrupole/octupole terms -- O((a/R)^2) of
a pair's force, a/R <= theta -- breaks the pair symmetry: bound 1e-9; the
wide FP32 form rounds whole pair terms in FP32 (u = 6e-8): bound 1e-6.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-6
FP32_FORMS = ["bulk", "wide"]
# (momentum, torque) bounds per form
RESID = {"fp64": (1e-14, 1e-12), "bulk": (1e-9, 1e-9), "wide": (1e-6, 1e-6)}


def prec_of(fmm, form):
    return {"fp64": fmm.OT_PRECISION_FP64, "bulk": fmm.OT_PRECISION_FP32_BULK,
            "wide": fmm.OT_PRECISION_FP32_WIDE}[form]


def error_metrics(phi, g, phi_o, g_o):
    """Errors against the oracle per field: max-norm relative (the parity
    bar), RMS relative, and the largest per-cell relative error with the
    reference floored at 1e-6 of its maximum (g per cell as a vector)."""
    out = {}
    for name, a, b in (("phi", np.asarray(phi).reshape(-1, 1), np.asarray(phi_o).reshape(-1, 1)),
                       ("g", np.moveaxis(np.asarray(g), -2, -1).reshape(-1, 3),
                        np.moveaxis(np.asarray(g_o), -2, -1).reshape(-1, 3))):
        d = np.linalg.norm(a - b, axis=1)
        r = np.linalg.norm(b, axis=1)
        out[name] = {"max": float(d.max() / r.max()),
                     "rms": float(np.sqrt((d ** 2).mean() / (r ** 2).mean())),
                     "cell": float((d / np.maximum(r, 1e-6 * r.max())).max())}
    return out


def residuals(lv, r, g):
    """(momentum, torque) residuals of F = m g over every leaf cell, on the
    device (r, g: device tensors [n, 512], [n, 3, 512])."""
    h = torch.from_numpy(1.0 / (8.0 * 2.0 ** lv[:, 0])).to(r.device)
    m = r * (h ** 3)[:, None]
    f = m[:, None, :] * g                                            # [n, 3, 512]
    x = torch.from_numpy(I.cell_centres(lv) - 0.5).to(r.device)      # [n, 512, 3]
    mom = (f.sum((0, 2)).abs().max() / f.abs().sum()).item()
    tq = torch.cross(x, f.permute(0, 2, 1), dim=2)
    ang = (tq.sum((0, 1)).abs().max() / tq.abs().sum()).item()
    return mom, ang


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


@pytest.mark.parametrize("form", FP32_FORMS)
@pytest.mark.parametrize("theta", [0.4, 1.0 / 3.0, 0.75])
def test_fp32_forms_other_theta(fmm, theta, form):
    # near sets other than theta = 0.5's run the lattice kernel's generic near
    # loop; theta = 1/3 also takes the widest far halo
    lv, rho = CASES["amr_l3_seams"]()
    phi, g = gpu_solve(fmm, lv, rho, theta=theta, precision=prec_of(fmm, form))
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


@pytest.mark.parametrize("form", FP32_FORMS)
def test_fp32_forms_binary_l3_and_conservation(fmm, binary_l3, form):
    lv, rho, phi_o, g_o = binary_l3
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    phi, g = tree.solve(r, precision=prec_of(fmm, form))
    torch.cuda.synchronize()
    assert rel(phi.cpu().numpy(), phi_o) < TOL32
    assert rel(g.cpu().numpy(), g_o) < TOL32
    mom, ang = residuals(lv, r, g)
    print(f"binary_l3 {form}: momentum {mom:.2e}, torque {ang:.2e}")
    assert mom < RESID[form][0] and ang < RESID[form][1]
    tree.close()


@pytest.mark.parametrize("form", FP32_FORMS)
@pytest.mark.parametrize("case", ["sphere_l1_shuffled", "amr_l3_seams", "amr_l2_ragged",
                                  "amr_l3_empty", "root_leaf"])
def test_fp32_forms_match_oracle(fmm, case, form):
    lv, rho = CASES[case]()
    phi, g = gpu_solve(fmm, lv, rho, precision=prec_of(fmm, form))
    phi_o, g_o = O.solve(lv, rho)
    assert rel(phi, phi_o) < TOL32
    assert rel(g, g_o) < TOL32


@pytest.mark.parametrize("am", [True, False])
def test_fp32_bulk_without_correction(fmm, am):
    lv, rho = CASES["amr_l3_seams"]()
    phi, g = gpu_solve(fmm, lv, rho, am_correction=am, precision=fmm.OT_PRECISION_FP32_BULK)
    phi_o, g_o = O.solve(lv, rho, am_correction=am)
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
    for prec, tol in ((fmm.OT_PRECISION_FP64, TOL64), (fmm.OT_PRECISION_FP32_BULK, TOL32),
                      (fmm.OT_PRECISION_FP32_WIDE, TOL32)):
        phi, g = tree.solve(r, precision=prec)
        torch.cuda.synchronize()
        phi = phi.cpu().numpy().reshape(-1)[sample]
        g = np.moveaxis(g.cpu().numpy(), 1, 2).reshape(-1, 3)[sample]
        assert rel(phi, phi_s) < tol, prec
        assert rel(g, g_s) < tol, prec
        print(f"errors binary_amr6 (3,000 sampled cells) precision {prec}: "
              f"{error_metrics(phi, np.swapaxes(g, -1, -2), phi_s, np.swapaxes(g_s, -1, -2))}")
    tree.close()


@pytest.mark.parametrize("form", FP32_FORMS)
def test_fp32_error_bounded_for_any_item_length(fmm, form):
    """The FP32 partial sums are flushed every 64 pairs whatever the plan's
    item length (their rounding error grows with the summation length: on
    this tree the wide form gives 8.6e-7 in g with 263-pair sums, 3.1e-7 with
    64).  The tree is tuned for the FP64 form first, which may choose the
    longest items; the FP32 solve is then compared with the FP64 GPU solve
    (itself within 1e-12 of the oracle)."""
    lv, rho = I.workload("binary_amr6")
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    tree.autotune(r)
    p64, g64 = tree.solve(r)
    p32, g32 = tree.solve(r, precision=prec_of(fmm, form))
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
    tree.solve_host(hr, hp, hg)    # pinned: read and written by the kernels
    torch.cuda.synchronize()
    assert rel(hp.numpy(), phi_o) < TOL64
    assert rel(hg.numpy(), g_o) < TOL64
    # the same pinned buffers with new contents replay their graph
    hr.copy_(torch.from_numpy(rho))
    tree.solve_host(hr, hp, hg)
    torch.cuda.synchronize()
    phi_r, g_r = O.solve(lv, rho)
    assert rel(hp.numpy(), phi_r) < TOL64
    assert rel(hg.numpy(), g_r) < TOL64
    # pageable buffers: staged through device copies; and the self term,
    # which reads the densities again in the evaluation
    pr = np.ascontiguousarray(rho2)
    pp = np.empty((lv.shape[0], 512))
    pg = np.empty((lv.shape[0], 3, 512))
    tree.solve_host(pr, pp, pg)
    torch.cuda.synchronize()
    assert rel(pp, phi_o) < TOL64
    assert rel(pg, g_o) < TOL64
    hr.copy_(torch.from_numpy(rho2))
    tree.solve_host(hr, hp, hg, self_term=True)
    torch.cuda.synchronize()
    phi_s, g_s = O.solve(lv, rho2, self_term=True)
    assert rel(hp.numpy(), phi_s) < TOL64
    assert rel(hg.numpy(), g_s) < TOL64
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
    launch configuration the benchmark times: every form on the GPU, the
    oracle on 2,000 seeded leaf cells (and the expansions of their
    ancestors); momentum and torque residuals over every cell."""
    lv, rho = I.workload("binary_amr8")
    rng = np.random.default_rng(12)
    sample = rng.choice(lv.shape[0] * 512, size=2000, replace=False)
    phi_s, g_s = O.solve_sample(lv, rho, sample)
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    resid = {"fp64": (1e-13, 1e-11), "bulk": RESID["bulk"], "wide": RESID["wide"]}
    for form, tol in (("fp64", TOL64), ("bulk", TOL32), ("wide", TOL32)):
        prec = prec_of(fmm, form)
        tree.autotune(r, precision=prec)
        phi, g = tree.solve(r, precision=prec)
        torch.cuda.synchronize()
        assert rel(phi.view(-1)[torch.from_numpy(sample).cuda()].cpu().numpy(), phi_s) < tol, form
        gs = g.permute(0, 2, 1).reshape(-1, 3)[torch.from_numpy(sample).cuda()].cpu().numpy()
        assert rel(gs, g_s) < tol, form
        ps = phi.view(-1)[torch.from_numpy(sample).cuda()].cpu().numpy()
        print(f"errors binary_amr8 (2,000 sampled cells) {form}: "
              f"{error_metrics(ps, np.swapaxes(gs, -1, -2), phi_s, np.swapaxes(g_s, -1, -2))}")
        mom, ang = residuals(lv, r, g)
        print(f"amr8 {form} residuals: momentum {mom:.2e}, torque {ang:.2e}")
        assert mom < resid[form][0] and ang < resid[form][1], form
    tree.close()


@pytest.mark.parametrize("form", ["fp64", "bulk"])
def test_six_resident_solves_equal_independent_solves(fmm, form):
    """The two solves per stage of an RK3 step on a resident tree: the
    density is updated in place on the device and the captured graph is
    replayed six times; each result equals an independent solve of the same
    density on a fresh tree to rounding (the expansion sums are FP64 atomics
    whose order varies from run to run: 1e-14 of the field's maximum)."""
    lv, rho = CASES["amr_l3_seams"]()
    prec = prec_of(fmm, form)
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    phi, g = tree.empty_outputs()
    tree.solve(r, phi, g, precision=prec)
    outs, dens = [], []
    for k in range(6):
        r.mul_(1.0 + 0.01 * (k + 1) * (-1) ** k)
        tree.solve(r, phi, g, precision=prec)   # graph replay on the updated density
        outs.append((phi.clone(), g.clone()))
        dens.append(r.clone())
    torch.cuda.synchronize()
    worst = 0.0
    for (p6, g6), d in zip(outs, dens):
        fresh = fmm.Tree(lv)
        p1, g1 = fresh.solve(d, precision=prec)
        torch.cuda.synchronize()
        worst = max(worst, float((p6 - p1).abs().max() / p1.abs().max()),
                    float((g6 - g1).abs().max() / g1.abs().max()))
        fresh.close()
    print(f"six resident solves ({form}) vs independent: {worst:.2e}")
    assert worst < 1e-14
    tree.close()


@pytest.mark.parametrize("workload", ["sphere_l1", "binary_l3"])
def test_error_metrics_every_form(fmm, workload):
    """Every form against the full oracle solve: max-norm, RMS and floored
    per-cell relative errors (printed; the max-norm bars asserted)."""
    lv, rho = I.workload(workload)
    phi_o, g_o = O.solve(lv, rho)
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    for form, tol in (("fp64", TOL64), ("bulk", TOL32), ("wide", TOL32)):
        phi, g = tree.solve(r, precision=prec_of(fmm, form))
        torch.cuda.synchronize()
        m = error_metrics(phi.cpu().numpy(), g.cpu().numpy(), phi_o, g_o)
        print(f"errors {workload} {form}: {m}")
        assert m["phi"]["max"] < tol and m["g"]["max"] < tol
    tree.close()
