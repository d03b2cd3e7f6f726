"""GPU tangent of the solve (ot_solve_gravity_tangent): the time derivative
of the potential and acceleration for densities changing at rho_dot.

* Against the oracle's dual-number solve (itself pinned by central
  differences of the whole solve): the tangents to 1e-11 of their field's
  maximum and the values to 1e-12, on the parity trees, with and without the
  correction, with the self term and another G.
* Against the GPU adjoint, an independent code: for J = <w1, phi> + <w2, g>,
  <w1, phi_dot> + <w2, g_dot> = <dJ/drho, rho_dot> (the directional
  derivative two ways) to 1e-11, on the level-3 binary and at full size on
  the level-8 AMR binary.
The direction is rho_dot = rho u with u uniform in [-1, 1] (seeded): a
relative rate of change, as the hydrodynamics would give.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOLT = 1e-11
TOL64 = 1e-12


@pytest.fixture(scope="module")
def fmm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_15518_gb300 import fmm as F
    return F


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def direction(rho, seed=31):
    return rho * np.random.default_rng(seed).uniform(-1.0, 1.0, rho.shape)


CASES = {
    "sphere_l1_shuffled": lambda: (lambda lv: (lv, I.density(lv, I.SPHERE, 0)))(I.uniform_leaves(1, seed=3)),
    "amr_l3_seams": lambda: (lambda lv: (lv, I.density(lv, I.BINARY, 5)))(I.amr_leaves(3, 2e-4, I.BINARY)),
    "amr_l2_ragged": lambda: (lambda lv: (lv, I.density(lv, I.BINARY, 4)))(
        I.amr_leaves(2, 5e-4, I.BINARY, lmin=1)),
    "root_leaf": lambda: (np.array([[0, 0, 0, 0]], np.int32),
                          I.density(np.array([[0, 0, 0, 0]], np.int32), I.SPHERE, 2)),
    "amr_l5": lambda: (lambda lv: (lv, I.density(lv, I.BINARY_Q07, 4)))(I.amr_leaves(5, 1e-4, I.BINARY_Q07)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("am", [True, False])
def test_tangent_matches_oracle_dual_solve(fmm, case, am):
    lv, rho = CASES[case]()
    v = direction(rho)
    tree = fmm.Tree(lv)
    r, rd = torch.from_numpy(rho).cuda(), torch.from_numpy(v).cuda()
    phi, g, pd, gd = tree.tangent(r, rd, with_values=True, am_correction=am)
    torch.cuda.synchronize()
    phi_o, g_o, pd_o, gd_o = O.solve_jvp(lv, rho, v, am_correction=am)
    assert rel(phi.cpu().numpy(), phi_o) < TOL64
    assert rel(g.cpu().numpy(), g_o) < TOL64
    ep, eg = rel(pd.cpu().numpy(), pd_o), rel(gd.cpu().numpy(), gd_o)
    print(f"tangent {case} am={am}: phi_dot {ep:.2e}, g_dot {eg:.2e}")
    assert ep < TOLT and eg < TOLT
    tree.close()


def test_tangent_self_term_and_G(fmm):
    lv, rho = CASES["amr_l3_seams"]()
    v = direction(rho, seed=5)
    tree = fmm.Tree(lv)
    pd, gd = tree.tangent(torch.from_numpy(rho).cuda(), torch.from_numpy(v).cuda(), self_term=True, G=2.5)
    torch.cuda.synchronize()
    _, _, pd_o, gd_o = O.solve_jvp(lv, rho, v, self_term=True, G=2.5)
    assert rel(pd.cpu().numpy(), pd_o) < TOLT and rel(gd.cpu().numpy(), gd_o) < TOLT
    tree.close()


@pytest.mark.parametrize("workload", ["binary_l3", "binary_amr8"])
def test_tangent_and_adjoint_agree(fmm, workload):
    lv, rho = I.workload(workload)
    w1, w2 = I.weights(lv.shape[0])
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    rd = torch.from_numpy(direction(rho, seed=7)).cuda()
    W1, W2 = torch.from_numpy(w1).cuda(), torch.from_numpy(w2).cuda()
    del w1, w2
    pd, gd = tree.tangent(r, rd)
    forward = float((W1 * pd).sum() + (W2 * gd).sum())
    del pd, gd
    grad = tree.backward(r, W1, W2)
    reverse = float((grad * rd).sum())
    torch.cuda.synchronize()
    e = abs(forward - reverse) / float((grad * rd).abs().sum())
    print(f"{workload}: <w, J_dot> = {forward:.12e}, <grad, rho_dot> = {reverse:.12e}, rel {e:.2e}")
    assert e < TOLT
    tree.close()


def test_tangent_rejects_fp32_forms(fmm):
    lv, rho = CASES["sphere_l1_shuffled"]()
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    with pytest.raises(fmm.OTError) as e:
        tree.tangent(r, r, precision=fmm.OT_PRECISION_FP32_BULK)
    assert e.value.code == -1
    tree.close()
