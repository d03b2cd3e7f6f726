"""GPU adjoint (ot_gravity_backward) against the oracle's reverse sweep,
central differences and the Euler identity.

Tolerance for the full gradient vector: max |gpu - oracle| / max |oracle|
< 1e-11.  Both sides are FP64; the adjoint sums run over every pair twice
(once per role) and through the L2L/M2M chains, so their rounding differs
by more operations than the forward's (measured error is printed by -rP).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOLG = 1e-11


@pytest.fixture(scope="module")
def fmm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_15518_gb300 import fmm as F
    return F


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def gpu_grad(fmm, lv, rho, w1, w2, **opts):
    tree = fmm.Tree(lv)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gr = tree.backward(d(rho), d(w1), d(w2), **opts)
    torch.cuda.synchronize()
    out = gr.cpu().numpy()
    tree.close()
    return out


CASES = {
    "sphere_l1_shuffled": lambda: (lambda lv: (lv, I.density(lv, I.SPHERE, 0)))(
        I.uniform_leaves(1, seed=3)),
    "amr_l3_seams": lambda: (lambda lv: (lv, I.density(lv, I.BINARY, 5)))(
        I.amr_leaves(3, 2e-4, I.BINARY)),
    "amr_l2_ragged": lambda: (lambda lv: (lv, I.density(lv, I.BINARY, 4)))(
        I.amr_leaves(2, 5e-4, I.BINARY, lmin=1)),
    # empty space outside the stars: cells and whole interior cells of zero mass
    "sphere_l1_empty": lambda: (lambda lv: (lv, I.density(lv, I.SPHERE, 0, atmosphere=0.0)))(
        I.uniform_leaves(1, seed=3)),
    "amr_l3_empty": lambda: (lambda lv: (lv, I.density(lv, I.BINARY, 5, atmosphere=0.0)))(
        I.amr_leaves(3, 2e-4, I.BINARY)),
    "root_leaf": lambda: (np.array([[0, 0, 0, 0]], np.int32),
                          I.density(np.array([[0, 0, 0, 0]], np.int32), I.SPHERE, 2)),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("am", [True, False])
def test_adjoint_matches_oracle(fmm, case, am):
    lv, rho = CASES[case]()
    w1, w2 = I.weights(lv.shape[0])
    g_gpu = gpu_grad(fmm, lv, rho, w1, w2, am_correction=am)
    g_orc = O.gradient(lv, rho, w1, w2, am_correction=am)
    e = rel(g_gpu, g_orc)
    print(f"{case} am={am}: max rel err {e:.2e}")
    assert e < TOLG


def test_adjoint_self_term(fmm):
    lv, rho = CASES["sphere_l1_shuffled"]()
    w1, w2 = I.weights(lv.shape[0])
    g_gpu = gpu_grad(fmm, lv, rho, w1, w2, self_term=True, G=2.5)
    g_orc = O.gradient(lv, rho, w1, w2, self_term=True, G=2.5)
    assert rel(g_gpu, g_orc) < TOLG


@pytest.fixture(scope="module")
def binary_l3_grad(fmm):
    lv, rho = I.workload("binary_l3")
    w1, w2 = I.weights(lv.shape[0])
    return lv, rho, w1, w2, gpu_grad(fmm, lv, rho, w1, w2)


def test_adjoint_binary_l3_matches_oracle(binary_l3_grad):
    lv, rho, w1, w2, g_gpu = binary_l3_grad
    g_orc = O.gradient(lv, rho, w1, w2)
    e = rel(g_gpu, g_orc)
    print(f"binary_l3: max rel err {e:.2e}")
    assert e < TOLG


def test_adjoint_binary_l3_central_differences(fmm, binary_l3_grad):
    """Central differences, h = 1e-6 (densities in units of the central
    density), at 64 seeded cells inside the stars, with the GPU forward."""
    lv, rho, w1, w2, g_gpu = binary_l3_grad
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda()
    W1, W2 = torch.from_numpy(w1).cuda(), torch.from_numpy(w2).cuda()
    phi, g = tree.empty_outputs()

    def J(rr):
        tree.solve(rr, phi, g)
        return float((W1 * phi).sum() + (W2 * g).sum())

    J0 = J(r)
    inside = np.nonzero(rho.reshape(-1) > 1e-2)[0]
    cells = np.random.default_rng(3).choice(inside, size=64, replace=False)
    h = 1e-6
    flat = r.view(-1)
    errs = []
    for c in cells:
        flat[c] += h
        jp = J(r)
        flat[c] -= 2 * h
        jm = J(r)
        flat[c] += h
        fd = (jp - jm) / (2 * h)
        errs.append(abs(fd - g_gpu.reshape(-1)[c]) / np.abs(g_gpu).max())
    tree.close()
    print(f"central differences: max err / max|grad| = {max(errs):.2e}, J = {J0:.6e}")
    assert max(errs) < 1e-6
    # Euler identity: J is homogeneous of degree 1 in rho
    assert abs((g_gpu * rho).sum() - J0) < 1e-12 * abs(J0) * 10


def test_autograd_function(fmm):
    lv, rho = CASES["amr_l3_seams"]()
    w1, w2 = I.weights(lv.shape[0])
    tree = fmm.Tree(lv)
    r = torch.from_numpy(rho).cuda().requires_grad_(True)
    phi, g = fmm.GravitySolve.apply(r, tree, {})
    J = (torch.from_numpy(w1).cuda() * phi).sum() + (torch.from_numpy(w2).cuda() * g).sum()
    J.backward()
    g_orc = O.gradient(lv, rho, w1, w2)
    assert rel(r.grad.cpu().numpy(), g_orc) < TOLG
    tree.close()


def test_backward_rejects_fp32_bulk(fmm):
    lv, rho = CASES["sphere_l1_shuffled"]()
    w1, w2 = I.weights(lv.shape[0])
    tree = fmm.Tree(lv)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with pytest.raises(fmm.OTError) as e:
        tree.backward(d(rho), d(w1), d(w2), precision=fmm.OT_PRECISION_FP32_BULK)
    assert e.value.code == -1
    tree.close()
