"""GPU hydro right-hand side (ot_hydro_rhs) against the oracles
(oracle/hydro.py on uniform trees, oracle/hydro_amr.py on adaptive ones),
element by element.

Both sides evaluate the same formulas operation by operation in FP64
without fused multiply-adds (PPM values, Rusanov fluxes, Simpson face rule,
divergence, gravity source), so the limiter and the wave-speed maxima take
the same branches and the rates agree bit for bit: the comparison is exact
equality.  At the bench's size (uniform level 4, 2.1M cells), where the
oracle would hold several GB of directional values, the tests check what
holds at any size: a uniform state feels the gravity source only, and a
linear state in uniform motion changes at its closed-form rate.
"""
import numpy as np
import pytest
import torch

from oracle import hydro as H
from oracle import hydro_amr as A
from paper_2412_15518_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def fmm():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_15518_gb300 import fmm as F
    return F


def rand_g(lv, seed):
    return np.random.default_rng(seed).standard_normal((lv.shape[0], 3, 512))


CASES = {
    # uniform level 1, shuffled leaf order, the binary's fields, gravity
    "l1_hydro_g": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=3), rand_g(lv, 4)))(
        I.uniform_leaves(1, seed=2)),
    # uniform level 2, no gravity
    "l2_hydro": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=1), None))(I.uniform_leaves(2)),
    # uniform level 3 (262,144 cells), gravity
    "l3_hydro_g": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=2), rand_g(lv, 5)))(
        I.uniform_leaves(3, seed=5)),
    # a lone root leaf: every face of the domain is transmissive
    "root_g": lambda: (np.array([[0, 0, 0, 0]], np.int32),
                       I.hydro_fields(np.array([[0, 0, 0, 0]], np.int32), seed=6),
                       rand_g(np.array([[0, 0, 0, 0]], np.int32), 7)),
}


def gpu_rhs(fmm, lv, u, g, gamma=GAMMA, size=1.0):
    tree = fmm.Tree(lv, size=size)
    ug = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    gg = None if g is None else torch.from_numpy(np.ascontiguousarray(g)).cuda()
    out = tree.hydro_rhs(ug, gg, gamma)
    torch.cuda.synchronize()
    res = out.cpu().numpy()
    tree.close()
    return res


@pytest.mark.parametrize("case", sorted(CASES))
def test_hydro_rhs_matches_oracle_bit_for_bit(fmm, case):
    lv, u, g = CASES[case]()
    got = gpu_rhs(fmm, lv, u, g)
    want = H.rhs(lv, u, g, GAMMA)
    diff = int((got != want).sum())
    print(f"hydro {case}: {got.size} values, {diff} differ, max |diff| {np.abs(got - want).max():.2e}")
    assert np.isfinite(got).all()
    assert diff == 0


def test_hydro_rhs_other_gamma_and_domain_size(fmm):
    lv = I.uniform_leaves(1)
    u = I.hydro_fields(lv, seed=8)
    g = rand_g(lv, 9)
    got = gpu_rhs(fmm, lv, u, g, gamma=1.4, size=3.0)
    want = H.rhs(lv, u, g, 1.4, size=3.0)
    assert int((got != want).sum()) == 0


def test_hydro_rhs_with_the_gravity_solve(fmm):
    """The two workloads coupled: g from the GPU gravity solve of the same
    density, both sides fed the same g."""
    lv = I.uniform_leaves(2)
    u = I.hydro_fields(lv, seed=10)
    tree = fmm.Tree(lv)
    ug = torch.from_numpy(u).cuda()
    rho = ug[:, 0].contiguous()
    phi, g = tree.solve(rho)
    out = tree.hydro_rhs(ug, g, GAMMA)
    torch.cuda.synchronize()
    got, gn = out.cpu().numpy(), g.cpu().numpy()
    tree.close()
    want = H.rhs(lv, u, gn, GAMMA)
    assert int((got != want).sum()) == 0


def test_level4_uniform_state_feels_the_source_only(fmm):
    lv = I.uniform_leaves(4)
    vel = (0.3, -0.2, 0.7)
    rho, p = 1.3, 0.8
    E = p / (GAMMA - 1.0) + 0.5 * rho * sum(v * v for v in vel)
    u = np.empty((lv.shape[0], 5, 512))
    for f, val in enumerate([rho, rho * vel[0], rho * vel[1], rho * vel[2], E]):
        u[:, f] = val
    g = rand_g(lv, 11)
    got = gpu_rhs(fmm, lv, u, g)
    assert np.all(got[:, 0] == 0.0)
    for b in range(3):
        assert np.all(got[:, 1 + b] == rho * g[:, b])
    assert np.allclose(got[:, 4], rho * (vel[0] * g[:, 0] + vel[1] * g[:, 1] + vel[2] * g[:, 2]),
                       rtol=1e-14, atol=1e-15)


def test_level4_linear_state_advects_at_the_closed_form_rate(fmm):
    lv = I.uniform_leaves(4)
    n, h = 128, 1.0 / 128
    b = np.array([0.0011, -0.0007, 0.0005])
    vel = (0.4, -0.3, 0.25)
    c = np.arange(8)
    kk, jj, ii = np.meshgrid(c, c, c, indexing="ij")
    u = np.empty((lv.shape[0], 5, 512))
    for m, (_, ix, iy, iz) in enumerate(lv):
        rho = 1.0 + b[0] * (8 * ix + ii) + b[1] * (8 * iy + jj) + b[2] * (8 * iz + kk)
        rho = rho.reshape(-1)
        u[m] = [rho, rho * vel[0], rho * vel[1], rho * vel[2],
                0.9 / (GAMMA - 1.0) + 0.5 * rho * sum(v * v for v in vel)]
    got = gpu_rhs(fmm, lv, u, None)
    vb = (vel[0] * b[0] + vel[1] * b[1] + vel[2] * b[2]) / h
    v2 = sum(v * v for v in vel)
    want = [-vb] + [-vel[a] * vb for a in range(3)] + [-0.5 * v2 * vb]
    # interior cells: three cells from the domain boundary
    lo = np.asarray(lv)[:, 1:4] * 8
    glob = np.stack([lo[:, 0:1] + ii.reshape(1, -1), lo[:, 1:2] + jj.reshape(1, -1),
                     lo[:, 2:3] + kk.reshape(1, -1)])
    inner = np.all((glob >= 3) & (glob < n - 3), axis=0)
    for f in range(5):
        assert np.abs(got[:, f][inner] - want[f]).max() < 1e-9, f


AMR_CASES = {
    # levels 1-2 and 1-3 refined on the binary: coarse-fine faces, restriction
    # and injection in the halos, flux matching
    "binary_l1_l2_g": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=12), rand_g(lv, 13)))(
        I.amr_leaves(2, 5e-4, I.BINARY, lmin=1)),
    "binary_l1_l3": lambda: (lambda lv: (lv, I.hydro_fields(lv, seed=14), None))(
        I.amr_leaves(3, 2e-4, I.BINARY)),
    "sphere_l2_l3_g": lambda: (lambda lv: (lv, I.hydro_fields(lv, I.SPHERE, seed=15), rand_g(lv, 16)))(
        I.amr_leaves(3, 1e-3, I.SPHERE, lmin=1)),
}


@pytest.mark.parametrize("case", sorted(AMR_CASES))
def test_hydro_rhs_on_adaptive_trees_matches_oracle_bit_for_bit(fmm, case):
    lv, u, g = AMR_CASES[case]()
    assert len(set(np.asarray(lv)[:, 0].tolist())) >= 2
    tree = fmm.Tree(lv)
    ug = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    gg = None if g is None else torch.from_numpy(np.ascontiguousarray(g)).cuda()
    out = tree.hydro_rhs(ug, gg, GAMMA)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert tree.info()["device_status"] == 0
    tree.close()
    want = A.rhs(lv, u, g, GAMMA)
    diff = int((got != want).sum())
    print(f"hydro amr {case}: {got.size} values, {diff} differ, max |diff| {np.abs(got - want).max():.2e}")
    assert np.isfinite(got).all()
    assert diff == 0


def test_hydro_rhs_on_an_adaptive_tree_with_the_gravity_solve(fmm):
    lv = I.amr_leaves(3, 2e-4, I.BINARY)
    u = I.hydro_fields(lv, seed=17)
    tree = fmm.Tree(lv)
    ug = torch.from_numpy(u).cuda()
    phi, g = tree.solve(ug[:, 0].contiguous())
    out = tree.hydro_rhs(ug, g, GAMMA)
    torch.cuda.synchronize()
    got, gn = out.cpu().numpy(), g.cpu().numpy()
    tree.close()
    assert int((got != A.rhs(lv, u, gn, GAMMA)).sum()) == 0


def test_hydro_rhs_rejects_bad_gamma(fmm):
    lv = I.uniform_leaves(1)
    tree = fmm.Tree(lv)
    u = torch.ones((lv.shape[0], 5, 512), dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    for bad in (1.0, 0.5, float("nan"), float("inf")):
        with pytest.raises(fmm.OTError) as e:
            fmm.ot_hydro_rhs(tree.handle, u, None, bad, out)
        assert e.value.code == -1
    tree.close()


def test_level8_adaptive_tree_properties(fmm):
    """At the bench's adaptive size (the level-8 binary's tree, 22.1M cells,
    levels 3-8): a uniform state is steady across every refinement jump, and
    a compact perturbation of a gas at rest conserves the totals of mass,
    momentum and energy (the fluxes matched at every jump); the device
    status word stays clear."""
    lv, _ = I.workload("binary_amr8")
    lv = np.asarray(lv)
    tree = fmm.Tree(lv)
    x = torch.from_numpy(I.cell_centres(lv)).cuda()                  # [n, 512, 3]
    u = torch.empty((lv.shape[0], 5, 512), dtype=torch.float64, device="cuda")
    vel = (0.3, -0.2, 0.7)
    u[:, 0] = 1.3
    for b in range(3):
        u[:, 1 + b] = 1.3 * vel[b]
    u[:, 4] = 0.8 / (GAMMA - 1.0) + 0.5 * 1.3 * sum(v * v for v in vel)
    d = tree.hydro_rhs(u, None, GAMMA)
    torch.cuda.synchronize()
    assert float(d.abs().max()) < 1e-8
    r2 = ((x[..., 0] - 0.45) ** 2 + (x[..., 1] - 0.5) ** 2 + (x[..., 2] - 0.52) ** 2) / 0.0625
    bump = torch.clamp(1.0 - r2, min=0.0) ** 4
    u[:, 0] = 1.0 + 0.5 * bump
    u[:, 1] = 0.3 * bump * (x[..., 1] - 0.5)
    u[:, 2] = -0.2 * bump * (x[..., 0] - 0.45)
    u[:, 3] = 0.1 * bump
    u[:, 4] = 1.5 + 0.8 * bump
    d = tree.hydro_rhs(u, None, GAMMA)
    torch.cuda.synchronize()
    h = 1.0 / (8.0 * 2.0 ** torch.from_numpy(lv[:, 0].astype(np.float64)).cuda())
    w = (h ** 3)[:, None, None]
    total = (d * w).sum(dim=(0, 2))
    scale = (d.abs() * w).sum(dim=(0, 2))
    assert bool((total.abs() < 1e-11 * scale).all()), (total / scale).tolist()
    assert tree.info()["device_status"] == 0
    tree.close()
