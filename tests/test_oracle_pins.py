"""Pins of the CPU oracle against facts that do not come from the oracle itself.

The paper (arXiv 2412.15518) gives the method only in prose: an FMM on an
octree of 8^3-cell subgrids (Sec. 4.3.2) that conserves linear momentum and,
with a special technique, angular momentum (Sec. 4.3.1).  The oracle's
formulas are a reading of that prose; these tests tie every step to
mathematics that holds independently of the reading:

* D-tensors against finite differences of 1/r and against tracelessness;
* M2M against moments taken directly from the point masses;
* L2L against direct evaluation of the shifted polynomial;
* M2L order (error ~ (a/R)^4 in phi) against direct summation;
* theta -> 0 (every pair near) against O(N^2) direct summation;
* the interaction partition against an independent pair-by-pair enumeration;
* conservation of momentum and angular momentum (Sec. 4.3.1);
* degree-1 homogeneity, the uniform-sphere closed form, the cube self
  potential closed form;
* the dual-number derivative against central differences;
* the sampled solve against the full solve at its cells;
* the pair reverse against central differences of the pair.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2412_15518_gb300 import inputs as I


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module")
def sphere():
    lv, r = I.workload("sphere_l1")
    return lv, r


@pytest.fixture(scope="module")
def small_amr():
    # level-3 AMR refined on the binary: leaves at levels 1..3 (2:1 balanced)
    lv = I.amr_leaves(3, 2e-4, I.BINARY)
    return lv, I.density(lv, I.BINARY, seed=5)


def masses_positions(lv, rho):
    x = I.cell_centres(lv)
    h = 1.0 / (8.0 * 2.0 ** lv[:, 0])
    return rho * h[:, None] ** 3, x


# --------------------------------------------------------------------------
# D-tensors
def test_dtensor_is_derivative_of_inverse_distance():
    rng = np.random.default_rng(0)
    for _ in range(5):
        R = rng.normal(size=3)
        D = O.dtensor(R)
        assert abs(D[0] - 1 / np.linalg.norm(R)) < 1e-15
        eps = 1e-5
        for n in range(1, 5):
            # D^(n)_{..., i} = d/dR_i D^(n-1)_{...}  (central differences)
            fd = np.zeros((3,) * n)
            for i in range(3):
                e = np.zeros(3)
                e[i] = eps
                fd[..., i] = (np.asarray(O.dtensor(R + e)[n - 1]) -
                              np.asarray(O.dtensor(R - e)[n - 1])) / (2 * eps)
            assert np.abs(fd - D[n]).max() < 1e-8 * max(1.0, np.abs(D[n]).max())
        # harmonic: every trace vanishes; every tensor is symmetric
        for n in range(2, 5):
            T = np.asarray(D[n])
            assert np.abs(np.trace(T, axis1=0, axis2=1)).max() < 1e-12 * np.abs(T).max()
            for p in itertools.permutations(range(n)):
                assert np.abs(T - np.transpose(T, p)).max() < 1e-13 * np.abs(T).max()


# --------------------------------------------------------------------------
# Upward pass: U1 + U2 must reproduce the moments of the point masses exactly.
def direct_moments(m, x):
    M0 = m.sum()
    X = (m[:, None] * x).sum(0) / M0
    y = x - X
    M2 = np.einsum("n,ni,nj->ij", m, y, y)
    M3 = np.einsum("n,ni,nj,nk->ijk", m, y, y, y)
    return M0, X, M2, M3


def test_m2m_matches_direct_moments_of_points():
    rng = np.random.default_rng(1)
    pts = rng.uniform(size=(37, 3))
    m = rng.uniform(0.1, 1.0, size=37)
    got = O.unpack_mom(O.p2m_m2m(pts, m))
    M0, X, M2, M3 = direct_moments(m, pts)
    assert abs(got["m"] - M0) < 1e-14 * M0
    assert np.abs(got["X"] - X).max() < 1e-14
    assert np.abs(got["M2"] - M2).max() < 1e-13 * np.abs(M2).max()
    assert np.abs(got["M3"] - M3).max() < 1e-13 * np.abs(M3).max()
    # two-stage M2M (points -> 4 groups -> 1) equals one stage
    groups = [O.p2m_m2m(pts[i::4], m[i::4]) for i in range(4)]
    two = O.unpack_mom(O.m2m(np.stack(groups)))
    assert np.abs(two["M3"] - M3).max() < 1e-13 * np.abs(M3).max()
    assert np.abs(two["M2"] - M2).max() < 1e-13 * np.abs(M2).max()


@pytest.mark.parametrize("which", ["sphere", "small_amr"])
def test_tree_moments_match_point_masses(which, request):
    lv, rho = request.getfixturevalue(which)
    m, x = masses_positions(lv, rho)
    xyz, mom = O.level_moments(lv, rho, 0)
    assert xyz.shape == (1, 3)
    # level-0 cell c covers the leaf cells whose centres fall in it
    h0 = 1.0 / 8
    cell0 = np.floor(x / h0).astype(int)
    key = cell0[..., 0] + 8 * cell0[..., 1] + 64 * cell0[..., 2]
    for c in [0, 73, 219, 292, 511]:
        sel = key == c
        M0, X, M2, M3 = direct_moments(m[sel], x[sel])
        got = O.unpack_mom(mom[0, c])
        assert abs(got["m"] - M0) <= 1e-13 * M0
        assert np.abs(got["X"] - X).max() < 1e-14
        assert np.abs(got["M2"] - M2).max() <= 1e-12 * np.abs(M2).max()
        assert np.abs(got["M3"] - M3).max() <= 1e-11 * np.abs(M3).max() + 1e-30


# --------------------------------------------------------------------------
# Downward pass: L2L is the exact shift of a degree-3 polynomial.
def poly_eval(L0, L1, L2, L3, r):
    return (L0 + L1 @ r + 0.5 * r @ L2 @ r + np.einsum("ijk,i,j,k->", L3, r, r, r) / 6.0)


def poly_grad(L1, L2, L3, r):
    return L1 + L2 @ r + 0.5 * np.einsum("ijk,j,k->i", L3, r, r)


def sym(T):
    n = T.ndim
    return sum(np.transpose(T, p) for p in itertools.permutations(range(n))) / len(
        list(itertools.permutations(range(n))))


def test_l2l_is_exact_polynomial_shift():
    rng = np.random.default_rng(2)
    L0 = rng.normal()
    L1 = rng.normal(size=3)
    L2 = sym(rng.normal(size=(3, 3)))
    L3 = sym(rng.normal(size=(3, 3, 3)))
    ac = rng.normal(size=3)
    loc = np.concatenate([[L0], L1, L2.ravel(), L3.ravel(), ac])
    for _ in range(5):
        d = rng.normal(size=3)
        s = O.unpack_loc(O.l2l(loc, d))
        r = rng.normal(size=3)
        # shifted polynomial at r equals the original at d + r
        assert abs(poly_eval(s["L0"], s["L1"], s["L2"], s["L3"], r) -
                   poly_eval(L0, L1, L2, L3, d + r)) < 1e-12
        assert np.abs(poly_grad(s["L1"], s["L2"], s["L3"], r) -
                      poly_grad(L1, L2, L3, d + r)).max() < 1e-12
        assert np.abs(s["ac"] - ac).max() == 0.0


# --------------------------------------------------------------------------
# M2L: order-3 truncation => phi error ~ (a/R)^4 against direct summation.
def test_m2l_truncation_order_against_direct_sum():
    rng = np.random.default_rng(3)
    a = 0.05
    pa = rng.uniform(-a, a, size=(20, 3))
    pb = rng.uniform(-a, a, size=(20, 3))
    ma = rng.uniform(0.5, 1.5, 20)
    mb = rng.uniform(0.5, 1.5, 20)
    errs_phi, errs_g, Rs = [], [], []
    for R in [0.4, 0.8, 1.6, 3.2]:
        off = np.array([R, 0.3 * R, -0.2 * R])
        A = O.p2m_m2m(pa + off, ma)
        B = O.p2m_m2m(pb, mb)
        loc = O.m2l(A, B, G=1.0, am_correction=False)
        XA = A[1:4]
        ephi, eg = 0.0, 0.0
        for i in range(20):
            xi = pa[i] + off
            s = O.unpack_loc(O.l2l(loc, xi - XA))
            r = xi - pb
            d = np.linalg.norm(r, axis=1)
            phi_ex = -(mb / d).sum()
            g_ex = -(mb[:, None] * r / d[:, None] ** 3).sum(0)
            ephi = max(ephi, abs(s["L0"] - phi_ex) / abs(phi_ex))
            eg = max(eg, np.linalg.norm(-s["L1"] - g_ex) / np.linalg.norm(g_ex))
        errs_phi.append(ephi)
        errs_g.append(eg)
        Rs.append(R)
    sp = np.polyfit(np.log(Rs), np.log(errs_phi), 1)[0]
    sg = np.polyfit(np.log(Rs), np.log(errs_g), 1)[0]
    # phi: first omitted terms have total order 4 -> relative error (a/R)^4;
    # g: pointwise the (2,2) and (4,0) terms are of relative order (a/R)^3.
    assert -4.5 < sp < -3.5, sp
    assert -3.5 < sg < -2.5, sg


def test_am_correction_gives_the_top_order_mean_force():
    """The mass-weighted mean acceleration of cluster A from L1 + ac equals
    the exact mean force to order (a/R)^4 (the correction supplies the
    missing total-order-3 orbital term), versus (a/R)^3 without it."""
    rng = np.random.default_rng(4)
    a = 0.05
    pa = rng.uniform(-a, a, size=(30, 3))
    pb = rng.uniform(-a, a, size=(30, 3))
    ma = rng.uniform(0.5, 1.5, 30)
    mb = rng.uniform(0.5, 1.5, 30)
    slopes = {}
    for am in (True, False):
        errs, Rs = [], []
        for R in [0.4, 0.8, 1.6, 3.2]:
            off = np.array([R, 0.3 * R, -0.2 * R])
            A = O.p2m_m2m(pa + off, ma)
            B = O.p2m_m2m(pb, mb)
            loc = O.m2l(A, B, G=1.0, am_correction=am)
            XA = A[1:4]
            F = np.zeros(3)
            Fex = np.zeros(3)
            for i in range(30):
                xi = pa[i] + off
                s = O.unpack_loc(O.l2l(loc, xi - XA))
                F += ma[i] * (-s["L1"] + s["ac"])
                r = xi - pb
                d = np.linalg.norm(r, axis=1)
                Fex += ma[i] * -(mb[:, None] * r / d[:, None] ** 3).sum(0)
            errs.append(np.linalg.norm(F - Fex) / np.linalg.norm(Fex))
            Rs.append(R)
        slopes[am] = np.polyfit(np.log(Rs), np.log(errs), 1)[0]
    assert slopes[True] < -3.5, slopes
    assert -3.5 < slopes[False] < -2.5, slopes


# --------------------------------------------------------------------------
# Whole solve against direct summation.
def test_theta_to_zero_equals_direct_sum(sphere):
    """With 1/theta above the grid diameter every pair is near, so the FMM
    reduces to exact point-mass summation."""
    lv, rho = sphere
    phi_d, g_d = O.direct(lv, rho)
    phi, g, cnt = O.solve(lv, rho, theta=0.03, return_counts=True)
    assert cnt["m2l"] == 0 and cnt["seam"] == 0
    assert cnt["p2p"] == 4096 * 4095
    assert rel(phi, phi_d) < 1e-13
    assert rel(g, g_d) < 1e-13


def test_error_against_direct_sum_shrinks_with_theta(sphere):
    lv, rho = sphere
    phi_d, g_d = O.direct(lv, rho)
    e = []
    for th in (0.5, 0.4, 1.0 / 3.0):
        phi, g = O.solve(lv, rho, theta=th)
        e.append((rel(phi, phi_d), rel(g, g_d)))
    # measured at theta = 0.5: phi 2.3e-4, g 7.1e-3 (max-norm relative)
    assert e[0][0] < 5e-4 and e[0][1] < 1.5e-2
    assert e[0][0] > e[1][0] > e[2][0]
    assert e[0][1] > e[1][1] > e[2][1]


def test_amr_error_against_direct_sum(small_amr):
    """Mixed leaf/interior near pairs interact through the interior cell's
    multipole at distances down to one cell, so the AMR error is larger than
    the uniform one (measured at theta = 0.5: phi 4.0e-3, g 5.4e-2) and
    shrinks with theta."""
    lv, rho = small_amr
    phi_d, g_d = O.direct(lv, rho)
    e = []
    for th in (0.5, 0.4, 1.0 / 3.0):
        phi, g, cnt = O.solve(lv, rho, theta=th, return_counts=True)
        assert cnt["seam"] > 0
        e.append((rel(phi, phi_d), rel(g, g_d)))
    assert e[0][0] < 8e-3 and e[0][1] < 0.1
    assert e[0][0] > e[1][0] > e[2][0]
    assert e[0][1] > e[1][1] > e[2][1]


# --------------------------------------------------------------------------
# Interaction partition: each unordered pair of leaf cells is covered by
# exactly one ancestor pair, found here pair by pair (top-down walk) and
# counted independently of the oracle's stencil loops.
def partition_counts(lv, theta):
    x = I.cell_centres(lv).reshape(-1, 3)
    L = np.repeat(lv[:, 0], 512).astype(np.int64)
    h = 1.0 / (8.0 * 2.0 ** L)
    c = np.floor(x / h[:, None]).astype(np.int64)  # cell index at its own level
    n = c.shape[0]
    it2 = 1.0 / theta ** 2
    keys = {1: [], 2: [], 3: []}
    for a in range(n):
        b = np.arange(a + 1, n)
        done = np.zeros(b.size, bool)
        for q in range(0, int(L.max()) + 1):
            act = np.nonzero(~done)[0]
            if act.size == 0:
                break
            bb = b[act]
            ca = c[a] >> (L[a] - q)
            cb = c[bb] >> (L[bb] - q)[:, None]
            leaf_a = L[a] == q
            leaf_b = L[bb] == q
            near = ((cb - ca) ** 2).sum(1) <= it2
            cls = np.where(near, np.where(leaf_b & leaf_a, 2, np.where(leaf_b | leaf_a, 3, 0)), 1)
            # an unordered ancestor pair, encoded as one integer
            ka = ca[0] + 64 * ca[1] + 4096 * ca[2]
            kb = cb[:, 0] + 64 * cb[:, 1] + 4096 * cb[:, 2]
            key = (q * 2 ** 18 + np.minimum(ka, kb)) * 2 ** 18 + np.maximum(ka, kb)
            for k in (1, 2, 3):
                keys[k].append(key[cls == k])
            done[act[cls > 0]] = True
        assert done.all()
    return {k: 2 * np.unique(np.concatenate(v)).size for k, v in keys.items()}


def test_partition_counts_match_independent_enumeration():
    lv = np.array([[1, x, y, z] for z in range(2) for y in range(2) for x in range(2)], np.int32)
    # a level-2 refinement of one corner keeps a small but non-uniform tree
    lv = np.concatenate([lv[1:], [[2, x, y, z] for z in range(2) for y in range(2)
                                  for x in range(2)]]).astype(np.int32)
    rho = I.density(lv, I.SPHERE, seed=1)
    _, _, cnt = O.solve(lv, rho, return_counts=True)
    want = partition_counts(lv, 0.5)
    assert cnt == {"m2l": want[1], "p2p": want[2], "seam": want[3]}, (cnt, want)


def test_uniform_counts_level1():
    # directed pairs of the uniform level-1 tree at theta = 0.5
    _, _, c1 = O.solve(*I.workload("sphere_l1"), return_counts=True)
    assert c1 == {"m2l": 959280, "p2p": 114744, "seam": 0}


# --------------------------------------------------------------------------
# Conservation (Sec. 4.3.1).
def residuals(lv, rho, g):
    m, x = masses_positions(lv, rho)
    f = m[:, :, None] * np.moveaxis(g, 1, 2)           # [n, 512, 3]
    mom = np.abs(f.sum((0, 1))).max() / np.abs(f).sum()
    tq = np.cross(x - 0.5, f)
    ang = np.abs(tq.sum((0, 1))).max() / np.abs(tq).sum()
    return mom, ang


@pytest.mark.parametrize("which", ["sphere", "small_amr"])
def test_momentum_and_angular_momentum_conserved(which, request):
    lv, rho = request.getfixturevalue(which)
    _, g = O.solve(lv, rho)
    mom, ang = residuals(lv, rho, g)
    assert mom < 1e-14
    assert ang < 1e-12
    _, g0 = O.solve(lv, rho, am_correction=False)
    mom0, ang0 = residuals(lv, rho, g0)
    assert mom0 < 1e-14          # linear momentum needs no correction
    assert ang0 > 1e3 * ang      # without the correction torque is not conserved


def test_homogeneity_degree_one(small_amr):
    lv, rho = small_amr
    phi, g = O.solve(lv, rho)
    phi3, g3 = O.solve(lv, 3.0 * rho)
    assert rel(phi3, 3.0 * phi) < 1e-14
    assert rel(g3, 3.0 * g) < 1e-14


def test_uniform_sphere_closed_form():
    """Outside a spherically symmetric mass phi = -G M / r; inside a uniform
    ball g = -G M r / R^3 (up to voxelisation of the ball on the grid)."""
    lv = I.uniform_leaves(2)
    x = I.cell_centres(lv)
    R = 0.3
    r = np.linalg.norm(x - 0.5, axis=-1)
    rho = np.where(r < R, 1.0, 1e-10)
    m, _ = masses_positions(lv, rho)
    M = m.sum()
    phi, g = O.solve(lv, rho)
    out = r > 0.42
    assert np.abs(phi[out] + M / r[out]).max() / np.abs(M / r[out]).max() < 3e-3
    inner = (r < 0.2) & (r > 0.05)
    gin = np.moveaxis(g, 1, 2)[inner]
    gex = -M * (x[inner] - 0.5) / R ** 3
    assert np.linalg.norm(gin - gex, axis=1).max() / np.linalg.norm(gex, axis=1).max() < 0.1


def test_cube_self_constant_closed_form():
    """int_{[-1/2,1/2]^3} dV/|r| = 3 (ln(2 + sqrt 3) - pi/6): the pyramid
    reduction gives 3 int_0^1 int_0^1 du dv / sqrt(1+u^2+v^2), whose value
    follows from int_0^1 asinh(1/sqrt(1+u^2)) du by parts."""
    assert abs(O.cube_self_constant() - 3 * (np.log(2 + np.sqrt(3)) - np.pi / 6)) < 1e-13


def test_self_term_adds_cube_self_potential(sphere):
    lv, rho = sphere
    phi, g = O.solve(lv, rho)
    phis, gs = O.solve(lv, rho, self_term=True)
    h = 1.0 / 16
    C = 3 * (np.log(2 + np.sqrt(3)) - np.pi / 6)
    assert np.abs(phis - phi + rho * h * h * C).max() < 1e-14 * np.abs(phi).max()
    assert np.array_equal(gs, g)


# --------------------------------------------------------------------------
def test_dual_number_derivative_matches_central_differences(small_amr):
    lv, rho = small_amr
    rng = np.random.default_rng(7)
    v = rng.normal(size=rho.shape) * rho
    phi, g, dphi, dg = O.solve_jvp(lv, rho, v)
    p0, g0 = O.solve(lv, rho)
    assert np.array_equal(phi, p0) and np.array_equal(g, g0)
    eps = 1e-4
    pp, gp = O.solve(lv, rho + eps * v)
    pm, gm = O.solve(lv, rho - eps * v)
    assert rel(dphi, (pp - pm) / (2 * eps)) < 1e-7
    assert rel(dg, (gp - gm) / (2 * eps)) < 1e-6


def test_invalid_trees_are_rejected():
    good = I.uniform_leaves(1)
    assert O.check_tree(good) == 0
    assert O.check_tree(good[1:]) == -3                                # hole
    assert O.check_tree(np.concatenate([good, good[:1]])) == -2          # duplicate
    assert O.check_tree(np.concatenate([good, [[2, 0, 0, 0]]])) == -2    # leaf inside a leaf
    assert O.check_tree(np.array([[1, 2, 0, 0]], np.int32)) == -1        # out of range


# --------------------------------------------------------------------------
# Adjoint of the solve (hand-written reverse sweep in the oracle).
def test_dtensor5_is_derivative_of_d4():
    rng = np.random.default_rng(8)
    for _ in range(3):
        R = rng.normal(size=3)
        D5 = O.dtensor5(R)
        eps = 1e-5
        fd = np.zeros((3,) * 5)
        for i in range(3):
            e = np.zeros(3)
            e[i] = eps
            fd[..., i] = (O.dtensor(R + e)[4] - O.dtensor(R - e)[4]) / (2 * eps)
        assert np.abs(fd - D5).max() < 1e-8 * np.abs(D5).max()
        assert np.abs(np.trace(D5, axis1=1, axis2=3)).max() < 1e-12 * np.abs(D5).max()
        for p in itertools.permutations(range(5)):
            assert np.abs(D5 - np.transpose(D5, p)).max() < 1e-13 * np.abs(D5).max()


def J_of(lv, rho, w1, w2, **kw):
    phi, g = O.solve(lv, rho, **kw)
    return float((w1 * phi).sum() + (w2 * g).sum())


@pytest.mark.parametrize("which", ["sphere", "small_amr"])
@pytest.mark.parametrize("am", [True, False])
def test_gradient_matches_dual_number_directional_derivative(which, am, request):
    """<dJ/drho, v> from the reverse sweep equals the forward-mode (dual
    number) derivative of J along v: two independent differentiations of the
    same discrete solve (through centres of mass and the mass ratio)."""
    lv, rho = request.getfixturevalue(which)
    w1, w2 = I.weights(lv.shape[0])
    gr = O.gradient(lv, rho, w1, w2, am_correction=am)
    for seed in (3, 4):
        v = np.random.default_rng(seed).normal(size=rho.shape) * rho
        _, _, dphi, dg = O.solve_jvp(lv, rho, v, am_correction=am)
        jvp = (w1 * dphi).sum() + (w2 * dg).sum()
        assert abs((gr * v).sum() - jvp) < 1e-12 * abs(jvp)


def test_gradient_euler_identity(small_amr):
    """J is homogeneous of degree 1 in rho, so sum rho dJ/drho = J."""
    lv, rho = small_amr
    w1, w2 = I.weights(lv.shape[0])
    gr = O.gradient(lv, rho, w1, w2)
    J = J_of(lv, rho, w1, w2)
    assert abs((gr * rho).sum() - J) < 1e-13 * abs(J)


def test_gradient_central_differences(sphere):
    """Central differences with h = 1e-6 (densities in units of the central
    density) at 16 seeded cells inside the star."""
    lv, rho = sphere
    w1, w2 = I.weights(lv.shape[0])
    gr = O.gradient(lv, rho, w1, w2).reshape(-1)
    inside = np.nonzero(rho.reshape(-1) > 1e-2)[0]
    cells = np.random.default_rng(3).choice(inside, size=16, replace=False)
    h = 1e-6
    for c in cells:
        rp = rho.copy().reshape(-1)
        rm = rho.copy().reshape(-1)
        rp[c] += h
        rm[c] -= h
        fd = (J_of(lv, rp.reshape(rho.shape), w1, w2) - J_of(lv, rm.reshape(rho.shape), w1, w2)) / (2 * h)
        assert abs(fd - gr[c]) < 1e-6 * abs(gr).max(), (c, fd, gr[c])


def test_gradient_self_term(sphere):
    lv, rho = sphere
    w1, w2 = I.weights(lv.shape[0])
    g0 = O.gradient(lv, rho, w1, w2)
    g1 = O.gradient(lv, rho, w1, w2, self_term=True)
    C = 3 * (np.log(2 + np.sqrt(3)) - np.pi / 6)
    assert np.abs(g1 - g0 + w1 * (1.0 / 16) ** 2 * C).max() < 1e-12 * np.abs(g0).max()


# --------------------------------------------------------------------------
# Empty space.  A cell of zero total mass has no centre of mass and no mass
# ratio; the readings are: its moments are taken about its geometric centre,
# and the correction's target term -(m_B / m_A) M3_A (M3_A = 0 for
# non-negative densities) is zero.  Both must be the limit of a vanishing
# uniform atmosphere, where every quantity is defined.
EPS_ATM = 1e-150


def empty_and_limit(lv, stars, seed):
    rho0 = I.density(lv, stars, seed, atmosphere=0.0)
    rho_eps = np.where(rho0 == 0.0, EPS_ATM, rho0)   # uniform: no noise outside the stars
    return rho0, rho_eps


@pytest.fixture(scope="module")
def empty_sphere():
    lv = I.uniform_leaves(1)
    rho0, rho_eps = empty_and_limit(lv, I.SPHERE, 0)
    assert (rho0 == 0.0).mean() > 0.4      # most of the cube is empty
    return lv, rho0, rho_eps


@pytest.fixture(scope="module")
def empty_amr():
    lv = I.amr_leaves(3, 2e-4, I.BINARY)
    rho0, rho_eps = empty_and_limit(lv, I.BINARY, 5)
    return lv, rho0, rho_eps


@pytest.mark.parametrize("which", ["empty_sphere", "empty_amr"])
@pytest.mark.parametrize("am", [True, False])
def test_zero_mass_cells_are_the_vanishing_atmosphere_limit(which, am, request):
    lv, rho0, rho_eps = request.getfixturevalue(which)
    phi0, g0 = O.solve(lv, rho0, am_correction=am)
    phie, ge = O.solve(lv, rho_eps, am_correction=am)
    assert np.isfinite(phi0).all() and np.isfinite(g0).all()
    assert rel(phi0, phie) < 1e-13
    assert rel(g0, ge) < 1e-13


def test_zero_mass_cells_theta_to_zero_equals_direct_sum(empty_sphere):
    lv, rho0, _ = empty_sphere
    phi_d, g_d = O.direct(lv, rho0)
    phi, g = O.solve(lv, rho0, theta=0.03)
    assert rel(phi, phi_d) < 1e-13
    assert rel(g, g_d) < 1e-13


@pytest.mark.parametrize("which", ["empty_sphere", "empty_amr"])
def test_zero_mass_cells_conserve_momentum_and_angular_momentum(which, request):
    lv, rho0, _ = request.getfixturevalue(which)
    _, g = O.solve(lv, rho0)
    mom, ang = residuals(lv, rho0, g)
    assert mom < 1e-14
    assert ang < 1e-12


@pytest.mark.parametrize("which", ["empty_sphere", "empty_amr"])
def test_zero_mass_gradient(which, request):
    """The gradient is finite; on cells inside the stars it equals the
    gradient of the vanishing-atmosphere field, and it agrees with the
    forward-mode derivative along directions inside the stars."""
    lv, rho0, rho_eps = request.getfixturevalue(which)
    w1, w2 = I.weights(lv.shape[0])
    gr0 = O.gradient(lv, rho0, w1, w2)
    assert np.isfinite(gr0).all()
    star = rho0 > 0.0
    gre = O.gradient(lv, rho_eps, w1, w2)
    assert np.abs(gr0 - gre)[star].max() < 1e-12 * np.abs(gre[star]).max()
    v = np.random.default_rng(3).normal(size=rho0.shape) * rho0
    _, _, dphi, dg = O.solve_jvp(lv, rho0, v)
    jvp = (w1 * dphi).sum() + (w2 * dg).sum()
    assert abs((gr0 * v).sum() - jvp) < 1e-12 * abs(jvp)


# --------------------------------------------------------------------------
# the sampled solve and the pair reverse


def test_sampled_solve_equals_the_full_solve_at_its_cells(small_amr):
    # the sampled solve (used at full sizes, where the full oracle is too slow)
    # evaluates the same algorithm for the sampled leaf cells only
    lv, rho = small_amr
    phi, g = O.solve(lv, rho)
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(lv.shape[0] * 512, size=200, replace=False))
    phi_s, g_s = O.solve_sample(lv, rho, sample)
    assert rel(phi_s, phi.reshape(-1)[sample]) < 1e-13
    g_full = np.moveaxis(g, 1, 2).reshape(-1, 3)[sample]
    assert rel(g_s, g_full) < 1e-13


def _sym_moment_direction(rng):
    # a direction in moment space (m, X[3], M2[9], M3[27]) with symmetric M2, M3
    v = np.zeros(40)
    v[0] = rng.standard_normal()
    v[1:4] = rng.standard_normal(3)
    a = rng.standard_normal((3, 3))
    v[4:13] = ((a + a.T) / 2).reshape(-1)
    b = rng.standard_normal((3, 3, 3))
    s = sum(np.transpose(b, p) for p in itertools.permutations(range(3))) / 6.0
    v[13:40] = s.reshape(-1)
    return v


@pytest.mark.parametrize("am", [True, False])
def test_pair_reverse_is_the_gradient_of_the_pair(am):
    # J = Ebar . m2l(A, B); the pair reverse must give dJ/dA and dJ/dB, checked
    # by central differences along random symmetric directions
    rng = np.random.default_rng(11)
    pa = rng.uniform(-0.05, 0.05, (6, 3)) + np.array([0.1, 0.2, 0.3])
    pb = rng.uniform(-0.05, 0.05, (6, 3)) + np.array([0.9, 0.6, 0.45])
    A = O.p2m_m2m(pa, rng.uniform(0.5, 1.5, 6))
    B = O.p2m_m2m(pb, rng.uniform(0.5, 1.5, 6))
    E = rng.standard_normal(43)
    J = lambda a, b: float(E @ O.m2l(a, b, am_correction=am))
    ga, gb = O.m2l_reverse(A, B, E, am_correction=am)
    for _ in range(4):
        va, vb = _sym_moment_direction(rng), _sym_moment_direction(rng)
        eps = 1e-5
        da = (J(A + eps * va, B) - J(A - eps * va, B)) / (2 * eps)
        db = (J(A, B + eps * vb) - J(A, B - eps * vb)) / (2 * eps)
        assert abs(ga @ va - da) <= 1e-7 * (abs(da) + np.abs(ga).max())
        assert abs(gb @ vb - db) <= 1e-7 * (abs(db) + np.abs(gb).max())
