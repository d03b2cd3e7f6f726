"""Pins of the adaptive-tree hydro right-hand-side oracle
(oracle/hydro_amr.py) against facts that do not come from it: equality with
the grid-wide oracle on uniform trees, steady uniform states across
refinement jumps, conservation of mass, momentum and energy across them
(flux matching), the closed-form rate of a linear state in uniform motion on
every level away from the jumps, and reflection symmetry."""
import numpy as np
import pytest

from oracle import hydro as H
from oracle import hydro_amr as A
from paper_2412_15518_gb300 import inputs as I

GAMMA = 5.0 / 3.0


def cells_of(leaves, fns, size=1.0):
    """Values of fns(x, y, z) at the cell centres (physical coordinates):
    [n_leaf, len(fns), 512]."""
    x = I.cell_centres(leaves, size=size)              # [n, 512, 3]
    return np.stack([np.broadcast_to(f(x[..., 0], x[..., 1], x[..., 2]), x.shape[:2]) for f in fns],
                    axis=1).astype(np.float64)


def conserved(rho, vel, p):
    def s(b):
        return lambda x, y, z: rho(x, y, z) * vel[b]

    def E(x, y, z):
        return p(x, y, z) / (GAMMA - 1.0) + 0.5 * rho(x, y, z) * sum(v * v for v in vel)
    return [rho, s(0), s(1), s(2), E]


def const(v):
    return lambda x, y, z: np.full(np.shape(x), v)


def levels_of(lv):
    return sorted(set(int(v) for v in np.asarray(lv)[:, 0]))


AMR_TREES = {
    "binary_l1_l2": lambda: I.amr_leaves(2, 5e-4, I.BINARY, lmin=1),
    "binary_l1_l3": lambda: I.amr_leaves(3, 2e-4, I.BINARY),
}


@pytest.mark.parametrize("level", [1, 2])
def test_equals_the_grid_oracle_on_uniform_trees(level):
    lv = I.uniform_leaves(level, seed=3)
    u = I.hydro_fields(lv, seed=level)
    g = np.random.default_rng(level).standard_normal((lv.shape[0], 3, 512))
    assert np.array_equal(A.rhs(lv, u, g, GAMMA), H.rhs(lv, u, g, GAMMA))


@pytest.mark.parametrize("tree", sorted(AMR_TREES))
def test_trees_have_refinement_jumps(tree):
    assert len(levels_of(AMR_TREES[tree]())) >= 2


@pytest.mark.parametrize("tree", sorted(AMR_TREES))
@pytest.mark.parametrize("vel", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.7)])
def test_uniform_state_is_steady_across_refinement_jumps(tree, vel):
    lv = AMR_TREES[tree]()
    u = cells_of(lv, conserved(const(1.3), vel, const(0.8)))
    d = A.rhs(lv, u)
    # the restriction's mean of 8 equal values may round by an ulp
    assert np.abs(d).max() < 1e-10


@pytest.mark.parametrize("tree", sorted(AMR_TREES))
def test_totals_are_conserved_across_refinement_jumps(tree):
    """A smooth perturbation of a gas at rest, zero beyond 0.25 of its centre
    (more than 3 level-1 cells from the domain boundary): the volume-weighted sum of the rates (mass, momentum, energy)
    is the boundary flux of the background, which cancels; the fine and
    coarse sides of every level jump exchange the same flux."""
    lv = AMR_TREES[tree]()
    bump = lambda x, y, z: np.maximum(
        1.0 - ((x - 0.45) ** 2 + (y - 0.5) ** 2 + (z - 0.52) ** 2) / 0.0625, 0.0) ** 4
    fns = [lambda x, y, z: 1.0 + 0.5 * bump(x, y, z),
           lambda x, y, z: 0.3 * bump(x, y, z) * (y - 0.5),
           lambda x, y, z: -0.2 * bump(x, y, z) * (x - 0.45),
           lambda x, y, z: 0.1 * bump(x, y, z),
           lambda x, y, z: 1.5 + 0.8 * bump(x, y, z)]
    u = cells_of(lv, fns)
    d = A.rhs(lv, u)
    vol = (1.0 / (8 << np.asarray(lv)[:, 0].astype(np.int64))) ** 3        # cell volume per leaf
    total = (d * vol[:, None, None]).sum(axis=(0, 2))
    scale = (np.abs(d) * vol[:, None, None]).sum(axis=(0, 2))
    assert np.all(np.abs(total) < 1e-12 * scale), total / scale
    assert np.abs(d).max() > 0.1


def test_flux_matching_is_what_conserves():
    """The same state without matching (each leaf's own fluxes) does not
    conserve mass: the pin above is not trivially satisfied."""
    lv = AMR_TREES["binary_l1_l3"]()
    bump = lambda x, y, z: np.maximum(
        1.0 - ((x - 0.45) ** 2 + (y - 0.5) ** 2 + (z - 0.52) ** 2) / 0.0625, 0.0) ** 4
    u = cells_of(lv, [lambda x, y, z: 1.0 + 0.5 * bump(x, y, z), lambda x, y, z: 0.2 * bump(x, y, z),
                      const(0.0), const(0.0), lambda x, y, z: 1.5 + 0.8 * bump(x, y, z)])
    leaves = np.asarray(lv)
    lm = A.leaf_map(leaves)
    vol = (1.0 / (8 << leaves[:, 0].astype(np.int64))) ** 3
    own = 0.0
    for i in range(leaves.shape[0]):
        F = A.leaf_fluxes(leaves, A.block_values(A.halo(leaves, lm, u, i)), i, GAMMA)
        h = 1.0 / (8 << int(leaves[i, 0]))
        d = sum(F[a][0].take(range(8), axis=2 - a) - F[a][0].take(range(1, 9), axis=2 - a)
                for a in range(3)) / h
        own += d.sum() * vol[i]
    scale = np.abs(A.rhs(lv, u)[:, 0] * vol[:, None]).sum()
    assert abs(own) > 1e-8 * scale


@pytest.mark.parametrize("tree", sorted(AMR_TREES))
def test_linear_state_advects_at_the_closed_form_rate_away_from_jumps(tree):
    """rho = 1 + b.x, uniform v and p: every cell at least 3 cells (of its
    level) from the domain boundary and from a leaf of another level changes
    at d rho/dt = -v.b, d s/dt = -v (v.b), dE/dt = -|v|^2 (v.b) / 2."""
    lv = np.asarray(AMR_TREES[tree]())
    b = np.array([0.3, -0.2, 0.15])
    vel = (0.4, -0.3, 0.25)
    u = cells_of(lv, conserved(lambda x, y, z: 1.0 + b[0] * x + b[1] * y + b[2] * z, vel, const(0.9)))
    d = A.rhs(lv, u)
    vb = vel[0] * b[0] + vel[1] * b[1] + vel[2] * b[2]
    v2 = sum(v * v for v in vel)
    want = np.array([-vb] + [-vel[a] * vb for a in range(3)] + [-0.5 * v2 * vb])
    lm = A.leaf_map(lv)
    c = np.arange(8)
    kk, jj, ii = np.meshgrid(c, c, c, indexing="ij")
    checked = 0
    for i, (L, nx, ny, nz) in enumerate(lv):
        N = 8 << int(L)
        gl = np.stack([8 * nx + ii, 8 * ny + jj, 8 * nz + kk]).reshape(3, -1)
        ok = np.all((gl >= 3) & (gl < N - 3), axis=0)
        # cells within 3 cells of a neighbour node at another level are excluded
        for s in np.ndindex(3, 3, 3):
            o = np.array(s) - 1
            if not o.any():
                continue
            key = (int(L), nx + o[0], ny + o[1], nz + o[2])
            if min(key[1:]) < 0 or max(key[1:]) >= (1 << int(L)) or key in lm:
                continue
            loc = gl - 8 * np.array([nx, ny, nz])[:, None]
            near = np.ones(512, bool)
            for a in range(3):
                if o[a] < 0:
                    near &= loc[a] < 3
                elif o[a] > 0:
                    near &= loc[a] > 4
            ok &= ~near
        if ok.any():
            checked += int(ok.sum())
            assert np.abs(d[i][:, ok] - want[:, None]).max() < 1e-11
    assert checked > 0


def test_reflection_reflects_the_rates():
    """A tree refined on a centred sphere is symmetric under x -> -x; the
    rates of the reflected state (s_x negated) are the reflected rates."""
    lv = np.asarray(I.amr_leaves(3, 1e-3, I.SPHERE, lmin=1))
    assert len(levels_of(lv)) >= 2
    u = I.hydro_fields(lv, I.SPHERE, seed=4)
    lm = A.leaf_map(lv)
    perm = np.array([lm[(int(L), (1 << int(L)) - 1 - int(x), int(y), int(z))] for L, x, y, z in lv])
    ur = u[perm].reshape(-1, 5, 8, 8, 8)[..., ::-1].copy()
    ur[:, 1] = -ur[:, 1]
    a = A.rhs(lv, u)
    b = A.rhs(lv, ur.reshape(-1, 5, 512))[perm].reshape(-1, 5, 8, 8, 8)[..., ::-1].copy()
    b[:, 1] = -b[:, 1]
    scale = np.abs(a).max()
    assert np.abs(a - b.reshape(a.shape)).max() <= 1e-12 * scale
