"""Pins of the hydro right-hand-side oracle (oracle/hydro.py) against facts
that do not come from it: steady uniform states, the gravity source alone,
the Euler flux written out independently, the face rule's exactness on a
bicubic advected density (the integral by calculus), the exact rate of
change of a linear state in uniform motion (a closed form), conservation (interior
fluxes telescope), the reduction to a 1-D finite-volume scheme on one axis,
and reflection symmetry."""
import numpy as np
import pytest

from oracle import hydro as H
from oracle import ppm as P
from paper_2412_15518_gb300 import inputs as I

GAMMA = 5.0 / 3.0


def field_of(leaves, fns):
    """Cell values of the functions fns(i, j, k) (global cell indices) laid
    out per leaf: [n_leaf, len(fns), 512]."""
    leaves = np.asarray(leaves)
    c = np.arange(8)
    kk, jj, ii = np.meshgrid(c, c, c, indexing="ij")
    out = np.empty((leaves.shape[0], len(fns), 512))
    for n, (_, ix, iy, iz) in enumerate(leaves):
        for f, fn in enumerate(fns):
            v = fn(8 * ix + ii, 8 * iy + jj, 8 * iz + kk)
            out[n, f] = np.broadcast_to(v, ii.shape).reshape(-1)
    return out


def conserved(rho, vel, p):
    """Conserved fields from primitive functions of (i, j, k)."""
    def s(b):
        return lambda i, j, k: rho(i, j, k) * vel[b]

    def E(i, j, k):
        r = rho(i, j, k)
        return p(i, j, k) / (GAMMA - 1.0) + 0.5 * r * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    return [rho, s(0), s(1), s(2), E]


def const(v):
    return lambda i, j, k: np.full(np.shape(i), v, dtype=float)


@pytest.mark.parametrize("vel", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.7)])
def test_uniform_state_is_steady(vel):
    lv = I.uniform_leaves(1)
    u = field_of(lv, conserved(const(1.3), vel, const(0.8)))
    assert np.all(H.rhs(lv, u) == 0.0)


def test_uniform_state_under_gravity_feels_the_source_only():
    lv = I.uniform_leaves(1)
    vel = (0.3, -0.2, 0.7)
    u = field_of(lv, conserved(const(1.3), vel, const(0.8)))
    g = np.random.default_rng(3).standard_normal((lv.shape[0], 3, 512))
    d = H.rhs(lv, u, g)
    assert np.all(d[:, 0] == 0.0)
    for b in range(3):
        assert np.allclose(d[:, 1 + b], 1.3 * g[:, b], rtol=1e-15, atol=0)
    work = 1.3 * (vel[0] * g[:, 0] + vel[1] * g[:, 1] + vel[2] * g[:, 2])
    assert np.allclose(d[:, 4], work, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("a", [0, 1, 2])
def test_flux_of_equal_states_is_the_euler_flux(a):
    rng = np.random.default_rng(11 + a)
    rho = rng.uniform(0.5, 2.0, 50)
    v = rng.uniform(-1.0, 1.0, (3, 50))
    p = rng.uniform(0.1, 3.0, 50)
    E = p / (GAMMA - 1.0) + 0.5 * rho * (v ** 2).sum(axis=0)
    U = np.stack([rho, rho * v[0], rho * v[1], rho * v[2], E])
    F = np.stack(H.rusanov(U, U, a, GAMMA))
    # the Euler flux: mass rho v_a, momentum rho v_a v + p e_a, energy (E + p) v_a
    want = np.stack([rho * v[a]] + [rho * v[a] * v[b] + (p if b == a else 0.0) for b in range(3)]
                    + [(E + p) * v[a]])
    assert np.allclose(F, want, rtol=1e-13, atol=1e-14)


def test_linear_state_in_uniform_motion_advects_exactly():
    """rho = rho0 + b.x, uniform v and p: the reconstruction is exact and
    continuous at every face point, the Simpson rule integrates the linear
    fluxes exactly, so away from the boundary (three cells, where the ghost
    values are clamped) d rho/dt = -v.b, d s/dt = -v (v.b) and
    dE/dt = -|v|^2 (v.b) / 2, with h = 1/32 and b in cell units."""
    lv = I.uniform_leaves(2)
    n, h = 32, 1.0 / 32
    b = np.array([0.011, -0.007, 0.005])
    vel = (0.4, -0.3, 0.25)
    rho = lambda i, j, k: 1.0 + b[0] * i + b[1] * j + b[2] * k
    u = field_of(lv, conserved(rho, vel, const(0.9)))
    d = P.grid_of(lv, H.rhs(lv, u, gamma=GAMMA))
    vb = (vel[0] * b[0] + vel[1] * b[1] + vel[2] * b[2]) / h
    v2 = vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2
    s = slice(3, n - 3)
    want = [-vb] + [-vel[c] * vb for c in range(3)] + [-0.5 * v2 * vb]
    for f in range(5):
        assert np.abs(d[f][s, s, s] - want[f]).max() < 1e-11, f


def test_interior_fluxes_telescope():
    """A perturbation away from the boundary in a uniform gas at rest: the
    boundary fluxes are the background's on every side and cancel, so the
    totals of mass, momentum and energy do not change."""
    lv = I.uniform_leaves(2)
    rng = np.random.default_rng(5)
    pert = rng.uniform(-0.2, 0.2, (5, 32, 32, 32))
    mask = np.zeros((32, 32, 32))
    mask[6:26, 6:26, 6:26] = 1.0
    base = [1.0, 0.0, 0.0, 0.0, 1.0 / (GAMMA - 1.0)]
    g = np.stack([base[f] + (0.5 if f in (0, 4) else 0.3) * pert[f] * mask for f in range(5)])
    u = np.empty((lv.shape[0], 5, 512))
    for m, (_, ix, iy, iz) in enumerate(lv):
        u[m] = g[:, 8 * iz:8 * iz + 8, 8 * iy:8 * iy + 8, 8 * ix:8 * ix + 8].reshape(5, 512)
    d = H.rhs(lv, u)
    scale = np.abs(d).max(axis=(0, 2))
    assert np.all(np.abs(d.sum(axis=(0, 2))) < 1e-11 * scale * d.shape[0] * 512)
    assert np.abs(d).max() > 1.0  # the perturbation does evolve


def line_rhs_1d(q, h):
    """Independent 1-D statement: PPM (Colella & Woodward 1984) on a line of
    cells with clamped ends, Rusanov fluxes at the interfaces (transmissive
    ends), conservative update; q [5, n] conserved fields along x."""
    nf, n = q.shape

    def at(f, i):
        return q[f, min(max(i, 0), n - 1)]

    def iface(f, i):  # between cells i and i + 1
        v = 7.0 / 12.0 * (at(f, i) + at(f, i + 1)) - 1.0 / 12.0 * (at(f, i - 1) + at(f, i + 2))
        return min(max(v, min(at(f, i), at(f, i + 1))), max(at(f, i), at(f, i + 1)))

    left = np.empty((nf, n))
    right = np.empty((nf, n))
    for f in range(nf):
        for i in range(n):
            a, aL, aR = at(f, i), iface(f, i - 1), iface(f, i)
            if (aR - a) * (a - aL) <= 0.0:
                aL = aR = a
            else:
                dd = aR - aL
                if dd * (a - 0.5 * (aL + aR)) > dd * dd / 6.0:
                    aL = 3.0 * a - 2.0 * aR
                elif -dd * dd / 6.0 > dd * (a - 0.5 * (aL + aR)):
                    aR = 3.0 * a - 2.0 * aL
            left[f, i], right[f, i] = aL, aR

    def euler(U):
        r, sx, sy, sz, E = U
        vx, vy, vz = sx / r, sy / r, sz / r
        p = (GAMMA - 1.0) * (E - 0.5 * r * (vx * vx + vy * vy + vz * vz))
        c = np.sqrt(max(GAMMA * p / r, 0.0))
        return np.array([sx, sx * vx + p, sx * vy, sx * vz, (E + p) * vx]), abs(vx) + c

    flux = np.empty((nf, n + 1))
    for i in range(n + 1):
        UL = right[:, i - 1] if i > 0 else left[:, 0]
        UR = left[:, i] if i < n else right[:, n - 1]
        FL, cl = euler(UL)
        FR, cr = euler(UR)
        flux[:, i] = 0.5 * (FL + FR) - 0.5 * max(cl, cr) * (UR - UL)
    return (flux[:, :-1] - flux[:, 1:]) / h


def test_state_varying_along_one_axis_follows_the_1d_scheme():
    lv = I.uniform_leaves(1)
    n, h = 16, 1.0 / 16
    rho = lambda i, j, k: 1.0 + 0.5 * np.sin(0.7 * i) + 0.2 * (i > 9)
    vx = lambda i, j, k: 0.3 * np.cos(0.4 * i)
    p = lambda i, j, k: 1.0 + 0.3 * np.cos(0.9 * i)
    fns = [rho, lambda i, j, k: rho(i, j, k) * vx(i, j, k), const(0.0), const(0.0),
           lambda i, j, k: p(i, j, k) / (GAMMA - 1.0) + 0.5 * rho(i, j, k) * vx(i, j, k) ** 2]
    u = field_of(lv, fns)
    d = P.grid_of(lv, H.rhs(lv, u))                    # [5, z, y, x]
    line = P.grid_of(lv, u)[:, 0, 0, :]                 # [5, x]
    want = line_rhs_1d(line, h)
    scale = np.abs(want).max(axis=1, keepdims=True)
    for z in (0, 7, 15):
        for y in (0, 5, 15):
            assert np.all(np.abs(d[:, z, y, :] - want) <= 1e-13 * scale + 1e-15), (z, y)


def test_reflection_reflects_the_rate():
    """x -> -x with s_x -> -s_x maps the rates the same way."""
    lv = I.uniform_leaves(1)
    u = I.hydro_fields(lv, I.BINARY, seed=2)
    g = P.grid_of(lv, u)                                # [5, z, y, x]
    gr = g[:, :, :, ::-1].copy()
    gr[1] = -gr[1]
    ur = np.empty_like(u)
    for m, (_, ix, iy, iz) in enumerate(lv):
        ur[m] = gr[:, 8 * iz:8 * iz + 8, 8 * iy:8 * iy + 8, 8 * ix:8 * ix + 8].reshape(5, 512)
    a = P.grid_of(lv, H.rhs(lv, u))
    b = P.grid_of(lv, H.rhs(lv, ur))[:, :, :, ::-1].copy()
    b[1] = -b[1]
    scale = np.abs(a).max(axis=(1, 2, 3), keepdims=True)
    assert np.all(np.abs(a - b) <= 1e-12 * scale)


@pytest.mark.parametrize("a", [0, 1, 2])
def test_face_rule_integrates_bicubic_states_exactly(a):
    """Face points carry an advected density rho = 1 + q(y1, y2) of a
    bicubic q in the face's tangential coordinates (y1 along e_{a+1}, y2
    along e_{a+2}, in cell units, the face spanning [-1/2, 1/2]^2) with
    uniform velocity and pressure, the same on both sides: the mass flux
    through the face is v_a times the integral of rho over the face,
    1 + 1/12 + 1/144 + 0 for q = y1^2 + y1^2 y2^2 + y1 y2^3 (calculus)."""
    n = 2
    V = np.zeros((5, 26, n, n, n))
    va, p = 0.5, 1.0
    t1, t2 = (a + 1) % 3, (a + 2) % 3
    for s1 in (-1, 0, 1):
        for s2 in (-1, 0, 1):
            y1, y2 = 0.5 * s1, 0.5 * s2
            rho = 1.0 + y1 ** 2 + y1 ** 2 * y2 ** 2 + y1 * y2 ** 3
            vel = [0.0, 0.0, 0.0]
            vel[a] = va
            U = [rho, rho * vel[0], rho * vel[1], rho * vel[2], p / (GAMMA - 1.0) + 0.5 * rho * va * va]
            for sign in (1, -1):
                o = [0, 0, 0]
                o[a] = sign
                o[t1] += s1
                o[t2] += s2
                k = P.direction_index(tuple(o))
                for f in range(5):
                    V[f, k] = U[f]
    F = H.face_fluxes(V, a, GAMMA)
    want = va * (1.0 + 1.0 / 12.0 + 1.0 / 144.0)
    assert np.allclose(F[0], want, rtol=1e-14, atol=0)
