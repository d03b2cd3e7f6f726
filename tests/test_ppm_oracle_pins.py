"""Pins of the PPM reconstruction oracle (oracle/ppm.py) against facts that
do not come from it: exactness on constants, on linear fields along every
line direction and (before limiting) on cubic cell averages; the flattening
of a local extremum (Colella & Woodward 1984); the values' confinement
between a cell's average and its neighbour's; and the reflection symmetry of
the 26 directions."""
import numpy as np
import pytest

from oracle import ppm as P
from paper_2412_15518_gb300 import inputs as I


def field_of(leaves, fn, nf=1):
    """Cell values fn(i, j, k) (global cell indices) laid out per leaf."""
    leaves = np.asarray(leaves)
    c = np.arange(8)
    kk, jj, ii = np.meshgrid(c, c, c, indexing="ij")
    out = np.empty((leaves.shape[0], nf, 512))
    for n, (_, ix, iy, iz) in enumerate(leaves):
        v = fn(8 * ix + ii, 8 * iy + jj, 8 * iz + kk)
        out[n] = np.broadcast_to(v.reshape(-1), (nf, 512))
    return out


def test_constant_field_is_reproduced_in_every_direction():
    lv = I.uniform_leaves(1)
    u = field_of(lv, lambda i, j, k: np.full(i.shape, 2.75), nf=2)
    out = P.reconstruct(lv, u)
    assert np.all(out == 2.75)


@pytest.mark.parametrize("o", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 1, 1),
                               (-1, 1, -1), (0, 1, -1)])
def test_linear_field_gives_exact_boundary_values(o):
    """For u = a + b.x the average of a cell is its centre value and the value
    at the boundary point in direction o is u(centre + o h / 2); away from
    the domain edge (two cells, where the ghosts are clamped) the
    reconstruction is exact up to rounding."""
    lv = I.uniform_leaves(2)
    b = np.array([0.3, -0.7, 0.45])
    u = field_of(lv, lambda i, j, k: 1.0 + b[0] * i + b[1] * j + b[2] * k)
    out = P.reconstruct(lv, u)
    g = P.grid_of(lv, out.reshape(lv.shape[0], -1, 512))  # [26, n, n, n]
    k = P.direction_index(o)
    n = 32
    c = np.arange(n)
    kk, jj, ii = np.meshgrid(c, c, c, indexing="ij")
    want = 1.0 + b[0] * (ii + 0.5 * o[0]) + b[1] * (jj + 0.5 * o[1]) + b[2] * (kk + 0.5 * o[2])
    s = slice(2, n - 2)
    assert np.abs(g[k][s, s, s] - want[s, s, s]).max() < 1e-13


def test_interface_formula_is_exact_for_cubic_averages():
    """Cell averages of a cubic p(x) over [i, i+1]: the fourth-order
    interpolation returns p at the interfaces exactly (before the limiter,
    which a monotone convex cubic with small curvature does not trigger)."""
    p = lambda x: 0.01 * x ** 3 + 0.2 * x ** 2 + 3.0 * x + 1.0
    P4 = lambda x: 0.0025 * x ** 4 + 0.2 / 3.0 * x ** 3 + 1.5 * x ** 2 + x  # antiderivative
    i = np.arange(-2.0, 6.0)
    avg = P4(i + 1) - P4(i)
    v = P.interface(avg[0:4], avg[1:5], avg[2:6], avg[3:7])
    assert np.allclose(v, p(i[1:5] + 1.0), rtol=0, atol=1e-12)


def test_local_extremum_is_flattened():
    lv = I.uniform_leaves(1)
    u = field_of(lv, lambda i, j, k: -((i - 7.0) ** 2 + (j - 7.0) ** 2 + (k - 7.0) ** 2))
    out = P.reconstruct(lv, u)
    g = P.grid_of(lv, out.reshape(lv.shape[0], -1, 512))
    # the maximum sits at cell (7, 7, 7): every direction returns its average
    assert np.all(g[:, 7, 7, 7] == 0.0)


def test_values_lie_between_neighbouring_averages():
    lv = I.uniform_leaves(1)
    rng = np.random.default_rng(4)
    u = rng.standard_normal((lv.shape[0], 3, 512))
    out = P.reconstruct(lv, u)
    g = P.grid_of(lv, u)
    r = P.grid_of(lv, out.reshape(lv.shape[0], -1, 512)).reshape(3, 26, 16, 16, 16)
    pad = np.pad(g, ((0, 0), (1, 1), (1, 1), (1, 1)), mode="edge")
    for o in P.OFFSETS:
        nb = pad[:, 1 + o[2]:17 + o[2], 1 + o[1]:17 + o[1], 1 + o[0]:17 + o[0]]
        v = r[:, P.direction_index(o)]
        assert np.all(v >= np.minimum(g, nb) - 1e-15) and np.all(v <= np.maximum(g, nb) + 1e-15), o


def test_reflection_swaps_opposite_directions():
    lv = I.uniform_leaves(1)
    rng = np.random.default_rng(6)
    u = rng.standard_normal((lv.shape[0], 1, 512))
    g = P.grid_of(lv, u)
    gr = g[:, :, :, ::-1]  # x -> -x
    lv_sorted = lv
    ur = np.empty_like(u)
    for n, (_, ix, iy, iz) in enumerate(lv_sorted):
        ur[n] = gr[:, 8 * iz:8 * iz + 8, 8 * iy:8 * iy + 8, 8 * ix:8 * ix + 8].reshape(1, 512)
    a = P.grid_of(lv, P.reconstruct(lv, u).reshape(lv.shape[0], -1, 512)).reshape(26, 16, 16, 16)
    b = P.grid_of(lv, P.reconstruct(lv, ur).reshape(lv.shape[0], -1, 512)).reshape(26, 16, 16, 16)
    for o in P.OFFSETS:
        m = (-o[0], o[1], o[2])
        assert np.array_equal(a[P.direction_index(o)], b[P.direction_index(m)][:, :, ::-1]), o
