"""Oracle of the PPM reconstruction of the hydro solver's 26 directional cell
values (arXiv 2412.15518, Sec. 2: Octo-Tiger's finite-volume hydrodynamics
uses the piecewise parabolic method to compute the values at all 26 spatial
directions of a grid cell).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: a plain numpy
statement of what ``ot_ppm_reconstruct`` computes, on the whole uniform grid
at once, sharing no code with the GPU library.  Only ``tests/`` may import it.

Reading (the paper names the method and the 26 directions, nothing more):

* the tree's leaves are all at one level L, so the leaf sub-grids tile a
  uniform grid of n = 8 * 2^L cells per axis; each of the ``n_fields`` fields
  holds cell averages;
* for each of the 13 line directions e (the 26 neighbour offsets up to
  sign), the cells along the line through a cell are reconstructed by 1-D PPM
  (Colella & Woodward 1984): the value at the boundary point between
  neighbours i and i+1 is the fourth-order interpolation
  a_{i+1/2} = 7/12 (a_i + a_{i+1}) - 1/12 (a_{i-1} + a_{i+2}), held between
  a_i and a_{i+1}; then, with a_L, a_R the cell's values toward -e and +e:
  a_L = a_R = a at a local extremum ((a_R - a)(a - a_L) <= 0), else
  a_L = 3a - 2a_R if the parabola overshoots on the left
  ((a_R - a_L)(a - (a_L + a_R)/2) > (a_R - a_L)^2 / 6, evaluated as
  6 (a_R - a_L)(a - (a_L + a_R)/2) > (a_R - a_L)^2), else a_R = 3a - 2a_L
  if it overshoots on the right;
* the value in direction o (o in {-1,0,1}^3 minus 0) is a_R of the line
  e = o if o is the first of the pair (o, -o) in the order below, else a_L;
  direction index k of o = (ox+1) + 3 (oy+1) + 9 (oz+1), minus 1 above 13;
* outside the domain the cell averages are continued by clamping each index
  into the grid (zero-gradient ghost cells).

Every arithmetic step is written in the order the GPU path follows, in
FP64 without fused multiply-adds, so that both take the same branches and
agree bit for bit.

Pinned by ``tests/test_ppm_oracle_pins.py``: a constant field is reproduced
exactly in every direction; linear fields along any of the 13 lines give the
exact boundary values; cubic cell averages give exact interface values
before limiting; a local extremum is flattened; every value lies between the
cell's average and its neighbour's in that direction; reflecting the grid
swaps the opposite directions.
"""
from __future__ import annotations

import numpy as np

# the 26 offsets in direction-index order
OFFSETS = [(ox, oy, oz) for oz in (-1, 0, 1) for oy in (-1, 0, 1) for ox in (-1, 0, 1)
           if (ox, oy, oz) != (0, 0, 0)]


def direction_index(o) -> int:
    s = (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1)
    return s if s < 13 else s - 1


def interface(am1, a0, a1, a2):
    """Fourth-order value between a0 and a1, held between them."""
    v = (7.0 / 12.0) * (a0 + a1) - (1.0 / 12.0) * (am1 + a2)
    lo = np.minimum(a0, a1)
    hi = np.maximum(a0, a1)
    return np.minimum(np.maximum(v, lo), hi)


def limit(aL, a, aR):
    """The parabola constraints of Colella & Woodward (their eq. 1.10)."""
    aL = aL.copy()
    aR = aR.copy()
    ext = (aR - a) * (a - aL) <= 0.0
    d = aR - aL
    c6 = 6.0 * (d * (a - 0.5 * (aL + aR)))
    q6 = d * d
    left = ~ext & (c6 > q6)
    right = ~ext & ~left & (-q6 > c6)
    aL = np.where(ext, a, np.where(left, 3.0 * a - 2.0 * aR, aL))
    aR = np.where(ext, a, np.where(right, 3.0 * a - 2.0 * aL, aR))
    return aL, aR


def grid_of(leaves, u):
    """Assembles the leaf sub-grids into the uniform grid [nf, n, n, n] (z, y, x)."""
    leaves = np.asarray(leaves)
    L = int(leaves[0, 0])
    assert (leaves[:, 0] == L).all(), "all leaves at one level"
    n = 8 << L
    u = np.asarray(u, dtype=np.float64)
    nf = u.shape[1]
    g = np.empty((nf, n, n, n))
    for idx, (_, ix, iy, iz) in enumerate(leaves):
        g[:, 8 * iz:8 * iz + 8, 8 * iy:8 * iy + 8, 8 * ix:8 * ix + 8] = u[idx].reshape(nf, 8, 8, 8)
    return g


def reconstruct(leaves, u):
    """The 26 directional values: [n_leaf, n_fields, 26, 512] for u
    [n_leaf, n_fields, 512]."""
    leaves = np.asarray(leaves)
    g = grid_of(leaves, u)
    nf, n = g.shape[0], g.shape[1]
    pad = np.pad(g, ((0, 0), (2, 2), (2, 2), (2, 2)), mode="edge")

    def shifted(k, e):
        # the field at cell + k e for every cell of the grid
        ex, ey, ez = e
        return pad[:, 2 + k * ez:2 + k * ez + n, 2 + k * ey:2 + k * ey + n, 2 + k * ex:2 + k * ex + n]

    full = np.empty((nf, 26, n, n, n))
    for o in OFFSETS:
        if direction_index(o) > direction_index(tuple(-c for c in o)):
            continue  # each line once, from its first offset
        e = o
        am2, am1, a0, a1, a2 = (shifted(k, e) for k in (-2, -1, 0, 1, 2))
        aR = interface(am1, a0, a1, a2)
        aL = interface(am2, am1, a0, a1)
        aL, aR = limit(aL, a0, aR)
        full[:, direction_index(o)] = aR
        full[:, direction_index(tuple(-c for c in o))] = aL
    out = np.empty((leaves.shape[0], nf, 26, 512))
    for idx, (_, ix, iy, iz) in enumerate(leaves):
        out[idx] = full[:, :, 8 * iz:8 * iz + 8, 8 * iy:8 * iy + 8, 8 * ix:8 * ix + 8].reshape(nf, 26, 512)
    return out
