"""Oracle of the hydro solver's right-hand side on a uniform grid of 8^3
sub-grids (arXiv 2412.15518, Sec. 2: Octo-Tiger's finite-volume
hydrodynamics computes the values at all 26 spatial directions of a grid
cell with the piecewise parabolic method; Sec. 4.3.1: the hydro solver is
the second solver of every Runge-Kutta stage, beside the gravity solve).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: a plain numpy
statement of what ``ot_hydro_rhs`` computes, on the whole uniform grid at
once, sharing no code with the GPU library.  Only ``tests/`` and the CPU
baseline of ``bench.py`` may import it.

Reading (the paper names finite volumes, PPM in 26 directions and the
Runge-Kutta stages; the flux formula and the face quadrature are this
build's reading, each a published textbook method):

* the state of a cell is the conserved vector U = (rho, s_x, s_y, s_z, E)
  (density, momentum density, total energy density) of an ideal gas with
  adiabatic index gamma: v = s / rho, p = (gamma - 1) (E - s.v / 2);
* each conserved field is reconstructed independently by PPM in the 26
  directions (``oracle.ppm``), so a cell has a value of U at the centre of
  each of its 6 faces, 12 edges and 8 corners;
* the flux through the face between cells c and c + e_a is the 2-D Simpson
  rule over the face (weights 1/6, 4/6, 1/6 per tangential axis, so 16/36 at
  the face centre, 4/36 at the edge midpoints, 1/36 at the corners): the
  point at offset e_a / 2 + (s1 t1 + s2 t2) / 2 from c's centre sees c's
  value in direction e_a + s1 t1 + s2 t2 on the left and the neighbour's
  value in direction -e_a + s1 t1 + s2 t2 on the right (t1 = e_{a+1},
  t2 = e_{a+2} cyclically);
* the flux at a point is the local Lax-Friedrichs (Rusanov) flux, the
  first member of the Kurganov-Tadmor family of central schemes:
  F* = (F(U_L) + F(U_R)) / 2 - a (U_R - U_L) / 2 with
  a = max(|v_a| + c) over the two states and c = sqrt(max(gamma p / rho, 0))
  (the sound speed, zero where the reconstructed pressure is negative);
* at a face on the domain boundary the outside state equals the inside one
  (a transmissive boundary), so the flux there is F(U_inside);
* dU/dt = (sum over the three axes of (F at the cell's low face - F at its
  high face)) / h + (0, rho g, s.g) with g the gravitational acceleration
  (the FMM solve's output) at the cell, h the cell side.

Every arithmetic step is written in the order the GPU path follows, in
FP64 without fused multiply-adds, so that both take the same branches and
agree bit for bit.

Pinned by ``tests/test_hydro_oracle_pins.py``: a uniform state at rest or in
uniform motion is steady without gravity; with gravity its rate of change is
exactly the source term; the Rusanov flux of two equal states is the Euler
flux written out independently; the face rule integrates a bicubic advected
density exactly (the integral by calculus); a linear state in uniform motion
changes at the closed-form rate; a state that varies along one axis only
evolves as the 1-D finite-volume scheme on that axis (a separate loop over
one line of cells); the interior fluxes telescope (the total rate of change
is the boundary flux alone); and reflecting the grid reflects the rate.
"""
from __future__ import annotations

import numpy as np

from . import ppm

NF = 5  # conserved fields: rho, s_x, s_y, s_z, E

# Simpson weights of a face point with tangential offsets (s1, s2)
_W1 = {-1: 1.0, 0: 4.0, 1: 1.0}


def point_weight(s1: int, s2: int) -> float:
    return (_W1[s1] * _W1[s2]) / 36.0


def state_flux(U, a: int, gamma: float):
    """Euler flux along axis a of the states U [5, ...] and their wave speed
    |v_a| + c, in the order the GPU path evaluates them."""
    rho, sx, sy, sz, E = U
    rinv = 1.0 / rho
    vx = sx * rinv
    vy = sy * rinv
    vz = sz * rinv
    ke = 0.5 * ((sx * vx + sy * vy) + sz * vz)
    p = (gamma - 1.0) * (E - ke)
    c = np.sqrt(np.maximum((gamma * p) * rinv, 0.0))
    s = (sx, sy, sz)[a]
    v = (vx, vy, vz)[a]
    F = [s, s * vx, s * vy, s * vz, (E + p) * v]
    F[1 + a] = F[1 + a] + p
    return F, np.abs(v) + c


def rusanov(UL, UR, a: int, gamma: float):
    """Local Lax-Friedrichs flux along axis a between left and right states."""
    FL, cl = state_flux(UL, a, gamma)
    FR, cr = state_flux(UR, a, gamma)
    half_a = 0.5 * np.maximum(cl, cr)
    return [0.5 * (FL[f] + FR[f]) - half_a * (UR[f] - UL[f]) for f in range(NF)]


def face_fluxes(V, a: int, gamma: float):
    """Fluxes [5, faces along a (n + 1), n, n] (axes in grid order z, y, x
    with the face axis in place of a's) from the directional values
    V [5, 26, n, n, n]."""
    n = V.shape[2]
    ax = 2 - a  # array axis of grid axis a (arrays are [z, y, x])
    t1, t2 = (a + 1) % 3, (a + 2) % 3
    acc = None
    for s2 in (-1, 0, 1):
        for s1 in (-1, 0, 1):
            o = [0, 0, 0]
            o[a] = 1
            o[t1] += s1
            o[t2] += s2
            om = list(o)
            om[a] = -1
            kL = ppm.direction_index(tuple(o))
            kR = ppm.direction_index(tuple(om))
            left = V[:, kL]   # value of cell c toward the face point on its high side
            right = V[:, kR]  # value of cell c toward the face point on its low side
            # faces f = 0..n along a: left state from cell f - 1, right from
            # cell f; the boundary faces take the inside state on both sides
            lo = np.take(right, [0], axis=1 + ax)
            hi = np.take(left, [n - 1], axis=1 + ax)
            UL = np.concatenate([lo, left], axis=1 + ax)
            UR = np.concatenate([right, hi], axis=1 + ax)
            F = rusanov(UL, UR, a, gamma)
            w = point_weight(s1, s2)
            term = [w * F[f] for f in range(NF)]
            acc = term if acc is None else [acc[f] + term[f] for f in range(NF)]
    return np.stack(acc)


def rhs(leaves, u, g=None, gamma: float = 5.0 / 3.0, size: float = 1.0):
    """dU/dt [n_leaf, 5, 512] of the conserved fields u [n_leaf, 5, 512] on
    leaves all at one level, with the gravitational acceleration
    g [n_leaf, 3, 512] (None: no gravity) in the domain cube of side size."""
    leaves = np.asarray(leaves)
    L = int(leaves[0, 0])
    n = 8 << L
    h = size / n
    U = ppm.grid_of(leaves, u)                                          # [5, n, n, n]
    V = ppm.grid_of(leaves, ppm.reconstruct(leaves, u).reshape(leaves.shape[0], -1, 512))
    V = V.reshape(NF, 26, n, n, n)
    d = np.zeros_like(U)
    for a in range(3):
        F = face_fluxes(V, a, gamma)
        ax = 1 + (2 - a)
        Fm = np.take(F, np.arange(n), axis=ax)        # the cell's low face
        Fp = np.take(F, np.arange(1, n + 1), axis=ax)  # its high face
        d = d + (Fm - Fp)
    out = d * (1.0 / h)
    if g is not None:
        G = ppm.grid_of(leaves, g)                                      # [3, n, n, n]
        rho, sx, sy, sz = U[0], U[1], U[2], U[3]
        out[1] = out[1] + rho * G[0]
        out[2] = out[2] + rho * G[1]
        out[3] = out[3] + rho * G[2]
        out[4] = out[4] + ((sx * G[0] + sy * G[1]) + sz * G[2])
    res = np.empty((leaves.shape[0], NF, 512))
    for idx, (_, ix, iy, iz) in enumerate(leaves):
        res[idx] = out[:, 8 * iz:8 * iz + 8, 8 * iy:8 * iy + 8, 8 * ix:8 * ix + 8].reshape(NF, 512)
    return res
