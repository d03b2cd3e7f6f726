"""Oracle of the hydro right-hand side on an adaptive octree of 8^3
sub-grids (arXiv 2412.15518, Sec. 2: finite-volume hydrodynamics with PPM
values at all 26 directions of a cell; Sec. 4.3.1: Octo-Tiger conserves mass,
momentum and energy across jumps in refinement level by matching the fluxes
there; Sec. 4.3.2: the octree of sub-grids with ghost layers).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: a plain numpy
statement of what ``ot_hydro_rhs`` computes on a 2:1-balanced tree, leaf by
leaf, sharing no code with the GPU library.  Only ``tests/`` may import it.

Reading (beyond ``oracle.hydro``, which it equals on uniform trees):

* every leaf sees a halo of 3 ghost layers of cell averages at its own
  level.  A ghost cell's global index is first clamped into the domain (zero
  gradient at the domain boundary); then its average is the same-level leaf
  cell's, or, where the region is refined, the mean of the 8 finer cells it
  covers (restriction, summed in z, y, x order), or, where the region is
  coarser, the average of the coarser cell that contains it (injection);
  2:1 balance makes those the only cases;
* PPM (``oracle.ppm``) on the halo gives the 26 values of the leaf's cells
  and of the ghost cells next to its faces (the ghost values toward the
  leaf), so every face of the leaf has both states at its own level;
* each leaf computes the fluxes of its 3 x 9 x 8 x 8 faces like
  ``oracle.hydro`` (Simpson rule of Rusanov fluxes, transmissive domain
  boundary);
* flux matching: a face of a leaf that borders a finer region takes, in
  place of its own flux, the mean of the 4 finer faces that cover it as the
  finer leaves computed them ((F00 + F10) + F01 + F11) / 4 over the two
  tangential axes), so that what leaves the fine cells enters the coarse
  one;
* dU/dt = sum over axes of (F_low - F_high) / h_L + (0, rho g, s.g), h_L the
  leaf's cell side.

Pinned by ``tests/test_hydro_amr_oracle_pins.py``: on uniform trees it
equals the grid-wide ``oracle.hydro`` bit for bit; a uniform state on an AMR
tree is steady; the totals of mass, momentum and energy are conserved across
refinement jumps (the volume-weighted sum of the rates vanishes for a
perturbation away from the domain boundary); a linear state in uniform
motion changes at its closed-form rate away from the level jumps on every
level; and reflecting a symmetric tree reflects the rates.
"""
from __future__ import annotations

import numpy as np

from . import hydro as H
from . import ppm

NF = 5
W = 3  # ghost layers of the halo


def leaf_map(leaves):
    return {tuple(int(v) for v in row): i for i, row in enumerate(np.asarray(leaves))}


def _values(lm, u, L, gx, gy, gz):
    """Averages [5, len] of the level-L cells at clamped global indices
    (gx, gy, gz), by the leaf that covers each: same level, finer
    (restriction) or coarser (injection)."""
    out = np.empty((NF, gx.size))
    nodes = np.stack([gx >> 3, gy >> 3, gz >> 3], axis=1)
    for key in {tuple(r) for r in nodes}:
        m = np.all(nodes == np.array(key), axis=1)
        x, y, z = gx[m], gy[m], gz[m]
        leaf = lm.get((L,) + key)
        if leaf is not None:
            out[:, m] = u[leaf][:, (x & 7) + 8 * (y & 7) + 64 * (z & 7)]
            continue
        coarse = lm.get((L - 1, key[0] >> 1, key[1] >> 1, key[2] >> 1)) if L > 0 else None
        if coarse is not None:
            cx, cy, cz = x >> 1, y >> 1, z >> 1
            out[:, m] = u[coarse][:, (cx & 7) + 8 * (cy & 7) + 64 * (cz & 7)]
            continue
        s = np.zeros((NF, x.size))
        for dz in (0, 1):
            for dy in (0, 1):
                for dx in (0, 1):
                    fx, fy, fz = 2 * x + dx, 2 * y + dy, 2 * z + dz
                    fine = np.empty((NF, x.size))
                    fn = np.stack([fx >> 3, fy >> 3, fz >> 3], axis=1)
                    for fk in {tuple(r) for r in fn}:
                        fm = np.all(fn == np.array(fk), axis=1)
                        fl = lm[(L + 1,) + fk]  # 2:1 balance: the finer cells are leaf cells
                        fine[:, fm] = u[fl][:, (fx[fm] & 7) + 8 * (fy[fm] & 7) + 64 * (fz[fm] & 7)]
                    s = s + fine
        out[:, m] = s * 0.125
    return out


def halo(leaves, lm, u, idx):
    """Cell averages [5, 14, 14, 14] (z, y, x; local -3..10) around leaf idx."""
    L, nx, ny, nz = (int(v) for v in leaves[idx])
    N = 8 << L
    r = np.arange(-W, 8 + W)
    gz, gy, gx = np.meshgrid(8 * nz + r, 8 * ny + r, 8 * nx + r, indexing="ij")
    g = [np.clip(a.reshape(-1), 0, N - 1) for a in (gx, gy, gz)]
    return _values(lm, u, L, *g).reshape(NF, 8 + 2 * W, 8 + 2 * W, 8 + 2 * W)


def block_values(Hb):
    """The 26 PPM values [5, 26, 10, 10, 10] of the halo's cells at local
    -1..8 (z, y, x), each field on its own (``oracle.ppm``'s steps)."""
    out = np.empty((NF, 26, 10, 10, 10))

    def shifted(k, e):
        ex, ey, ez = e
        lo = W - 1
        return Hb[:, lo + k * ez:lo + k * ez + 10, lo + k * ey:lo + k * ey + 10, lo + k * ex:lo + k * ex + 10]

    for o in ppm.OFFSETS:
        mo = tuple(-c for c in o)
        if ppm.direction_index(o) > ppm.direction_index(mo):
            continue
        am2, am1, a0, a1, a2 = (shifted(k, o) for k in (-2, -1, 0, 1, 2))
        aR = ppm.interface(am1, a0, a1, a2)
        aL = ppm.interface(am2, am1, a0, a1)
        aL, aR = ppm.limit(aL, a0, aR)
        out[:, ppm.direction_index(o)] = aR
        out[:, ppm.direction_index(mo)] = aL
    return out


def leaf_fluxes(leaves, V, idx, gamma):
    """The leaf's face fluxes per axis a: [5, ...] with 9 faces along a and
    8 cells along the other axes (arrays z, y, x), from its block values V
    [5, 26, 10, 10, 10] (local -1..8)."""
    L, nx, ny, nz = (int(v) for v in leaves[idx])
    top = (1 << L) - 1
    node = (nx, ny, nz)
    out = []
    for a in range(3):
        ax = 2 - a
        t1, t2 = (a + 1) % 3, (a + 2) % 3
        sl_lo = [slice(1, 9)] * 3
        sl_hi = [slice(1, 9)] * 3
        sl_lo[ax] = slice(0, 9)   # cells -1..7: left of faces 0..8
        sl_hi[ax] = slice(1, 10)  # cells 0..8: right of faces 0..8
        acc = None
        for s2 in (-1, 0, 1):
            for s1 in (-1, 0, 1):
                o = [0, 0, 0]
                o[a] = 1
                o[t1] += s1
                o[t2] += s2
                om = list(o)
                om[a] = -1
                kL, kR = ppm.direction_index(tuple(o)), ppm.direction_index(tuple(om))
                UL = V[(slice(None), kL) + tuple(sl_lo)].copy()
                UR = V[(slice(None), kR) + tuple(sl_hi)].copy()
                first = [slice(None)] * 4
                last = [slice(None)] * 4
                first[1 + ax] = slice(0, 1)
                last[1 + ax] = slice(8, 9)
                if node[a] == 0:      # low domain boundary: the inside state on both sides
                    UL[tuple(first)] = UR[tuple(first)]
                if node[a] == top:    # high domain boundary
                    UR[tuple(last)] = UL[tuple(last)]
                F = H.rusanov(UL, UR, a, gamma)
                w = H.point_weight(s1, s2)
                term = [w * F[f] for f in range(NF)]
                acc = term if acc is None else [acc[f] + term[f] for f in range(NF)]
        out.append(np.stack(acc))
    return out


def rhs(leaves, u, g=None, gamma: float = 5.0 / 3.0, size: float = 1.0):
    """dU/dt [n_leaf, 5, 512] of the conserved fields u [n_leaf, 5, 512] on a
    2:1-balanced tree, with the gravitational acceleration g [n_leaf, 3, 512]
    (None: no gravity)."""
    leaves = np.asarray(leaves)
    u = np.asarray(u, dtype=np.float64)
    lm = leaf_map(leaves)
    n = leaves.shape[0]
    F = [leaf_fluxes(leaves, block_values(halo(leaves, lm, u, i)), i, gamma) for i in range(n)]
    res = np.empty((n, NF, 512))
    for i in range(n):
        L, nx, ny, nz = (int(v) for v in leaves[i])
        node = (nx, ny, nz)
        h = size / (8 << L)
        d = np.zeros((NF, 8, 8, 8))
        for a in range(3):
            ax = 2 - a
            t1, t2 = (a + 1) % 3, (a + 2) % 3
            Fa = F[i][a].copy()
            for side in (0, 1):  # the leaf's low and high boundary faces along a
                nb = list(node)
                nb[a] += -1 if side == 0 else 1
                if nb[a] < 0 or nb[a] > (1 << L) - 1 or (L,) + tuple(nb) in lm:
                    continue
                if L > 0 and (L - 1, nb[0] >> 1, nb[1] >> 1, nb[2] >> 1) in lm:
                    continue  # coarser neighbour: this leaf's own flux stands
                # finer neighbour: the mean of the 4 finer faces over each face
                X = 8 * node[a] + (0 if side == 0 else 8)      # global face index at level L
                fa_fine = 8 if side == 0 else 0                 # its index in the finer leaf
                fcell = 2 * X - 1 if side == 0 else 2 * X       # the finer cell next to it
                for c2 in range(8):
                    for c1 in range(8):
                        s = np.zeros(NF)
                        for d2 in (0, 1):
                            for d1 in (0, 1):
                                gf = [0, 0, 0]
                                gf[a] = fcell
                                gf[t1] = 2 * (8 * node[t1] + c1) + d1
                                gf[t2] = 2 * (8 * node[t2] + c2) + d2
                                fl = lm[(L + 1, gf[0] >> 3, gf[1] >> 3, gf[2] >> 3)]
                                loc = [gf[0] & 7, gf[1] & 7, gf[2] & 7]
                                loc[a] = fa_fine
                                s = s + F[fl][a][:, loc[2], loc[1], loc[0]]
                        loc = [0, 0, 0]
                        loc[a] = 0 if side == 0 else 8
                        loc[t1], loc[t2] = c1, c2
                        Fa[:, loc[2], loc[1], loc[0]] = s * 0.25
            lo = [slice(None)] * 4
            hi = [slice(None)] * 4
            lo[1 + ax] = slice(0, 8)
            hi[1 + ax] = slice(1, 9)
            d = d + (Fa[tuple(lo)] - Fa[tuple(hi)])
        out = d * (1.0 / h)
        if g is not None:
            U = u[i].reshape(NF, 8, 8, 8)
            G = np.asarray(g[i]).reshape(3, 8, 8, 8)
            out[1] = out[1] + U[0] * G[0]
            out[2] = out[2] + U[0] * G[1]
            out[3] = out[3] + U[0] * G[2]
            out[4] = out[4] + ((U[1] * G[0] + U[2] * G[1]) + U[3] * G[2])
        res[i] = out.reshape(NF, 512)
    return res
