"""Seeded synthetic inputs: octree leaf lists, density fields and weights.

This module holds no arithmetic of the gravity solve.  It builds the inputs
that both the GPU library and the CPU oracle are run on: binary-star density
fields on octrees of 8x8x8-cell subgrids (the paper's workloads are double
white dwarf binaries with the AMR refined on the stars and the region between
them, Sec. 1 and Sec. 3.1, Fig. 2; the production restart files are not
available, so polytrope-like spheres stand in for the stars).

Leaves are int32 ``[n_leaf, 4]`` = (level, ix, iy, iz); densities are float64
``[n_leaf, 512]`` with cell (i, j, k) of a leaf at ``i + 8 j + 64 k``.
"""
from __future__ import annotations

import numpy as np

ATMOSPHERE = 1e-10

# (centre, central density, radius) of the stars of each workload
SPHERE = [((0.5, 0.5, 0.5), 1.0, 0.4)]                              # R^2 = 0.16
BINARY = [((0.25, 0.5, 0.5), 1.0, 0.18), ((0.75, 0.5, 0.5), 0.6, 0.12)]
# mass ratio 0.7 with the same radii: rho_c2 = 0.7 (0.18 / 0.12)^3
BINARY_Q07 = [((0.25, 0.5, 0.5), 1.0, 0.18), ((0.75, 0.5, 0.5), 0.7 * (0.18 / 0.12) ** 3, 0.12)]


def uniform_leaves(level: int, order: str = "zyx", seed: int | None = None) -> np.ndarray:
    """All 8**level nodes of one level as leaves (lexicographic, z slowest),
    optionally shuffled with a seeded permutation."""
    n = 1 << level
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    leaves = np.stack([np.full(x.size, level), x.ravel(), y.ravel(), z.ravel()], 1)
    leaves = leaves.astype(np.int32)
    if seed is not None:
        leaves = leaves[np.random.default_rng(seed).permutation(leaves.shape[0])]
    return np.ascontiguousarray(leaves)


def cell_centres(leaves, origin=(0.0, 0.0, 0.0), size=1.0) -> np.ndarray:
    """Cell centres [n_leaf, 512, 3] of every leaf's 8^3 cells."""
    leaves = np.asarray(leaves)
    L = leaves[:, 0].astype(np.float64)
    h = size / (8.0 * 2.0 ** L)
    l = np.arange(512)
    loc = np.stack([l & 7, (l >> 3) & 7, l >> 6], 1).astype(np.float64)  # [512, 3]
    base = 8.0 * leaves[:, 1:4].astype(np.float64)                        # [n, 3]
    return np.asarray(origin) + (base[:, None, :] + loc[None] + 0.5) * h[:, None, None]


def star_density(x: np.ndarray, stars, atmosphere: float = ATMOSPHERE) -> np.ndarray:
    """max(atmosphere, sum_s rho_s (1 - |x - c_s|^2 / R_s^2)_+^1.5) at points x [..., 3]."""
    rho = np.zeros(x.shape[:-1])
    for c, rc, R in stars:
        q = 1.0 - np.sum((x - np.asarray(c)) ** 2, -1) / (R * R)
        rho += rc * np.clip(q, 0.0, None) ** 1.5
    return np.maximum(rho, atmosphere)


def density(leaves, stars, seed: int = 0, noise: float = 1e-3, origin=(0.0, 0.0, 0.0),
            size=1.0, atmosphere: float = ATMOSPHERE) -> np.ndarray:
    """Star densities at cell centres times (1 + noise * u), u ~ U[-1, 1] drawn
    from PCG64(seed) in leaf order.  atmosphere = 0 leaves the space outside
    the stars empty (cells of exactly zero mass)."""
    rho = star_density(cell_centres(leaves, origin, size), stars, atmosphere)
    u = np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, size=rho.shape)
    return np.ascontiguousarray(rho * (1.0 + noise * u))


def _node_mass(nodes: np.ndarray, stars) -> np.ndarray:
    """Sum of rho h^3 over the 8^3 cells of each node (no noise): the
    refinement indicator of the synthetic AMR trees."""
    rho = star_density(cell_centres(nodes), stars)
    h = 1.0 / (8.0 * 2.0 ** nodes[:, 0].astype(np.float64))
    return rho.sum(1) * h ** 3


def _covering_level(leafset: set, L: int, x: int, y: int, z: int) -> int:
    """Level of the leaf that covers node position (L, x, y, z), or L+1 if the
    region is refined below L."""
    for q in range(L, -1, -1):
        s = L - q
        if (q, x >> s, y >> s, z >> s) in leafset:
            return q
    return L + 1


def _code(x, y, z):
    return x.astype(np.int64) | (y.astype(np.int64) << 20) | (z.astype(np.int64) << 40)


def _decode(c):
    m = (1 << 20) - 1
    return c & m, (c >> 20) & m, (c >> 40) & m


def balance(leaves) -> np.ndarray:
    """Refine leaves until every pair of face/edge/corner-adjacent leaves
    differs by at most one level (2:1 balance): a leaf of level l that covers
    a same-level neighbour position of a leaf of level L >= l + 2 is split,
    until nothing changes (the minimal balanced refinement)."""
    leaves = np.asarray(leaves, dtype=np.int64)
    lmax = int(leaves[:, 0].max())
    levels = {L: np.unique(_code(*leaves[leaves[:, 0] == L, 1:4].T)) for L in range(lmax + 1)}
    offs = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                     if (dx, dy, dz) != (0, 0, 0)], dtype=np.int64)
    changed = True
    while changed:
        changed = False
        for L in range(lmax, 1, -1):
            if levels[L].size == 0:
                continue
            x, y, z = _decode(levels[L])
            n = 1 << L
            q = np.stack([x, y, z], 1)[:, None, :] + offs[None]
            q = q.reshape(-1, 3)
            q = q[np.all((q >= 0) & (q < n), 1)]
            for l in range(L - 2, -1, -1):
                s = L - l
                cand = np.unique(_code(q[:, 0] >> s, q[:, 1] >> s, q[:, 2] >> s))
                hit = cand[np.isin(cand, levels[l], assume_unique=True)]
                if hit.size == 0:
                    continue
                changed = True
                levels[l] = np.setdiff1d(levels[l], hit, assume_unique=True)
                hx, hy, hz = _decode(hit)
                kids = [_code(2 * hx + (c & 1), 2 * hy + ((c >> 1) & 1), 2 * hz + (c >> 2))
                        for c in range(8)]
                levels[l + 1] = np.union1d(levels[l + 1], np.concatenate(kids))
    out = []
    for L in range(lmax + 1):
        x, y, z = _decode(levels[L])
        out.append(np.stack([np.full(x.size, L), x, y, z], 1))
    out = np.concatenate(out).astype(np.int32)
    order = np.lexsort((out[:, 3], out[:, 2], out[:, 1], out[:, 0]))
    return np.ascontiguousarray(out[order])


def is_balanced(leaves) -> bool:
    leafset = set(map(tuple, np.asarray(leaves).tolist()))
    for (L, x, y, z) in leafset:
        n = 1 << L
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    qx, qy, qz = x + dx, y + dy, z + dz
                    if (dx | dy | dz) == 0 or min(qx, qy, qz) < 0 or max(qx, qy, qz) >= n:
                        continue
                    if _covering_level(leafset, L, qx, qy, qz) < L - 1:
                        return False
    return True


def amr_leaves(lmax: int, m_thr: float, stars, lmin: int = 1, do_balance: bool = True):
    """Refine from the root: a node below lmax is split iff its mass exceeds
    m_thr (nodes above lmin are always split), then 2:1 balance."""
    leaves = []
    front = np.array([[0, 0, 0, 0]], dtype=np.int64)
    while front.shape[0]:
        L = front[:, 0]
        split = L < lmin
        can = (L < lmax) & ~split
        if np.any(can):
            split[can] = _node_mass(front[can], stars) > m_thr
        leaves.append(front[~split])
        par = front[split]
        kids = []
        for c in range(8):
            k = par.copy()
            k[:, 0] += 1
            k[:, 1] = 2 * par[:, 1] + (c & 1)
            k[:, 2] = 2 * par[:, 2] + ((c >> 1) & 1)
            k[:, 3] = 2 * par[:, 3] + (c >> 2)
            kids.append(k)
        front = np.concatenate(kids) if par.shape[0] else np.zeros((0, 4), np.int64)
    out = np.concatenate(leaves).astype(np.int32)
    if do_balance:
        out = balance(out)
    return np.ascontiguousarray(out)


def hydro_fields(leaves, stars=BINARY, seed: int = 0, omega: float = 2.0):
    """Five conserved fields [n_leaf, 5, 512] for the hydro reconstruction:
    density (the binary's polytropes in the atmosphere, with noise), momentum
    of a rigid rotation about the z axis through the domain centre at angular
    speed omega (the binary's orbit) with 1e-3 relative noise, and the total
    energy of a polytropic gas, p = rho^(5/3) (gamma = 5/3), plus the kinetic
    energy."""
    rho = density(leaves, stars, seed)
    x = cell_centres(leaves) - 0.5                                    # [n, 512, 3]
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    vx = -omega * x[..., 1] * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, rho.shape))
    vy = omega * x[..., 0] * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, rho.shape))
    vz = 1e-3 * omega * rng.uniform(-1.0, 1.0, rho.shape) * np.abs(x[..., 2])
    e_int = rho ** (5.0 / 3.0) / (5.0 / 3.0 - 1.0)
    E = e_int + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return np.ascontiguousarray(np.stack([rho, rho * vx, rho * vy, rho * vz, E], axis=1))


def weights(n_leaf: int, seed_w1: int = 1, seed_w2: int = 2):
    """Gaussian weights w1 [n_leaf, 512] and w2 [n_leaf, 3, 512] of the
    functional J = sum(w1 phi + w2 . g)."""
    w1 = np.random.Generator(np.random.PCG64(seed_w1)).standard_normal((n_leaf, 512))
    w2 = np.random.Generator(np.random.PCG64(seed_w2)).standard_normal((n_leaf, 3, 512))
    return w1, w2


# Named workloads (sizes as in the project's configuration list).
WORKLOADS = {
    "sphere_l1": "uniform level-1 octree, 8 leaves of 8^3 (16^3 = 4,096 cells), one sphere",
    "binary_l3": "uniform level-3 octree, 512 leaves of 8^3 (64^3 = 262,144 cells), binary",
    "binary_amr6": "AMR octree to level 6 refined on the binary, ~4,000 leaves (~2M cells)",
    "binary_amr8": "AMR octree to level 8, mass ratio 0.7 binary, ~40,000 leaves (~20M cells)",
}

# the stars of each workload's density (hydro_fields builds the workload's
# density with them, plus momentum and energy)
WORKLOAD_STARS = {"sphere_l1": SPHERE, "binary_l3": BINARY, "binary_amr6": BINARY,
                  "binary_amr8": BINARY_Q07}

AMR6_MTHR = 1e-5
AMR8_MTHR = 1e-6


def workload(name: str, seed: int = 0):
    """(leaves, rho) of a named workload."""
    if name == "sphere_l1":
        lv = uniform_leaves(1)
        return lv, density(lv, SPHERE, seed)
    if name == "binary_l3":
        lv = uniform_leaves(3)
        return lv, density(lv, BINARY, seed)
    if name == "binary_amr6":
        lv = amr_leaves(6, AMR6_MTHR, BINARY)
        return lv, density(lv, BINARY, seed)
    if name == "binary_amr8":
        lv = amr_leaves(8, AMR8_MTHR, BINARY_Q07)
        return lv, density(lv, BINARY_Q07, seed)
    raise KeyError(name)
