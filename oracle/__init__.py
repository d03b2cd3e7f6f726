"""Oracle for the FMM self-gravity solve (arXiv 2412.15518, Sec. 4.3).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow FP64 CPU statement
of what the GPU library computes (``fmm_oracle.cpp``: the method's steps in
the order the paper's prose implies, every tensor unpacked, every sum in a
fixed order).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It imports nothing from the
GPU package and shares no code with it.

Every function here is pinned by ``tests/test_oracle_pins.py`` (and the
tree checks by ``tests/test_abi_host.py``) against facts that do not come
from the oracle: direct summation, closed forms, finite differences of the
D tensors, of the pair and of the whole solve, moments taken directly from
point masses, an independent pair enumeration, and momentum and angular
momentum conservation.  None is parity-unpinned.

Every function takes plain numpy arrays:

* ``leaves``: int32 ``[n_leaf, 4]`` = (level, ix, iy, iz) of each leaf node;
  a level-L node covers ``[ix, ix+1) * size / 2**L`` per axis and holds 8^3
  cells (Sec. 4.3.2).
* ``rho``: float64 ``[n_leaf, 512]`` cell densities, cell (i, j, k) of a leaf
  at index ``i + 8 j + 64 k``.
* outputs ``phi`` ``[n_leaf, 512]`` and ``g`` ``[n_leaf, 3, 512]``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import build as _build_lib, lib_path

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)

ERRORS = {-1: "bad leaf (level or coordinates out of range)",
          -2: "duplicate or overlapping leaves",
          -3: "incomplete octree (an interior node lacks a child, or no root)"}


class OracleError(RuntimeError):
    pass


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(
            os.path.join(os.path.dirname(__file__), "fmm_oracle.cpp")):
        _build_lib()
    lib = ctypes.CDLL(path)
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_solve.argtypes = [ctypes.c_int, _I32, _D, ctypes.c_double, _D, ctypes.c_double,
                              ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D, _I64]
    lib.orc_solve_sample.argtypes = [ctypes.c_int, _I32, _D, ctypes.c_double, _D,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_long, _I64, _D, _D, _I64]
    lib.orc_solve_jvp.argtypes = [ctypes.c_int, _I32, _D, ctypes.c_double, _D, _D,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  _D, _D, _D, _D]
    lib.orc_direct.argtypes = [ctypes.c_int, _I32, _D, ctypes.c_double, _D, ctypes.c_double,
                               _D, _D]
    lib.orc_level_moments.argtypes = [ctypes.c_int, _I32, _D, ctypes.c_double, _D,
                                      ctypes.c_int, _D, _I32]
    lib.orc_level_moments.restype = ctypes.c_long
    lib.orc_check_tree.argtypes = [ctypes.c_int, _I32]
    lib.orc_dtensor.argtypes = [_D, _D]
    lib.orc_dtensor.restype = None
    lib.orc_p2m_m2m.argtypes = [ctypes.c_int, _D, _D, _D]
    lib.orc_p2m_m2m.restype = None
    lib.orc_m2m.argtypes = [ctypes.c_int, _D, _D]
    lib.orc_m2m.restype = None
    lib.orc_m2l.argtypes = [_D, _D, ctypes.c_double, ctypes.c_int, _D]
    lib.orc_m2l.restype = None
    lib.orc_l2l.argtypes = [_D, _D, _D]
    lib.orc_l2l.restype = None
    lib.orc_cube_self_constant.restype = ctypes.c_double
    lib.orc_gradient.argtypes = [ctypes.c_int, _I32, _D, ctypes.c_double, _D, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D, _D]
    lib.orc_m2l_reverse.argtypes = [_D, _D, ctypes.c_double, ctypes.c_int, _D, _D, _D]
    lib.orc_m2l_reverse.restype = None
    lib.orc_dtensor5.argtypes = [_D, _D]
    lib.orc_dtensor5.restype = None
    _lib = lib
    return lib


def _p(a, t=_D):
    return a.ctypes.data_as(t)


def _prep(leaves, rho=None, origin=(0.0, 0.0, 0.0)):
    leaves = np.ascontiguousarray(leaves, dtype=np.int32).reshape(-1, 4)
    org = np.ascontiguousarray(origin, dtype=np.float64)
    if rho is not None:
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(leaves.shape[0], 512)
    return leaves, rho, org


def _check(e):
    if e < 0:
        raise OracleError(ERRORS.get(int(e), f"oracle error {e}"))


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave as is); returns the count in use."""
    return int(_load().orc_set_threads(int(n)))


def solve(leaves, rho, theta=0.5, G=1.0, am_correction=True, self_term=False,
          origin=(0.0, 0.0, 0.0), size=1.0, return_counts=False):
    """Full FMM solve; returns (phi, g[, counts]).

    counts = dict(m2l=far pairs, p2p=exact near leaf pairs, seam=mixed near pairs).
    """
    lib = _load()
    leaves, rho, org = _prep(leaves, rho, origin)
    n = leaves.shape[0]
    phi = np.empty((n, 512))
    g = np.empty((n, 3, 512))
    cnt = np.zeros(3, dtype=np.int64)
    _check(lib.orc_solve(n, _p(leaves, _I32), _p(org), size, _p(rho), theta, G,
                         int(bool(am_correction)), int(bool(self_term)), _p(phi), _p(g),
                         _p(cnt, _I64)))
    if return_counts:
        return phi, g, dict(m2l=int(cnt[0]), p2p=int(cnt[1]), seam=int(cnt[2]))
    return phi, g


def solve_sample(leaves, rho, sample, theta=0.5, G=1.0, am_correction=True, self_term=False,
                 origin=(0.0, 0.0, 0.0), size=1.0, return_counts=False):
    """Solve for sampled leaf cells only (sample = leaf * 512 + cell); returns
    (phi [n_sample], g [n_sample, 3][, counts of the pairs evaluated])."""
    lib = _load()
    leaves, rho, org = _prep(leaves, rho, origin)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    phi = np.empty(sample.shape[0])
    g = np.empty((sample.shape[0], 3))
    cnt = np.zeros(3, dtype=np.int64)
    _check(lib.orc_solve_sample(leaves.shape[0], _p(leaves, _I32), _p(org), size, _p(rho),
                                theta, G, int(bool(am_correction)), int(bool(self_term)),
                                sample.shape[0], _p(sample, _I64), _p(phi), _p(g),
                                _p(cnt, _I64)))
    if return_counts:
        return phi, g, dict(m2l=int(cnt[0]), p2p=int(cnt[1]), seam=int(cnt[2]))
    return phi, g


def solve_jvp(leaves, rho, v, theta=0.5, G=1.0, am_correction=True, self_term=False,
              origin=(0.0, 0.0, 0.0), size=1.0):
    """Forward-mode (dual-number) derivative of the solve along v; returns
    (phi, g, dphi, dg)."""
    lib = _load()
    leaves, rho, org = _prep(leaves, rho, origin)
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(rho.shape)
    n = leaves.shape[0]
    phi, dphi = np.empty((n, 512)), np.empty((n, 512))
    g, dg = np.empty((n, 3, 512)), np.empty((n, 3, 512))
    _check(lib.orc_solve_jvp(n, _p(leaves, _I32), _p(org), size, _p(rho), _p(v), theta, G,
                             int(bool(am_correction)), int(bool(self_term)), _p(phi), _p(g),
                             _p(dphi), _p(dg)))
    return phi, g, dphi, dg


def gradient(leaves, rho, w1, w2, theta=0.5, G=1.0, am_correction=True, self_term=False,
             origin=(0.0, 0.0, 0.0), size=1.0):
    """Hand-written adjoint: dJ/drho for J = sum(w1 * phi + w2 * g)."""
    lib = _load()
    leaves, rho, org = _prep(leaves, rho, origin)
    w1 = np.ascontiguousarray(w1, dtype=np.float64).reshape(rho.shape)
    w2 = np.ascontiguousarray(w2, dtype=np.float64).reshape(rho.shape[0], 3, 512)
    drho = np.empty_like(rho)
    _check(lib.orc_gradient(leaves.shape[0], _p(leaves, _I32), _p(org), size, _p(rho), theta, G,
                            int(bool(am_correction)), int(bool(self_term)), _p(w1), _p(w2),
                            _p(drho)))
    return drho


def m2l_reverse(momA, momB, Ebar, G=1.0, am_correction=True):
    """Reverse of one pair: adjoints (packed 40 each) of A and of B given the
    adjoint Ebar (43) of A's expansion."""
    a = np.ascontiguousarray(momA, dtype=np.float64)
    b = np.ascontiguousarray(momB, dtype=np.float64)
    e = np.ascontiguousarray(Ebar, dtype=np.float64)
    oa, ob = np.empty(40), np.empty(40)
    _load().orc_m2l_reverse(_p(a), _p(b), G, int(bool(am_correction)), _p(e), _p(oa), _p(ob))
    return oa, ob


def dtensor5(R):
    """D^(5) of 1/|R| at R, [3, 3, 3, 3, 3]."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.empty(243)
    _load().orc_dtensor5(_p(R), _p(out))
    return out.reshape(3, 3, 3, 3, 3)


def direct(leaves, rho, G=1.0, origin=(0.0, 0.0, 0.0), size=1.0):
    """O(N^2) direct summation over all leaf cells as point masses."""
    lib = _load()
    leaves, rho, org = _prep(leaves, rho, origin)
    n = leaves.shape[0]
    phi = np.empty((n, 512))
    g = np.empty((n, 3, 512))
    _check(lib.orc_direct(n, _p(leaves, _I32), _p(org), size, _p(rho), G, _p(phi), _p(g)))
    return phi, g


def level_moments(leaves, rho, L, origin=(0.0, 0.0, 0.0), size=1.0):
    """Moments of every level-L cell: (node_xyz [n, 3], mom [n, 512, 40]) with
    mom = (m, X[3], M2[9], M3[27]) about the cell's centre of mass."""
    lib = _load()
    leaves, rho, org = _prep(leaves, rho, origin)
    nn = lib.orc_level_moments(leaves.shape[0], _p(leaves, _I32), _p(org), size, _p(rho), L,
                               None, None)
    _check(nn)
    out = np.empty((nn, 512, 40))
    xyz = np.empty((nn, 3), dtype=np.int32)
    _check(lib.orc_level_moments(leaves.shape[0], _p(leaves, _I32), _p(org), size, _p(rho), L,
                                 _p(out), _p(xyz, _I32)))
    return xyz, out


def check_tree(leaves) -> int:
    """0 for a valid complete octree, else a negative error code (see ERRORS)."""
    leaves, _, _ = _prep(leaves)
    return int(_load().orc_check_tree(leaves.shape[0], _p(leaves, _I32)))


def dtensor(R):
    """(D0, D1[3], D2[3,3], D3[3,3,3], D4[3,3,3,3]) of 1/|R| at R."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.empty(121)
    _load().orc_dtensor(_p(R), _p(out))
    return (out[0], out[1:4], out[4:13].reshape(3, 3), out[13:40].reshape(3, 3, 3),
            out[40:121].reshape(3, 3, 3, 3))


def p2m_m2m(points, masses):
    """Moments (packed, 40) of point masses via leaf moments plus one M2M step."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    m = np.ascontiguousarray(masses, dtype=np.float64)
    out = np.empty(40)
    _load().orc_p2m_m2m(pts.shape[0], _p(pts), _p(m), _p(out))
    return out


def m2m(moms):
    moms = np.ascontiguousarray(moms, dtype=np.float64).reshape(-1, 40)
    out = np.empty(40)
    _load().orc_m2m(moms.shape[0], _p(moms), _p(out))
    return out


def m2l(momA, momB, G=1.0, am_correction=True):
    """Expansion (packed, 43 = L0, L1[3], L2[9], L3[27], ac[3]) at A due to B."""
    a = np.ascontiguousarray(momA, dtype=np.float64)
    b = np.ascontiguousarray(momB, dtype=np.float64)
    out = np.empty(43)
    _load().orc_m2l(_p(a), _p(b), G, int(bool(am_correction)), _p(out))
    return out


def l2l(loc, delta):
    loc = np.ascontiguousarray(loc, dtype=np.float64)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    out = np.empty(43)
    _load().orc_l2l(_p(loc), _p(d), _p(out))
    return out


def cube_self_constant() -> float:
    """int over the unit cube of 1/|r| about its centre, by quadrature."""
    return float(_load().orc_cube_self_constant())


def unpack_loc(v):
    v = np.asarray(v)
    return dict(L0=v[0], L1=v[1:4], L2=v[4:13].reshape(3, 3), L3=v[13:40].reshape(3, 3, 3),
                ac=v[40:43])


def unpack_mom(v):
    v = np.asarray(v)
    return dict(m=v[..., 0], X=v[..., 1:4], M2=v[..., 4:13].reshape(v.shape[:-1] + (3, 3)),
                M3=v[..., 13:40].reshape(v.shape[:-1] + (3, 3, 3)))
