"""Thin Python binding of the GB300 FMM gravity library (``include/octofmm.h``).

Argument marshalling only: every step of the solve runs in ``libotfmm.so``.
PyTorch supplies device memory (tensors) and streams.  The functions named
``ot_*`` mirror the C entry points one to one; :class:`Tree` and
:class:`GravitySolve` are conveniences on top of them.

The library must be built (``__graft_entry__.build()`` or
``python -m paper_2412_15518_gb300._build``); importing this module without
it raises ``ImportError`` -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libotfmm.so")

OT_OK = 0
OT_ERR_DEVICE_STATUS = -8
# bits of the device status word (ot_tree_info's device_status)
OT_STATUS_BAD_INDEX = 1
OT_STATUS_BAD_ITEM = 2  # reserved: no kernel of this version latches it
OT_STATUS_BAD_DENSITY = 4
OT_PRECISION_FP64 = 0
OT_PRECISION_FP32_BULK = 1
OT_PRECISION_FP32_WIDE = 2
OT_MAX_LEVELS = 16

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")
_lib = ctypes.CDLL(LIB_PATH)


class ot_tree_desc(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("size", ctypes.c_double),
                ("n_leaf", ctypes.c_int32), ("leaves", ctypes.POINTER(ctypes.c_int32))]


class ot_solve_opts(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("G", ctypes.c_double),
                ("precision", ctypes.c_int32), ("am_correction", ctypes.c_int32),
                ("self_term", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ot_tree_stats(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("n_leaf", ctypes.c_int32),
                ("n_nodes", ctypes.c_int64 * OT_MAX_LEVELS),
                ("n_leaf_nodes", ctypes.c_int64 * OT_MAX_LEVELS),
                ("n_m2l", ctypes.c_int64), ("n_p2p", ctypes.c_int64),
                ("n_seam", ctypes.c_int64), ("n_lattice", ctypes.c_int64),
                ("n_m2p", ctypes.c_int64), ("n_p2m", ctypes.c_int64), ("n_mm", ctypes.c_int64),
                ("flops_am", ctypes.c_double), ("flops_noam", ctypes.c_double),
                ("flops_near", ctypes.c_double),
                ("n_work_items", ctypes.c_int64), ("tuned_chunk", ctypes.c_int32),
                ("tuned_ctas_per_sm", ctypes.c_int32), ("tuned_warps_per_cta", ctypes.c_int32),
                ("tuned_lattice_ctas_per_sm", ctypes.c_int32),
                ("device_status", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64),
                ("flops_bulk64", ctypes.c_double), ("flops_bulk32", ctypes.c_double),
                ("flops_adjoint", ctypes.c_double), ("flops_tangent", ctypes.c_double)]


_P = ctypes.c_void_p
_lib.ot_build_tree.argtypes = [ctypes.POINTER(ot_tree_desc), ctypes.c_int, ctypes.POINTER(_P)]
_lib.ot_compute_moments.argtypes = [_P, _P, _P]
_lib.ot_solve_gravity.argtypes = [_P, _P, _P, _P, ctypes.POINTER(ot_solve_opts), _P]
_lib.ot_solve_gravity_host.argtypes = [_P, _P, _P, _P, ctypes.POINTER(ot_solve_opts), _P]
_lib.ot_gravity_backward.argtypes = [_P, _P, _P, _P, _P, ctypes.POINTER(ot_solve_opts), _P]
_lib.ot_autotune.argtypes = [_P, _P, _P, _P, ctypes.POINTER(ot_solve_opts), _P]
_lib.ot_tree_info.argtypes = [_P, ctypes.POINTER(ot_tree_stats)]
_lib.ot_last_solve_times.argtypes = [_P, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(ctypes.c_float)]
_lib.ot_solve_gravity_static.argtypes = [ctypes.POINTER(ot_tree_desc), _P, _P, _P,
                                         ctypes.POINTER(ot_solve_opts), _P]
_lib.ot_solve_gravity_tangent.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(ot_solve_opts), _P]
_lib.ot_ppm_reconstruct.argtypes = [_P, _P, ctypes.c_int, _P, _P]
_lib.ot_hydro_rhs.argtypes = [_P, _P, _P, ctypes.c_double, _P, _P]
_lib.ot_hydro_rk3_step.argtypes = [_P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(ot_solve_opts), _P]
_lib.ot_get_moments.argtypes = [_P, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int32), _P]
_lib.ot_set_launch_shape.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
_lib.ot_alu_peaks.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
_lib.ot_destroy_tree.argtypes = [_P]
_lib.ot_destroy_tree.restype = None
_lib.ot_error_string.argtypes = [ctypes.c_int]
_lib.ot_error_string.restype = ctypes.c_char_p

EXPORTS = ["ot_build_tree", "ot_compute_moments", "ot_solve_gravity", "ot_solve_gravity_host",
           "ot_gravity_backward", "ot_autotune", "ot_last_solve_times", "ot_tree_info",
           "ot_destroy_tree", "ot_error_string", "ot_solve_gravity_static", "ot_get_moments",
           "ot_set_launch_shape", "ot_alu_peaks", "ot_solve_gravity_tangent",
           "ot_ppm_reconstruct", "ot_hydro_rhs", "ot_hydro_rk3_step"]


class OTError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__(f"{what}: {ot_error_string(code)} ({code})")


def _check(code: int, what: str):
    if code != OT_OK:
        raise OTError(code, what)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_opts(theta=0.5, G=1.0, precision=OT_PRECISION_FP64, am_correction=True,
              self_term=False) -> ot_solve_opts:
    return ot_solve_opts(float(theta), float(G), int(precision), int(bool(am_correction)),
                         int(bool(self_term)), 0)


# --- the C entry points, one to one -----------------------------------------
def ot_error_string(code: int) -> str:
    return _lib.ot_error_string(int(code)).decode()


def ot_build_tree(leaves, device: int = 0, origin=(0.0, 0.0, 0.0), size: float = 1.0):
    """Returns an opaque tree handle (int); leaves int32 [n_leaf, 4]."""
    lv = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32).reshape(-1, 4))
    desc = ot_tree_desc((ctypes.c_double * 3)(*origin), float(size), lv.shape[0],
                        lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    h = ctypes.c_void_p()
    _check(_lib.ot_build_tree(ctypes.byref(desc), int(device), ctypes.byref(h)), "ot_build_tree")
    return h.value


def ot_compute_moments(tree, rho, stream=None):
    _check(_lib.ot_compute_moments(_P(tree), _ptr(rho), _stream(stream)), "ot_compute_moments")


def ot_solve_gravity(tree, rho, phi, g, opts: ot_solve_opts | None = None, stream=None):
    _check(_lib.ot_solve_gravity(_P(tree), _ptr(rho), _ptr(phi), _ptr(g),
                                 ctypes.byref(opts) if opts is not None else None,
                                 _stream(stream)), "ot_solve_gravity")


def ot_solve_gravity_host(tree, rho, phi, g, opts: ot_solve_opts | None = None, stream=None):
    _check(_lib.ot_solve_gravity_host(_P(tree), _ptr(rho), _ptr(phi), _ptr(g),
                                      ctypes.byref(opts) if opts is not None else None,
                                      _stream(stream)), "ot_solve_gravity_host")


def ot_gravity_backward(tree, rho, w1, w2, drho, opts: ot_solve_opts | None = None,
                        stream=None):
    _check(_lib.ot_gravity_backward(_P(tree), _ptr(rho), _ptr(w1), _ptr(w2), _ptr(drho),
                                    ctypes.byref(opts) if opts is not None else None,
                                    _stream(stream)), "ot_gravity_backward")


def ot_solve_gravity_tangent(tree, rho, rho_dot, phi, g, phi_dot, g_dot,
                             opts: ot_solve_opts | None = None, stream=None):
    _check(_lib.ot_solve_gravity_tangent(_P(tree), _ptr(rho), _ptr(rho_dot), _ptr(phi), _ptr(g),
                                         _ptr(phi_dot), _ptr(g_dot),
                                         ctypes.byref(opts) if opts is not None else None,
                                         _stream(stream)), "ot_solve_gravity_tangent")


def ot_hydro_rhs(tree, u, g, gamma, dudt, stream=None):
    _check(_lib.ot_hydro_rhs(_P(tree), _ptr(u), _ptr(g), float(gamma), _ptr(dudt), _stream(stream)),
           "ot_hydro_rhs")


def ot_hydro_rk3_step(tree, u, dt, gamma, gravity, opts=None, stream=None):
    o = ctypes.byref(opts) if opts is not None else None
    _check(_lib.ot_hydro_rk3_step(_P(tree), _ptr(u), float(dt), float(gamma), int(gravity), o,
                                  _stream(stream)), "ot_hydro_rk3_step")


def ot_ppm_reconstruct(tree, u, out, stream=None):
    """u: device [n_leaf, n_fields, 512] -> out: device [n_leaf, n_fields, 26, 512]."""
    _check(_lib.ot_ppm_reconstruct(_P(tree), _ptr(u), int(u.shape[1]), _ptr(out), _stream(stream)),
           "ot_ppm_reconstruct")


def ot_autotune(tree, rho, phi, g, opts: ot_solve_opts | None = None, stream=None):
    _check(_lib.ot_autotune(_P(tree), _ptr(rho), _ptr(phi), _ptr(g),
                            ctypes.byref(opts) if opts is not None else None, _stream(stream)),
           "ot_autotune")


def ot_solve_gravity_static(leaves, rho, phi, g, opts: ot_solve_opts | None = None, stream=None,
                            origin=(0.0, 0.0, 0.0), size: float = 1.0):
    """Allocation-free solve of a small tree (at most 9 nodes) on the current
    device, for callers that cannot allocate device memory (a plug-in whose
    host application owns all device memory, a loop that forbids allocation
    after start-up).  All scratch is a fixed array inside the library; calls
    share it, so do not overlap them on the GPU."""
    lv = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32).reshape(-1, 4))
    desc = ot_tree_desc((ctypes.c_double * 3)(*origin), float(size), lv.shape[0],
                        lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    _check(_lib.ot_solve_gravity_static(ctypes.byref(desc), _ptr(rho), _ptr(phi), _ptr(g),
                                        ctypes.byref(opts) if opts is not None else None,
                                        _stream(stream)), "ot_solve_gravity_static")


def ot_get_moments(tree, level: int, out, stream=None):
    """Moments of every cell of `level` in physical units into the device
    tensor out [n_nodes(level), 20, 512] (m, X[3], M2[6], M3[10] packed);
    returns the nodes' coordinates at that level, int32 [n_nodes(level), 3]."""
    n = int(out.shape[0])
    xyz = np.zeros((n, 3), dtype=np.int32)
    _check(_lib.ot_get_moments(_P(tree), int(level), _ptr(out),
                               xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream(stream)),
           "ot_get_moments")
    return xyz


def ot_set_launch_shape(tree, chunk: int, ctas_per_sm: int, lattice_ctas_per_sm: int = 0):
    _check(_lib.ot_set_launch_shape(_P(tree), int(chunk), int(ctas_per_sm), int(lattice_ctas_per_sm)),
           "ot_set_launch_shape")


def ot_alu_peaks(device: int = 0, reps: int = 5) -> dict:
    """Measured CUDA-core peaks of `device` in TFLOP/s: FP64 FMA, FP32 FMA and
    paired FP32 FMA."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.ot_alu_peaks(int(device), int(reps), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "ot_alu_peaks")
    return {"fp64_tflops": a.value, "fp32_tflops": b.value, "fp32x2_tflops": c.value}


def ot_last_solve_times(tree):
    """(interaction launch ms, whole solve ms) of the last solve on the tree."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(_lib.ot_last_solve_times(_P(tree), ctypes.byref(a), ctypes.byref(b)),
           "ot_last_solve_times")
    return a.value, b.value


def ot_tree_info(tree) -> dict:
    st = ot_tree_stats()
    code = _lib.ot_tree_info(_P(tree), ctypes.byref(st))
    n = st.n_levels
    info = dict(n_levels=n, n_leaf=st.n_leaf, n_nodes=list(st.n_nodes[:n]),
                n_leaf_nodes=list(st.n_leaf_nodes[:n]), n_m2l=st.n_m2l, n_p2p=st.n_p2p,
                n_seam=st.n_seam, n_lattice=st.n_lattice, n_m2p=st.n_m2p, n_p2m=st.n_p2m,
                n_mm=st.n_mm, flops_am=st.flops_am, flops_noam=st.flops_noam,
                flops_near=st.flops_near, n_work_items=st.n_work_items,
                tuned_chunk=st.tuned_chunk, tuned_ctas_per_sm=st.tuned_ctas_per_sm,
                tuned_warps_per_cta=st.tuned_warps_per_cta,
                tuned_lattice_ctas_per_sm=st.tuned_lattice_ctas_per_sm, device_status=st.device_status,
                workspace_bytes=st.workspace_bytes, flops_bulk64=st.flops_bulk64,
                flops_bulk32=st.flops_bulk32, flops_adjoint=st.flops_adjoint,
                flops_tangent=st.flops_tangent)
    if code == OT_ERR_DEVICE_STATUS:
        # the latched bits travel with the error (reading them cleared them)
        err = OTError(code, "ot_tree_info")
        err.info = info
        raise err
    _check(code, "ot_tree_info")
    return info


def ot_destroy_tree(tree):
    _lib.ot_destroy_tree(_P(tree))


# --- conveniences --------------------------------------------------------------
class Tree:
    """An octree of 8^3-cell leaf subgrids resident on one GPU."""

    def __init__(self, leaves, device: int = 0, origin=(0.0, 0.0, 0.0), size: float = 1.0):
        self.leaves = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32).reshape(-1, 4))
        self.n_leaf = self.leaves.shape[0]
        self.device = device
        self.handle = ot_build_tree(self.leaves, device, origin, size)

    def close(self):
        if self.handle:
            ot_destroy_tree(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        return torch.device("cuda", self.device)

    def empty_outputs(self):
        phi = torch.empty((self.n_leaf, 512), dtype=torch.float64, device=self._dev())
        g = torch.empty((self.n_leaf, 3, 512), dtype=torch.float64, device=self._dev())
        return phi, g

    def solve(self, rho, phi=None, g=None, stream=None, **opts):
        if phi is None or g is None:
            phi, g = self.empty_outputs()
        ot_solve_gravity(self.handle, rho, phi, g, make_opts(**opts), stream)
        return phi, g

    def solve_host(self, rho, phi, g, stream=None, **opts):
        ot_solve_gravity_host(self.handle, rho, phi, g, make_opts(**opts), stream)

    def backward(self, rho, w1, w2, drho=None, stream=None, **opts):
        if drho is None:
            drho = torch.empty_like(rho)
        ot_gravity_backward(self.handle, rho, w1, w2, drho, make_opts(**opts), stream)
        return drho

    def tangent(self, rho, rho_dot, stream=None, with_values=False, **opts):
        """(phi_dot, g_dot) -- or (phi, g, phi_dot, g_dot) with with_values --
        the solve's derivative along rho_dot (the time derivative of the
        potential and acceleration for densities changing at rho_dot)."""
        pd, gd = self.empty_outputs()
        phi, g = self.empty_outputs() if with_values else (None, None)
        ot_solve_gravity_tangent(self.handle, rho, rho_dot, phi, g, pd, gd, make_opts(**opts), stream)
        return (phi, g, pd, gd) if with_values else (pd, gd)

    def ppm(self, u, stream=None):
        """The 26 directional PPM values [n_leaf, n_fields, 26, 512] of the
        cell averages u [n_leaf, n_fields, 512] (leaves all at one level)."""
        out = torch.empty((u.shape[0], u.shape[1], 26, 512), dtype=torch.float64, device=u.device)
        ot_ppm_reconstruct(self.handle, u, out, stream)
        return out

    def hydro_rhs(self, u, g=None, gamma=5.0 / 3.0, stream=None):
        """dU/dt [n_leaf, 5, 512] of the conserved fields u [n_leaf, 5, 512]
        (rho, s, E; leaves all at one level) with the gravitational
        acceleration g [n_leaf, 3, 512] or None."""
        out = torch.empty_like(u)
        ot_hydro_rhs(self.handle, u, g, gamma, out, stream)
        return out

    def hydro_step(self, u, dt, gamma=5.0 / 3.0, gravity=True, stream=None, **opts):
        """One third-order Runge-Kutta step of the conserved fields u
        [n_leaf, 5, 512] in place, each stage with the gravity solve of its
        own density (gravity=True) or without gravity."""
        ot_hydro_rk3_step(self.handle, u, dt, gamma, 1 if gravity else 0, make_opts(**opts), stream)
        return u

    def compute_moments(self, rho, stream=None):
        ot_compute_moments(self.handle, rho, stream)

    def moments(self, level: int, stream=None):
        """(node_xyz [n, 3], moments [n, 20, 512]) of every cell of `level`."""
        n = self.info()["n_nodes"][level]
        out = torch.empty((n, 20, 512), dtype=torch.float64, device=self._dev())
        xyz = ot_get_moments(self.handle, level, out, stream)
        return xyz, out

    def set_launch_shape(self, chunk: int, ctas_per_sm: int, lattice_ctas_per_sm: int = 0):
        ot_set_launch_shape(self.handle, chunk, ctas_per_sm, lattice_ctas_per_sm)

    def autotune(self, rho, stream=None, **opts):
        phi, g = self.empty_outputs()
        ot_autotune(self.handle, rho, phi, g, make_opts(**opts), stream)

    def info(self) -> dict:
        return ot_tree_info(self.handle)

    def last_times(self):
        return ot_last_solve_times(self.handle)


class GravitySolve(torch.autograd.Function):
    """phi, g = GravitySolve.apply(rho, tree, opts_dict); the backward pass is
    the library's hand-written adjoint (dJ/drho for J = <w1, phi> + <w2, g>)."""

    @staticmethod
    def forward(ctx, rho, tree: Tree, opts: dict | None = None):
        opts = dict(opts or {})
        rho = rho.contiguous()
        phi, g = tree.solve(rho, **opts)
        ctx.tree = tree
        ctx.opts = opts
        ctx.save_for_backward(rho)
        return phi, g

    @staticmethod
    def backward(ctx, gphi, gg):
        (rho,) = ctx.saved_tensors
        w1 = gphi.contiguous() if gphi is not None else torch.zeros_like(rho)
        w2 = (gg.contiguous() if gg is not None else
              torch.zeros((rho.shape[0], 3, 512), dtype=rho.dtype, device=rho.device))
        drho = ctx.tree.backward(rho, w1, w2, **ctx.opts)
        return drho, None, None


def host_only_counts(leaves, theta: float = 0.5) -> dict:
    """Validates a leaf list and counts its interactions on the host
    (ot_build_tree with device -1: no CUDA call)."""
    h = ot_build_tree(leaves, -1)
    try:
        return ot_tree_info(h)
    finally:
        ot_destroy_tree(h)
