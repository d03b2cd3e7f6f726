"""Oracle of one time step of the coupled hydro-gravity system on an octree of
8^3 sub-grids (arXiv 2412.15518, Sec. 4.3.1: a third-order Runge-Kutta
scheme, each of whose three stages runs the hydro solver together with the
FMM gravity solve; Sec. 2: finite-volume hydrodynamics with PPM values at
all 26 directions of a cell, and FMM self-gravity).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: a plain statement
of what ``ot_hydro_rk3_step`` computes, sharing no code with the GPU
library.  Only ``tests/`` may import it.

Reading (the paper names the third-order Runge-Kutta scheme and the solvers
of each stage, not the scheme's coefficients):

* the scheme is the strong-stability-preserving third-order Runge-Kutta
  method of Shu & Osher (1988):
  U1 = U0 + dt L(U0),
  U2 = 3/4 U0 + 1/4 (U1 + dt L(U1)),
  U3 = 1/3 U0 + 2/3 (U2 + dt L(U2));
* L(U) is the hydro right-hand side (``oracle.hydro_amr``) with the
  gravitational acceleration of the stage's own density U[:, 0] from one
  FMM solve (``oracle.solve``), or without gravity;
* each combination is evaluated in the order written, in FP64.

Pinned by ``tests/test_hydro_step_oracle_pins.py``: on dU/dt = lambda U
the step multiplies U by the cubic Taylor polynomial of lambda dt (the
amplification factor of every three-stage third-order method); on
dU/dt = U^2 its local error falls as dt^4; a uniform state without gravity
is unchanged; mass, momentum and energy totals are conserved without
gravity; and gravity enters through its source (0, rho g, s.g) at first
order in dt.
"""
from __future__ import annotations

import numpy as np

from . import hydro_amr as A


def rhs(leaves, U, gamma, gravity, G, theta, am_correction, size):
    """L(U): the hydro right-hand side with the stage's own gravity."""
    from . import solve
    g = None
    if gravity:
        _, g = solve(leaves, np.ascontiguousarray(U[:, 0]), theta=theta, G=G,
                     am_correction=am_correction, size=size)
    return A.rhs(leaves, U, g, gamma, size)


def rk3_step(leaves, u, dt, gamma=5.0 / 3.0, gravity=True, G=1.0, theta=0.5, am_correction=True,
             size=1.0):
    """U^{n+1} [n_leaf, 5, 512] from U^n = u after one step of size dt."""
    U0 = np.asarray(u, dtype=np.float64)
    args = (gamma, gravity, G, theta, am_correction, size)
    U1 = U0 + dt * rhs(leaves, U0, *args)
    U2 = 0.75 * U0 + 0.25 * (U1 + dt * rhs(leaves, U1, *args))
    return (1.0 / 3.0) * U0 + (2.0 / 3.0) * (U2 + dt * rhs(leaves, U2, *args))
