"""Pins of the coupled time-step oracle (oracle/hydro_step.py) against facts
that do not come from it: the amplification factor of a three-stage
third-order Runge-Kutta method on a linear equation (the cubic Taylor
polynomial), fourth-order local error on a nonlinear equation with a known
solution, an unchanged uniform state, the conservation of mass, momentum
and energy, and gravity entering through its source at first order in dt."""
import numpy as np
import pytest

from oracle import hydro_step as S
from paper_2412_15518_gb300 import inputs as I

GAMMA = 5.0 / 3.0


def with_rhs(monkeypatch, fn):
    monkeypatch.setattr(S, "rhs", lambda leaves, U, *args: fn(U))


@pytest.mark.parametrize("lam_dt", [-0.3, 0.2, -1.1])
def test_linear_equation_gets_the_cubic_taylor_factor(monkeypatch, lam_dt):
    """dU/dt = lambda U: any three-stage third-order Runge-Kutta method
    multiplies U by 1 + z + z^2/2 + z^3/6, z = lambda dt."""
    lam = 2.5
    dt = lam_dt / lam
    with_rhs(monkeypatch, lambda U: lam * U)
    u = np.random.default_rng(1).uniform(0.5, 2.0, (2, 5, 512))
    z = lam * dt
    want = u * (1.0 + z + z * z / 2.0 + z ** 3 / 6.0)
    assert np.allclose(S.rk3_step(None, u, dt), want, rtol=1e-14, atol=0)


def test_nonlinear_equation_has_fourth_order_local_error(monkeypatch):
    """dU/dt = U^2 from U0 = 1: U(t) = 1 / (1 - t); one step's error scales
    as dt^4 (halving dt divides it by about 16)."""
    with_rhs(monkeypatch, lambda U: U * U)
    u = np.ones((1, 5, 512))
    err = []
    for dt in (0.02, 0.01, 0.005):
        got = S.rk3_step(None, u, dt)[0, 0, 0]
        err.append(abs(got - 1.0 / (1.0 - dt)))
    r1, r2 = err[0] / err[1], err[1] / err[2]
    assert 14.0 < r1 < 18.0 and 14.0 < r2 < 18.0, (r1, r2)


def test_uniform_state_without_gravity_is_unchanged():
    lv = I.uniform_leaves(1)
    u = np.empty((lv.shape[0], 5, 512))
    for f, v in enumerate([1.3, 0.39, -0.26, 0.91, 2.0]):
        u[:, f] = v
    out = S.rk3_step(lv, u, 0.01, gravity=False)
    assert np.abs(out - u).max() <= 1e-15 * np.abs(u).max()


def bump_state(lv):
    x = I.cell_centres(lv)
    r2 = ((x[..., 0] - 0.45) ** 2 + (x[..., 1] - 0.5) ** 2 + (x[..., 2] - 0.52) ** 2) / 0.0625
    b = np.maximum(1.0 - r2, 0.0) ** 4
    return np.stack([1.0 + 0.5 * b, 0.3 * b * (x[..., 1] - 0.5), -0.2 * b * (x[..., 0] - 0.45),
                     0.1 * b, 1.5 + 0.8 * b], axis=1)


def totals(lv, u):
    vol = (1.0 / (8 << np.asarray(lv)[:, 0].astype(np.int64))) ** 3
    return (u * vol[:, None, None]).sum(axis=(0, 2))


def test_totals_are_conserved_without_gravity():
    lv = I.amr_leaves(2, 5e-4, I.BINARY, lmin=1)
    u = bump_state(lv)
    out = S.rk3_step(lv, u, 0.005, gravity=False)
    before, after = totals(lv, u), totals(lv, out)
    assert np.all(np.abs(after - before) < 1e-13 * np.abs(before).max())
    assert np.abs(out - u).max() > 1e-3  # the state does move


def test_gravity_enters_through_the_source_at_first_order():
    """The step with gravity minus the step without it, divided by dt, tends
    to the gravity source (0, rho g, s.g) of the initial state, g the FMM
    solve of its density (oracle.solve), with an error proportional to dt."""
    from oracle import solve
    lv = I.amr_leaves(2, 5e-4, I.BINARY, lmin=1)
    u = bump_state(lv)
    _, g = solve(lv, np.ascontiguousarray(u[:, 0]))
    src = np.zeros_like(u)
    src[:, 1:4] = u[:, 0:1] * g
    src[:, 4] = (u[:, 1:4] * g).sum(axis=1)
    err = []
    for dt in (2e-3, 1e-3):
        d = (S.rk3_step(lv, u, dt, gravity=True) - S.rk3_step(lv, u, dt, gravity=False)) / dt
        err.append(np.abs(d - src).max())
    assert err[1] < 5e-2 * np.abs(src).max()
    assert 1.6 < err[0] / err[1] < 2.4, err
