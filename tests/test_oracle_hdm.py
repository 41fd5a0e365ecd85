"""Pins of the oracle's HDM (Sec. 2.1-2.2, Sec. 3.1) against facts fixed
outside the oracle: discrete conservation, exact Riemann solutions (Euler
and Burgers), Rankine-Hugoniot shock speed, x/y symmetry, Newton's
residual.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import hdm
from tests import riemann_exact as RX


def test_normal_shock_states_satisfy_rankine_hugoniot():
    g = 1.4
    rho2, u2, p2, s = W.normal_shock_states(g, 3.0, 1.4, 1.0)
    rho1, u1, p1 = 1.4, 0.0, 1.0
    E1 = p1 / (g - 1) + 0.5 * rho1 * u1 ** 2
    E2 = p2 / (g - 1) + 0.5 * rho2 * u2 ** 2
    # jump conditions s [q] = [f(q)] for mass, momentum, energy
    assert math.isclose(s * (rho2 - rho1), rho2 * u2 - rho1 * u1, rel_tol=1e-13)
    assert math.isclose(s * (rho2 * u2 - rho1 * u1), (rho2 * u2 ** 2 + p2) - (rho1 * u1 ** 2 + p1), rel_tol=1e-13)
    assert math.isclose(s * (E2 - E1), (E2 + p2) * u2 - (E1 + p1) * u1, rel_tol=1e-13)
    assert math.isclose(s, 3.0, rel_tol=1e-15)


def test_periodic_conservation_rk2_and_be():
    q0, cfg, _ = W.euler_vortex(n=24, seed=5)
    q = q0.reshape(4, 24, 24)
    tot0 = q.sum(axis=(1, 2))
    for k in range(1, 6):
        q = hdm.rk2_step(q, cfg, k)
    assert np.allclose(q.sum(axis=(1, 2)), tot0, rtol=1e-13, atol=1e-12)
    u0, bcfg, _ = W.burgers_sine(n=128, seed=3)
    u = u0.reshape(1, 1, 128)
    m0 = u.sum()
    for k in range(1, 6):
        u, it, ok = hdm.newton_be(u, bcfg, k * bcfg.dt)
        assert ok
    assert abs(u.sum() - m0) < 1e-10


def test_newton_solves_the_bdf1_residual():
    u0, cfg, _ = W.burgers_sine(n=64, seed=7)
    q0 = u0.reshape(1, 1, 64)
    q, it, ok = hdm.newton_be(q0, cfg, cfg.dt)
    assert ok and it >= 1
    R = hdm.residual_be(q, q0, cfg, cfg.dt)
    assert np.abs(R).max() <= cfg.newton_tol * 2.0


@pytest.mark.parametrize("scheme", [W.SCHEME_RK2, W.SCHEME_BE])
def test_burgers_riemann_converges_to_entropy_solution(scheme):
    errs = []
    T = 0.1
    for n in (100, 200, 400):
        x = (np.arange(n) + 0.5) / n
        u0 = np.where((x >= 0.25) & (x < 0.5), 2.0, 0.0)
        dx = 1.0 / n
        cfg = W.ArConfig(pde=W.PDE_BURGERS, scheme=scheme, nx=n, ny=1, dx=dx, dy=1.0,
                         dt=0.4 * dx / 2.0, bc=(W.BC_PERIODIC,) * 4)
        steps = int(round(T / cfg.dt))
        q = u0.reshape(1, 1, n)
        for k in range(1, steps + 1):
            q = hdm.full_step(q, cfg, k)
        exact = RX.burgers_step_exact(x, steps * cfg.dt)
        errs.append(np.abs(q.reshape(-1) - exact).mean())
    # first-order scheme: L1 error small and shrinking under refinement
    assert errs[0] < 0.06
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1]


def test_burgers_shock_moves_at_rankine_hugoniot_speed():
    n = 1000
    x = (np.arange(n) + 0.5) / n
    uL, uR = 1.5, 0.5
    u0 = np.where(x < 0.3, uL, uR)
    dx = 1.0 / n
    cfg = W.ArConfig(pde=W.PDE_BURGERS, scheme=W.SCHEME_RK2, nx=n, ny=1, dx=dx, dy=1.0,
                     dt=0.4 * dx / uL, bc=(W.BC_OUTFLOW,) * 4)
    steps = 500
    q = u0.reshape(1, 1, n)
    for k in range(1, steps + 1):
        q = hdm.full_step(q, cfg, k)
    t = steps * cfg.dt
    # mass-based shock location: int u dx = uL xs + uR (1 - xs) (+ inflow)
    mass = q.sum() * dx
    inflow = (0.5 * uL * uL - 0.5 * uR * uR) * t
    xs = (mass - uR) / (uL - uR)
    assert abs(mass - (uL * 0.3 + uR * 0.7 + inflow)) < 1e-12
    assert abs(xs - (0.3 + 0.5 * (uL + uR) * t)) < 1e-9


def _euler_sod_error(n, axis):
    q0, cfg = W.euler_riemann_x(n=n)
    T = 0.2
    if axis == 1:  # same problem along y: swap momenta, grid is 1 x n
        q0 = q0[[0, 2, 1, 3]]
        cfg = cfg.with_(nx=1, ny=n, dx=1.0, dy=1.0 / n)
        shape = (4, n, 1)
    else:
        shape = (4, 1, n)
    steps = int(round(T / cfg.dt))
    q = q0.reshape(shape)
    for k in range(1, steps + 1):
        q = hdm.full_step(q, cfg, k)
    x = (np.arange(n) + 0.5) / n
    ex = RX.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / (steps * cfg.dt))
    rho = q[0].reshape(-1)
    return np.abs(rho - ex[0]).mean(), q


@pytest.mark.parametrize("n", [100, 400])
def test_euler_sod_matches_exact_riemann_solution(n):
    e, _ = _euler_sod_error(n, 0)
    # first-order Rusanov: L1 density error ~ C / sqrt(n) at the contact
    assert e < {100: 0.03, 400: 0.014}[n]


def test_euler_y_direction_matches_x_direction():
    ex_, qx = _euler_sod_error(100, 0)
    ey_, qy = _euler_sod_error(100, 1)
    assert ex_ == ey_
    assert np.array_equal(qx[0].reshape(-1), qy[0].reshape(-1))
    assert np.array_equal(qx[1].reshape(-1), qy[2].reshape(-1))


def test_oblique_shock_front_moves_at_shock_speed():
    q0, cfg, _ = W.euler_oblique_shock(n=96, seed=11, k=4)
    n = 96
    q = q0.reshape(4, n, n)
    steps = 60
    for k in range(1, steps + 1):
        q = hdm.full_step(q, cfg, k)
    t = steps * cfg.dt
    # density along the normal through the domain centre region: the front
    # (mid-density crossing) sits near d0 + speed t
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    proj = cfg.shock_n[0] * X + cfg.shock_n[1] * Y
    rho1, rho2 = cfg.shock_pre[0], cfg.shock_post[0]
    mid = 0.5 * (rho1 + rho2)
    band = (X > 0.2) & (X < 0.8) & (Y > 0.2) & (Y < 0.8)
    behind = (q[0] > mid) & band
    ahead = (q[0] <= mid) & band
    front = cfg.shock_d0 + cfg.shock_speed * t
    # every cell clearly behind the exact front is post-shock and vice versa
    assert np.all(proj[ahead] > front - 4.0 / n)
    assert np.all(proj[behind] < front + 4.0 / n)


def test_uniform_flow_is_a_steady_state():
    n = 16
    cfg = W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=n, ny=n, dx=0.1, dy=0.1, dt=0.01,
                     bc=(W.BC_PERIODIC,) * 4)
    q = np.empty((4, n, n))
    q[0], q[1], q[2], q[3] = 1.2, 0.3, -0.2, 3.0
    r = hdm.rhs(q, cfg, 0.0)
    assert np.abs(r).max() < 1e-13
