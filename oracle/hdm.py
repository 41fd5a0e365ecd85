"""High-dimensional model (HDM): Sec. 2.1 (conservation law, Eq. cons),
Sec. 2.2 (semi-discrete ODE Eq. semi_disc, BDF Eq. bdf, residual Eq. hdm),
Sec. 2.3 (partial residual Eq. partial_hdm2) and Sec. 3.1 (Euler equations
with the ideal-gas law).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Fluxes are first-order finite volume (the HDMs of the run configurations):
  Burgers  f(u) = u^2/2 with the Godunov flux
           F(uL, uR) = max(f(max(uL, 0)), f(min(uR, 0)))
  Euler    Rusanov flux  F = (f(qL) + f(qR))/2 - a (qR - qL)/2,
           a = max(|u_n| + c) over the two sides, c = sqrt(max(gamma p/rho, 0))
Time integration:
  BDF1 (backward Euler, Eq. bdf with s = 1): R(q) = q - q_prev - dt f*(q)
  SSP-RK2:  q1 = q + dt L(q);  q_new = q/2 + (q1 + dt L(q1))/2

Each scalar expression is written in one fixed evaluation order (left to
right, no fused multiply-add), so that a GPU kernel evaluating the same
expression in the same order reproduces these FP64 values exactly.

Arrays: a state is q[v, j, i] (variable, row y, column x), i.e. the SoA
layout q[v*Nc + j*nx + i] reshaped.  Burgers has one variable and ny = 1.
"""
from __future__ import annotations

import numpy as np

import workloads as W


# ----------------------------------------------------------------------------
# boundary (ghost) values
# ----------------------------------------------------------------------------

def _shock_state(cfg, xg, yg, t):
    """Exact planar-shock state at points (xg, yg) and time t, shape (4, ...).
    Post-shock where n.x < d0 + speed*t (evaluated in that order)."""
    n0, n1 = cfg.shock_n
    proj = n0 * xg + n1 * yg
    front = cfg.shock_d0 + cfg.shock_speed * t
    post = proj < front
    pre = np.asarray(cfg.shock_pre, dtype=np.float64)
    pst = np.asarray(cfg.shock_post, dtype=np.float64)
    return np.where(post[None], pst.reshape(4, *([1] * post.ndim)),
                    pre.reshape(4, *([1] * post.ndim)))


def pad_ghost(q, cfg, t, g):
    """Return q extended by g ghost layers on each side of each active axis.

    left/right sides pad axis x, bottom/top pad axis y (only when ny > 1).
    Periodic sides wrap; outflow sides copy the boundary cell (zero
    gradient); shock sides take the exact planar-shock state at the ghost
    cell centre at time t.
    """
    c, ny, nx = q.shape
    dx, dy = cfg.dx, cfg.dy
    # x direction
    if cfg.bc[0] == W.BC_PERIODIC or cfg.bc[1] == W.BC_PERIODIC:
        assert cfg.bc[0] == cfg.bc[1] == W.BC_PERIODIC
        qx = np.concatenate([q[:, :, nx - g:], q, q[:, :, :g]], axis=2)
    else:
        yc = (np.arange(ny) + 0.5) * dy
        parts = []
        for side in (0, 1):
            if cfg.bc[side] == W.BC_OUTFLOW:
                src = q[:, :, :1] if side == 0 else q[:, :, nx - 1:]
                parts.append(np.repeat(src, g, axis=2))
            else:
                if side == 0:
                    xg = (np.arange(-g, 0) + 0.5) * dx
                else:
                    xg = (np.arange(nx, nx + g) + 0.5) * dx
                XG, YG = np.meshgrid(xg, yc, indexing="xy")
                parts.append(_shock_state(cfg, XG, YG, t))
        qx = np.concatenate([parts[0], q, parts[1]], axis=2)
    if ny == 1:
        return qx
    # y direction (pads the x-extended array; corners are never read by the
    # 5-point stencils used here)
    nxg = nx + 2 * g
    if cfg.bc[2] == W.BC_PERIODIC or cfg.bc[3] == W.BC_PERIODIC:
        assert cfg.bc[2] == cfg.bc[3] == W.BC_PERIODIC
        return np.concatenate([qx[:, ny - g:, :], qx, qx[:, :g, :]], axis=1)
    xc = (np.arange(-g, nx + g) + 0.5) * dx
    parts = []
    for side in (2, 3):
        if cfg.bc[side] == W.BC_OUTFLOW:
            src = qx[:, :1, :] if side == 2 else qx[:, ny - 1:, :]
            parts.append(np.repeat(src, g, axis=1))
        else:
            if side == 2:
                yg = (np.arange(-g, 0) + 0.5) * dy
            else:
                yg = (np.arange(ny, ny + g) + 0.5) * dy
            XG, YG = np.meshgrid(xc, yg, indexing="xy")
            parts.append(_shock_state(cfg, XG, YG, t))
    assert parts[0].shape[2] == nxg
    return np.concatenate([parts[0], qx, parts[1]], axis=1)


# ----------------------------------------------------------------------------
# fluxes and the semi-discrete operator f*(q, t)   (Eq. semi_disc)
# ----------------------------------------------------------------------------

def burgers_godunov(uL, uR):
    """Godunov flux of f(u) = u^2/2 (exact Riemann solution at the face)."""
    a = np.maximum(uL, 0.0)
    b = np.minimum(uR, 0.0)
    fa = 0.5 * a * a
    fb = 0.5 * b * b
    return np.maximum(fa, fb)


def _euler_prims(q, gamma):
    rho, mx, my, en = q
    u = mx / rho
    v = my / rho
    p = (gamma - 1.0) * (en - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(np.maximum(gamma * p / rho, 0.0))
    return u, v, p, c


def euler_rusanov(qL, qR, gamma, axis):
    """Rusanov (local Lax-Friedrichs) flux across a face normal to x
    (axis = 0) or y (axis = 1)."""
    uL, vL, pL, cL = _euler_prims(qL, gamma)
    uR, vR, pR, cR = _euler_prims(qR, gamma)
    if axis == 0:
        fL = np.stack([qL[1], qL[1] * uL + pL, qL[2] * uL, (qL[3] + pL) * uL])
        fR = np.stack([qR[1], qR[1] * uR + pR, qR[2] * uR, (qR[3] + pR) * uR])
        a = np.maximum(np.abs(uL) + cL, np.abs(uR) + cR)
    else:
        fL = np.stack([qL[2], qL[1] * vL, qL[2] * vL + pL, (qL[3] + pL) * vL])
        fR = np.stack([qR[2], qR[1] * vR, qR[2] * vR + pR, (qR[3] + pR) * vR])
        a = np.maximum(np.abs(vL) + cL, np.abs(vR) + cR)
    return 0.5 * (fL + fR) - 0.5 * a * (qR - qL)


def rhs(q, cfg, t):
    """f*(q, t): the FV spatial operator, -(F_{i+1/2} - F_{i-1/2})/dx
    - (G_{j+1/2} - G_{j-1/2})/dy  (y terms only when ny > 1)."""
    c, ny, nx = q.shape
    qg = pad_ghost(q, cfg, t, 1)
    if ny > 1:
        core_x = qg[:, 1:ny + 1, :]          # rows of the domain, x padded
    else:
        core_x = qg
    if cfg.pde == W.PDE_BURGERS:
        F = burgers_godunov(core_x[0, :, :-1], core_x[0, :, 1:])[None]
    else:
        F = euler_rusanov(core_x[:, :, :-1], core_x[:, :, 1:], cfg.gamma, 0)
    out = -(F[:, :, 1:] - F[:, :, :-1]) / cfg.dx
    if ny > 1:
        core_y = qg[:, :, 1:nx + 1]          # columns of the domain, y padded
        G = euler_rusanov(core_y[:, :-1, :], core_y[:, 1:, :], cfg.gamma, 1)
        out = out - (G[:, 1:, :] - G[:, :-1, :]) / cfg.dy
    return out


# ----------------------------------------------------------------------------
# time integration: residual (Eq. hdm with BDF1) and explicit SSP-RK2
# ----------------------------------------------------------------------------

def residual_be(q, q_prev, cfg, t):
    """R(q) = q - q_prev - dt f*(q, t): Eq. hdm for BDF1 (a0 = -1, a1 = 1,
    beta = 1).  Also the filter's residual for every scheme."""
    return (q - q_prev) - cfg.dt * rhs(q, cfg, t)


def rk2_step(q, cfg, k):
    """One SSP-RK2 step from t_{k-1} = (k-1) dt to t_k = k dt (stage 1 is
    evaluated at t_{k-1}, stage 2 at t_k)."""
    q1 = q + cfg.dt * rhs(q, cfg, (k - 1) * cfg.dt)
    return 0.5 * q + 0.5 * (q1 + cfg.dt * rhs(q1, cfg, k * cfg.dt))


def _burgers_dF(uL, uR):
    """(dF/duL, dF/duR) of the Godunov flux; the uL branch wins ties."""
    a = np.maximum(uL, 0.0)
    b = np.minimum(uR, 0.0)
    left = 0.5 * a * a >= 0.5 * b * b
    return np.where(left, a, 0.0), np.where(left, 0.0, b)


def burgers_be_jacobian(u, cfg):
    """Dense dR/du of the BDF1 Burgers residual on the periodic grid."""
    n = u.size
    um = np.roll(u, 1)
    up = np.roll(u, -1)
    dLm, dRm = _burgers_dF(um, u)      # face i-1/2
    dLp, dRp = _burgers_dF(u, up)      # face i+1/2
    lam = cfg.dt / cfg.dx
    J = np.eye(n)
    idx = np.arange(n)
    # f*_i = -(F_{i+1/2} - F_{i-1/2})/dx
    J[idx, (idx - 1) % n] += -lam * dLm
    J[idx, idx] += lam * (dLp - dRm)
    J[idx, (idx + 1) % n] += lam * dRp
    return J


def newton_be(q_prev, cfg, t, active=None, q_init=None):
    """Solve the BDF1 residual R(q) = 0 by Newton's method.

    active: boolean mask over cells of the unknowns (Eq. partial_hdm2 with
    the other cells frozen at q_init); None means all cells (the full HDM
    solve, the full HDM step of Algorithm 1).  Stops when max|R_active| <= newton_tol *
    max(1, max|q_prev|) or after newton_max iterations.
    Returns (q, iterations, converged).  Burgers only.
    """
    if cfg.pde != W.PDE_BURGERS:
        raise NotImplementedError("implicit HDM is defined for Burgers only")
    q = (q_prev if q_init is None else q_init).copy()
    u = q.reshape(-1)
    up = q_prev.reshape(-1)
    act = np.ones(u.size, bool) if active is None else active.reshape(-1)
    tol = cfg.newton_tol * max(1.0, float(np.abs(up).max()))
    it = 0
    while True:
        R = residual_be(u.reshape(q.shape), q_prev, cfg, t).reshape(-1)
        if np.abs(R[act]).max(initial=0.0) <= tol:
            return u.reshape(q.shape), it, True
        if it >= cfg.newton_max:
            return u.reshape(q.shape), it, False
        J = burgers_be_jacobian(u, cfg)
        Ja = J[np.ix_(act, act)]
        u = u.copy()
        u[act] = u[act] - np.linalg.solve(Ja, R[act])
        it += 1


def full_step(q_prev, cfg, k):
    """Full HDM snapshot at step k (Algorithm 1): gamma_k = F_k(gamma_k)."""
    t = k * cfg.dt
    if cfg.scheme == W.SCHEME_BE:
        q, _, _ = newton_be(q_prev, cfg, t)
        return q
    return rk2_step(q_prev, cfg, k)
