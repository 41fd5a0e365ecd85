"""The paper's own HDM (Sec. 3.1): a second-order MUSCL finite-volume
discretisation of the Euler equations with the Roe flux and the minmod
limiter on a Cartesian mesh, integrated by the second-order BDF scheme
(a0 = 1/3, a1 = -4/3, a2 = 1, beta = 2/3 in Eq. bdf), each implicit step
R_k(q_k) = 0 (Eq. hdm) solved by Newton's method with GMRES.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings where the paper is silent:
  * MUSCL reconstructs the primitive variables (rho, u, v, p), component
    by component: the slope of cell i is minmod(w_i - w_{i-1}, w_{i+1} - w_i)
    (zero when the two differences differ in sign, else the one of smaller
    magnitude), the face states are w_i + slope_i / 2 and
    w_{i+1} - slope_{i+1} / 2, converted back to conserved variables for the
    flux.  The paper does not say which variables MUSCL reconstructs; the
    primitive ones are taken because, with minmod slopes, every reconstructed
    density and pressure then lies between the values of the two cells it
    comes from, so a face state of positive neighbours is itself physical
    (a conserved reconstruction can give a negative face pressure at a
    strong shock).
  * the Roe flux has no entropy fix;
  * in two dimensions each direction is reconstructed and fluxed
    separately (dimension by dimension);
  * ghost cells are two layers of hdm.pad_ghost (periodic, outflow or exact
    shock state);
  * the first step, which has no q_{k-2}, is BDF1 (backward Euler);
  * the Newton solve is Jacobian-free (scipy's newton_krylov with GMRES)
    and stops at max |R| <= tol * max(1, max |q_{k-1}|); a start that
    already meets the test is the solution (no Newton step is taken).
    Algorithm 1 (oracle/arom.py) passes the run parameter newton_tol, as for
    the BDF1 HDM.
"""
from __future__ import annotations

import numpy as np
from scipy import optimize

import workloads as W
from . import hdm


def minmod(a, b):
    return np.where(a * b > 0.0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)


def _flux(q, gamma, axis):
    rho, mx, my, en = q
    u, v = mx / rho, my / rho
    p = (gamma - 1.0) * (en - 0.5 * rho * (u * u + v * v))
    if axis == 0:
        return np.stack([mx, mx * u + p, my * u, (en + p) * u])
    return np.stack([my, mx * v, my * v + p, (en + p) * v])


def roe_flux(qL, qR, gamma, axis):
    """Roe's approximate Riemann solver across a face normal to x (axis 0) or
    y (axis 1): F = (f(qL) + f(qR))/2 - sum_k |lambda_k| alpha_k r_k / 2 with
    the Roe-averaged eigen-decomposition of the Euler flux Jacobian."""
    rL, rR = qL[0], qR[0]
    uL, uR = qL[1] / rL, qR[1] / rR
    vL, vR = qL[2] / rL, qR[2] / rR
    pL = (gamma - 1.0) * (qL[3] - 0.5 * rL * (uL * uL + vL * vL))
    pR = (gamma - 1.0) * (qR[3] - 0.5 * rR * (uR * uR + vR * vR))
    HL, HR = (qL[3] + pL) / rL, (qR[3] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    w = sL + sR
    u = (sL * uL + sR * uR) / w
    v = (sL * vL + sR * vR) / w
    H = (sL * HL + sR * HR) / w
    c = np.sqrt((gamma - 1.0) * (H - 0.5 * (u * u + v * v)))
    rho = sL * sR
    # normal / tangential velocity and their jumps
    un, ut = (u, v) if axis == 0 else (v, u)
    dr = rR - rL
    dp = pR - pL
    dun = (uR - uL) if axis == 0 else (vR - vL)
    dut = (vR - vL) if axis == 0 else (uR - uL)
    # wave strengths: acoustic (un - c, un + c), entropy, shear
    a1 = (dp - rho * c * dun) / (2.0 * c * c)
    a3 = (dp + rho * c * dun) / (2.0 * c * c)
    a2 = dr - dp / (c * c)
    a4 = rho * dut
    l1, l2, l3 = np.abs(un - c), np.abs(un), np.abs(un + c)
    one = np.ones_like(u)
    if axis == 0:
        r1 = np.stack([one, u - c, v, H - u * c])
        r3 = np.stack([one, u + c, v, H + u * c])
        r2 = np.stack([one, u, v, 0.5 * (u * u + v * v)])
        r4 = np.stack([0.0 * one, 0.0 * one, one, v])
    else:
        r1 = np.stack([one, u, v - c, H - v * c])
        r3 = np.stack([one, u, v + c, H + v * c])
        r2 = np.stack([one, u, v, 0.5 * (u * u + v * v)])
        r4 = np.stack([0.0 * one, one, 0.0 * one, u])
    diss = l1 * a1 * r1 + l2 * a2 * r2 + l3 * a3 * r3 + l2 * a4 * r4
    return 0.5 * (_flux(qL, gamma, axis) + _flux(qR, gamma, axis)) - 0.5 * diss


def to_primitive(q, gamma):
    rho, mx, my, en = q
    u, v = mx / rho, my / rho
    return np.stack([rho, u, v, (gamma - 1.0) * (en - 0.5 * rho * (u * u + v * v))])


def to_conserved(w, gamma):
    rho, u, v, p = w
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def _faces(w, axis):
    """MUSCL face states along `axis` (1 = y, 2 = x) of a primitive array
    with two ghost layers on that axis: face f lies between padded cells
    f + 1 and f + 2 (f = 0..n), the slopes are those of padded cells 1..n+2."""
    n = w.shape[axis] - 4
    d = np.diff(w, axis=axis)                             # n + 3 differences
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[axis], hi[axis] = slice(0, n + 2), slice(1, n + 3)
    s = minmod(d[tuple(lo)], d[tuple(hi)])                # slopes of padded cells 1..n+2
    a = [slice(None)] * 3
    b = [slice(None)] * 3
    sa = [slice(None)] * 3
    sb = [slice(None)] * 3
    a[axis], b[axis] = slice(1, n + 2), slice(2, n + 3)
    sa[axis], sb[axis] = slice(0, n + 1), slice(1, n + 2)
    return w[tuple(a)] + 0.5 * s[tuple(sa)], w[tuple(b)] - 0.5 * s[tuple(sb)]


def rhs(q, cfg, t):
    """f*(q, t) of the MUSCL-Roe-minmod discretisation (Euler, 1D or 2D)."""
    c, ny, nx = q.shape
    g = cfg.gamma
    qg = hdm.pad_ghost(q, cfg, t, 2)
    rows = slice(2, ny + 2) if ny > 1 else slice(None)
    wL, wR = _faces(to_primitive(qg[:, rows, :], g), 2)  # domain rows, 2 ghosts in x
    F = roe_flux(to_conserved(wL, g), to_conserved(wR, g), g, 0)
    out = -(F[:, :, 1:] - F[:, :, :-1]) / cfg.dx
    if ny > 1:
        wL, wR = _faces(to_primitive(qg[:, :, 2:nx + 2], g), 1)
        G = roe_flux(to_conserved(wL, g), to_conserved(wR, g), g, 1)
        out = out - (G[:, 1:, :] - G[:, :-1, :]) / cfg.dy
    return out


BDF2 = (1.0 / 3.0, -4.0 / 3.0, 1.0, 2.0 / 3.0)     # a0, a1, a2, beta


def residual(q, q_prev, q_prev2, cfg, t):
    """R_k(q) = q - F_k(q) of Eq. hdm for BDF2 (BDF1 when q_prev2 is None)."""
    if q_prev2 is None:
        return (q - q_prev) - cfg.dt * rhs(q, cfg, t)
    a0, a1, a2, beta = BDF2
    return a2 * q + a1 * q_prev + a0 * q_prev2 - cfg.dt * beta * rhs(q, cfg, t)


def step(q_prev, q_prev2, cfg, k, tol=1e-11):
    """One implicit step k: the q with R_k(q) = 0, by Newton-GMRES from the
    previous state."""
    t = k * cfg.dt
    shape = q_prev.shape
    scale = max(1.0, float(np.abs(q_prev).max()))

    def F(x):
        return residual(x.reshape(shape), q_prev, q_prev2, cfg, t).reshape(-1)

    x0 = q_prev.reshape(-1).copy()
    if np.abs(F(x0)).max() <= tol * scale:     # the start already solves it
        return x0.reshape(shape)
    x = optimize.newton_krylov(F, x0, method="gmres", f_tol=tol * scale, maxiter=50)
    return x.reshape(shape)


def partial_step(q_prev, q_prev2, cfg, k, active, q_init, tol=1e-11):
    """The partial HDM of Sec. 2.3 (Eq. partial_hdm2) for this HDM: the
    cells of `active` (bool [ny, nx]) solve their rows of R_k(q) = 0, every
    other cell keeps its value in q_init."""
    t = k * cfg.dt
    shape = q_prev.shape
    act = np.broadcast_to(active[None], shape)
    scale = max(1.0, float(np.abs(q_prev).max()))
    base = q_init.copy()
    if not act.any():
        return base

    def F(x):
        q = base.copy()
        q[act] = x
        return residual(q, q_prev, q_prev2, cfg, t)[act]

    x0 = base[act].copy()
    if np.abs(F(x0)).max() <= tol * scale:     # the start already solves it
        return base
    x = optimize.newton_krylov(F, x0, method="gmres", f_tol=tol * scale, maxiter=50)
    out = base.copy()
    out[act] = x
    return out


def trajectory(q0, cfg, steps):
    """q_1..q_steps: BDF1 for the first step, BDF2 after."""
    qs = [np.asarray(q0, np.float64).reshape(cfg.nvar, cfg.ny, cfg.nx)]
    for k in range(1, steps + 1):
        q2 = qs[-2] if len(qs) >= 2 else None
        qs.append(step(qs[-1], q2, cfg, k))
    return qs[1:]
