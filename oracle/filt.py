"""Spatial low-pass filters with the residual gate: Sec. 2.3.4.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings where the paper is silent:
  * the explicit Shapiro filter of order 2n has the frequency response
    1 - sin^{2n}(theta/2):  u~ = u - (-1)^n (delta^2)^n u / 4^n with
    delta^2 u_i = u_{i-1} - 2 u_i + u_{i+1}.  Weights (times 4^n):
      n = 1: (1, 2, 1)            n = 2: (-1, 4, 10, 4, -1)
      n = 3: (1, -6, 15, 44, 15, -6, 1)
    evaluated as a left-to-right weighted sum, then scaled by 4^-n.
  * multi-D: x direction first, then y (the remark on filtering by
    direction).  Boundaries: zeroth-order extrapolation (ghost = boundary
    value) on non-periodic sides, wrap on periodic sides.
  * residual: R(v) = v - gamma_{k-1} - dt f*(v, t_k) (Eq. hdm with BDF1) for
    every scheme; per-cell measure rho_i = sum_v |R_{v,i}|.
  * one pass: filter the whole state, keep the filtered value on cells
    whose rho strictly decreases.  Passes repeat until no cell is kept, the
    kept cells' total decrease is below eps_f times their previous total,
    or jmax_f passes ran.  Orders are applied in the configured sequence
    (2, 4, 6), each with its own pass loop.
"""
from __future__ import annotations

import numpy as np

import workloads as W
from . import hdm

SHAPIRO = {
    1: [1.0, 2.0, 1.0],
    2: [-1.0, 4.0, 10.0, 4.0, -1.0],
    3: [1.0, -6.0, 15.0, 44.0, 15.0, -6.0, 1.0],
}


def _pad_axis(u, g, axis, periodic):
    n = u.shape[axis]
    if periodic:
        lo = np.take(u, np.arange(n - g, n), axis=axis)
        hi = np.take(u, np.arange(0, g), axis=axis)
    else:
        lo = np.repeat(np.take(u, [0], axis=axis), g, axis=axis)
        hi = np.repeat(np.take(u, [n - 1], axis=axis), g, axis=axis)
    return np.concatenate([lo, u, hi], axis=axis)


def shapiro_1d(u, n, axis, periodic):
    """Order-2n Shapiro filter of array u along `axis`."""
    wts = SHAPIRO[n]
    g = n
    up = _pad_axis(u, g, axis, periodic)
    L = u.shape[axis]
    acc = None
    for t, wgt in enumerate(wts):
        sl = np.take(up, np.arange(t, t + L), axis=axis)
        term = sl if wgt == 1.0 else (-sl if wgt == -1.0 else wgt * sl)
        acc = term if acc is None else acc + term
    return acc * (0.25 ** n)


def shapiro(q, n, cfg):
    """Apply the 1D filter along x, then along y (when ny > 1)."""
    out = shapiro_1d(q, n, 2, cfg.bc[0] == W.BC_PERIODIC)
    if cfg.ny > 1:
        out = shapiro_1d(out, n, 1, cfg.bc[2] == W.BC_PERIODIC)
    return out


def cell_residual(q, q_prev, cfg, t, resid=None):
    """rho_i = sum_v |R_{v,i}(q)|, R the BDF1 residual at time t (or
    resid(q), the residual of the HDM in use)."""
    R = np.abs(hdm.residual_be(q, q_prev, cfg, t) if resid is None else resid(q))
    acc = R[0].copy()
    for v in range(1, R.shape[0]):
        acc = acc + R[v]
    return acc


def spatial_filter(q, q_prev, cfg, t, resid=None):
    """SpatialFilter of Algorithm 1.  Returns (q_filtered,
    passes_run, cells_kept_total).  resid: the residual of the HDM in use
    (default the BDF1 form)."""
    q = q.copy()
    passes = 0
    kept_total = 0
    for n in cfg.filt_orders:
        rho_old = cell_residual(q, q_prev, cfg, t, resid)
        for _ in range(cfg.jmax_f):
            g = shapiro(q, n, cfg)
            rho_new = cell_residual(g, q_prev, cfg, t, resid)
            keep = rho_new < rho_old
            passes += 1
            nk = int(np.count_nonzero(keep))
            if nk == 0:
                break
            kept_total += nk
            q[:, keep] = g[:, keep]
            dec = float(np.sum(rho_old[keep] - rho_new[keep]))
            tot = float(np.sum(rho_old[keep]))
            if dec < cfg.eps_f * tot:
                break
            rho_old = cell_residual(q, q_prev, cfg, t, resid)
    return q, passes, kept_total
