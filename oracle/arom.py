"""Algorithm 1 (hybrid snapshot AROM) of the paper, step by step, and the
metrics of Sec. 3.1 (relative L1 error, sampling averages).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

State kept between steps: the last w+1 snapshots gamma_{k-w}..gamma_k, the
basis Phi, points P, reference state psi and sampling sets in effect.

Readings where the paper is silent:
  * explicit schemes (SSP-RK2): the partial HDM is S-hat^T gamma_k =
    S-hat^T RK2(gamma_{k-1}), exact with no subiterations (the remark on
    explicit time marching); its stencil reaches two cells.
  * implicit schemes (BDF1, and the paper's MUSCL-Roe-BDF2 HDM of
    oracle/hdm_muscl.py): subiterations j = 1..J stop when
    ||y^(j) - y^(j-1)||_2 < eps_y (checked from j = 2) or j = jmax; with the
    MUSCL HDM the filter's gate is that HDM's own residual R_k of Eq. hdm
    (BDF2; BDF1 at the first step), the residual Sec. 2.3.4 names.
  * psi, Phi, P "in effect": when a rebuild was skipped (mod(k+1, z) = 0)
    the most recent ones are used by the next RRE and POD.  The RRE needs a
    basis; before the first rebuild G is empty.
  * y for the RRE is recomputed from the final (filtered) gamma_k.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import workloads as W
from . import hdm, hdm_muscl, rom, select, filt


@dataclass
class StepInfo:
    k: int
    was_full: bool
    J: int = 0
    n_s: int = 0
    n_g: int = 0
    n_p: int = 0
    m_eff: int = 0
    filt_passes: int = 0
    rebuilt: bool = False


class Arom:
    """Algorithm 1.  `q0` has shape [c, Nc] (SoA, cell index x-fastest)."""

    def __init__(self, q0, cfg: W.ArConfig):
        self.cfg = cfg
        c, ny, nx = cfg.nvar, cfg.ny, cfg.nx
        self.shape = (c, ny, nx)
        g0 = np.asarray(q0, dtype=np.float64).reshape(self.shape).copy()
        self.snaps = {0: g0}                 # gamma_j for the last w+1 steps
        self.k = 0
        self.psi = None
        self.Phi = None                      # N x m_eff (rows v*Nc + cell)
        self.P = []                          # row indices, order chosen
        self.s_hat = None                    # bool [ny, nx]
        self.s_tilde = None
        self.G = np.zeros(0, np.int64)
        self.y = None
        self.history = []

    # -- helpers -------------------------------------------------------------
    @property
    def gamma(self):
        return self.snaps[self.k]

    def _flat(self, q):
        return q.reshape(-1)

    def _is_full(self, k):
        cfg = self.cfg
        return (k + 1 <= cfg.w) or (cfg.z > 0 and k % cfg.z == 0)

    def _rebuild_due(self, k):
        cfg = self.cfg
        return k >= cfg.w - 1 and (cfg.z <= 0 or (k + 1) % cfg.z != 0)

    def _rec(self, y):
        """psi + Phi y as a state array."""
        r = self._flat(self.psi).copy()
        if self.Phi.shape[1]:
            r = r + self.Phi @ y
        return r.reshape(self.shape)

    def _gappy(self, v):
        rows = self._sample_rows() if self.cfg.regress_rows == W.ROWS_SAMPLE else self.P
        return rom.gappy_coords(self.Phi, rows, self._flat(v), self._flat(self.psi))

    def _sample_rows(self):
        """All dof rows of the cells of S-hat in effect (variable-major): the
        regression rows of the sample-row form of the reduced solve, which
        contain P (P is a subset of S-hat, Sec. 2.2)."""
        cells = np.flatnonzero(self.s_hat)
        return np.concatenate([v * self.cfg.ncell + cells for v in range(self.cfg.nvar)])

    # -- one iteration of Algorithm 1's loop ----------------------------------
    def step(self):
        cfg = self.cfg
        k = self.k + 1
        prev = self.snaps[k - 1]
        info = StepInfo(k=k, was_full=self._is_full(k))
        t = k * cfg.dt
        muscl = cfg.scheme == W.SCHEME_BDF2_MUSCL
        prev2 = self.snaps.get(k - 2) if muscl else None
        # the filter's gate (Sec. 2.3.4): the residual R_k of Eq. hdm, i.e. for
        # the paper's HDM the BDF2 residual (BDF1 at the first step)
        resid = (lambda q: hdm_muscl.residual(q, prev, prev2, cfg, t)) if muscl else None
        if info.was_full:
            if muscl:                                             # the paper's HDM
                gam = hdm_muscl.step(prev, prev2, cfg, k, tol=cfg.newton_tol)
            else:
                gam = hdm.full_step(prev, cfg, k)                 # full HDM step
            info.n_s = cfg.ncell
        else:
            s_hat = self.s_hat
            s_breve = ~s_hat
            info.n_s = int(s_hat.sum())
            if cfg.scheme == W.SCHEME_RK2:
                full = hdm.rk2_step(prev, cfg, k)
                v = prev.copy()
                v[:, s_hat] = full[:, s_hat]
                y = self._gappy(v)
                info.J = 1
            else:
                v = prev.copy()                                   # predictor
                y = None
                for j in range(1, cfg.jmax + 1):                  # subiterations
                    if muscl:
                        v = hdm_muscl.partial_step(prev, prev2, cfg, k, s_hat, v,
                                                   tol=cfg.newton_tol)
                    else:
                        v, _, _ = hdm.newton_be(prev, cfg, t, active=s_hat, q_init=v)
                    y_new = self._gappy(v)
                    conv = y is not None and np.linalg.norm(y_new - y) < cfg.eps_y
                    y = y_new
                    info.J = j
                    if conv:
                        break
                    rec = self._rec(y)
                    v = v.copy()
                    v[:, self.s_tilde] = rec[:, self.s_tilde]
            rec = self._rec(y)                                    # reconstruction
            v = v.copy()
            v[:, s_breve] = rec[:, s_breve]
            gam, info.filt_passes, _ = filt.spatial_filter(v, prev, cfg, t, resid)  # SpatialFilter
            self.y = y
        self.snaps[k] = gam
        self.k = k
        self.snaps.pop(k - cfg.w - 1, None)

        if k == cfg.w - 1:                                        # psi initialisation
            self.psi = rom.window_mean([self.snaps[j] for j in range(0, cfg.w)])
        if self._rebuild_due(k):                                  # rebuild test
            info.rebuilt = True
            if k >= cfg.w and self.Phi is not None:               # error indicator
                y2 = self._gappy(gam)
                eps = select.cell_error(self._flat(gam), self._flat(self.psi),
                                        self.Phi, y2, cfg.nvar)
                self.G, info.n_g = select.select_cells(eps, cfg.sel_mode,
                                                       cfg.delta, cfg.top_frac)
            else:
                self.G, info.n_g = np.zeros(0, np.int64), 0      # no previous basis
            win = [self.snaps[j] for j in range(k - cfg.w + 1, k + 1)]
            Xc = np.stack([self._flat(g) - self._flat(self.psi) for g in win], axis=1)
            raw = float(np.sqrt(sum(float(np.sum(g * g)) for g in win)))
            self.Phi, _ = rom.pod(Xc, cfg.m, cfg.pod_tol, cfg.pod_abs * raw)  # POD
            b = getattr(cfg, "odeim_batch", 1)
            if b > 1:   # the cheaper variant (not the paper's): b points per pass
                self.P = rom.odeim_batched(self.Phi, cfg.n_p, cfg.tie_tol, b)
            else:
                self.P = rom.odeim(self.Phi, cfg.n_p, cfg.tie_tol)    # ODEIM
            self.s_hat, self.s_tilde = select.build_masks(self.G, self.P, cfg)  # sampling sets
            self.psi = rom.window_mean(win)                       # psi update
        info.n_p = len(self.P)
        info.m_eff = 0 if self.Phi is None else self.Phi.shape[1]
        self.history.append(info)
        return info

    def run(self, steps):
        for _ in range(steps):
            self.step()
        return self.gamma


def hdm_trajectory(q0, cfg, steps):
    """Full-HDM-only trajectory q_1..q_steps (reference for e_k)."""
    q = np.asarray(q0, dtype=np.float64).reshape(cfg.nvar, cfg.ny, cfg.nx)
    out = []
    for k in range(1, steps + 1):
        q = hdm.full_step(q, cfg, k)
        out.append(q)
    return out


def rel_l1(gam, q):
    """e_k = int |gamma_k - q_k|_1 dV / int |q_k|_1 dV on a uniform grid."""
    return float(np.abs(gam - q).sum() / np.abs(q).sum())


def sampling_averages(history, ncell, ndof):
    """s-bar over the steps from the first hybrid step on (the warm-up full
    steps are excluded, which makes s-bar = s-bar* when z is infinite, as the
    paper's z = infinity results show), s-bar* over hybrid steps and p-bar
    (ODEIM points per dof) over hybrid steps; percentages (Sec. 3.1)."""
    first = next((h.k for h in history if not h.was_full), None)
    if first is None:
        return float("nan"), float("nan"), float("nan")
    post = [h for h in history if h.k >= first]
    hyb = [h for h in history if not h.was_full]
    sbar = 100.0 * float(np.mean([h.n_s / ncell for h in post]))
    sstar = 100.0 * float(np.mean([h.n_s / ncell for h in hyb]))
    pbar = 100.0 * float(np.mean([h.n_p / ndof for h in hyb]))
    return sbar, sstar, pbar
