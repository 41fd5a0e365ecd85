"""Tangent-linear model of Algorithm 1: the derivative of the hybrid
trajectory, and of a time-integrated output, with respect to parameters of
the initial state (the differentiation form).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The method is piecewise smooth.  Its discrete decisions are:

  * the sampled sets;
  * the selection G;
  * the ODEIM points;
  * the filter's keep masks and stopping;
  * the POD rank m_eff;
  * the entry that fixes each mode's sign.

They are taken by the forward run, and the derivative is the one of the
smooth map they leave.  A small enough perturbation of the parameters does
not change them; the finite-difference pins check that it did not (the
decision log of this module).  Everything else is differentiated:

  * the HDM steps (SSP-RK2 with the Rusanov or Godunov flux), by the JVP of
    the flux at each face;
  * the gappy coordinates (Eq. red_coord), by the derivative of the least
    squares solution;
  * the reconstruction psi + Phi y;
  * the filter passes, which are linear once their keep masks are fixed;
  * POD_m (Eq. pod), by the derivative of the thin SVD's left singular
    vectors (distinct singular values);
  * the window means psi (Eq. mean).

Ghost values of a shock side are exact states that do not depend on the
parameters (zero tangent); outflow and periodic ghosts carry the tangent of
the cell they copy.  Readings:

  * the output is J = sum_k dt sum_{cells of the box} p(gamma_k) dx dy over
    the steps 1..K (a fixed box of cells; p the ideal-gas pressure);
  * at a tie of the two wave speeds in the Rusanov flux the left one is
    differentiated (np.maximum keeps the first argument on ties);
  * explicit schemes only (the differentiation form's SSP-RK2); the BDF1
    Burgers HDM raises.
"""
from __future__ import annotations

import numpy as np

import workloads as W
from . import arom, filt, hdm, rom, select


# ----------------------------------------------------------------------------
# HDM: JVP of the FV operator and of the SSP-RK2 step
# ----------------------------------------------------------------------------

def _zero_shock(cfg):
    """cfg with the shock states zeroed: hdm.pad_ghost of a tangent then
    gives zero on shock sides and copies on outflow and periodic sides."""
    z = (0.0, 0.0, 0.0, 0.0)
    return cfg.with_(shock_pre=z, shock_post=z)


def euler_prims_jvp(q, dq, gamma):
    """(u, v, p, c) of hdm's _euler_prims and their tangents."""
    rho, mx, my, en = q
    drho, dmx, dmy, den = dq
    u = mx / rho
    v = my / rho
    du = (dmx - u * drho) / rho
    dv = (dmy - v * drho) / rho
    p = (gamma - 1.0) * (en - 0.5 * rho * (u * u + v * v))
    dp = (gamma - 1.0) * (den - 0.5 * drho * (u * u + v * v) - rho * (u * du + v * dv))
    a2 = gamma * p / rho
    da2 = gamma * (dp - p * drho / rho) / rho
    c = np.sqrt(np.maximum(a2, 0.0))
    dc = np.where(a2 > 0.0, 0.5 * da2 / np.where(c > 0.0, c, 1.0), 0.0)
    return (u, v, p, c), (du, dv, dp, dc)


def euler_rusanov_jvp(qL, dqL, qR, dqR, gamma, axis):
    """Tangent of hdm.euler_rusanov(qL, qR, gamma, axis)."""
    (uL, vL, pL, cL), (duL, dvL, dpL, dcL) = euler_prims_jvp(qL, dqL, gamma)
    (uR, vR, pR, cR), (duR, dvR, dpR, dcR) = euler_prims_jvp(qR, dqR, gamma)

    def flux_jvp(q, dq, u, v, p, du, dv, dp):
        if axis == 0:
            return np.stack([dq[1], dq[1] * u + q[1] * du + dp, dq[2] * u + q[2] * du,
                             (dq[3] + dp) * u + (q[3] + p) * du])
        return np.stack([dq[2], dq[1] * v + q[1] * dv, dq[2] * v + q[2] * dv + dp,
                         (dq[3] + dp) * v + (q[3] + p) * dv])

    dfL = flux_jvp(qL, dqL, uL, vL, pL, duL, dvL, dpL)
    dfR = flux_jvp(qR, dqR, uR, vR, pR, duR, dvR, dpR)
    nL, dnL = (uL, duL) if axis == 0 else (vL, dvL)
    nR, dnR = (uR, duR) if axis == 0 else (vR, dvR)
    sL, sR = np.abs(nL) + cL, np.abs(nR) + cR
    dsL, dsR = np.sign(nL) * dnL + dcL, np.sign(nR) * dnR + dcR
    a = np.maximum(sL, sR)
    da = np.where(sL >= sR, dsL, dsR)
    return 0.5 * (dfL + dfR) - 0.5 * (da * (qR - qL) + a * (dqR - dqL))


def burgers_godunov_jvp(uL, duL, uR, duR):
    dL, dR = hdm._burgers_dF(uL, uR)
    return dL * duL + dR * duR


def rhs_jvp(q, dq, cfg, t):
    """Tangent of hdm.rhs(q, cfg, t) along dq."""
    c, ny, nx = q.shape
    qg = hdm.pad_ghost(q, cfg, t, 1)
    dg = hdm.pad_ghost(dq, _zero_shock(cfg), t, 1)
    qx = qg[:, 1:ny + 1, :] if ny > 1 else qg
    dx_ = dg[:, 1:ny + 1, :] if ny > 1 else dg
    if cfg.pde == W.PDE_BURGERS:
        dF = burgers_godunov_jvp(qx[0, :, :-1], dx_[0, :, :-1], qx[0, :, 1:], dx_[0, :, 1:])[None]
    else:
        dF = euler_rusanov_jvp(qx[:, :, :-1], dx_[:, :, :-1], qx[:, :, 1:], dx_[:, :, 1:],
                               cfg.gamma, 0)
    out = -(dF[:, :, 1:] - dF[:, :, :-1]) / cfg.dx
    if ny > 1:
        qy = qg[:, :, 1:nx + 1]
        dy_ = dg[:, :, 1:nx + 1]
        dG = euler_rusanov_jvp(qy[:, :-1, :], dy_[:, :-1, :], qy[:, 1:, :], dy_[:, 1:, :],
                               cfg.gamma, 1)
        out = out - (dG[:, 1:, :] - dG[:, :-1, :]) / cfg.dy
    return out


def rk2_step_jvp(q, dq, cfg, k):
    """hdm.rk2_step(q, cfg, k) and its tangent along dq."""
    t0, t1 = (k - 1) * cfg.dt, k * cfg.dt
    q1 = q + cfg.dt * hdm.rhs(q, cfg, t0)
    dq1 = dq + cfg.dt * rhs_jvp(q, dq, cfg, t0)
    qn = 0.5 * q + 0.5 * (q1 + cfg.dt * hdm.rhs(q1, cfg, t1))
    dqn = 0.5 * dq + 0.5 * (dq1 + cfg.dt * rhs_jvp(q1, dq1, cfg, t1))
    return qn, dqn


# ----------------------------------------------------------------------------
# reduced basis: gappy coordinates, POD, filter
# ----------------------------------------------------------------------------

def gappy_coords_jvp(Phi, dPhi, rows, v, dv, psi, dpsi):
    """rom.gappy_coords and its tangent: with A = Phi[rows], b = (v - psi)[rows],
    y = argmin |A y - b| (full column rank) has
    dy = (A^T A)^{-1} (dA^T r + A^T (db - dA y)),  r = b - A y."""
    y = rom.gappy_coords(Phi, rows, v, psi)
    if Phi.shape[1] == 0:
        return y, np.zeros(0)
    A, dA = Phi[rows, :], dPhi[rows, :]
    b, db = v[rows] - psi[rows], dv[rows] - dpsi[rows]
    r = b - A @ y
    dy = np.linalg.solve(A.T @ A, dA.T @ r + A.T @ (db - dA @ y))
    return y, dy


def pod_jvp(Xc, dXc, m, pod_tol, abs_floor):
    """rom.pod and the tangent of its Phi along dXc.  For the thin SVD
    X = U S V^T with distinct singular values, column j of U moves by
      sum_{i != j} u_i (s_j (U^T dX V)_ij + s_i (U^T dX V)_ji) / (s_j^2 - s_i^2)
      + (I - U U^T) dX v_j / s_j;
    each kept column carries the sign rom.pod gave it.  Also returns the
    index of each column's largest-magnitude entry (a decision)."""
    Phi, s = rom.pod(Xc, m, pod_tol, abs_floor)
    me = Phi.shape[1]
    if me == 0:
        return Phi, np.zeros_like(Phi), ()
    U, s, Vt = np.linalg.svd(Xc, full_matrices=False)
    V = Vt.T
    K = U.T @ dXc @ V                       # w x w
    dPhi = np.empty_like(Phi)
    resid = dXc @ V[:, :me] - U @ (U.T @ (dXc @ V[:, :me]))
    for j in range(me):
        sj = s[j]
        col = resid[:, j] / sj
        for i in range(s.size):
            if i == j:
                continue
            col = col + U[:, i] * ((sj * K[i, j] + s[i] * K[j, i]) / (sj * sj - s[i] * s[i]))
        sign = 1.0 if np.dot(Phi[:, j], U[:, j]) > 0.0 else -1.0
        dPhi[:, j] = sign * col
    piv = tuple(int(np.argmax(np.abs(Phi[:, j]))) for j in range(me))
    return Phi, dPhi, piv


def spatial_filter_jvp(q, dqs, q_prev, cfg, t):
    """filt.spatial_filter(q, q_prev, cfg, t) and the tangents dqs (a list)
    carried through it: the same passes and gates, and on the kept cells
    of each pass the filtered tangent (the filter is linear).  Also returns
    the decisions: each pass's keep mask."""
    q = q.copy()
    dqs = [d.copy() for d in dqs]
    keeps = []
    for n in cfg.filt_orders:
        rho_old = filt.cell_residual(q, q_prev, cfg, t)
        for _ in range(cfg.jmax_f):
            g = filt.shapiro(q, n, cfg)
            rho_new = filt.cell_residual(g, q_prev, cfg, t)
            keep = rho_new < rho_old
            keeps.append(keep.copy())
            nk = int(np.count_nonzero(keep))
            if nk == 0:
                break
            q[:, keep] = g[:, keep]
            for d in dqs:
                d[:, keep] = filt.shapiro(d, n, cfg)[:, keep]
            dec = float(np.sum(rho_old[keep] - rho_new[keep]))
            tot = float(np.sum(rho_old[keep]))
            if dec < cfg.eps_f * tot:
                break
            rho_old = filt.cell_residual(q, q_prev, cfg, t)
    return q, dqs, keeps


# ----------------------------------------------------------------------------
# Algorithm 1 with tangents
# ----------------------------------------------------------------------------

def pressure(q, gamma):
    rho, mx, my, en = q
    return (gamma - 1.0) * (en - 0.5 * (mx * mx + my * my) / rho)


def pressure_jvp(q, dq, gamma):
    rho, mx, my, en = q
    drho, dmx, dmy, den = dq
    kin = (mx * mx + my * my) / rho
    dkin = (2.0 * (mx * dmx + my * dmy) - kin * drho) / rho
    return (gamma - 1.0) * (den - 0.5 * dkin)


class TangentArom(arom.Arom):
    """arom.Arom carrying tangents dq0 (a list of directions, each shaped
    like q0) through every step, and the output
    J = sum_k dt sum_box p(gamma_k) dx dy with its tangents.  The forward
    values are arom.Arom's (the same oracle calls in the same order); with
    no directions it is the plain method plus the decision log."""

    def __init__(self, q0, cfg, dq0=(), box=None):
        if cfg.scheme != W.SCHEME_RK2 or cfg.pde != W.PDE_EULER:
            raise NotImplementedError("the tangent model covers the Euler SSP-RK2 HDM")
        super().__init__(q0, cfg)
        self.dsnaps = {0: [np.asarray(d, np.float64).reshape(self.shape).copy() for d in dq0]}
        self.nd = len(dq0)
        self.dpsi = None
        self.dPhi = None
        self.box = box if box is not None else (0, cfg.nx, 0, cfg.ny)   # i0, i1, j0, j1
        self.J = 0.0
        self.dJ = np.zeros(self.nd)
        self.decisions = []

    def _output(self, gam, dgs):
        cfg = self.cfg
        i0, i1, j0, j1 = self.box
        w = cfg.dt * cfg.dx * cfg.dy
        self.J += w * float(np.sum(pressure(gam, cfg.gamma)[j0:j1, i0:i1]))
        for d in range(self.nd):
            self.dJ[d] += w * float(np.sum(pressure_jvp(gam, dgs[d], cfg.gamma)[j0:j1, i0:i1]))

    def _dflat(self, d):
        return d.reshape(-1)

    def step(self):
        cfg = self.cfg
        k = self.k + 1
        prev, dprev = self.snaps[k - 1], self.dsnaps[k - 1]
        info = arom.StepInfo(k=k, was_full=self._is_full(k))
        t = k * cfg.dt
        dec = {"k": k}
        if info.was_full:
            outs = [rk2_step_jvp(prev, d, cfg, k) for d in dprev]
            gam = hdm.full_step(prev, cfg, k)
            dgs = [o[1] for o in outs]
            info.n_s = cfg.ncell
        else:
            s_hat = self.s_hat
            s_breve = ~s_hat
            info.n_s = int(s_hat.sum())
            full = hdm.rk2_step(prev, cfg, k)
            v = prev.copy()
            v[:, s_hat] = full[:, s_hat]
            dvs = []
            for d in dprev:
                _, dfull = rk2_step_jvp(prev, d, cfg, k)
                dv = d.copy()
                dv[:, s_hat] = dfull[:, s_hat]
                dvs.append(dv)
            rows = self._sample_rows() if cfg.regress_rows == W.ROWS_SAMPLE else self.P
            y = self._gappy(v)
            info.J = 1
            for i, dv in enumerate(dvs):                          # before v changes
                _, dy = gappy_coords_jvp(self.Phi, self.dPhi[i], rows, self._flat(v),
                                         self._dflat(dv), self._flat(self.psi),
                                         self._dflat(self.dpsi[i]))
                drec = self._dflat(self.dpsi[i]).copy()
                if self.Phi.shape[1]:
                    drec = drec + self.dPhi[i] @ y + self.Phi @ dy
                dv[:, s_breve] = drec.reshape(self.shape)[:, s_breve]
            rec = self._rec(y)
            v = v.copy()
            v[:, s_breve] = rec[:, s_breve]
            gam, dgs, keeps = spatial_filter_jvp(v, dvs, prev, cfg, t)
            info.filt_passes = len(keeps)
            dec["keeps"] = keeps
            self.y = y
        self.snaps[k] = gam
        self.dsnaps[k] = dgs
        self.k = k
        self.snaps.pop(k - cfg.w - 1, None)
        self.dsnaps.pop(k - cfg.w - 1, None)
        self._output(gam, dgs)

        if k == cfg.w - 1:
            self.psi = rom.window_mean([self.snaps[j] for j in range(0, cfg.w)])
            self.dpsi = [rom.window_mean([self.dsnaps[j][d] for j in range(0, cfg.w)])
                         for d in range(self.nd)]
        if self._rebuild_due(k):
            info.rebuilt = True
            if k >= cfg.w and self.Phi is not None:
                y2 = self._gappy(gam)
                eps = select.cell_error(self._flat(gam), self._flat(self.psi),
                                        self.Phi, y2, cfg.nvar)
                self.G, info.n_g = select.select_cells(eps, cfg.sel_mode,
                                                       cfg.delta, cfg.top_frac)
            else:
                self.G, info.n_g = np.zeros(0, np.int64), 0
            js = range(k - cfg.w + 1, k + 1)
            win = [self.snaps[j] for j in js]
            Xc = np.stack([self._flat(g) - self._flat(self.psi) for g in win], axis=1)
            raw = float(np.sqrt(sum(float(np.sum(g * g)) for g in win)))
            dPhis = []
            piv = ()
            for d in range(self.nd):
                dXc = np.stack([self._dflat(self.dsnaps[j][d]) - self._dflat(self.dpsi[d])
                                for j in js], axis=1)
                Phi, dPhi, piv = pod_jvp(Xc, dXc, cfg.m, cfg.pod_tol, cfg.pod_abs * raw)
                dPhis.append(dPhi)
            self.Phi, _ = rom.pod(Xc, cfg.m, cfg.pod_tol, cfg.pod_abs * raw)
            if self.nd == 0 and self.Phi.shape[1]:
                piv = tuple(int(np.argmax(np.abs(self.Phi[:, j])))
                            for j in range(self.Phi.shape[1]))
            self.dPhi = dPhis
            self.P = rom.odeim(self.Phi, cfg.n_p, cfg.tie_tol)
            self.s_hat, self.s_tilde = select.build_masks(self.G, self.P, cfg)
            self.psi = rom.window_mean(win)
            self.dpsi = [rom.window_mean([self.dsnaps[j][d] for j in js])
                         for d in range(self.nd)]
            dec.update(G=np.asarray(self.G).copy(), P=tuple(int(p) for p in self.P),
                       m_eff=self.Phi.shape[1], piv=piv)
        info.n_p = len(self.P)
        info.m_eff = 0 if self.Phi is None else self.Phi.shape[1]
        self.history.append(info)
        self.decisions.append(dec)
        return info
