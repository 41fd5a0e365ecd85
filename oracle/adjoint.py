"""Reverse mode of the tangent-linear model (oracle/tangent.py): the adjoint
of Algorithm 1 with the forward run's decisions held, and the gradient of
the time-integrated output J by one reverse sweep.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Each function is the transpose of the tangent of the same name in
oracle/tangent.py: for every direction d and cotangent w,
<w, T(d)> = <T^T(w), d>, which is how each one is pinned.  The sweep walks
the recorded steps backwards.

  * A step's cotangent goes through the filter passes in reverse order.
  * It then goes through the reconstruction on S-breve, the gappy
    coordinates on the regression rows, and the partial or full RK2 step.
  * A rebuild's basis and reference-state cotangents go back to the window
    snapshots through the transposed thin-SVD derivative and the window
    means.

Ghost values follow the tangent's rules: a shock ghost is fixed, an outflow
ghost hands its cotangent to the boundary cell it copies, periodic ghosts
fold back onto the cells they wrap.
"""
from __future__ import annotations

import numpy as np

import workloads as W
from . import filt, hdm, rom, select, tangent as T


# ----------------------------------------------------------------------------
# HDM
# ----------------------------------------------------------------------------

def _pad_T(gq, shape, cfg, g):
    """Transpose of hdm.pad_ghost(., cfg, t, g) for a tangent (shock ghosts
    carry nothing): fold the ghost layers of gq back onto the cells."""
    c, ny, nx = shape
    twoD = ny > 1
    if twoD:
        core = gq[:, g:g + ny, :].copy()
        lo, hi = gq[:, :g, :], gq[:, g + ny:, :]
        if cfg.bc[2] == W.BC_PERIODIC:
            core[:, ny - g:, :] += lo
            core[:, :g, :] += hi
        else:
            if cfg.bc[2] == W.BC_OUTFLOW:
                core[:, :1, :] += lo.sum(axis=1, keepdims=True)
            if cfg.bc[3] == W.BC_OUTFLOW:
                core[:, ny - 1:, :] += hi.sum(axis=1, keepdims=True)
    else:
        core = gq.copy()
    out = core[:, :, g:g + nx].copy()
    lo, hi = core[:, :, :g], core[:, :, g + nx:]
    if cfg.bc[0] == W.BC_PERIODIC:
        out[:, :, nx - g:] += lo
        out[:, :, :g] += hi
    else:
        if cfg.bc[0] == W.BC_OUTFLOW:
            out[:, :, :1] += lo.sum(axis=2, keepdims=True)
        if cfg.bc[1] == W.BC_OUTFLOW:
            out[:, :, nx - 1:] += hi.sum(axis=2, keepdims=True)
    return out


def _face_T(qL, qR, Fbar, gamma, axis):
    """(dF/dqL)^T Fbar and (dF/dqR)^T Fbar of the Rusanov flux, faces along
    the trailing axes, from the tangent applied to the unit vectors."""
    gL = np.zeros_like(qL)
    gR = np.zeros_like(qR)
    z = np.zeros_like(qL)
    for c in range(4):
        e = np.zeros_like(qL)
        e[c] = 1.0
        gL[c] = np.sum(T.euler_rusanov_jvp(qL, e, qR, z, gamma, axis) * Fbar, axis=0)
        gR[c] = np.sum(T.euler_rusanov_jvp(qL, z, qR, e, gamma, axis) * Fbar, axis=0)
    return gL, gR


def rhs_vjp(q, mu, cfg, t):
    """L'(q, t)^T mu, L = hdm.rhs (Euler)."""
    c, ny, nx = q.shape
    qg = hdm.pad_ghost(q, cfg, t, 1)
    gq = np.zeros_like(qg)
    # x faces of the domain rows: F[:, :, f] between padded columns f, f + 1
    rows = slice(1, ny + 1) if ny > 1 else slice(None)
    qx = qg[:, rows, :]
    Fbar = np.zeros((4, ny, nx + 1))
    Fbar[:, :, :nx] += mu / cfg.dx          # L_i = -(F_{i+1/2} - F_{i-1/2})/dx
    Fbar[:, :, 1:] -= mu / cfg.dx
    gL, gR = _face_T(qx[:, :, :-1], qx[:, :, 1:], Fbar, cfg.gamma, 0)
    gq[:, rows, :-1] += gL
    gq[:, rows, 1:] += gR
    if ny > 1:
        qy = qg[:, :, 1:nx + 1]
        Gbar = np.zeros((4, ny + 1, nx))
        Gbar[:, :ny, :] += mu / cfg.dy
        Gbar[:, 1:, :] -= mu / cfg.dy
        gL, gR = _face_T(qy[:, :-1, :], qy[:, 1:, :], Gbar, cfg.gamma, 1)
        gq[:, :, 1:nx + 1][:, :-1, :] += gL
        gq[:, :, 1:nx + 1][:, 1:, :] += gR
    return _pad_T(gq, q.shape, cfg, 1)


def rk2_step_vjp(q, lam, cfg, k):
    """(d rk2_step(q, cfg, k) / dq)^T lam."""
    t0, t1 = (k - 1) * cfg.dt, k * cfg.dt
    q1 = q + cfg.dt * hdm.rhs(q, cfg, t0)
    lam1 = 0.5 * lam + 0.5 * cfg.dt * rhs_vjp(q1, lam, cfg, t1)
    return 0.5 * lam + lam1 + cfg.dt * rhs_vjp(q, lam1, cfg, t0)


# ----------------------------------------------------------------------------
# reduced basis
# ----------------------------------------------------------------------------

def gappy_coords_vjp(Phi, rows, v, psi, lam_y):
    """Transpose of tangent.gappy_coords_jvp: returns (lam_Phi, lam_v, lam_psi)
    with y = (A^T A)^{-1} A^T b, A = Phi[rows], b = (v - psi)[rows]:
    z = (A^T A)^{-1} lam_y, lam_A = r z^T - A z y^T, lam_b = A z."""
    N = Phi.shape[0]
    lam_Phi = np.zeros_like(Phi)
    lam_v = np.zeros(N)
    if Phi.shape[1] == 0:
        return lam_Phi, lam_v, np.zeros(N)
    y = rom.gappy_coords(Phi, rows, v, psi)
    A = Phi[rows, :]
    b = v[rows] - psi[rows]
    r = b - A @ y
    zz = np.linalg.solve(A.T @ A, lam_y)
    np.add.at(lam_Phi, rows, np.outer(r, zz) - np.outer(A @ zz, y))
    lb = A @ zz
    np.add.at(lam_v, rows, lb)
    return lam_Phi, lam_v, -lam_v.copy()


def pod_vjp(Xc, lam_Phi, m, pod_tol, abs_floor):
    """Transpose of tangent.pod_jvp's Phi tangent: lam_X for the cotangent
    lam_Phi of the kept (signed) columns."""
    Phi, _ = rom.pod(Xc, m, pod_tol, abs_floor)
    me = Phi.shape[1]
    lam_X = np.zeros_like(Xc)
    if me == 0:
        return lam_X
    U, s, Vt = np.linalg.svd(Xc, full_matrices=False)
    V = Vt.T
    for j in range(me):
        sign = 1.0 if np.dot(Phi[:, j], U[:, j]) > 0.0 else -1.0
        lj = sign * lam_Phi[:, j]
        sj = s[j]
        proj = lj - U @ (U.T @ lj)
        lam_X += np.outer(proj / sj, V[:, j])
        for i in range(s.size):
            if i == j:
                continue
            cij = np.dot(lj, U[:, i]) / (sj * sj - s[i] * s[i])
            lam_X += cij * (sj * np.outer(U[:, i], V[:, j]) + s[i] * np.outer(U[:, j], V[:, i]))
    return lam_X


def _shapiro_1d_T(w, n, axis, periodic):
    """Transpose of filt.shapiro_1d along `axis`."""
    wts = filt.SHAPIRO[n]
    g = n
    L = w.shape[axis]
    shp = list(w.shape)
    shp[axis] = L + 2 * g
    up = np.zeros(shp)
    for t, wgt in enumerate(wts):
        idx = [slice(None)] * w.ndim
        idx[axis] = slice(t, t + L)
        up[tuple(idx)] += wgt * w * (0.25 ** n)
    # fold the padding back (transpose of filt._pad_axis)
    core = np.take(up, np.arange(g, g + L), axis=axis).copy()
    lo = np.take(up, np.arange(0, g), axis=axis)
    hi = np.take(up, np.arange(g + L, L + 2 * g), axis=axis)
    if periodic:
        idx = [slice(None)] * w.ndim
        idx[axis] = slice(L - g, L)
        core[tuple(idx)] += lo
        idx[axis] = slice(0, g)
        core[tuple(idx)] += hi
    else:
        idx = [slice(None)] * w.ndim
        idx[axis] = slice(0, 1)
        core[tuple(idx)] += lo.sum(axis=axis, keepdims=True)
        idx[axis] = slice(L - 1, L)
        core[tuple(idx)] += hi.sum(axis=axis, keepdims=True)
    return core


def shapiro_T(w, n, cfg):
    """Transpose of filt.shapiro (x then y): y^T, then x^T."""
    out = w
    if cfg.ny > 1:
        out = _shapiro_1d_T(out, n, 1, cfg.bc[2] == W.BC_PERIODIC)
    return _shapiro_1d_T(out, n, 2, cfg.bc[0] == W.BC_PERIODIC)


def spatial_filter_vjp(lam, orders, keeps, cfg):
    """Transpose of the kept filter passes (tangent.spatial_filter_jvp with
    its keep masks; orders[i] is the Shapiro n of pass i): the passes in
    reverse order, each lam <- lam off the kept cells + F^T(lam on them)."""
    lam = lam.copy()
    for n, keep in zip(reversed(orders), reversed(keeps)):
        if not keep.any():
            continue
        kept = np.where(keep[None], lam, 0.0)
        lam = np.where(keep[None], 0.0, lam) + shapiro_T(kept, n, cfg)
    return lam


def _filter_logged(q, q_prev, cfg, t):
    """filt.spatial_filter with each pass's order and keep mask logged (the
    same loop, the same values)."""
    q = q.copy()
    keeps, orders = [], []
    for n in cfg.filt_orders:
        rho_old = filt.cell_residual(q, q_prev, cfg, t)
        for _ in range(cfg.jmax_f):
            g = filt.shapiro(q, n, cfg)
            rho_new = filt.cell_residual(g, q_prev, cfg, t)
            keep = rho_new < rho_old
            keeps.append(keep)
            orders.append(n)
            if not keep.any():
                break
            q[:, keep] = g[:, keep]
            dec = float(np.sum(rho_old[keep] - rho_new[keep]))
            tot = float(np.sum(rho_old[keep]))
            if dec < cfg.eps_f * tot:
                break
            rho_old = filt.cell_residual(q, q_prev, cfg, t)
    return q, keeps, orders


def _pressure_vjp(q, lp, gamma):
    """(dp/dq)^T lp for p = (gamma - 1)(E - |m|^2 / (2 rho))."""
    rho, mx, my, en = q
    kin = (mx * mx + my * my) / rho
    return (gamma - 1.0) * np.stack([0.5 * kin / rho * lp, -mx / rho * lp,
                                     -my / rho * lp, lp])


# ----------------------------------------------------------------------------
# the reverse sweep
# ----------------------------------------------------------------------------

def forward_tape(q0, cfg, steps, box=None):
    """Algorithm 1 (the arom.Arom loop, Euler SSP-RK2) recording what the
    reverse sweep needs.  Bases and reference states are numbered versions:
    a hybrid step reads the versions in effect, a rebuild makes new ones
    from its window and the reference state in effect.  Returns (J, tape)."""
    if cfg.scheme != W.SCHEME_RK2 or cfg.pde != W.PDE_EULER:
        raise NotImplementedError("the adjoint covers the Euler SSP-RK2 HDM")
    shape = (cfg.nvar, cfg.ny, cfg.nx)
    i0, i1, j0, j1 = box if box is not None else (0, cfg.nx, 0, cfg.ny)
    wgt = cfg.dt * cfg.dx * cfg.dy
    snaps = {0: np.asarray(q0, np.float64).reshape(shape).copy()}
    Phis, psis = [], []          # versions
    cur_phi = cur_psi = None
    s_hat = s_tilde = None
    P = []
    G = np.zeros(0, np.int64)
    J = 0.0
    tape = []
    flat = lambda a: a.reshape(-1)  # noqa: E731
    for k in range(1, steps + 1):
        prev = snaps[k - 1]
        full = (k + 1 <= cfg.w) or (cfg.z > 0 and k % cfg.z == 0)
        rec = {"k": k, "full": full}
        t = k * cfg.dt
        if full:
            gam = hdm.full_step(prev, cfg, k)
        else:
            Phi, psi = Phis[cur_phi], psis[cur_psi]
            v = prev.copy()
            v[:, s_hat] = hdm.rk2_step(prev, cfg, k)[:, s_hat]
            if cfg.regress_rows == W.ROWS_SAMPLE:
                cells = np.flatnonzero(s_hat)
                rows = np.concatenate([c * cfg.ncell + cells for c in range(cfg.nvar)])
            else:
                rows = np.asarray(P)
            y = rom.gappy_coords(Phi, rows, flat(v), flat(psi))
            rec.update(phi=cur_phi, psi=cur_psi, s_hat=s_hat, rows=rows, vpred=v.copy(), y=y)
            r = flat(psi).copy()
            if Phi.shape[1]:
                r = r + Phi @ y
            v[:, ~s_hat] = r.reshape(shape)[:, ~s_hat]
            gam, keeps, orders = _filter_logged(v, prev, cfg, t)
            rec.update(keeps=keeps, orders=orders)
        snaps[k] = gam
        J += wgt * float(np.sum(T.pressure(gam, cfg.gamma)[j0:j1, i0:i1]))
        if k == cfg.w - 1:
            psis.append(rom.window_mean([snaps[j] for j in range(0, cfg.w)]))
            cur_psi = len(psis) - 1
            rec["psi_init"] = cur_psi
        if k >= cfg.w - 1 and (cfg.z <= 0 or (k + 1) % cfg.z != 0):
            if k >= cfg.w and cur_phi is not None:
                Phi, psi = Phis[cur_phi], psis[cur_psi]
                rows_e = np.asarray(P) if cfg.regress_rows != W.ROWS_SAMPLE else np.concatenate(
                    [c * cfg.ncell + np.flatnonzero(s_hat) for c in range(cfg.nvar)])
                y2 = rom.gappy_coords(Phi, rows_e, flat(gam), flat(psi))
                eps = select.cell_error(flat(gam), flat(psi), Phi, y2, cfg.nvar)
                G, _ = select.select_cells(eps, cfg.sel_mode, cfg.delta, cfg.top_frac)
            else:
                G = np.zeros(0, np.int64)
            win = list(range(k - cfg.w + 1, k + 1))
            Xc = np.stack([flat(snaps[j]) - flat(psis[cur_psi]) for j in win], axis=1)
            raw = float(np.sqrt(sum(float(np.sum(snaps[j] * snaps[j])) for j in win)))
            Phi_new, _ = rom.pod(Xc, cfg.m, cfg.pod_tol, cfg.pod_abs * raw)
            Phis.append(Phi_new)
            P = rom.odeim(Phi_new, cfg.n_p, cfg.tie_tol)
            s_hat, s_tilde = select.build_masks(G, P, cfg)
            psis.append(rom.window_mean([snaps[j] for j in win]))
            rec.update(rebuild=True, window=win, psi_cur=cur_psi, Xc=Xc,
                       floor=cfg.pod_abs * raw, new_phi=len(Phis) - 1, new_psi=len(psis) - 1)
            cur_phi, cur_psi = len(Phis) - 1, len(psis) - 1
        tape.append(rec)
    return J, {"snaps": snaps, "Phis": Phis, "psis": psis, "steps": tape, "box": (i0, i1, j0, j1),
               "shape": shape}


def gradient(q0, cfg, steps, box=None):
    """J and dJ/dq0 by forward_tape and one reverse sweep."""
    J, tp = forward_tape(q0, cfg, steps, box)
    shape = tp["shape"]
    snaps, Phis, psis = tp["snaps"], tp["Phis"], tp["psis"]
    i0, i1, j0, j1 = tp["box"]
    wgt = cfg.dt * cfg.dx * cfg.dy
    lam = {k: np.zeros(shape) for k in snaps}
    lPhi = [np.zeros_like(P) for P in Phis]
    lpsi = [np.zeros(np.prod(shape)) for _ in psis]
    nvar = cfg.nvar
    for rec in reversed(tp["steps"]):
        k = rec["k"]
        if rec.get("rebuild"):                     # the rebuild after step k
            w = len(rec["window"])
            lX = pod_vjp(rec["Xc"], lPhi[rec["new_phi"]], cfg.m, cfg.pod_tol, rec["floor"])
            for c, j in enumerate(rec["window"]):
                lam[j] += lX[:, c].reshape(shape)
                lam[j] += lpsi[rec["new_psi"]].reshape(shape) / w
            lpsi[rec["psi_cur"]] -= lX.sum(axis=1)
        if "psi_init" in rec:                      # psi_{w-1} = mean(gamma_0..gamma_{w-1})
            for j in range(0, cfg.w):
                lam[j] += lpsi[rec["psi_init"]].reshape(shape) / cfg.w
        lp = np.zeros(shape[1:])                    # the output term of step k
        lp[j0:j1, i0:i1] = wgt
        lk = lam.pop(k) + _pressure_vjp(snaps[k], lp, cfg.gamma)
        prev = snaps[k - 1]
        if rec["full"]:
            lam[k - 1] += rk2_step_vjp(prev, lk, cfg, k)
            continue
        Phi, psi = Phis[rec["phi"]], psis[rec["psi"]]
        lv = spatial_filter_vjp(lk, rec["orders"], rec["keeps"], cfg).reshape(-1)
        sb = np.tile(~rec["s_hat"].reshape(-1), nvar)
        lrec = np.where(sb, lv, 0.0)
        lpsi[rec["psi"]] += lrec
        ly = np.zeros(0)
        if Phi.shape[1]:
            lPhi[rec["phi"]] += np.outer(lrec, rec["y"])
            ly = Phi.T @ lrec
        lvp = np.where(sb, 0.0, lv)
        gP, gv, gpsi = gappy_coords_vjp(Phi, rec["rows"], rec["vpred"].reshape(-1),
                                        psi.reshape(-1), ly)
        lPhi[rec["phi"]] += gP
        lpsi[rec["psi"]] += gpsi
        lvp = (lvp + gv).reshape(shape)
        m3 = np.broadcast_to(rec["s_hat"][None], shape)
        lam[k - 1] += np.where(m3, 0.0, lvp) + rk2_step_vjp(prev, np.where(m3, lvp, 0.0), cfg, k)
    return J, lam[0]
