"""Error indicator, sample selection and sampling-set algebra: Sec. 2.3.3
(pointwise reconstruction error, RRE ordering, Eq. rre, the union defining
S-hat) and Sec. 2.4 / Algorithm 1 (union, setdiff, Neighbors; Fig. 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings where the paper is silent:
  * the selection unit is the cell: eps_cell = sum over the c variables of
    the pointwise squared error (the paper indexes dofs; a FV cell is solved
    with all its variables).
  * ordering: descending eps, ties by ascending cell id.
  * exact sums: eps is mapped to integers key = floor(eps * 2^s) with
    s = 63 - ceil(log2 Nc) - e, where eps_max = f 2^e, f in [0.5, 1), so that
    every partial sum of keys fits in 63 bits and the RRE threshold test is
    exact integer arithmetic.  The map is exact (a power-of-two scaling and a
    floor), so equal eps give equal keys on any machine.
  * RRE rule (Eq. rre): n_g = smallest n with sum_{top n} key >= delta * S,
    tested exactly as sum * 2^(53 - E) >= a * S where delta = a 2^(E - 53).
    All-zero keys (S = 0) give n_g = 0.
  * top-fraction rule (run configurations): n_g = ceil(top_frac * Nc).
  * the "halo" of a run configuration dilates the sampled set by that many
    cells (diamond |di| + |dj| <= halo) before Neighbors is taken.
  * Neighbors(S-hat) = cells within the scheme's dependency radius that are
    not in S-hat: radius 1 (BDF1 5-point residual) or 2 (two RK2 stages).
    Non-periodic sides clip at the boundary.
"""
from __future__ import annotations

import math

import numpy as np

import workloads as W


def cell_error(gamma, psi, Phi, y, nvar):
    """eps_cell = sum_v (gamma - psi - Phi y)_{v,cell}^2  (Sec. 2.3.3)."""
    if Phi.shape[1]:
        rec = Phi @ y
    else:
        rec = np.zeros_like(gamma)
    r = (gamma - psi) - rec
    r2 = (r * r).reshape(nvar, -1)
    e = r2[0].copy()
    for v in range(1, nvar):
        e = e + r2[v]
    return e


def ceil_log2(n):
    return 0 if n <= 1 else (int(n) - 1).bit_length()


def fixed_point_keys(eps):
    """Exact integer keys of the error values (see module docstring)."""
    eps = np.asarray(eps, dtype=np.float64)
    nc = eps.size
    emax = float(eps.max()) if nc else 0.0
    if emax <= 0.0:
        return [0] * nc, 0
    _, e = math.frexp(emax)
    s = 63 - ceil_log2(nc) - e
    keys = [int(math.floor(math.ldexp(float(x), s))) for x in eps]
    return keys, s


def select_cells(eps, sel_mode, delta=0.9, top_frac=0.1):
    """G: the first n_g cells in (descending eps, ascending id) order.
    Returns (sorted cell ids of G, n_g)."""
    keys, _ = fixed_point_keys(eps)
    nc = len(keys)
    order = sorted(range(nc), key=lambda i: (-keys[i], i))
    if sel_mode == W.SEL_TOPFRAC:
        n_g = min(nc, int(math.ceil(top_frac * nc)))
    else:
        S = sum(keys)
        if S == 0:
            n_g = 0
        else:
            f, E = math.frexp(delta)
            a = int(f * (1 << 53))
            shift = 53 - E
            acc = 0
            n_g = nc
            for n, i in enumerate(order, start=1):
                acc += keys[i]
                if (acc << shift) >= a * S:
                    n_g = n
                    break
    return np.sort(np.asarray(order[:n_g], dtype=np.int64)), n_g


def _offsets(radius, two_d):
    if not two_d:
        return [(0, d) for d in range(-radius, radius + 1)]
    return [(dj, di) for dj in range(-radius, radius + 1)
            for di in range(-radius, radius + 1) if abs(di) + abs(dj) <= radius]


def dilate(mask, radius, cfg):
    """Cells within diamond distance `radius` of a marked cell.
    mask: bool [ny, nx]."""
    if radius <= 0:
        return mask.copy()
    ny, nx = mask.shape
    px = cfg.bc[0] == W.BC_PERIODIC
    py = cfg.bc[2] == W.BC_PERIODIC
    out = np.zeros_like(mask)
    js, is_ = np.nonzero(mask)
    for dj, di in _offsets(radius, ny > 1):
        jj = js + dj
        ii = is_ + di
        if px:
            ii = ii % nx
        if py:
            jj = jj % ny
        ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny)
        out[jj[ok], ii[ok]] = True
    return out


def stencil_radius(cfg):
    """Cells a partial solve on S-hat reads around it: one for the
    first-order implicit residual, two for SSP-RK2's two stages and for the
    MUSCL residual (its face states use the neighbours' slopes)."""
    return 1 if cfg.scheme == W.SCHEME_BE else 2


def build_masks(G_cells, P_rows, cfg):
    """S-hat = union(G, cells of P) dilated by the halo; S-tilde =
    Neighbors(S-hat); S-breve = setdiff(all, S-hat).  Returns bool [ny, nx]
    arrays (S_hat, S_tilde)."""
    ny, nx = cfg.ny, cfg.nx
    nc = nx * ny
    base = np.zeros(nc, bool)
    base[np.asarray(G_cells, dtype=np.int64)] = True
    if len(P_rows):
        base[np.asarray(P_rows, dtype=np.int64) % nc] = True
    s_hat = dilate(base.reshape(ny, nx), cfg.halo, cfg)
    ring = dilate(s_hat, stencil_radius(cfg), cfg)
    s_tilde = ring & ~s_hat
    return s_hat, s_tilde
