"""Reduced-basis approximation: Sec. 2.3.1 of the paper.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  pod            POD_m (Eq. pod): thin SVD of the centred window, first m
                 left singular vectors.
  gappy_coords   y = (P^T Phi)^+ P^T (v - psi)   (Eq. red_coord)
  deim           DEIM greedy points (the interpolation points that ODEIM
                 starts from)
  odeim          ODEIM_{n_p} (Eq. odeim): DEIM points, then oversampling
  window_mean    psi = (1/w) sum of w snapshots   (Eq. mean)
  gappy_coords_normal
                 the same coordinates on the rows given, from the normal
                 equations with the normal matrix formed from inputs rounded
                 to TF32, BF16 or a TF32 hi/lo pair (the reduced-precision
                 form of the sample-row solve); round_tf32, round_bf16 and
                 split_tf32 are those roundings, bit for bit

Readings where the paper is silent:
  * numerical rank: mode j is kept when sigma_j > pod_tol * sigma_1 and
    sigma_j > pod_abs * ||X_raw||_F (the Frobenius norm of the uncentred
    window), so a window that differs from psi only by rounding noise has
    rank 0; m_eff <= m.  Each kept column is signed so that its
    largest-magnitude entry (first one on ties) is positive.
  * ODEIM oversampling picks, among rows not yet chosen, the row phi_i that
    maximises lambda_min(A^T A + phi_i phi_i^T), A = P^T Phi: the smallest
    eigenvalue after adding that row, i.e. the smallest squared singular
    value of the augmented sampled basis.
  * arg-max ties: among rows whose score is >= s_max (1 - tie_tol) the
    lowest row index wins, so rounding-order differences below tie_tol
    cannot change a choice.
  * rows are degrees of freedom (v*Nc + cell); a cell is sampled when any of
    its rows is.
"""
from __future__ import annotations

import numpy as np

import workloads as W


def pod(Xc, m, pod_tol, abs_floor=0.0):
    """POD_m of a centred snapshot matrix Xc (N x w) by LAPACK's thin SVD.
    abs_floor = pod_abs * ||X_raw||_F.

    Returns (Phi [N x m_eff], sigma [min(N, w)])."""
    U, s, _ = np.linalg.svd(Xc, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros((Xc.shape[0], 0)), s
    keep = (s[:m] > pod_tol * s[0]) & (s[:m] > abs_floor)
    m_eff = int(np.count_nonzero(keep))
    Phi = U[:, :m_eff].copy()
    for j in range(m_eff):
        i = int(np.argmax(np.abs(Phi[:, j])))
        if Phi[i, j] < 0.0:
            Phi[:, j] = -Phi[:, j]
    return Phi, s


def window_mean(snaps):
    """psi = (1/w) sum_j gamma_j (Eq. mean); snaps is a list of states."""
    return np.mean(np.stack(snaps, axis=0), axis=0)


def gappy_coords(Phi, P, v, psi):
    """Least-squares reduced coordinates on the sampled rows P (Eq. red_coord).
    Phi: N x m, P: row indices, v, psi: length-N vectors."""
    if Phi.shape[1] == 0:
        return np.zeros(0)
    A = Phi[P, :]
    b = v[P] - psi[P]
    y, *_ = np.linalg.lstsq(A, b, rcond=None)
    return y


def round_tf32(x):
    """FP32 values rounded to TF32 (10 stored mantissa bits; FP32 exponent
    range), to nearest with ties away from zero: half of the dropped 13-bit
    field is added to the magnitude bits, which are then cut.  Finite inputs
    whose magnitude rounds below FP32's largest finite value."""
    b = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def round_bf16(x):
    """FP32 values rounded to BF16 (7 stored mantissa bits), to nearest with
    ties to even (the kept field's lowest bit decides a tie).  Finite
    inputs."""
    b = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def split_tf32(x):
    """x = hi + lo with hi = x's 13 low mantissa bits cleared (a TF32 value)
    and lo = round_tf32(x - hi) (x - hi is exact in FP32): hi + lo is within
    2^-21 |x| of x."""
    x32 = np.ascontiguousarray(np.asarray(x, np.float32))
    hi = (x32.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)
    return hi.astype(np.float64), round_tf32(x32 - hi)


def gappy_coords_normal(Phi, rows, v, psi, red):
    """Reduced coordinates (Eq. red_coord) on `rows` from the normal
    equations (X^T X) y = X^T (v - psi)_rows, X = Phi[rows], where the
    normal matrix is formed from X rounded as `red` says (workloads.RED_*:
    F32 = the FP32 values as given, TF32 / BF16 = round_tf32 / round_bf16,
    TF32_SPLIT = hi + lo of split_tf32), and the right-hand side from X as
    given; everything in FP64, solved by Cholesky."""
    X = np.asarray(Phi, np.float64)[rows, :]
    if red == W.RED_TF32:
        Xr = round_tf32(X)
    elif red == W.RED_BF16:
        Xr = round_bf16(X)
    elif red == W.RED_TF32_SPLIT:
        hi, lo = split_tf32(X)
        Xr = hi + lo
    else:
        Xr = X
    G = Xr.T @ Xr
    b = X.T @ (np.asarray(v, np.float64)[rows] - np.asarray(psi, np.float64)[rows])
    L = np.linalg.cholesky(G)
    return np.linalg.solve(L.T, np.linalg.solve(L, b))


def argmax_tie(score, tie_tol, exclude=()):
    """Lowest index among the rows whose score is within tie_tol (relative)
    of the maximum; rows in `exclude` never win."""
    s = np.array(score, dtype=np.float64, copy=True)
    if len(exclude):
        s[np.asarray(list(exclude), dtype=np.int64)] = -np.inf
    smax = s.max()
    return int(np.flatnonzero(s >= smax * (1.0 - tie_tol))[0])


def deim(Phi, tie_tol):
    """DEIM interpolation points (Chaturantabut & Sorensen): the first point
    maximises |phi_1|; point l maximises the residual of phi_l after
    interpolating it from phi_1..phi_{l-1} at the points chosen so far."""
    N, m = Phi.shape
    if m == 0:
        return []
    p = [argmax_tie(np.abs(Phi[:, 0]), tie_tol)]
    for l in range(1, m):
        c = np.linalg.solve(Phi[p, :l], Phi[p, l])
        r = Phi[:, l] - Phi[:, :l] @ c
        p.append(argmax_tie(np.abs(r), tie_tol, exclude=p))
    return p


def lambda_min_update_eig(M, rows):
    """lambda_min(M + phi phi^T) for each phi in rows, by a dense symmetric
    eigensolve per row (the definition; for small inputs)."""
    out = np.empty(rows.shape[0])
    for i in range(rows.shape[0]):
        phi = rows[i]
        out[i] = np.linalg.eigvalsh(M + np.outer(phi, phi))[0]
    return out


def lambda_min_update_secular(M, rows, chunk=4096):
    """lambda_min(M + phi phi^T) for each phi in rows, as the smallest root
    of the secular equation 1 + sum_j z_j^2 / (lambda_j - mu) = 0 with
    M = W diag(lambda) W^T and z = W^T phi (Golub's rank-one modification
    of the symmetric eigenproblem).  The root lies in [lambda_1,
    min(lambda_2, lambda_1 + |z|^2)]; it is found by bisection to the last
    bit: a row stops when the midpoint of its bracket rounds to one of the
    ends, and the upper end is returned.  The secular function is only
    evaluated strictly inside (lambda_1, lambda_2), so no pole is touched.
    When it has no root there the answer is lambda_1: z_1 = 0 (lambda_1
    stays an eigenvalue and none falls below it) or a double eigenvalue
    lambda_1 = lambda_2 (an empty bracket).  Rows are taken in chunks so the
    work arrays stay small."""
    lam, Wm = np.linalg.eigh(M)
    Z = rows @ Wm
    z2 = Z * Z
    if lam.size == 1:
        return lam[0] + z2[:, 0]
    out = np.empty(rows.shape[0])
    for a in range(0, rows.shape[0], chunk):
        zc = z2[a:a + chunk]
        lo = np.full(zc.shape[0], lam[0])
        hi = np.minimum(lam[1], lam[0] + zc.sum(axis=1))
        hi[zc[:, 0] == 0.0] = lam[0]
        live = np.flatnonzero(lo < hi)
        for _ in range(200):
            if live.size == 0:
                break
            l, h = lo[live], hi[live]
            mid = 0.5 * (l + h)
            inside = (mid > l) & (mid < h)
            live, l, h, mid = live[inside], l[inside], h[inside], mid[inside]
            if live.size == 0:
                break
            f = 1.0 + (zc[live] / (lam[None, :] - mid[:, None])).sum(axis=1)
            below = f < 0.0
            lo[live] = np.where(below, mid, l)
            hi[live] = np.where(below, h, mid)
        out[a:a + chunk] = hi
    return out


def odeim_batched(Phi, n_p, tie_tol, b):
    """A cheaper variant of ODEIM for study (not the paper's method): after
    the DEIM points, each oversampling pass scores every row once against
    the current sampled Gram matrix and takes the b best rows (in score
    order, ties to the lowest index) instead of one.  b = 1 is odeim()."""
    N, m = Phi.shape
    p = deim(Phi, tie_tol)
    if m == 0:
        return p
    n_p = min(n_p, N)
    while len(p) < n_p:
        A = Phi[p, :]
        score = lambda_min_update_secular(A.T @ A, Phi)
        for _ in range(min(b, n_p - len(p))):
            p.append(argmax_tie(score, tie_tol, exclude=p))
    return p


def odeim(Phi, n_p, tie_tol, method="secular"):
    """ODEIM_{n_p}(Phi) (Eq. odeim): the DEIM points, then n_p - m greedy
    oversampling points, each maximising the smallest eigenvalue of the
    sampled Gram matrix after adding the row.  Returns row indices in the
    order chosen."""
    N, m = Phi.shape
    p = deim(Phi, tie_tol)
    if m == 0:
        return p
    n_p = min(n_p, N)
    f = lambda_min_update_secular if method == "secular" else lambda_min_update_eig
    while len(p) < n_p:
        A = Phi[p, :]
        M = A.T @ A
        score = f(M, Phi)
        p.append(argmax_tie(score, tie_tol, exclude=p))
    return p
