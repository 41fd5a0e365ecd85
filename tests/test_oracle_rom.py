"""Pins of the oracle's reduced-basis part (Sec. 2.3.1): POD against a
window of known spectrum, gappy least squares against exact
representations and the normal equations, DEIM against the pivots of
Gaussian elimination with partial pivoting, ODEIM against brute-force
smallest singular values.  CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import rom


def test_pod_recovers_known_spectrum_and_subspace():
    N, w, m = 300, 12, 5
    g = np.random.Generator(np.random.PCG64(7))
    U, _ = np.linalg.qr(g.standard_normal((N, w)))
    V, _ = np.linalg.qr(g.standard_normal((w, w)))
    sig = 0.5 ** np.arange(w)
    Xc = (U * sig) @ V.T
    Phi, s = rom.pod(Xc, m, 1e-7)
    assert Phi.shape == (N, m)
    assert np.allclose(s, sig, rtol=1e-12, atol=1e-15)
    assert np.abs(Phi.T @ Phi - np.eye(m)).max() < 1e-13
    P_true = U[:, :m] @ U[:, :m].T
    assert np.abs(Phi @ Phi.T - P_true).max() < 1e-12
    # sign convention: largest-magnitude entry of each column is positive
    for j in range(m):
        i = np.argmax(np.abs(Phi[:, j]))
        assert Phi[i, j] > 0


def test_pod_numerical_rank_truncation():
    N, w = 200, 8
    g = np.random.Generator(np.random.PCG64(8))
    U, _ = np.linalg.qr(g.standard_normal((N, w)))
    V, _ = np.linalg.qr(g.standard_normal((w, w)))
    sig = np.array([1.0, 0.3, 1e-3, 1e-9, 0, 0, 0, 0])
    Phi, s = rom.pod((U * sig) @ V.T, 6, 1e-7)
    assert Phi.shape[1] == 3
    Phi0, _ = rom.pod(np.zeros((N, w)), 4, 1e-7)
    assert Phi0.shape == (N, 0)


def test_gappy_reconstructs_states_in_the_affine_subspace():
    N, m = 120, 4
    g = np.random.Generator(np.random.PCG64(9))
    Phi, _ = np.linalg.qr(g.standard_normal((N, m)))
    psi = g.standard_normal(N)
    a = g.standard_normal(m)
    v = psi + Phi @ a
    P = rom.odeim(Phi, 9, 1e-12)
    y = rom.gappy_coords(Phi, P, v, psi)
    assert np.abs(y - a).max() < 1e-12
    assert np.abs(psi + Phi @ y - v).max() < 1e-12
    # generic data: y solves the normal equations on the sampled rows
    v2 = g.standard_normal(N)
    y2 = rom.gappy_coords(Phi, P, v2, psi)
    A = Phi[P]
    b = v2[P] - psi[P]
    assert np.abs(A.T @ (A @ y2 - b)).max() < 1e-12


def _gepp_pivots(A):
    """Row pivots of Gaussian elimination with partial pivoting on A (N x m)."""
    A = A.copy()
    N, m = A.shape
    rows = np.arange(N)
    piv = []
    for j in range(m):
        i = j + int(np.argmax(np.abs(A[j:, j])))
        A[[j, i]] = A[[i, j]]
        rows[[j, i]] = rows[[i, j]]
        piv.append(int(rows[j]))
        A[j + 1:, j:] -= np.outer(A[j + 1:, j] / A[j, j], A[j, j:])
    return piv


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_deim_points_are_gepp_pivots(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    Phi, _ = np.linalg.qr(g.standard_normal((80, 7)))
    assert rom.deim(Phi, 1e-12) == _gepp_pivots(Phi)


def test_deim_tie_goes_to_lowest_index():
    Phi = np.zeros((6, 1))
    Phi[[1, 4], 0] = [0.5, -0.5]
    Phi[2, 0] = 0.5 * (1 - 1e-14)
    assert rom.deim(Phi, 1e-12) == [1]


@pytest.mark.parametrize("seed", [4, 5])
def test_odeim_matches_brute_force_smallest_singular_value(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    N, m, n_p = 40, 4, 11
    Phi, _ = np.linalg.qr(g.standard_normal((N, m)))
    p = rom.odeim(Phi, n_p, 1e-12, method="secular")
    assert p[:m] == rom.deim(Phi, 1e-12)
    assert len(set(p)) == n_p
    # brute force: each oversampling pick maximises sigma_min of the
    # augmented sampled matrix over all rows not yet chosen
    for l in range(m, n_p):
        chosen = p[:l]
        best, arg = -1.0, None
        for i in range(N):
            if i in chosen:
                continue
            smin = np.linalg.svd(Phi[chosen + [i]], compute_uv=False)[-1] ** 2
            if smin > best * (1 + 1e-12):
                best, arg = smin, i
        assert p[l] == arg
    assert rom.odeim(Phi, n_p, 1e-12, method="eig") == p


def test_secular_root_matches_dense_eigensolve():
    g = np.random.Generator(np.random.PCG64(12))
    A = g.standard_normal((9, 5))
    M = A.T @ A
    rows = g.standard_normal((50, 5))
    rows[3] = 0.0                       # no change: lambda_min stays
    a = rom.lambda_min_update_secular(M, rows)
    b = rom.lambda_min_update_eig(M, rows)
    assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()
    assert a[3] == pytest.approx(np.linalg.eigvalsh(M)[0], rel=1e-14)


def test_window_mean_is_the_average():
    snaps = [np.full(5, float(j)) for j in range(4)]
    assert np.array_equal(rom.window_mean(snaps), np.full(5, 1.5))
