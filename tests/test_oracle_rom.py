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


# ---- the reduced-precision form of the sample-row solve ---------------------

def test_round_bf16_is_torch_bfloat16():
    """round_bf16 against PyTorch's FP32 -> bfloat16 conversion (round to
    nearest even), on random values and on constructed ties."""
    torch = pytest.importorskip("torch")
    g = np.random.Generator(np.random.PCG64(70))
    x = (g.standard_normal(200000) * 10.0 ** g.uniform(-6, 6, 200000)).astype(np.float32)
    bits = x.view(np.uint32)
    ties = ((bits & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)[:5000]
    x = np.concatenate([x, ties, -ties])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(rom.round_bf16(x), want)


def test_round_tf32_cases_and_bound():
    """TF32 rounding: hand-worked cases (a tie goes away from zero, below half
    goes down, above half goes up, a carry into the exponent), the result
    keeps 10 mantissa bits, and |round(x) - x| <= 2^-11 |x|."""
    e = 2.0 ** -10   # one TF32 unit in the last place at 1
    cases = {1 + e / 2: 1 + e, -(1 + e / 2): -(1 + e), 1 + e / 4: 1.0, 1 + e / 2 + 2 ** -20: 1 + e,
             1 + 3 * e / 2: 1 + 2 * e, 2 - e / 2: 2.0, 0.0: 0.0, 3.0: 3.0}
    for x, want in cases.items():
        assert rom.round_tf32(np.float32(x)) == want, (x, rom.round_tf32(np.float32(x)), want)
    g = np.random.Generator(np.random.PCG64(71))
    x = (g.standard_normal(100000) * 10.0 ** g.uniform(-8, 8, 100000)).astype(np.float32)
    r = rom.round_tf32(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -11 * np.abs(x.astype(np.float64)))
    assert np.all(r.astype(np.float32).view(np.uint32) & np.uint32(0x1FFF) == 0)


def test_split_tf32_reconstructs_to_2_pow_21():
    g = np.random.Generator(np.random.PCG64(72))
    x = (g.standard_normal(100000) * 10.0 ** g.uniform(-8, 8, 100000)).astype(np.float32)
    hi, lo = rom.split_tf32(x)
    xd = x.astype(np.float64)
    assert np.all(hi.astype(np.float32).view(np.uint32) & np.uint32(0x1FFF) == 0)
    assert np.all(lo.astype(np.float32).view(np.uint32) & np.uint32(0x1FFF) == 0)
    assert np.all(np.abs(hi + lo - xd) <= 2.0 ** -21 * np.abs(xd))
    assert np.all(np.abs(hi) <= np.abs(xd))


@pytest.mark.parametrize("red", [W.RED_F32, W.RED_TF32, W.RED_BF16, W.RED_TF32_SPLIT])
def test_normal_equations_exact_on_representable_inputs(red):
    """With a basis whose entries are already BF16 (hence TF32) values, no
    rounding changes anything: every precision's normal-equation solution is
    the least-squares solution of gappy_coords."""
    g = np.random.Generator(np.random.PCG64(73))
    N, m = 400, 7
    Phi = g.integers(-64, 65, size=(N, m)) / 64.0      # 7-bit integers over 2^6
    rows = np.sort(g.choice(N, 90, replace=False))
    psi = g.standard_normal(N)
    v = psi + Phi @ g.standard_normal(m) + 0.1 * g.standard_normal(N)
    want = rom.gappy_coords(Phi, rows, v, psi)
    got = rom.gappy_coords_normal(Phi, rows, v, psi, red)
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


def test_normal_equations_follow_the_rounded_matrix():
    """TF32 and BF16 normal matrices move y by about kappa times their input
    rounding (and by no more than the first-order bound), BF16 more than
    TF32, the split form by no more than FP32 rounding."""
    g = np.random.Generator(np.random.PCG64(74))
    N, m = 3000, 12
    Phi, _ = np.linalg.qr(g.standard_normal((N, m)))
    Phi = Phi.astype(np.float32).astype(np.float64)
    rows = np.sort(g.choice(N, 600, replace=False))
    psi = g.standard_normal(N)
    v = psi + Phi @ g.standard_normal(m)
    exact = rom.gappy_coords(Phi, rows, v, psi)
    X = Phi[rows]
    kappa = np.linalg.cond(X.T @ X)
    errs = {}
    for red, u in ((W.RED_TF32, 2.0 ** -11), (W.RED_BF16, 2.0 ** -8),
                   (W.RED_TF32_SPLIT, 2.0 ** -21)):
        y = rom.gappy_coords_normal(Phi, rows, v, psi, red)
        errs[red] = np.linalg.norm(y - exact) / np.linalg.norm(exact)
        # |E| <= (2u + u^2) |X|^T |X| entrywise
        eta = (2 * u + u * u) * np.linalg.norm(np.abs(X).T @ np.abs(X), 2) / \
            np.linalg.norm(X.T @ X, 2)
        assert errs[red] <= kappa * eta / (1 - kappa * eta) + 1e-12, (red, errs[red])
    assert errs[W.RED_BF16] > 4 * errs[W.RED_TF32] > 0
    assert errs[W.RED_TF32_SPLIT] < 1e-6


def test_batched_odeim_study_variant():
    """rom.odeim_batched (a cheaper variant for study, not the paper's
    method): with one point per pass it is ODEIM; with b per pass each pass
    takes the b best-scored unpicked rows of that pass."""
    g = np.random.Generator(np.random.PCG64(12))
    Phi, _ = np.linalg.qr(g.standard_normal((300, 6)))
    assert rom.odeim_batched(Phi, 20, 1e-12, 1) == rom.odeim(Phi, 20, 1e-12)
    P = rom.odeim_batched(Phi, 20, 1e-12, 4)
    assert len(P) == 20 and len(set(P)) == 20
    first = rom.deim(Phi, 1e-12)
    assert P[:6] == first
    A = Phi[first, :]
    score = rom.lambda_min_update_secular(A.T @ A, Phi)
    score[first] = -np.inf
    assert sorted(P[6:10]) == sorted(np.argsort(-score, kind="stable")[:4].tolist())
