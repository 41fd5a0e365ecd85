"""Pins of the oracle's selection (Sec. 2.3.3, Eq. rre), sampling-set algebra
(Algorithm 1, Fig. 1) and residual-gated Shapiro filtering (Sec. 2.3.4):
brute force on small inputs, exact integer sums, closed-form Fourier
responses.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import select, filt, hdm


def test_fixed_point_keys_are_exact_and_order_preserving():
    g = np.random.Generator(np.random.PCG64(3))
    eps = g.exponential(size=1000) ** 3
    keys, s = select.fixed_point_keys(eps)
    assert sum(keys) < 2 ** 63
    order_e = np.argsort(-eps, kind="stable")
    k = np.array(keys, dtype=object)
    assert all(k[order_e[i]] >= k[order_e[i + 1]] for i in range(999))
    # a power-of-two scaling then floor: exact for representable values
    assert keys[int(np.argmax(eps))] == math.floor(eps.max() * 2.0 ** s)
    assert 2 ** (62 - select.ceil_log2(1000)) <= max(keys) < 2 ** (63 - select.ceil_log2(1000))


def test_top_fraction_selects_largest_with_index_ties():
    eps = np.array([0.5, 3.0, 3.0, 0.1, 2.0, 3.0, 0.0, 2.0])
    G, n = select.select_cells(eps, W.SEL_TOPFRAC, top_frac=0.5)
    assert n == 4
    assert list(G) == [1, 2, 4, 5]     # the three 3.0s, then the lower-id 2.0
    G, n = select.select_cells(eps, W.SEL_TOPFRAC, top_frac=0.3)
    assert n == 3 and list(G) == [1, 2, 5]


@pytest.mark.parametrize("delta", [0.5, 0.8, 0.9, 0.99])
def test_rre_threshold_matches_float_brute_force(delta):
    g = np.random.Generator(np.random.PCG64(int(delta * 100)))
    eps = g.uniform(0.0, 1.0, size=257) ** 4
    order = np.argsort(-eps, kind="stable")
    cs = np.cumsum(eps[order]) / eps.sum()
    n_ref = int(np.argmax(cs >= delta)) + 1
    # brute force is trustworthy only away from the threshold
    assert abs(cs[n_ref - 1] - delta) > 1e-9 and (n_ref == 1 or abs(cs[n_ref - 2] - delta) > 1e-9)
    G, n = select.select_cells(eps, W.SEL_RRE, delta=delta)
    assert n == n_ref
    assert set(G) == set(order[:n_ref].tolist())


def test_rre_delta_one_takes_every_nonzero_and_zero_error_takes_none():
    eps = np.array([0.0, 1e-3, 0.0, 2.0, 5e-7])
    G, n = select.select_cells(eps, W.SEL_RRE, delta=1.0)
    assert list(G) == [1, 3, 4]
    G, n = select.select_cells(np.zeros(6), W.SEL_RRE, delta=0.9)
    assert n == 0 and G.size == 0


def _brute_dilate(mask, r, periodic):
    ny, nx = mask.shape
    out = np.zeros_like(mask)
    for j in range(ny):
        for i in range(nx):
            for jj in range(ny):
                for ii in range(nx):
                    if not mask[jj, ii]:
                        continue
                    di, dj = i - ii, j - jj
                    if periodic:
                        di = min(abs(di), nx - abs(di))
                        dj = min(abs(dj), ny - abs(dj)) if ny > 1 else abs(dj)
                    if abs(di) + abs(dj) <= r:
                        out[j, i] = True
    return out


@pytest.mark.parametrize("periodic", [True, False])
def test_masks_match_brute_force_distances(periodic):
    bc = (W.BC_PERIODIC,) * 4 if periodic else (W.BC_OUTFLOW,) * 4
    cfg = W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=9, ny=7, bc=bc, halo=1)
    G = np.array([0, 8, 30, 62])
    P = [4 * 63 + 17, 2 * 63 + 17, 63 + 45]        # rows of two cells (17, 45)
    s_hat, s_tilde = select.build_masks(G, P, cfg)
    base = np.zeros(63, bool)
    base[[0, 8, 30, 62, 17, 45]] = True
    base = base.reshape(7, 9)
    want_hat = _brute_dilate(base, 1, periodic)
    want_ring = _brute_dilate(want_hat, 2, periodic) & ~want_hat
    assert np.array_equal(s_hat, want_hat)
    assert np.array_equal(s_tilde, want_ring)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_shapiro_fourier_response(n):
    N = 64
    i = np.arange(N)
    for kw in (1, 5, 16, 31, 32):
        th = 2 * np.pi * kw / N
        u = np.cos(th * i).reshape(1, 1, N)
        out = filt.shapiro_1d(u, n, 2, True)
        want = (1.0 - np.sin(th / 2) ** (2 * n)) * u
        assert np.abs(out - want).max() < 1e-14


def test_shapiro_2d_is_separable_and_constant_preserving():
    cfg = W.ArConfig(pde=W.PDE_EULER, nx=32, ny=16, bc=(W.BC_PERIODIC,) * 4)
    x = np.arange(32)
    y = np.arange(16)
    tx, ty = 2 * np.pi * 3 / 32, 2 * np.pi * 2 / 16
    u = np.outer(np.cos(ty * y), np.cos(tx * x))[None].repeat(4, axis=0)
    out = filt.shapiro(u, 2, cfg)
    want = (1 - np.sin(tx / 2) ** 4) * (1 - np.sin(ty / 2) ** 4) * u
    assert np.abs(out - want).max() < 1e-14
    c = np.full((4, 16, 32), 0.7)
    assert np.abs(filt.shapiro(c, 3, cfg) - c).max() < 1e-15


def test_shapiro_zeroth_order_extrapolation_at_walls():
    u = np.arange(8, dtype=float).reshape(1, 1, 8)
    out = filt.shapiro_1d(u, 1, 2, False)
    # interior: a linear ramp is preserved; ends see a repeated boundary value
    assert np.array_equal(out[0, 0, 1:7], u[0, 0, 1:7])
    assert out[0, 0, 0] == 0.25 and out[0, 0, 7] == 6.75


def test_gate_rejects_filtering_of_an_exact_hdm_solution():
    u0, cfg, _ = W.burgers_sine(n=128, seed=4)
    q0 = u0.reshape(1, 1, 128)
    q1, _, ok = hdm.newton_be(q0, cfg, cfg.dt)
    assert ok
    out, passes, kept = filt.spatial_filter(q1, q0, cfg, cfg.dt)
    # filtering a converged HDM state raises its residual (R ~ 1e-14) far
    # above the noise, so only noise-level decisions can keep a cell and the
    # state moves by rounding-level amounts at most (a filter pass moves
    # this state by ~1e-5)
    assert np.abs(out - q1).max() < 1e-10
    assert kept < 16


def test_gate_removes_grid_scale_noise():
    u0, cfg, _ = W.burgers_sine(n=128, seed=4)
    q0 = u0.reshape(1, 1, 128)
    q1, _, _ = hdm.newton_be(q0, cfg, cfg.dt)
    noisy = q1 + 1e-3 * (-1.0) ** np.arange(128)
    r0 = filt.cell_residual(noisy, q0, cfg, cfg.dt).sum()
    out, passes, kept = filt.spatial_filter(noisy, q0, cfg, cfg.dt)
    r1 = filt.cell_residual(out, q0, cfg, cfg.dt).sum()
    # the order-2 filter cancels the grid-scale mode in one pass; what is
    # left is the filter's own O(dx^2) smoothing of the sine
    assert kept > 0 and r1 < 0.2 * r0
    assert np.abs(out - q1).max() < 0.5e-3
