"""Pins of the oracle's Algorithm 1 driver: the full/hybrid/rebuild schedule
(an integer sequence fixed by the full-step and rebuild tests of the algorithm, written out
by hand below), the all-cells invariant (a hybrid step whose sampled set is
every cell, with the filter off, is the full HDM step), exact
reproduction of a state in the reduced affine subspace, and a steady state.
CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import arom, hdm, rom, select


def _tiny_burgers(**kw):
    u0, cfg, _ = W.burgers_sine(n=64, seed=5)
    base = dict(w=3, m=2, n_p=4, halo=1, top_frac=0.2)
    base.update(kw)
    cfg = cfg.with_(**base)
    return u0, cfg


@pytest.mark.parametrize("w,z,full,rebuild", [
    # w = 3, z = 4: full when k + 1 <= 3 or k mod 4 = 0; rebuild when
    # k >= 2 and (k + 1) mod 4 != 0
    (3, 4, [1, 2, 4, 8], [2, 4, 5, 6, 8, 9]),
    # w = 5, z = infinity: five warm-up full steps, rebuild from k = 4 on
    (5, 0, [1, 2, 3, 4], [4, 5, 6, 7, 8, 9]),
    # w = 2, z = 3
    (2, 3, [1, 3, 6, 9], [1, 3, 4, 6, 7, 9]),
])
def test_schedule_full_hybrid_rebuild(w, z, full, rebuild):
    u0, cfg = _tiny_burgers()
    cfg = cfg.with_(w=w, z=z, m=min(2, w))
    A = arom.Arom(u0, cfg)
    for _ in range(9):
        A.step()
    assert [h.k for h in A.history if h.was_full] == full
    assert [h.k for h in A.history if h.rebuilt] == rebuild


@pytest.mark.parametrize("scheme", [W.SCHEME_BE, W.SCHEME_RK2])
def test_all_cells_hybrid_step_is_the_full_hdm_step(scheme):
    u0, cfg = _tiny_burgers(scheme=scheme, top_frac=1.0, filt_orders=())
    if scheme == W.SCHEME_RK2:
        cfg = cfg.with_(dt=0.5 * cfg.dt)
    A = arom.Arom(u0, cfg)
    seen = 0
    for _ in range(8):
        prev = A.gamma.copy()
        info = A.step()
        if not info.was_full and info.n_s == cfg.ncell:
            assert np.array_equal(A.gamma, hdm.full_step(prev, cfg, info.k))
            seen += 1
    assert seen >= 3


def test_state_in_the_affine_subspace_is_reproduced():
    """Reconstruction on S-breve (Algorithm 1) from the gappy coordinates of a
    state psi + Phi a returns that state on every cell."""
    u0, cfg = _tiny_burgers()
    g = np.random.Generator(np.random.PCG64(1))
    N = cfg.ndof
    Phi, _ = np.linalg.qr(g.standard_normal((N, 3)))
    psi = g.standard_normal(N)
    a = g.standard_normal(3)
    truth = psi + Phi @ a
    P = rom.odeim(Phi, 6, 1e-12)
    y = rom.gappy_coords(Phi, P, truth, psi)
    assert np.abs((psi + Phi @ y) - truth).max() < 1e-13


def test_steady_state_is_reproduced_by_hybrid_steps():
    n = 12
    cfg = W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=n, ny=n, dx=0.1, dy=0.1, dt=0.01,
                     bc=(W.BC_PERIODIC,) * 4, w=3, m=2, n_p=4, top_frac=0.1)
    q0 = np.empty((4, n * n))
    q0[0], q0[1], q0[2], q0[3] = 1.2, 0.3, -0.2, 3.0
    A = arom.Arom(q0, cfg)
    for _ in range(7):
        info = A.step()
    assert not info.was_full and info.m_eff == 0
    assert all(h.m_eff == 0 for h in A.history if h.rebuilt)
    assert np.abs(A.gamma.reshape(4, -1) - q0).max() < 1e-13


def test_hybrid_trajectory_tracks_the_hdm():
    u0, cfg, _ = W.burgers_sine(n=128, seed=1)
    steps = 40
    A = arom.Arom(u0, cfg)
    A.run(steps)
    ref = arom.hdm_trajectory(u0, cfg, steps)
    assert arom.rel_l1(A.gamma, ref[-1]) < 1e-5
    sbar, sstar, pbar = arom.sampling_averages(A.history, cfg.ncell, cfg.ndof)
    assert sbar == sstar          # z = infinity: warm-up steps are excluded
    assert 0 < sstar < 100


def test_sample_rows_contain_the_points_and_reproduce_affine_states():
    """Sample-row form of the reduced solve: the regression rows are all dofs
    of S-hat, which contain the ODEIM rows P; a state psi + Phi a is
    reproduced exactly from them."""
    u0, cfg = _tiny_burgers(regress_rows=W.ROWS_SAMPLE)
    A = arom.Arom(u0, cfg)
    while True:
        info = A.step()
        if info.rebuilt and A.k >= cfg.w:
            break
    rows = A._sample_rows()
    assert set(int(p) for p in A.P) <= set(int(r) for r in rows)
    assert len(rows) == cfg.nvar * int(A.s_hat.sum())
    a = np.random.Generator(np.random.PCG64(2)).standard_normal(A.Phi.shape[1])
    truth = A._flat(A.psi) + A.Phi @ a
    assert np.abs(A._gappy(truth.reshape(A.shape)) - a).max() < 1e-12


def test_sample_row_hybrid_trajectory_tracks_the_hdm():
    u0, cfg, _ = W.burgers_sine(n=128, seed=1)
    cfg = cfg.with_(regress_rows=W.ROWS_SAMPLE)
    steps = 40
    A = arom.Arom(u0, cfg)
    A.run(steps)
    ref = arom.hdm_trajectory(u0, cfg, steps)
    assert arom.rel_l1(A.gamma, ref[-1]) < 1e-5


def test_rounding_order_differences_grow_in_hybrid_steps():
    """The premise of the GPU lockstep bound: two oracle runs that differ only
    in the rounding order of the POD (rows reversed) agree to rounding during
    the warm-up and early hybrid steps, then drift apart geometrically once
    the k = 3 basis tracks the shock (measured 9e-16 at step 10, 2.6e-11 at
    step 16); the full-step part of the run is unaffected."""
    from tests import oracle_spread
    q0, cfg, _ = W.euler_oblique_shock(n=64, seed=3, k=3)
    cfg = cfg.with_(precision=W.PREC_F64, pod_tol=1e-10, pod_abs=1e-13)
    A = arom.Arom(q0, cfg)
    ref = []
    for _ in range(16):
        A.step()
        ref.append(A.gamma.reshape(-1).copy())
    sp = oracle_spread.spread(q0, cfg, 16, ref)
    assert max(sp[: cfg.w - 1]) == 0.0          # warm-up full steps: no POD yet
    assert max(sp[: 10]) < 1e-14
    assert sp[15] > 1e-12 and sp[15] > 1e3 * sp[9]
