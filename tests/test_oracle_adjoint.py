"""Pins of the oracle's adjoint (reverse mode, oracle/adjoint.py): each
transpose against the tangent it transposes by the dot-product identity
<w, T d> = <T^T w, d> on random directions and cotangents (to rounding), and
the gradient of the time-integrated box pressure by one reverse sweep
against the tangent model's eight directional derivatives."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as A, filt, hdm, tangent as T


def _close(a, b, tol=1e-12):
    return abs(a - b) <= tol * max(abs(a), abs(b))


def _states():
    n = 12
    _, cv, _ = W.euler_vortex(n=n, seed=2)
    yield "vortex", W.euler_vortex_theta(n, W.VORTEX_THETA0).reshape(4, n, n), \
        cv.with_(precision=W.PREC_F64)
    q0, cs, _ = W.euler_oblique_shock(n=n, seed=3, k=2)
    cs = cs.with_(precision=W.PREC_F64)
    yield "shock", hdm.rk2_step(q0.reshape(4, n, n), cs, 1), cs
    q0, c1 = W.euler_riemann_x(n=30)
    yield "sod_x", hdm.rk2_step(q0.reshape(4, 1, 30), c1, 1), c1


@pytest.mark.parametrize("name,q,cfg", list(_states()), ids=[s[0] for s in _states()])
def test_rk2_step_transpose(name, q, cfg):
    g = np.random.Generator(np.random.PCG64(1))
    v, w = g.standard_normal(q.shape), g.standard_normal(q.shape)
    _, Jv = T.rk2_step_jvp(q, v, cfg, 2)
    assert _close(np.sum(w * Jv), np.sum(A.rk2_step_vjp(q, w, cfg, 2) * v))


@pytest.mark.parametrize("name,q,cfg", list(_states())[:2], ids=["periodic", "outflow"])
def test_filter_transpose(name, q, cfg):
    g = np.random.Generator(np.random.PCG64(2))
    noisy = q + 1e-3 * g.standard_normal(q.shape) * (g.random(q.shape[1:]) < 0.3)
    qp = q
    out, keeps, orders = A._filter_logged(noisy, qp, cfg, cfg.dt)
    assert np.array_equal(out, filt.spatial_filter(noisy, qp, cfg, cfg.dt)[0])
    assert sum(k.any() for k in keeps) > 1
    v, w = g.standard_normal(q.shape), g.standard_normal(q.shape)
    _, (Fv,), _ = T.spatial_filter_jvp(noisy, [v], qp, cfg, cfg.dt)
    assert _close(np.sum(w * Fv), np.sum(A.spatial_filter_vjp(w, orders, keeps, cfg) * v))


def test_gappy_coords_transpose():
    g = np.random.Generator(np.random.PCG64(3))
    N, m = 50, 4
    Phi, _ = np.linalg.qr(g.standard_normal((N, m)))
    dPhi = g.standard_normal((N, m))
    rows = np.array([1, 4, 7, 11, 20, 33, 41, 49])
    v, dv, psi, dpsi = (g.standard_normal(N) for _ in range(4))
    _, dy = T.gappy_coords_jvp(Phi, dPhi, rows, v, dv, psi, dpsi)
    ly = g.standard_normal(m)
    gP, gv, gpsi = A.gappy_coords_vjp(Phi, rows, v, psi, ly)
    assert _close(ly @ dy, np.sum(gP * dPhi) + gv @ dv + gpsi @ dpsi)


def test_pod_transpose():
    g = np.random.Generator(np.random.PCG64(4))
    N, w, m = 60, 8, 5
    U, _ = np.linalg.qr(g.standard_normal((N, w)))
    V, _ = np.linalg.qr(g.standard_normal((w, w)))
    X = U @ np.diag(2.0 ** -np.arange(w)) @ V.T
    dX = g.standard_normal((N, w))
    _, dP, _ = T.pod_jvp(X, dX, m, 1e-10, 0.0)
    lP = g.standard_normal((N, m))
    assert _close(np.sum(lP * dP), np.sum(A.pod_vjp(X, lP, m, 1e-10, 0.0) * dX))


@pytest.mark.parametrize("rows", [W.ROWS_ODEIM, W.ROWS_SAMPLE], ids=["odeim_rows", "sample_rows"])
def test_reverse_sweep_gradient_equals_the_tangent(rows):
    """dJ/dtheta = (dq0/dtheta)^T lambda_0 from one reverse sweep over warm-up
    full steps, rebuilds and hybrid steps equals the tangent model's eight
    directional derivatives (the gradient is unique), and the recorded
    forward run gives the same J; for both forms of the reduced solve."""
    _, cfg, _ = W.euler_vortex(n=20, seed=2)
    cfg = cfg.with_(precision=W.PREC_F64, w=6, m=3, n_p=6, top_frac=0.15, pod_tol=1e-10,
                    pod_abs=1e-13, regress_rows=rows)
    th0 = np.array(W.VORTEX_THETA0)
    box, steps = (6, 14, 6, 14), cfg.w + 5
    q0 = W.euler_vortex_theta(20, th0)
    dq0 = []
    for i in range(8):
        th = th0.astype(complex)
        th[i] += 1e-30j
        dq0.append(W.euler_vortex_theta(20, th).imag / 1e-30)
    TA = T.TangentArom(q0, cfg, dq0, box=box)
    for _ in range(steps):
        TA.step()
    J, lam0 = A.gradient(q0, cfg, steps, box)
    assert J == TA.J
    grad = np.array([np.sum(lam0.reshape(-1) * d.reshape(-1)) for d in dq0])
    scale = np.maximum(np.abs(TA.dJ), 1e-3 * abs(J))
    assert np.all(np.abs(grad - TA.dJ) <= 1e-12 * scale), (grad, TA.dJ)


def test_reverse_sweep_on_shock_and_outflow_sides():
    """The oblique-shock workload (exact-state inflow sides, outflow sides,
    zeroth-order filter ghosts): <lambda_0, d> from the reverse sweep equals
    the tangent's dJ along a smooth bump d, through warm-up, rebuilds and
    hybrid steps.  (Central differences are not a pin here: the piecewise
    constant states give exactly tied errors, whose order any perturbation
    changes.)"""
    n = 20
    q0, cfg, _ = W.euler_oblique_shock(n=n, seed=3, k=3)
    cfg = cfg.with_(precision=W.PREC_F64, w=6, m=3, n_p=6, top_frac=0.15, pod_tol=1e-10,
                    pod_abs=1e-13)
    q0 = q0.reshape(4, n, n)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    bump = np.exp(-((X - 0.6) ** 2 + (Y - 0.55) ** 2) / 0.02)
    d = np.stack([0.05 * bump, 0.02 * bump, -0.01 * bump, 0.1 * bump])
    steps, box = cfg.w + 5, (8, 16, 8, 16)
    TA = T.TangentArom(q0, cfg, [d], box=box)
    for _ in range(steps):
        TA.step()
    assert any(not h.was_full for h in TA.history)
    J, lam0 = A.gradient(q0, cfg, steps, box)
    assert J == TA.J
    assert _close(float(np.sum(lam0 * d)), float(TA.dJ[0]))
