"""Pins of the oracle's tangent-linear model (the differentiation form):
every JVP against central differences of the oracle function it
differentiates (h = 1e-6, at points away from the flux's and the method's
kinks), and the gradient of the time-integrated box pressure with respect to
the eight initial-state parameters against central differences of the whole
method, checked only where the perturbed runs took the same decisions."""
import numpy as np
import pytest

import workloads as W
from oracle import arom, filt, hdm, rom, tangent as T


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _states():
    n = 16
    _, cv, _ = W.euler_vortex(n=n, seed=2)
    yield "vortex", W.euler_vortex_theta(n, W.VORTEX_THETA0).reshape(4, n, n), \
        cv.with_(precision=W.PREC_F64)
    q0, cs, _ = W.euler_oblique_shock(n=n, seed=3, k=3)
    cs = cs.with_(precision=W.PREC_F64)
    yield "shock", hdm.rk2_step(q0.reshape(4, n, n), cs, 1), cs
    q0, c1 = W.euler_riemann_x(n=40)
    yield "sod_x", hdm.rk2_step(q0.reshape(4, 1, 40), c1, 1), c1


@pytest.mark.parametrize("name,q,cfg", list(_states()), ids=[s[0] for s in _states()])
def test_rk2_step_jvp_matches_central_differences(name, q, cfg):
    g = np.random.Generator(np.random.PCG64(1))
    dq = g.standard_normal(q.shape) * np.abs(q).mean(axis=(1, 2), keepdims=True) * 0.1
    qn, dn = T.rk2_step_jvp(q, dq, cfg, 2)
    assert np.array_equal(qn, hdm.rk2_step(q, cfg, 2))
    h = 1e-6
    fd = (hdm.rk2_step(q + h * dq, cfg, 2) - hdm.rk2_step(q - h * dq, cfg, 2)) / (2 * h)
    assert _rel(dn, fd) < 1e-6


def test_pod_jvp_matches_central_differences():
    g = np.random.Generator(np.random.PCG64(4))
    N, w, m = 60, 8, 5
    U, _ = np.linalg.qr(g.standard_normal((N, w)))
    V, _ = np.linalg.qr(g.standard_normal((w, w)))
    X = U @ np.diag(2.0 ** -np.arange(w)) @ V.T          # distinct singular values
    dX = g.standard_normal((N, w))
    Phi, dPhi, piv = T.pod_jvp(X, dX, m, 1e-10, 0.0)
    assert np.array_equal(Phi, rom.pod(X, m, 1e-10)[0]) and len(piv) == m
    h = 1e-6
    fd = (rom.pod(X + h * dX, m, 1e-10)[0] - rom.pod(X - h * dX, m, 1e-10)[0]) / (2 * h)
    assert _rel(dPhi, fd) < 1e-6
    # a rank-deficient window: the kept modes still differentiate
    X2 = X.copy()
    X2[:, -1] = X2[:, 0]
    Phi2, dPhi2, _ = T.pod_jvp(X2, dX, 3, 1e-10, 0.0)
    fd2 = (rom.pod(X2 + h * dX, 3, 1e-10)[0] - rom.pod(X2 - h * dX, 3, 1e-10)[0]) / (2 * h)
    assert _rel(dPhi2, fd2) < 1e-6


def test_gappy_coords_jvp_matches_central_differences():
    g = np.random.Generator(np.random.PCG64(5))
    N, m = 50, 4
    Phi, _ = np.linalg.qr(g.standard_normal((N, m)))
    dPhi = g.standard_normal((N, m))
    rows = np.array([1, 4, 7, 11, 20, 33, 41, 49])
    v, dv, psi, dpsi = (g.standard_normal(N) for _ in range(4))
    y, dy = T.gappy_coords_jvp(Phi, dPhi, rows, v, dv, psi, dpsi)
    h = 1e-6
    yp = rom.gappy_coords(Phi + h * dPhi, rows, v + h * dv, psi + h * dpsi)
    ym = rom.gappy_coords(Phi - h * dPhi, rows, v - h * dv, psi - h * dpsi)
    assert np.array_equal(y, rom.gappy_coords(Phi, rows, v, psi))
    assert _rel(dy, (yp - ym) / (2 * h)) < 1e-6


def test_filter_jvp_matches_central_differences_with_the_same_gates():
    n = 24
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    cfg = cfg.with_(precision=W.PREC_F64)
    qp = W.euler_vortex_theta(n, W.VORTEX_THETA0).reshape(4, n, n)
    q1 = hdm.rk2_step(qp, cfg, 1)
    g = np.random.Generator(np.random.PCG64(3))
    noisy = q1 + 1e-3 * g.standard_normal(q1.shape) * (g.random(q1.shape[1:]) < 0.3)
    dq = 1e-3 * g.standard_normal(q1.shape)
    out, (dout,), keeps = T.spatial_filter_jvp(noisy, [dq], qp, cfg, cfg.dt)
    want, passes, _ = filt.spatial_filter(noisy, qp, cfg, cfg.dt)
    assert np.array_equal(out, want) and len(keeps) == passes
    h = 1e-6
    _, _, kp = T.spatial_filter_jvp(noisy + h * dq, [], qp, cfg, cfg.dt)
    _, _, km = T.spatial_filter_jvp(noisy - h * dq, [], qp, cfg, cfg.dt)
    assert len(kp) == len(km) == len(keeps)
    assert all(np.array_equal(a, b) and np.array_equal(a, c) for a, b, c in zip(keeps, kp, km))
    fd = (filt.spatial_filter(noisy + h * dq, qp, cfg, cfg.dt)[0] -
          filt.spatial_filter(noisy - h * dq, qp, cfg, cfg.dt)[0]) / (2 * h)
    # 30 passes of rounding in a difference of 1e-9: about 1e-7 of noise
    assert _rel(dout, fd) < 2e-6


def _cfg(n=20):
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    return cfg.with_(precision=W.PREC_F64, w=6, m=3, n_p=6, top_frac=0.15, pod_tol=1e-10,
                     pod_abs=1e-13)


def test_tangent_model_runs_the_method_unchanged():
    cfg = _cfg()
    q0 = W.euler_vortex_theta(cfg.nx, W.VORTEX_THETA0)
    A, B = arom.Arom(q0, cfg), T.TangentArom(q0, cfg, [np.ones_like(q0)])
    for _ in range(cfg.w + 4):
        ia, ib = A.step(), B.step()
        assert ia == ib
        assert np.array_equal(A.gamma, B.gamma)


def test_vortex_parameters_reproduce_the_workload_and_differentiate():
    """R = 1 and the seeded pulse centre give euler_vortex bit for bit; the
    complex step through the initial state matches central differences."""
    rng = W.Rng(2)
    xp, yp = rng.uniform(2.0, 8.0), rng.uniform(2.0, 8.0)
    q0, _, _ = W.euler_vortex(n=24, seed=2)
    assert np.array_equal(q0, W.euler_vortex_theta(24, (5.0, 5.0, 5.0, 1.0, 0.2, xp, yp, 0.5)))
    th0 = np.array(W.VORTEX_THETA0)
    for i in range(8):
        th = th0.astype(complex)
        th[i] += 1e-30j
        d = W.euler_vortex_theta(24, th).imag / 1e-30
        h = 1e-6 * max(1.0, abs(th0[i]))
        tp, tm = th0.copy(), th0.copy()
        tp[i] += h
        tm[i] -= h
        fd = (W.euler_vortex_theta(24, tp) - W.euler_vortex_theta(24, tm)) / (2 * h)
        assert _rel(d, fd) < 1e-6


def _same_decisions(d1, d2):
    if len(d1) != len(d2):
        return False
    for a, b in zip(d1, d2):
        if a.keys() != b.keys():
            return False
        for key in a:
            x, y = a[key], b[key]
            if key == "keeps":
                if len(x) != len(y) or any(not np.array_equal(p, q) for p, q in zip(x, y)):
                    return False
            elif key == "G":
                if not np.array_equal(x, y):
                    return False
            elif x != y:
                return False
    return True


def test_output_gradient_matches_central_differences():
    """dJ/dtheta of J = sum_k dt sum_box p(gamma_k) dx dy over warm-up full
    steps, the first rebuilds and hybrid steps (20^2 vortex, w = 6, m = 3,
    n_p = 6, 15 % sample), all eight parameters, against central differences
    of the whole method with h = 1e-6 max(1, |theta_i|); every perturbed run
    took the same decisions (sets, G, points, filter keep masks, ranks,
    sign entries), so the difference quotient differentiates the same
    smooth map."""
    cfg = _cfg()
    n, steps, box = cfg.nx, cfg.w + 5, (6, 14, 6, 14)
    th0 = np.array(W.VORTEX_THETA0)

    def run(theta, tangents):
        dq0 = []
        if tangents:
            for i in range(8):
                th = theta.astype(complex)
                th[i] += 1e-30j
                dq0.append(W.euler_vortex_theta(n, th).imag / 1e-30)
        A = T.TangentArom(W.euler_vortex_theta(n, theta), cfg, dq0, box=box)
        for _ in range(steps):
            A.step()
        return A

    A = run(th0, True)
    assert any(not h.was_full for h in A.history) and A.history[-1].m_eff == 3
    for i in range(8):
        h = 1e-6 * max(1.0, abs(th0[i]))
        tp, tm = th0.copy(), th0.copy()
        tp[i] += h
        tm[i] -= h
        P, M = run(tp, False), run(tm, False)
        assert _same_decisions(A.decisions, P.decisions), W.VORTEX_THETA_NAMES[i]
        assert _same_decisions(A.decisions, M.decisions), W.VORTEX_THETA_NAMES[i]
        fd = (P.J - M.J) / (2 * h)
        scale = max(abs(A.dJ[i]), 1e-3 * abs(A.J))
        assert abs(fd - A.dJ[i]) <= 1e-6 * scale, (W.VORTEX_THETA_NAMES[i], A.dJ[i], fd)
