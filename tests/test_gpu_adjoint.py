"""The adjoint of the SSP-RK2 Euler step (hyrom_stage_rk2_vjp) against the
oracle's tangent: the transposed Jacobian assembled column by column from
the oracle's JVP (oracle/tangent.py) applied to a cotangent, element by
element (FP64, within 1e-12 of its largest entry), for periodic, shock and
outflow sides, one and two dimensions, the full step and the partial step
on S-hat; and the dot-product identity <w, J v> = <J^T w, v> on a grid of
several thread blocks."""
import numpy as np
import pytest

import workloads as W
from oracle import hdm, tangent as T
from tests.gpu_util import Ctx, H, dev, dev_bits, host, rel_err, torch

pytestmark = pytest.mark.gpu


def _cases():
    n = 12
    _, cv, _ = W.euler_vortex(n=n, seed=2)
    yield "vortex12", W.euler_vortex_theta(n, W.VORTEX_THETA0).reshape(4, n, n), \
        cv.with_(precision=W.PREC_F64, w=4, m=2, n_p=4), 3
    q0, cs, _ = W.euler_oblique_shock(n=n, seed=3, k=2)
    cs = cs.with_(precision=W.PREC_F64)
    yield "shock12", hdm.rk2_step(q0.reshape(4, n, n), cs, 1), cs, 2
    q0, c1 = W.euler_riemann_x(n=30)
    c1 = c1.with_(w=4, m=2, n_p=4)
    yield "sod30", hdm.rk2_step(q0.reshape(4, 1, 30), c1, 1), c1, 2


def _jt(q, cfg, k, w):
    """J^T w of the oracle's step, J assembled from the tangent's columns."""
    N = q.size
    out = np.empty(N)
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        _, col = T.rk2_step_jvp(q, e.reshape(q.shape), cfg, k)
        out[i] = np.dot(col.reshape(-1), w)
    return out


def _gpu_vjp(cfg, q, lam, k, mask=None):
    hy = H()
    ctx = hy.hyrom_init(cfg, dev(q.reshape(-1)))
    try:
        N = q.size
        lam_in = torch.zeros(N, dtype=torch.float64, device="cuda")
        work = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
        hy.hyrom_stage_rk2_vjp(ctx, dev(q.reshape(-1)), dev(lam), lam_in,
                               None if mask is None else dev_bits(mask), k, work)
        return host(lam_in)
    finally:
        hy.hyrom_destroy(ctx)


@pytest.mark.parametrize("name,q,cfg,k", list(_cases()), ids=[c[0] for c in _cases()])
def test_step_adjoint_matches_the_oracle_transpose(name, q, cfg, k):
    g = np.random.Generator(np.random.PCG64(7))
    w = g.standard_normal(q.size)
    want = _jt(q, cfg, k, w)
    got = _gpu_vjp(cfg, q, w, k)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_partial_step_adjoint_passes_the_other_cells_through():
    name, q, cfg, k = list(_cases())[1]
    g = np.random.Generator(np.random.PCG64(8))
    mask = g.random(cfg.ncell) < 0.3
    w = g.standard_normal(q.size)
    mrows = np.tile(mask, cfg.nvar)
    want = _jt(q, cfg, k, np.where(mrows, w, 0.0)) + np.where(mrows, 0.0, w)
    got = _gpu_vjp(cfg, q, w, k, mask)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_dot_product_identity_on_a_larger_grid():
    n = 40
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    cfg = cfg.with_(precision=W.PREC_F64, w=4, m=2, n_p=4)
    q = W.euler_vortex_theta(n, W.VORTEX_THETA0).reshape(4, n, n)
    g = np.random.Generator(np.random.PCG64(9))
    v = g.standard_normal(q.shape)
    w = g.standard_normal(q.size)
    _, Jv = T.rk2_step_jvp(q, v, cfg, 2)
    JTw = _gpu_vjp(cfg, q, w, 2)
    lhs, rhs = float(np.dot(w, Jv.reshape(-1))), float(np.dot(JTw, v.reshape(-1)))
    assert abs(lhs - rhs) <= 1e-12 * np.abs(w).sum() * np.abs(Jv).max()


def test_autograd_function_chains_steps():
    """Two steps through HdmStep (a full step, then a partial step on S-hat)
    and a weighted sum: q0.grad equals J1^T J2^T w from the oracle."""
    from paper_2301_01718_gb300.autograd import HdmStep
    hy = H()
    name, q, cfg, k = list(_cases())[1]
    g = np.random.Generator(np.random.PCG64(10))
    mask = g.random(cfg.ncell) < 0.4
    w = g.standard_normal(q.size)
    ctx = hy.hyrom_init(cfg, dev(q.reshape(-1)))
    try:
        q0 = dev(q.reshape(-1)).requires_grad_(True)
        q1 = HdmStep.apply(ctx, q0, k, None)
        q2 = HdmStep.apply(ctx, q1, k + 1, dev_bits(mask))
        (q2 * dev(w)).sum().backward()
        got = host(q0.grad)
        q1_host = host(q1.detach()).reshape(q.shape)
    finally:
        hy.hyrom_destroy(ctx)
    assert np.array_equal(q1_host, hdm.rk2_step(q, cfg, k))
    mrows = np.tile(mask, cfg.nvar)
    lam1 = _jt(q1_host, cfg, k + 1, np.where(mrows, w, 0.0)) + np.where(mrows, 0.0, w)
    want = _jt(q, cfg, k, lam1)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_reduced_step_adjoint_matches_the_oracle():
    """hyrom_stage_reduced_vjp against the oracle's transposes of the
    reconstruction on S-breve and the gappy coordinates (oracle/adjoint.py),
    element by element: lam_v, lam_psi and lam_phi within 1e-12 of their
    largest entries (20^2 Euler, m = 5, 12 regression rows inside S-hat)."""
    from oracle import adjoint as A, rom
    hy = H()
    n, m = 20, 5
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    cfg = cfg.with_(precision=W.PREC_F64, w=6, m=m, n_p=12)
    N, nc = cfg.ndof, cfg.ncell
    g = np.random.Generator(np.random.PCG64(11))
    Phi, _ = np.linalg.qr(g.standard_normal((N, m)))
    s_hat = g.random(nc) < 0.25
    cells = np.flatnonzero(s_hat)
    rows = np.sort(g.choice(np.concatenate([c * nc + cells for c in range(4)]), 12,
                            replace=False)).astype(np.int32)
    v, psi, lam = (g.standard_normal(N) for _ in range(3))
    y = rom.gappy_coords(Phi, rows, v, psi)
    # the oracle
    sb = np.tile(~s_hat, 4)
    lrec = np.where(sb, lam, 0.0)
    gP, gv, gpsi = A.gappy_coords_vjp(Phi, rows, v, psi, Phi.T @ lrec)
    want_v = np.where(sb, 0.0, lam) + gv
    want_psi = lrec + gpsi
    want_phi = np.outer(lrec, y) + gP
    # the library
    ctx = hy.hyrom_init(cfg, dev(np.zeros(N)))
    try:
        lv = torch.zeros(N, dtype=torch.float64, device="cuda")
        lp = torch.zeros(N, dtype=torch.float64, device="cuda")
        lphi = torch.zeros(N * m, dtype=torch.float64, device="cuda")
        work = torch.zeros(hy.hyrom_reduced_vjp_work_doubles(m, len(rows)), dtype=torch.float64,
                           device="cuda")
        phi_d = dev(Phi.T.reshape(-1))                     # column-major N x m
        hy.hyrom_stage_reduced_vjp(ctx, phi_d, m, dev(rows, torch.int32), len(rows), dev(v),
                                   dev(psi), dev(y), dev_bits(s_hat), dev(lam), lv, lp, lphi,
                                   work)
        got_v, got_psi = host(lv), host(lp)
        got_phi = host(lphi).reshape(m, N).T
    finally:
        hy.hyrom_destroy(ctx)
    for got, want in ((got_v, want_v), (got_psi, want_psi), (got_phi, want_phi)):
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def _theta_dirs(n, th0):
    """dq0/dtheta_i of the vortex initial state by the complex step (the
    workload's analytic map, no method arithmetic)."""
    out = []
    for i in range(len(th0)):
        th = np.asarray(th0, complex)
        th[i] += 1e-30j
        out.append(W.euler_vortex_theta(n, th).imag.reshape(-1) / 1e-30)
    return out


def test_adjoint_sweep_matches_the_oracle_reverse_sweep():
    """hyrom_adjoint against oracle.adjoint.gradient on the 20^2 vortex
    (warm-up full steps, rebuilds and hybrid steps): the same J to 1e-12 and
    dJ/dq0 within 1e-12 of its largest entry; and the eight dJ/dtheta =
    (dq0/dtheta)^T dJ/dq0 within 1e-12 of the oracle's."""
    from oracle import adjoint as A
    n = 20
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    cfg = cfg.with_(precision=W.PREC_F64, w=6, m=3, n_p=6, top_frac=0.15, pod_tol=1e-10,
                    pod_abs=1e-13)
    th0 = np.array(W.VORTEX_THETA0)
    box, steps = (6, 14, 6, 14), cfg.w + 5
    q0 = W.euler_vortex_theta(n, th0)
    J_o, lam_o = A.gradient(q0, cfg, steps, box)
    with Ctx(cfg, q0) as (hy, ctx):
        g = torch.zeros(cfg.ndof, dtype=torch.float64, device="cuda")
        J = hy.hyrom_adjoint(ctx, steps, box, g)
        lam = host(g)
    lam_o = lam_o.reshape(-1)
    print(f"J {J:.15e} vs {J_o:.15e}; dJ/dq0 rel err {rel_err(lam, lam_o):.2e}")
    assert abs(J - J_o) <= 1e-12 * abs(J_o)
    assert rel_err(lam, lam_o) < 1e-12
    dirs = _theta_dirs(n, th0)
    gg = np.array([lam @ d for d in dirs])
    go = np.array([lam_o @ d for d in dirs])
    scale = np.maximum(np.abs(go), 1e-3 * abs(J_o))
    assert np.all(np.abs(gg - go) <= 1e-12 * scale), (gg, go)


def test_adjoint_gradient_against_central_differences():
    """dJ/dtheta from hyrom_adjoint against central differences of the GPU's
    own J (h = 1e-6 relative, FP64) over the whole method: for each parameter
    whose +-h runs keep the same sampled sets as the base run, within 1e-6 of
    max(|dJ/dtheta|, 1e-3 |J|)."""
    n = 20
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    cfg = cfg.with_(precision=W.PREC_F64, w=6, m=3, n_p=6, top_frac=0.15, pod_tol=1e-10,
                    pod_abs=1e-13)
    th0 = np.array(W.VORTEX_THETA0)
    box, steps = (6, 14, 6, 14), cfg.w + 5

    def run(theta):
        q0 = W.euler_vortex_theta(n, theta)
        with Ctx(cfg, q0) as (hy, ctx):
            g = torch.zeros(cfg.ndof, dtype=torch.float64, device="cuda")
            J = hy.hyrom_adjoint(ctx, steps, box, g)
            nw = (cfg.ncell + 31) // 32
            bm = torch.zeros(nw, dtype=torch.int32, device="cuda")
            hy.hyrom_sample(ctx, bitmap_dev=bm)
            return J, host(g), host(bm).copy()
    J0, lam0, m0 = run(th0)
    dirs = _theta_dirs(n, th0)
    checked = 0
    for i in range(8):
        h = 1e-6 * max(1.0, abs(th0[i]))
        tp, tm = th0.copy(), th0.copy()
        tp[i] += h
        tm[i] -= h
        Jp, _, mp = run(tp)
        Jm, _, mm = run(tm)
        if not (np.array_equal(mp, m0) and np.array_equal(mm, m0)):
            continue
        fd = (Jp - Jm) / (2 * h)
        ad = float(lam0 @ dirs[i])
        scale = max(abs(ad), 1e-3 * abs(J0))
        print(f"theta_{i}: adjoint {ad:.9e}, central difference {fd:.9e}")
        assert abs(ad - fd) <= 1e-6 * scale, (i, ad, fd)
        checked += 1
    assert checked >= 6


def test_pod_vjp_stage_matches_the_oracle():
    """hyrom_stage_pod_vjp (the thin-SVD adjoint the sweep applies at each
    rebuild) against oracle.adjoint.pod_vjp on a window of known, distinct
    spectrum: window and reference-state cotangents within 1e-12."""
    from oracle import adjoint as A
    n, w, m = 20, 6, 3
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    cfg = cfg.with_(nx=n, ny=n, precision=W.PREC_F64, w=w, m=m, n_p=2 * m, pod_tol=1e-10,
                    pod_abs=1e-13)
    N = cfg.ndof
    X, _ = W.random_spectrum_window(N, w, 11, decay=0.6, offset=1.0)
    g = np.random.Generator(np.random.PCG64(12))
    psi = 1.0 + 0.1 * g.standard_normal(N)
    lphi = g.standard_normal((N, m))
    raw = float(np.sqrt((X * X).sum()))
    want = A.pod_vjp(X - psi[:, None], lphi, m, cfg.pod_tol, cfg.pod_abs * raw)
    with Ctx(cfg) as (hy, ctx):
        lw = torch.zeros(N * w, dtype=torch.float64, device="cuda")
        lp = torch.zeros(N, dtype=torch.float64, device="cuda")
        hy.hyrom_stage_pod_vjp(ctx, dev(X.T.copy()), w, dev(psi), dev(lphi.T.copy()), m, lw, lp)
        got = host(lw).reshape(w, N).T
        gotp = host(lp)
    print(f"pod vjp rel err {rel_err(got, want):.2e}")
    assert rel_err(got, want) < 1e-12
    assert rel_err(gotp, -want.sum(axis=1)) < 1e-12


def test_filter_vjp_stage_matches_the_oracle():
    """hyrom_stage_filter_vjp against oracle.adjoint.spatial_filter_vjp with
    the oracle's logged keep masks: the same passes, cotangent within 1e-12."""
    from oracle import adjoint as A
    n = 24
    q0, cfg, _ = W.euler_vortex(n=n, seed=3)
    cfg = cfg.with_(nx=n, ny=n, precision=W.PREC_F64)
    qp = q0.reshape(4, n, n)
    g = np.random.Generator(np.random.PCG64(13))
    k = 3
    q = hdm.rk2_step(qp, cfg, k) + 0.01 * g.standard_normal(qp.shape)
    lam = g.standard_normal(qp.shape)
    _, keeps, orders = A._filter_logged(q, qp, cfg, k * cfg.dt)
    want = A.spatial_filter_vjp(lam, orders, keeps, cfg)
    with Ctx(cfg, q0) as (hy, ctx):
        io = dev(lam.reshape(-1))
        hy.hyrom_stage_filter_vjp(ctx, dev(q.reshape(-1)), dev(qp.reshape(-1)), k, io)
        got = host(io)
    print(f"filter vjp: {len(orders)} passes, rel err {rel_err(got, want.reshape(-1)):.2e}")
    assert rel_err(got, want.reshape(-1)) < 1e-12
