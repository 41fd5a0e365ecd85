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
from tests.gpu_util import H, dev, dev_bits, host, torch

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
