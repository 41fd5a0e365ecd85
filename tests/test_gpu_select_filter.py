"""GPU parity of selection (Eq. rre and the top-fraction rule; bit-exact
masks from identical errors), sampling sets (union / dilation / Neighbors,
bit-exact) and the residual-gated filter (Sec. 2.3.4)."""
import numpy as np
import pytest

import workloads as W
from oracle import select, filt, hdm
from tests.gpu_util import Ctx, dev, host, dev_bits, bits_of, rel_err, torch

pytestmark = pytest.mark.gpu


def _cfg(prec=W.PREC_F64, nx=72, ny=40, **kw):
    base = dict(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=nx, ny=ny, dx=0.1, dy=0.1, dt=0.01,
                w=6, m=4, n_p=8, precision=prec)
    base.update(kw)
    return W.ArConfig(**base)


def _eps_cases(nc):
    g = np.random.Generator(np.random.PCG64(5))
    yield "smooth", g.exponential(size=nc) ** 3
    e = np.round(g.random(nc) * 8) / 8.0                 # many exact ties
    yield "ties", e
    e = np.zeros(nc)
    e[g.integers(0, nc, 30)] = g.random(30)
    yield "sparse", e
    yield "zeros", np.zeros(nc)
    yield "tiny", 1e-300 * g.random(nc)


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
@pytest.mark.parametrize("mode,delta,frac", [(W.SEL_TOPFRAC, 0.9, 0.1), (W.SEL_TOPFRAC, 0.9, 0.337),
                                             (W.SEL_RRE, 0.8, 0.1), (W.SEL_RRE, 0.99, 0.1),
                                             (W.SEL_RRE, 1.0, 0.1)])
def test_selection_bit_exact(prec, mode, delta, frac):
    cfg = _cfg(prec, sel_mode=mode, delta=delta, top_frac=frac)
    nc = cfg.ncell
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    npdt = np.float32 if prec == W.PREC_F32 else np.float64
    with Ctx(cfg) as (hy, ctx):
        for name, eps in _eps_cases(nc):
            eps = eps.astype(npdt).astype(np.float64)
            G, n_g = select.select_cells(eps, mode, delta, frac)
            bm = torch.zeros((nc + 31) // 32, dtype=torch.int32, device="cuda")
            ng = hy.hyrom_stage_select(ctx, dev(eps, dt), bm)
            got = np.flatnonzero(bits_of(bm, nc))
            assert ng == n_g, name
            assert np.array_equal(got, G), name


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("scheme,halo", [(W.SCHEME_RK2, 0), (W.SCHEME_RK2, 2), (W.SCHEME_BE, 1)])
@pytest.mark.parametrize("oned", [False, True])
def test_masks_bit_exact(periodic, scheme, halo, oned):
    bc = (W.BC_PERIODIC,) * 4 if periodic else (W.BC_OUTFLOW,) * 4
    if oned:
        cfg = W.ArConfig(pde=W.PDE_BURGERS, scheme=scheme, nx=333, ny=1, dx=0.01, dy=1, dt=1e-3,
                         bc=(W.BC_PERIODIC,) * 4 if (periodic or scheme == W.SCHEME_BE) else bc,
                         halo=halo, w=4, m=2, n_p=4)
    else:
        if scheme == W.SCHEME_BE:
            pytest.skip("BDF1 is Burgers-only")
        cfg = _cfg(nx=72, ny=40, bc=bc, halo=halo, scheme=scheme)
    nc = cfg.ncell
    g = np.random.Generator(np.random.PCG64(7 + halo))
    Gm = g.random(nc) < 0.03
    Gm[0] = Gm[nc - 1] = True
    P = g.integers(0, cfg.ndof, 9).astype(np.int32)
    s_hat, s_tilde = select.build_masks(np.flatnonzero(Gm), P.tolist(), cfg)
    with Ctx(cfg) as (hy, ctx):
        nw = (nc + 31) // 32
        sh = torch.zeros(nw, dtype=torch.int32, device="cuda")
        st = torch.zeros(nw, dtype=torch.int32, device="cuda")
        n_s = hy.hyrom_stage_masks(ctx, dev_bits(Gm), dev(P, torch.int32), len(P), sh, st)
        assert n_s == int(s_hat.sum())
        assert np.array_equal(bits_of(sh, nc), s_hat.reshape(-1))
        assert np.array_equal(bits_of(st, nc), s_tilde.reshape(-1))


@pytest.mark.parametrize("case", ["burgers", "vortex", "shock", "sod_x", "shock_ragged"])
def test_filter_matches_oracle(case):
    if case == "sod_x":     # Euler in one dimension: 256-cell tiles, a ragged last tile
        q0, cfg = W.euler_riemann_x(n=300)
        cfg = cfg.with_(w=4, m=2, n_p=4)
        qp = q0.reshape(4, 1, 300)
        k = 1
        q1 = hdm.rk2_step(qp, cfg, k)
    elif case == "shock_ragged":   # tiles ragged in both directions, shock and outflow sides
        q0, cfg, _ = W.euler_oblique_shock(n=45, seed=4, k=4)
        cfg = cfg.with_(precision=W.PREC_F64)
        qp = q0.reshape(4, 45, 45)
        k = 2
        q1 = hdm.rk2_step(hdm.rk2_step(qp, cfg, 1), cfg, k)
        qp = hdm.rk2_step(qp, cfg, 1)
    elif case == "burgers":
        u0, cfg, _ = W.burgers_sine(n=400, seed=3)
        qp = u0.reshape(1, 1, -1)
        q1, _, _ = hdm.newton_be(qp, cfg, cfg.dt)
        k = 1
    elif case == "vortex":
        q0, cfg, _ = W.euler_vortex(n=48, seed=2)
        cfg = cfg.with_(precision=W.PREC_F64, w=4, m=2, n_p=4)
        qp = q0.reshape(4, 48, 48)
        k = 1
        q1 = hdm.rk2_step(qp, cfg, k)
    else:
        q0, cfg, _ = W.euler_oblique_shock(n=72, seed=3, k=4)
        cfg = cfg.with_(precision=W.PREC_F64)
        qp = q0.reshape(4, 72, 72)
        k = 1
        q1 = hdm.rk2_step(qp, cfg, k)
    g = np.random.Generator(np.random.PCG64(3))
    noisy = q1 + 1e-3 * np.abs(q1).max() * g.standard_normal(q1.shape) * (g.random(q1.shape[1:]) < 0.2)
    want, passes, _ = filt.spatial_filter(noisy, qp, cfg, k * cfg.dt)
    with Ctx(cfg, qp) as (hy, ctx):
        qd = dev(noisy)
        p = hy.hyrom_stage_filter(ctx, qd, dev(qp), k)
        got = host(qd).reshape(want.shape)
    assert p == passes
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
