"""GPU parity of the HDM stages against the oracle (Sec. 2.2-2.3, Sec. 3.1):
full SSP-RK2 steps (FP64 bit-exact: both sides evaluate the same
expressions in the same order with correctly rounded IEEE operations; FP32
within 1e-5 relative), masked partial steps on S-hat, and BDF1 Newton
(full periodic and per-segment partial) within 1e-12."""
import numpy as np
import pytest

import workloads as W
from oracle import hdm
from tests.gpu_util import Ctx, dev, host, dev_bits, rel_err, tdtype, torch

pytestmark = pytest.mark.gpu


def _cases():
    q, c, _ = W.euler_vortex(n=40, seed=3)
    yield "vortex40", q, c.with_(nx=40, ny=40)
    q, c, _ = W.euler_vortex(n=45, seed=4)      # tiles ragged in x and y, periodic
    yield "vortex45", q, c
    q, c, _ = W.euler_oblique_shock(n=72, seed=4, k=4)
    yield "shock72", q, c
    q, c, _ = W.euler_oblique_shock(n=45, seed=6, k=4)   # ragged, shock and outflow sides
    yield "shock45", q, c
    # FP32 takes a register-sweep kernel (warp strips of 64 columns, 60 of
    # them written, and rows split so that the strips fill one wave): several
    # strips wide and high, ragged in both directions, with strips that
    # touch no side
    q, c, _ = W.euler_oblique_shock(n=300, seed=7, k=4)
    yield "shock300x203", q.reshape(4, 300, 300)[:, :203, :].reshape(4, -1).copy(), \
        c.with_(ny=203)
    q, c, _ = W.euler_vortex(n=131, seed=8)
    yield "vortex131", q, c
    q, c = W.euler_riemann_x(n=200)
    yield "sod200", q, c
    u, c, _ = W.burgers_sine(n=300, seed=2)
    yield "burgers_rk2", u, c.with_(scheme=W.SCHEME_RK2)


@pytest.mark.parametrize("name,q0,cfg", list(_cases()), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
def test_full_rk2_step(name, q0, cfg, prec):
    cfg = cfg.with_(precision=prec, w=4, m=2, n_p=4)
    if prec == W.PREC_F32:      # same input values on both sides
        q0 = np.asarray(q0).astype(np.float32).astype(np.float64)
    shape = (cfg.nvar, cfg.ny, cfg.nx)
    k = 7
    want = hdm.rk2_step(np.asarray(q0).reshape(shape), cfg, k).reshape(-1)
    with Ctx(cfg, q0) as (hy, ctx):
        qp = dev(np.asarray(q0).reshape(-1), tdtype(cfg))
        out = torch.zeros_like(qp)
        hy.hyrom_stage_full_step(ctx, qp, out, k)
        got = host(out)
    if prec == W.PREC_F64:
        assert np.array_equal(got, want), f"max diff {np.abs(got - want).max()}"
    else:
        assert rel_err(got, want) < 1e-5


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
def test_partial_rk2_step_on_sampled_cells(prec):
    q0, cfg, _ = W.euler_oblique_shock(n=72, seed=5, k=4)
    cfg = cfg.with_(precision=prec)
    if prec == W.PREC_F32:
        q0 = q0.astype(np.float32).astype(np.float64)
    g = np.random.Generator(np.random.PCG64(1))
    mask = g.random(cfg.ncell) < 0.07
    mask[:5] = True                        # a boundary row
    mask[cfg.nx * 30: cfg.nx * 30 + 20] = True
    shape = (4, cfg.ny, cfg.nx)
    k = 3
    full = hdm.rk2_step(q0.reshape(shape), cfg, k).reshape(4, -1)
    with Ctx(cfg, q0) as (hy, ctx):
        qp = dev(q0.reshape(-1), tdtype(cfg))
        sentinel = torch.full_like(qp, -7.0)
        hy.hyrom_stage_partial_step(ctx, qp, sentinel, dev_bits(mask), k)
        got = host(sentinel).reshape(4, -1)
    assert np.all(got[:, ~mask] == -7.0)
    if prec == W.PREC_F64:
        assert np.array_equal(got[:, mask], full[:, mask])
    else:
        assert rel_err(got[:, mask], full[:, mask]) < 1e-5


def test_burgers_newton_full_step():
    u0, cfg, _ = W.burgers_sine(n=1024, seed=6)
    want, _, ok = hdm.newton_be(u0.reshape(1, 1, -1), cfg, 5 * cfg.dt)
    assert ok
    with Ctx(cfg, u0) as (hy, ctx):
        qp = dev(u0.reshape(-1))
        out = torch.zeros_like(qp)
        hy.hyrom_stage_full_step(ctx, qp, out, 5)
        got = host(out)
    assert rel_err(got, want.reshape(-1)) < 1e-12


@pytest.mark.parametrize("frac", [0.1, 0.5, 0.97])
def test_burgers_newton_partial_segments(frac):
    u0, cfg, _ = W.burgers_sine(n=512, seed=7)
    n = cfg.nx
    g = np.random.Generator(np.random.PCG64(int(frac * 100)))
    mask = np.zeros(n, bool)
    # random contiguous segments, one wrapping around the periodic end
    for _ in range(12):
        a = int(g.integers(0, n))
        mask[np.arange(a, a + int(g.integers(1, int(frac * n / 6) + 2))) % n] = True
    mask[np.arange(n - 5, n + 4) % n] = True
    q_init = u0.reshape(-1) + 1e-3 * g.standard_normal(n)   # frozen neighbours
    want, _, ok = hdm.newton_be(u0.reshape(1, 1, -1), cfg, cfg.dt, active=mask,
                                q_init=q_init.reshape(1, 1, -1))
    assert ok
    with Ctx(cfg, u0) as (hy, ctx):
        qp = dev(u0.reshape(-1))
        qio = dev(q_init)
        hy.hyrom_stage_partial_step(ctx, qp, qio, dev_bits(mask), 1)
        got = host(qio)
    assert np.array_equal(got[~mask], q_init[~mask])
    assert rel_err(got, want.reshape(-1)) < 1e-12


def test_all_cells_partial_step_is_the_full_step():
    u0, cfg, _ = W.burgers_sine(n=256, seed=8)
    with Ctx(cfg, u0) as (hy, ctx):
        qp = dev(u0.reshape(-1))
        full = torch.zeros_like(qp)
        hy.hyrom_stage_full_step(ctx, qp, full, 2)
        part = qp.clone()
        hy.hyrom_stage_partial_step(ctx, qp, part, dev_bits(np.ones(256, bool)), 2)
        assert torch.equal(full, part)
