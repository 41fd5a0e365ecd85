"""Statuses of the C ABI that report on a completed call, triggered from
host-made inputs: HYROM_ERANK (a window of rank below m, Sec. 2.3.1; a
rank-deficient sampled basis P^T Phi) and HYROM_ENONPHYS (an Euler state
with rho <= 0 or p <= 0)."""
import numpy as np
import pytest

import workloads as W
from oracle import rom
from tests.gpu_util import Ctx, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


def test_erank_when_the_window_has_rank_below_m():
    """A uniform Euler state is steady: every centred window is zero, so the
    first rebuild keeps m_eff = 0 < m modes and reports HYROM_ERANK as
    information (the binding returns it in info["status"]); the run goes on."""
    n = 16
    q0 = np.zeros((4, n * n))
    q0[0], q0[1], q0[2], q0[3] = 1.0, 0.3, -0.2, 2.5
    cfg = W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=n, ny=n, dx=0.1, dy=0.1,
                     dt=0.01, w=4, m=2, n_p=4, precision=W.PREC_F64)
    with Ctx(cfg, q0) as (hy, ctx):
        infos = [hy.hyrom_step(ctx) for _ in range(cfg.w + 2)]
        q = torch.zeros(cfg.ndof, dtype=torch.float64, device="cuda")
        hy.hyrom_get_state(ctx, q)
        assert "rank 0 < m = 2" in hy.hyrom_last_error(ctx)
    reb = [i for i in infos if i["rebuilt"]]
    assert reb and all(i["status"] == hy.HYROM_ERANK and i["m_eff"] == 0 for i in reb)
    assert all(i["status"] == hy.HYROM_OK for i in infos if not i["rebuilt"])
    assert np.array_equal(host(q).reshape(4, -1), q0)


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
def test_erank_and_nan_for_a_rank_deficient_sampled_basis(prec):
    """hyrom_stage_gappy with two equal sample rows and n_p = m: every y_j is
    NaN and the status is HYROM_ERANK; a well-posed call afterwards matches
    the oracle."""
    cfg = W.ArConfig(pde=W.PDE_BURGERS, scheme=W.SCHEME_RK2, nx=500, ny=1, dx=0.002, dy=1.0,
                     dt=1e-3, w=8, m=6, n_p=12, precision=prec)
    g = np.random.Generator(np.random.PCG64(3))
    Phi, _ = np.linalg.qr(g.standard_normal((cfg.ndof, cfg.m)))
    psi = g.standard_normal(cfg.ndof)
    v = psi + Phi @ g.standard_normal(cfg.m)
    if prec == W.PREC_F32:
        Phi, psi, v = (x.astype(np.float32).astype(np.float64) for x in (Phi, psi, v))
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    P = np.array([10, 10, 50, 90, 200, 333], np.int32)
    with Ctx(cfg) as (hy, ctx):
        phid, vd, psid = dev(Phi.T.copy(), dt), dev(v, dt), dev(psi, dt)
        y = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
        with pytest.raises(hy.HyromError) as e:
            hy.hyrom_stage_gappy(ctx, phid, cfg.m, dev(P, torch.int32), len(P), vd, psid, y)
        assert e.value.status == hy.HYROM_ERANK
        assert np.all(np.isnan(host(y)))
        P2 = P.copy()
        P2[1] = 11
        hy.hyrom_stage_gappy(ctx, phid, cfg.m, dev(P2, torch.int32), len(P2), vd, psid, y)
        want = rom.gappy_coords(Phi, P2, v, psi)
        assert rel_err(host(y), want) < (1e-12 if prec == W.PREC_F64 else 1e-5)


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
def test_enonphys_for_a_negative_density(prec):
    """A vortex state with one cell's density made negative: the first full
    step reports HYROM_ENONPHYS, naming the count of bad cells; a physical
    state steps with HYROM_OK."""
    q0, cfg, _ = W.euler_vortex(n=24, seed=2)
    cfg = cfg.with_(w=4, m=2, n_p=4, precision=prec)
    with Ctx(cfg, q0) as (hy, ctx):
        assert hy.hyrom_step(ctx)["status"] == hy.HYROM_OK
    bad = q0.copy()
    bad[0, 300] = -0.5
    with Ctx(cfg, bad) as (hy, ctx):
        with pytest.raises(hy.HyromError) as e:
            hy.hyrom_step(ctx)
        assert e.value.status == hy.HYROM_ENONPHYS
        assert "rho <= 0 or p <= 0" in str(e.value)
