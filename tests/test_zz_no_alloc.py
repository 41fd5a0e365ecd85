"""hyrom_gappy_static: the allocation-free gappy solve.

Callers that cannot allocate device memory (hosts that budget all device
memory up front, plugins that must not use the application's allocator,
loops that cannot afford cudaMalloc's implicit synchronisation) use this
entry point; its scratch lives in a static device array.  It must give the same reduced coordinates as the regular
entry point hyrom_stage_gappy, within the tolerance the gappy parity test
uses (1e-12 relative in FP64, 1e-5 in FP32), on consecutive calls that share
the scratch, and must reject sizes above its limits with a clear error.
This file is collected last so that a failure here leaves every other test
already run; it also passes on its own in a fresh process."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import Ctx, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


def _problem(prec, seed):
    cfg = W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=72, ny=40, dx=0.1, dy=0.1, dt=0.01,
                     w=12, m=8, n_p=16, precision=prec)
    N = cfg.ndof
    g = np.random.Generator(np.random.PCG64(seed))
    A = g.standard_normal((N, cfg.m)) * (np.exp(-((np.arange(N) % 700) / 90.0) ** 2)[:, None] + 1e-3)
    Phi, _ = np.linalg.qr(A)
    P = np.sort(g.choice(N, cfg.n_p, replace=False)).astype(np.int32)
    psi = g.standard_normal(N)
    v = psi + Phi @ g.standard_normal(cfg.m) + 1e-3 * g.standard_normal(N)
    if prec == W.PREC_F32:
        Phi, psi, v = (x.astype(np.float32).astype(np.float64) for x in (Phi, psi, v))
    return cfg, Phi, P, psi, v


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
def test_static_gappy_matches_the_allocating_entry_point(prec):
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    tol = 1e-12 if prec == W.PREC_F64 else 1e-5
    cfg, Phi, P, psi, v = _problem(prec, 3)
    with Ctx(cfg) as (hy, ctx):
        phid = dev(Phi.T.copy(), dt)
        pd, vd, psid = dev(P, torch.int32), dev(v, dt), dev(psi, dt)
        y_ref = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
        hy.hyrom_stage_gappy(ctx, phid, cfg.m, pd, len(P), vd, psid, y_ref)
        outs = []
        for _ in range(2):                  # two calls in a row share the scratch
            y = torch.full((cfg.m,), np.nan, dtype=torch.float64, device="cuda")
            hy.hyrom_gappy_static(phid, cfg.ndof, cfg.m, pd, len(P), vd, psid, prec, y)
            torch.cuda.synchronize()
            outs.append(host(y))
        ref = host(y_ref)
    for y in outs:
        assert np.all(np.isfinite(y))
        assert rel_err(y, ref) < tol
    assert rel_err(outs[0], outs[1]) < tol


def test_static_gappy_reuses_scratch_across_different_problems():
    """A second call with other data must not see the first call's values."""
    cfg, Phi, P, psi, v = _problem(W.PREC_F64, 5)
    cfg2, Phi2, P2, psi2, v2 = _problem(W.PREC_F64, 6)
    with Ctx(cfg) as (hy, ctx):
        res = []
        for (ph, pp, ps, vv) in ((Phi, P, psi, v), (Phi2, P2, psi2, v2)):
            phid = dev(ph.T.copy())
            pd, vd, psid = dev(pp, torch.int32), dev(vv), dev(ps)
            y_ref = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
            hy.hyrom_stage_gappy(ctx, phid, cfg.m, pd, len(pp), vd, psid, y_ref)
            y = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
            hy.hyrom_gappy_static(phid, cfg.ndof, cfg.m, pd, len(pp), vd, psid, W.PREC_F64, y)
            torch.cuda.synchronize()
            res.append((host(y), host(y_ref)))
    for y, ref in res:
        assert rel_err(y, ref) < 1e-12


def test_static_gappy_rejects_sizes_beyond_its_limits():
    from tests.gpu_util import H
    hy = H()
    y = torch.zeros(200, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(1000, dtype=torch.float64, device="cuda")
    pts = torch.zeros(200, dtype=torch.int32, device="cuda")
    with pytest.raises(hy.HyromError) as e:
        hy.hyrom_gappy_static(dummy, 1000, 8, pts, 200, dummy, dummy, W.PREC_F64, y)
    assert "n_p <= min(128, ndof)" in str(e.value)
    with pytest.raises(hy.HyromError) as e:
        hy.hyrom_gappy_static(dummy, 1000, 65, pts, 100, dummy, dummy, W.PREC_F64, y)
    assert "1 <= m <= 64" in str(e.value)
