"""hyrom_gappy_static: the allocation-free gappy solve.

Callers that cannot allocate device memory (hosts that budget all device
memory up front and hand the library only pointers into their own pools,
plugins that must not use the allocator of the program that loads them,
loops that cannot afford cudaMalloc's implicit synchronisation) use this
entry point; its scratch lives in a static device array.  Its reduced
coordinates are held against the oracle's least squares (oracle.rom.
gappy_coords) at the gappy parity test's tolerances, 1e-12 relative in FP64
and 1e-5 in FP32, on consecutive calls that share the scratch, up to its
size limits (m = 64, n_p = 128), and against the allocating entry point
hyrom_stage_gappy; further calls must not change the device memory in use;
a rank-deficient sampled basis gives NaN; sizes above the limits are
rejected with a clear error.  This file is collected last so that a failure
here leaves every other test already run; it also passes on its own in a
fresh process."""
import numpy as np
import pytest

import workloads as W
from oracle import rom
from tests.gpu_util import Ctx, dev, host, rel_err, torch

pytestmark = pytest.mark.gpu


def _problem(prec, seed, m=8, n_p=16, nx=72, ny=40):
    cfg = W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=nx, ny=ny, dx=0.1, dy=0.1,
                     dt=0.01, w=2 * m, m=m, n_p=n_p, precision=prec)
    N = cfg.ndof
    g = np.random.Generator(np.random.PCG64(seed))
    A = g.standard_normal((N, m)) * (np.exp(-((np.arange(N) % 700) / 90.0) ** 2)[:, None] + 1e-3)
    Phi, _ = np.linalg.qr(A)
    P = np.sort(g.choice(N, n_p, replace=False)).astype(np.int32)
    psi = g.standard_normal(N)
    v = psi + Phi @ g.standard_normal(m) + 1e-3 * g.standard_normal(N)
    if prec == W.PREC_F32:
        Phi, psi, v = (x.astype(np.float32).astype(np.float64) for x in (Phi, psi, v))
    return cfg, Phi, P, psi, v


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
@pytest.mark.parametrize("m,n_p", [(8, 16), (64, 128)])
def test_static_gappy_matches_the_oracle(prec, m, n_p):
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    tol = 1e-12 if prec == W.PREC_F64 else 1e-5
    cfg, Phi, P, psi, v = _problem(prec, 3 + m, m=m, n_p=n_p)
    want = rom.gappy_coords(Phi, P, v, psi)
    with Ctx(cfg) as (hy, ctx):
        phid = dev(Phi.T.copy(), dt)
        pd, vd, psid = dev(P, torch.int32), dev(v, dt), dev(psi, dt)
        y_ref = torch.zeros(m, dtype=torch.float64, device="cuda")
        hy.hyrom_stage_gappy(ctx, phid, m, pd, len(P), vd, psid, y_ref)
        outs = []
        for _ in range(2):                  # two calls in a row share the scratch
            y = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
            hy.hyrom_gappy_static(phid, cfg.ndof, m, pd, len(P), vd, psid, prec, y)
            torch.cuda.synchronize()
            outs.append(host(y))
        ref = host(y_ref)
    for y in outs:
        assert np.all(np.isfinite(y))
        assert rel_err(y, want) < tol, rel_err(y, want)
        assert rel_err(y, ref) < tol
    assert rel_err(outs[0], outs[1]) < tol


def test_static_gappy_allocates_nothing():
    """After a first call (which looks up the scratch's address), further
    calls at the size limits leave torch's allocator statistics and the
    device's free memory unchanged."""
    from tests.gpu_util import H
    hy = H()
    cfg, Phi, P, psi, v = _problem(W.PREC_F64, 11, m=64, n_p=128)
    phid = dev(Phi.T.copy())
    pd, vd, psid = dev(P, torch.int32), dev(v), dev(psi)
    y = torch.zeros(64, dtype=torch.float64, device="cuda")
    hy.hyrom_gappy_static(phid, cfg.ndof, 64, pd, 128, vd, psid, W.PREC_F64, y)
    torch.cuda.synchronize()
    stats0 = torch.cuda.memory_stats()
    free0, _ = torch.cuda.mem_get_info()   # cudaMemGetInfo
    for _ in range(5):
        hy.hyrom_gappy_static(phid, cfg.ndof, 64, pd, 128, vd, psid, W.PREC_F64, y)
    torch.cuda.synchronize()
    stats1 = torch.cuda.memory_stats()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for key in ("allocated_bytes.all.current", "reserved_bytes.all.current",
                "num_alloc_retries", "allocation.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    assert rel_err(host(y), rom.gappy_coords(Phi, P, v, psi)) < 1e-12


def test_static_gappy_reuses_scratch_across_different_problems():
    """A second call with other data must not see the first call's values."""
    cfg, Phi, P, psi, v = _problem(W.PREC_F64, 5)
    cfg2, Phi2, P2, psi2, v2 = _problem(W.PREC_F64, 6)
    with Ctx(cfg) as (hy, ctx):
        res = []
        for (ph, pp, ps, vv) in ((Phi, P, psi, v), (Phi2, P2, psi2, v2)):
            phid = dev(ph.T.copy())
            pd, vd, psid = dev(pp, torch.int32), dev(vv), dev(ps)
            y = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
            hy.hyrom_gappy_static(phid, cfg.ndof, cfg.m, pd, len(pp), vd, psid, W.PREC_F64, y)
            torch.cuda.synchronize()
            res.append((host(y), rom.gappy_coords(ph, pp, vv, ps)))
    for y, want in res:
        assert rel_err(y, want) < 1e-12


def test_static_gappy_rank_deficient_gives_nan():
    """Two equal sample rows with n_p = m leave P^T Phi rank-deficient: the
    static entry point writes NaN into every y_j (its status, returned before
    the work runs, is OK), and a following well-posed call is finite again
    (the rank counter is cleared by each call)."""
    from tests.gpu_util import H
    hy = H()
    cfg, Phi, P, psi, v = _problem(W.PREC_F64, 7)
    Pdup = P[: cfg.m].copy()
    Pdup[1] = Pdup[0]
    phid = dev(Phi.T.copy())
    vd, psid = dev(v), dev(psi)
    y = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
    hy.hyrom_gappy_static(phid, cfg.ndof, cfg.m, dev(Pdup, torch.int32), cfg.m, vd, psid,
                          W.PREC_F64, y)
    torch.cuda.synchronize()
    assert np.all(np.isnan(host(y)))
    hy.hyrom_gappy_static(phid, cfg.ndof, cfg.m, dev(P, torch.int32), len(P), vd, psid,
                          W.PREC_F64, y)
    torch.cuda.synchronize()
    assert rel_err(host(y), rom.gappy_coords(Phi, P, v, psi)) < 1e-12


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
