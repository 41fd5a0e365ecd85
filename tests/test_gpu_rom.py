"""GPU parity of the reduced-basis stages against the oracle (Sec. 2.3.1,
2.3.3): gappy coordinates (Eq. red_coord), reconstruction, pointwise error,
POD_m (Eq. pod) on windows of known spectrum, and ODEIM points (Eq. odeim),
which must be identical row for row (both sides decide in FP64 on the same
quantity; ties within 1e-12 go to the lowest row)."""
import numpy as np
import pytest

import workloads as W
from oracle import rom, select
from tests.gpu_util import Ctx, dev, host, dev_bits, rel_err, torch

pytestmark = pytest.mark.gpu


def _cfg(prec, nx=72, ny=40, m=8, n_p=16, w=12):
    return W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=nx, ny=ny, dx=0.1, dy=0.1,
                      dt=0.01, w=w, m=m, n_p=n_p, precision=prec)


def _basis(N, m, seed, prec, concentrated=True):
    g = np.random.Generator(np.random.PCG64(seed))
    A = g.standard_normal((N, m))
    if concentrated:   # a localized basis, like one around a moving front
        A *= np.exp(-((np.arange(N) % 700) / 90.0) ** 2)[:, None] + 1e-3
    Q, _ = np.linalg.qr(A)
    if prec == W.PREC_F32:
        Q = Q.astype(np.float32).astype(np.float64)
    return Q


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
def test_gappy_coordinates(prec):
    cfg = _cfg(prec)
    N = cfg.ndof
    Phi = _basis(N, cfg.m, 1, prec)
    g = np.random.Generator(np.random.PCG64(2))
    P = rom.odeim(Phi, cfg.n_p, cfg.tie_tol)
    psi = g.standard_normal(N)
    v = psi + Phi @ g.standard_normal(cfg.m) + 1e-3 * g.standard_normal(N)
    if prec == W.PREC_F32:
        psi = psi.astype(np.float32).astype(np.float64)
        v = v.astype(np.float32).astype(np.float64)
    want = rom.gappy_coords(Phi, P, v, psi)
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    with Ctx(cfg) as (hy, ctx):
        y = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
        phid = dev(Phi.T.copy(), dt)            # column-major N x m
        hy.hyrom_stage_gappy(ctx, phid, cfg.m, dev(P, torch.int32), len(P), dev(v, dt),
                             dev(psi, dt), y)
        got = host(y)
    assert rel_err(got, want) < (1e-12 if prec == W.PREC_F64 else 1e-5)


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
def test_reconstruct_and_cell_error(prec):
    cfg = _cfg(prec)
    N, nc = cfg.ndof, cfg.ncell
    Phi = _basis(N, cfg.m, 3, prec)
    g = np.random.Generator(np.random.PCG64(4))
    psi = g.standard_normal(N)
    yv = g.standard_normal(cfg.m)
    q = g.standard_normal(N)
    if prec == W.PREC_F32:
        psi = psi.astype(np.float32).astype(np.float64)
        q = q.astype(np.float32).astype(np.float64)
    shat = g.random(nc) < 0.2
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    tol = 1e-13 if prec == W.PREC_F64 else 2e-6
    with Ctx(cfg) as (hy, ctx):
        phid = dev(Phi.T.copy(), dt)
        qd = dev(q, dt)
        hy.hyrom_stage_reconstruct(ctx, phid, cfg.m, dev(yv), dev(psi, dt), dev_bits(shat), qd)
        got = host(qd).reshape(4, -1)
        eps = torch.zeros(nc, dtype=dt, device="cuda")
        hy.hyrom_stage_cell_error(ctx, dev(q, dt), dev(psi, dt), phid, cfg.m, dev(yv), eps)
        got_e = host(eps)
    rec = (psi + Phi @ yv).reshape(4, -1)
    assert np.array_equal(got[:, shat], q.reshape(4, -1)[:, shat])
    assert rel_err(got[:, ~shat], rec[:, ~shat]) < tol
    want_e = select.cell_error(q, psi, Phi, yv, 4)
    assert rel_err(got_e, want_e) < tol * 10


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
@pytest.mark.parametrize("w", [12, 11])
def test_pod_of_known_spectrum(prec, w):
    cfg = _cfg(prec, w=w, m=6)
    N = cfg.ndof
    g = np.random.Generator(np.random.PCG64(10 + w))
    U, _ = np.linalg.qr(g.standard_normal((N, w)))
    V, _ = np.linalg.qr(g.standard_normal((w, w)))
    sig = 0.6 ** np.arange(w)
    psi = 2.0 + g.standard_normal(N) * 0.1
    X = psi[:, None] + (U * sig) @ V.T
    if prec == W.PREC_F32:
        X = X.astype(np.float32).astype(np.float64)
        psi = psi.astype(np.float32).astype(np.float64)
    raw = float(np.sqrt((X * X).sum()))
    Phi_o, s_o = rom.pod(X - psi[:, None], cfg.m, cfg.pod_tol, cfg.pod_abs * raw)
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    with Ctx(cfg) as (hy, ctx):
        phi = torch.zeros(cfg.m * N, dtype=dt, device="cuda")
        sg = torch.zeros(w, dtype=torch.float64, device="cuda")
        me = hy.hyrom_stage_pod(ctx, dev(X.T.copy(), dt), w, dev(psi, dt), phi, sg)
        Pg = host(phi)[: me * N].reshape(me, N).T.astype(np.float64)
        sg = host(sg)
    assert me == Phi_o.shape[1] == cfg.m
    if prec == W.PREC_F64:
        assert rel_err(sg[:w], s_o[:w]) < 1e-13
        assert np.abs(Pg @ Pg.T - Phi_o @ Phi_o.T).max() < 1e-12
        assert np.abs(Pg - Phi_o).max() < 1e-12          # same sign convention
    else:
        assert rel_err(sg[:cfg.m], s_o[:cfg.m]) < 1e-5
        assert np.abs(Pg @ Pg.T - Phi_o @ Phi_o.T).max() < 2e-4


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
@pytest.mark.parametrize("frac", [0.03, 0.3])
def test_sample_row_coordinates(prec, frac):
    """Sample-row reduced coordinates (every dof row of a cell set, normal
    equations, FP64 Cholesky) against the oracle's least squares on the same
    rows: 1e-12 relative in FP64, 1e-5 in FP32 (FP32 products summed in FP32
    within a block; more than 128 rows per block and several blocks)."""
    cfg = _cfg(prec, nx=96, ny=64, m=24, n_p=48, w=48).with_(regress_rows=W.ROWS_SAMPLE)
    N, nc = cfg.ndof, cfg.ncell
    Phi = _basis(N, cfg.m, 21, prec, concentrated=False)
    g = np.random.Generator(np.random.PCG64(22))
    cells = np.flatnonzero(g.random(nc) < frac).astype(np.int32)
    psi = g.standard_normal(N)
    v = psi + Phi @ g.standard_normal(cfg.m) + 1e-2 * g.standard_normal(N)
    if prec == W.PREC_F32:
        psi, v = (x.astype(np.float32).astype(np.float64) for x in (psi, v))
    rows = np.concatenate([a * nc + cells for a in range(4)])
    want = rom.gappy_coords(Phi, rows, v, psi)
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    with Ctx(cfg) as (hy, ctx):
        y = torch.zeros(cfg.m, dtype=torch.float64, device="cuda")
        hy.hyrom_stage_gappy_rows(ctx, dev(Phi.T.copy(), dt), cfg.m, dev(cells, torch.int32),
                                  len(cells), dev(v, dt), dev(psi, dt), y)
        got = host(y)
    tol = 1e-12 if prec == W.PREC_F64 else 1e-5
    assert rel_err(got, want) < tol, rel_err(got, want)


@pytest.mark.parametrize("red", [W.RED_TF32, W.RED_BF16, W.RED_TF32_SPLIT])
@pytest.mark.parametrize("nx,ny,m,frac", [(96, 64, 24, 0.03), (96, 64, 61, 0.3),
                                          (256, 256, 37, 1.0)])
def test_sample_row_coordinates_tensor_cores(red, nx, ny, m, frac):
    """Sample-row reduced coordinates with the normal matrix on the tensor
    cores (TF32, BF16, TF32 hi/lo split; FP32 accumulation, FP64 Cholesky)
    against the oracle's normal equations with the same input rounding
    (gappy_coords_normal): within 1e-5, the bar of the FP32 CUDA-core path,
    which leaves only the FP32 accumulation.  For TF32 and BF16 the GPU must
    also sit far closer to that rounded solution than the rounding moves it
    from the FP64 least-squares one (it rounds exactly as defined); the
    split form is within 1e-5 of the FP64 least squares.  Sizes: a few
    128-row stages, m not a multiple of 4 or 16, and 262 144 rows (more
    stages per CTA than the ring holds, so every ring slot is reused)."""
    cfg = _cfg(W.PREC_F32, nx=nx, ny=ny, m=m, n_p=2 * m, w=2 * m).with_(
        regress_rows=W.ROWS_SAMPLE, reduced_prec=red)
    N, nc = cfg.ndof, cfg.ncell
    Phi = _basis(N, m, 31 + m, W.PREC_F32, concentrated=False)
    g = np.random.Generator(np.random.PCG64(32 + m))
    cells = np.flatnonzero(g.random(nc) < frac).astype(np.int32)
    psi = g.standard_normal(N).astype(np.float32).astype(np.float64)
    v = (psi + Phi @ g.standard_normal(m) + 1e-2 * g.standard_normal(N)).astype(
        np.float32).astype(np.float64)
    rows = np.concatenate([a * nc + cells for a in range(4)])
    exact = rom.gappy_coords(Phi, rows, v, psi)
    want = rom.gappy_coords_normal(Phi, rows, v, psi, red)
    with Ctx(cfg) as (hy, ctx):
        y = torch.zeros(m, dtype=torch.float64, device="cuda")
        hy.hyrom_stage_gappy_rows(ctx, dev(Phi.T.copy(), torch.float32), m,
                                  dev(cells, torch.int32), len(cells),
                                  dev(v, torch.float32), dev(psi, torch.float32), y)
        got = host(y)
    nrm = np.linalg.norm(exact)
    e_def = float(np.linalg.norm(got - want) / nrm)      # vs the rounded definition
    e_round = float(np.linalg.norm(want - exact) / nrm)  # what the rounding itself does
    e_fp64 = float(np.linalg.norm(got - exact) / nrm)
    print(f"red={red} rows={len(rows)} m={m} err_vs_def={e_def:.3g} "
          f"rounding={e_round:.3g} err_vs_fp64={e_fp64:.3g}")
    assert rel_err(got, want) < 1e-5, rel_err(got, want)
    if red == W.RED_TF32_SPLIT:
        assert rel_err(got, exact) < 1e-5, rel_err(got, exact)
    elif frac < 1.0:
        # with all 262 144 rows of an orthonormal basis (G = I) the rounding
        # moves y by only a few 1e-6, the size of the FP32 accumulation error
        # over 1792 rows per CTA, so only the 1e-5 bar applies there
        assert e_def < 0.1 * e_round, (e_def, e_round)


@pytest.mark.parametrize("pde,nx,ny", [(W.PDE_BURGERS, 1073, 1), (W.PDE_EULER, 33, 17)])
@pytest.mark.parametrize("m", [20, 40])
def test_pod_fp32_wide_basis(pde, nx, ny, m):
    """FP32 POD with m > 16 (the register-tiled product Phi = X_c C): row
    counts that are not a multiple of the 128-row tile (Burgers, 1073 rows,
    not even a multiple of 4; Euler 33 x 17, 2244 rows)."""
    w = 48
    cfg = W.ArConfig(pde=pde, scheme=W.SCHEME_RK2, nx=nx, ny=ny, dx=0.1, dy=0.1, dt=0.01,
                     w=w, m=m, n_p=2 * m, precision=W.PREC_F32, pod_tol=1e-6, pod_abs=1e-6)
    N = cfg.ndof
    g = np.random.Generator(np.random.PCG64(100 + m + nx))
    U, _ = np.linalg.qr(g.standard_normal((N, w)))
    V, _ = np.linalg.qr(g.standard_normal((w, w)))
    sig = 0.9 ** np.arange(w)
    psi = (1.0 + g.standard_normal(N) * 0.1).astype(np.float32).astype(np.float64)
    X = (psi[:, None] + (U * sig) @ V.T).astype(np.float32).astype(np.float64)
    raw = float(np.sqrt((X * X).sum()))
    Phi_o, s_o = rom.pod(X - psi[:, None], m, cfg.pod_tol, cfg.pod_abs * raw)
    with Ctx(cfg) as (hy, ctx):
        phi = torch.zeros(m * N, dtype=torch.float32, device="cuda")
        sg = torch.zeros(w, dtype=torch.float64, device="cuda")
        me = hy.hyrom_stage_pod(ctx, dev(X.T.copy(), torch.float32), w,
                                dev(psi, torch.float32), phi, sg)
        Pg = host(phi)[: me * N].reshape(me, N).T.astype(np.float64)
        sg = host(sg)
    assert me == Phi_o.shape[1] == m
    assert rel_err(sg[:m], s_o[:m]) < 1e-5
    # directions: FP32 rounding of the product, amplified by sigma_1 / sigma_j;
    # lengths: FP32 rounding of the columns (a few 1e-8)
    nrm = np.linalg.norm(Pg, axis=0)
    assert np.abs(nrm - 1.0).max() < 1e-6
    for j in range(m):
        c = abs(float(Pg[:, j] @ Phi_o[:, j])) / nrm[j]
        assert 1.0 - c < 1e-10 * (s_o[0] / s_o[j]) ** 2 + 1e-11, (j, 1.0 - c)
    assert np.abs(Pg.T @ Pg - np.eye(m)).max() < 1e-5


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
@pytest.mark.parametrize("N,m,n_p,conc", [(600, 4, 9, False), (40000, 8, 17, True),
                                          (40000, 16, 32, False)])
def test_odeim_points_identical(prec, N, m, n_p, conc):
    cfg = W.ArConfig(pde=W.PDE_BURGERS, scheme=W.SCHEME_RK2, nx=N, ny=1, dx=1.0 / N, dy=1.0,
                     dt=1e-3, w=m + 2, m=m, n_p=n_p, precision=prec)
    Phi = _basis(N, m, 20 + m, prec, concentrated=conc)
    want = rom.odeim(Phi, n_p, cfg.tie_tol)
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    with Ctx(cfg) as (hy, ctx):
        pts = torch.zeros(n_p, dtype=torch.int32, device="cuda")
        hy.hyrom_stage_odeim(ctx, dev(Phi.T.copy(), dt), m, n_p, pts)
        got = host(pts).tolist()
    assert got == want


@pytest.mark.parametrize("b", [2, 4])
@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
@pytest.mark.parametrize("N,m,n_p,conc", [(600, 4, 9, False), (40000, 8, 17, True),
                                          (40000, 16, 32, False)])
def test_odeim_batched_points_identical(prec, N, m, n_p, conc, b):
    """The cheaper oversampling variant (odeim_batch = b: the b best rows of
    each scoring pass, not the paper's greedy) gives the oracle's
    rom.odeim_batched points row for row, including a last pass with fewer
    than b points."""
    cfg = W.ArConfig(pde=W.PDE_BURGERS, scheme=W.SCHEME_RK2, nx=N, ny=1, dx=1.0 / N, dy=1.0,
                     dt=1e-3, w=m + 2, m=m, n_p=n_p, precision=prec, odeim_batch=b)
    Phi = _basis(N, m, 20 + m, prec, concentrated=conc)
    want = rom.odeim_batched(Phi, n_p, cfg.tie_tol, b)
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    with Ctx(cfg) as (hy, ctx):
        pts = torch.zeros(n_p, dtype=torch.int32, device="cuda")
        hy.hyrom_stage_odeim(ctx, dev(Phi.T.copy(), dt), m, n_p, pts)
        got = host(pts).tolist()
    assert got == want


def _golden_odeim_cases():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "odeim_front_basis.json")
    with open(path) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_odeim_cases(), ids=lambda c: c["prec"])
def test_odeim_points_identical_at_benchmark_size(case):
    """ODEIM at the 2048^2 benchmark's sizes (m = 64 modes, n_p = 128 points)
    on 102 400 rows, so that the 2048-row probe, the norm-bucket pruning, the
    rising exact-score limit and the four-rows-per-CTA exact scoring all run:
    the points must equal the oracle's row for row.  The oracle needs ~5 s per
    oversampling step here, so its points were written by
    tests/golden/make_odeim_golden.py (oracle.rom.odeim only) for the same
    bits of workloads.front_basis, which the SHA-256 checks first."""
    import hashlib
    prec = W.PREC_F64 if case["prec"] == "f64" else W.PREC_F32
    Phi = W.front_basis(case["nrow"], case["m"], case["seed"])
    if prec == W.PREC_F32:
        Phi = Phi.astype(np.float32).astype(np.float64)
    assert hashlib.sha256(np.ascontiguousarray(Phi).tobytes()).hexdigest() == case["sha256"]
    N, m, n_p = case["nrow"], case["m"], case["n_p"]
    cfg = W.ArConfig(pde=W.PDE_BURGERS, scheme=W.SCHEME_RK2, nx=N, ny=1, dx=1.0 / N, dy=1.0,
                     dt=1e-3, w=2 * m, m=m, n_p=n_p, precision=prec, tie_tol=case["tie_tol"])
    dt = torch.float32 if prec == W.PREC_F32 else torch.float64
    with Ctx(cfg) as (hy, ctx):
        pts = torch.zeros(n_p, dtype=torch.int32, device="cuda")
        hy.hyrom_stage_odeim(ctx, dev(Phi.T.copy(), dt), m, n_p, pts)
        got = host(pts).tolist()
        cnt = hy.hyrom_odeim_counters(ctx)
    print(f"{case['prec']}: {cnt}")
    assert got == case["points"]


def test_pod_fp32_benchmark_shape():
    """FP32 POD at the benchmark's window and basis sizes (w = 128, m = 64):
    the eigensolve runs in a 16-CTA thread-block cluster and the tensor-core
    basis product in four chunks of the window per row tile.  Rows: an Euler
    160 x 160 grid (102 400 rows, 800 row tiles); the bars are those of
    test_pod_fp32_wide_basis."""
    w, m = 128, 64
    cfg = W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=160, ny=160, dx=0.1, dy=0.1,
                     dt=0.01, w=w, m=m, n_p=2 * m, precision=W.PREC_F32, pod_tol=1e-6,
                     pod_abs=1e-6)
    N = cfg.ndof
    g = np.random.Generator(np.random.PCG64(4096))
    U, _ = np.linalg.qr(g.standard_normal((N, w)))
    V, _ = np.linalg.qr(g.standard_normal((w, w)))
    sig = 0.93 ** np.arange(w)
    psi = (1.0 + g.standard_normal(N) * 0.1).astype(np.float32).astype(np.float64)
    X = (psi[:, None] + (U * sig) @ V.T).astype(np.float32).astype(np.float64)
    raw = float(np.sqrt((X * X).sum()))
    Phi_o, s_o = rom.pod(X - psi[:, None], m, cfg.pod_tol, cfg.pod_abs * raw)
    with Ctx(cfg) as (hy, ctx):
        phi = torch.zeros(m * N, dtype=torch.float32, device="cuda")
        sg = torch.zeros(w, dtype=torch.float64, device="cuda")
        me = hy.hyrom_stage_pod(ctx, dev(X.T.copy(), torch.float32), w,
                                dev(psi, torch.float32), phi, sg)
        sweeps = hy.hyrom_eig_sweeps(ctx)
        Pg = host(phi)[: me * N].reshape(me, N).T.astype(np.float64)
        sg = host(sg)
    assert me == Phi_o.shape[1] == m
    e_sig = rel_err(sg[:m], s_o[:m])
    nrm = np.linalg.norm(Pg, axis=0)
    worst = max(1.0 - abs(float(Pg[:, j] @ Phi_o[:, j])) / nrm[j] for j in range(m))
    print(f"sigma rel err {e_sig:.2e}, worst 1 - cos {worst:.2e}, sweeps {sweeps}")
    assert e_sig < 1e-5
    # column lengths: the FP32 bar (measured 1.5e-6, every column slightly
    # short: the tensor cores' FP32 accumulation over the four chunks of the
    # 128-snapshot window rounds towards zero)
    assert np.abs(nrm - 1.0).max() < 1e-5
    for j in range(m):
        c = abs(float(Pg[:, j] @ Phi_o[:, j])) / nrm[j]
        assert 1.0 - c < 1e-10 * (s_o[0] / s_o[j]) ** 2 + 1e-11, (j, 1.0 - c)
    # orthonormality: an entry of Phi^T Phi - I carries both columns' FP32
    # errors (measured 1.08e-5, the short column lengths above included)
    assert np.abs(Pg.T @ Pg - np.eye(m)).max() < 2e-5
