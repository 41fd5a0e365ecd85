"""End-to-end parity of Algorithm 1 on the GPU (FP64) against the oracle,
step by step: states, the full/hybrid/rebuild schedule and the sampled sets.
FP32 runs are compared to the FP64 oracle with a looser, measured bound."""
import numpy as np
import pytest

import workloads as W
from oracle import arom, hdm
from tests.gpu_util import Ctx, dev, host, bits_of, rel_err, tdtype, torch
from tests import oracle_spread

pytestmark = pytest.mark.gpu


def _cases():
    u, c, _ = W.burgers_sine(n=256, seed=1)
    yield "burgers", u, c.with_(w=8, m=4, n_p=8), 30
    q, c, _ = W.euler_vortex(n=48, seed=2)
    yield "vortex", q, c.with_(w=6, m=4, n_p=8, precision=W.PREC_F64, pod_tol=1e-10,
                               pod_abs=1e-13, top_frac=0.05), 16
    q, c, _ = W.euler_oblique_shock(n=64, seed=3, k=3)
    yield "shock", q, c.with_(precision=W.PREC_F64, pod_tol=1e-10, pod_abs=1e-13), 16
    # the benchmark's problem at 128^2 with k = 16, w = 32, n_p = 32: six
    # rebuilds after the warm-up
    q, c, _ = W.euler_oblique_shock(n=128, seed=3, k=16)
    yield "shock128_k16", q, c.with_(precision=W.PREC_F64, pod_tol=1e-10, pod_abs=1e-13), 38
    # the cheaper oversampling variant (three points per scoring pass; the
    # oracle takes the same variant)
    q, c, _ = W.euler_oblique_shock(n=64, seed=3, k=4)
    yield "shock_odeim_batch3", q, c.with_(precision=W.PREC_F64, pod_tol=1e-10, pod_abs=1e-13,
                                           odeim_batch=3), 16
    # the sample-row form of the reduced solve (all dof rows of S-hat)
    u, c, _ = W.burgers_sine(n=256, seed=1)
    yield "burgers_sample_rows", u, c.with_(w=8, m=4, n_p=8, regress_rows=W.ROWS_SAMPLE), 30
    q, c, _ = W.euler_vortex(n=48, seed=2)
    yield "vortex_sample_rows", q, c.with_(w=6, m=4, n_p=8, precision=W.PREC_F64,
                                           pod_tol=1e-10, pod_abs=1e-13, top_frac=0.05,
                                           regress_rows=W.ROWS_SAMPLE), 16


def _lockstep(q0, cfg, steps):
    A = arom.Arom(q0, cfg)
    out = []
    with Ctx(cfg, q0) as (hy, ctx):
        nw = (cfg.ncell + 31) // 32
        bm = torch.zeros(nw, dtype=torch.int32, device="cuda")
        q = torch.zeros(cfg.ndof, dtype=tdtype(cfg), device="cuda")
        for _ in range(steps):
            info = hy.hyrom_step(ctx)
            oi = A.step()
            hy.hyrom_get_state(ctx, q)
            rec = dict(k=oi.k, info=info, oinfo=oi, state=host(q).astype(np.float64),
                       want=A.gamma.reshape(-1).copy())
            if oi.rebuilt:
                hy.hyrom_sample(ctx, bitmap_dev=bm)
                rec["mask"] = bits_of(bm, cfg.ncell)
                rec["want_mask"] = A.s_hat.reshape(-1).copy()
            out.append(rec)
    return out


@pytest.mark.parametrize("name,q0,cfg,steps", list(_cases()), ids=[c[0] for c in _cases()])
def test_fp64_lockstep_with_oracle(name, q0, cfg, steps):
    """Every step: the same schedule and rank, identical sampled sets at every
    rebuild, full steps bit for bit, and states within 1e-12 relative of the
    oracle, or within 100x the drift between two oracle runs that differ
    only in the rounding order of their POD once the method has amplified
    that drift beyond 1e-14 (tests/oracle_spread.py; measured worst GPU
    drift: 2.5e-10 after 11 hybrid steps of the 64^2 shock with k = 3,
    where two oracle runs drift 2.6e-11 apart)."""
    recs = _lockstep(q0, cfg, steps)
    spread = oracle_spread.spread(q0, cfg, steps, [r["want"] for r in recs])
    worst_full = worst_hyb = 0.0
    per_step = []
    for r, sp in zip(recs, spread):
        assert bool(r["info"]["was_full"]) == r["oinfo"].was_full
        assert bool(r["info"]["rebuilt"]) == r["oinfo"].rebuilt
        assert r["info"]["m_eff"] == r["oinfo"].m_eff
        e = rel_err(r["state"], r["want"])
        per_step.append((e, sp))
        if r["oinfo"].was_full:
            worst_full = max(worst_full, e)
            assert e == 0.0, f"full step {r['k']}: rel err {e}"
        else:
            worst_hyb = max(worst_hyb, e)
        assert e <= oracle_spread.bar(sp), f"step {r['k']}: rel err {e}, oracle spread {sp}"
        if "mask" in r:
            assert np.array_equal(r["mask"], r["want_mask"]), f"step {r['k']}: masks differ"
    print(f"{name}: worst rel err full steps {worst_full:.3e}, hybrid steps {worst_hyb:.3e}; "
          f"per step (gpu, oracle spread) {['%.1e/%.1e' % p for p in per_step]}")


def test_fp32_vortex_tracks_fp64_oracle():
    """FP32 states against the FP64 oracle.  Single stages agree to 1e-5
    (stage tests); over many hybrid steps the FP32 run takes its own filter
    and sampling decisions near ties and the difference grows (measured:
    1e-7 during the full warm-up steps, ~1e-3 max-relative after 14 steps;
    the relative L1 deviation reached 0.21 of the method error with the
    FP32 flux kernels that round like the FP64 ones, 0.51 with the
    contracted FP32 sweep kernel: the hybrid steps amplify whichever FP32
    rounding they start from).  Criterion: full steps stay at FP32 rounding,
    and the FP32 deviation in the paper's relative L1 error (Sec. 3.1) stays
    below the method's own error against the full-HDM trajectory."""
    q0, cfg, _ = W.euler_vortex(n=48, seed=2)
    cfg = cfg.with_(w=6, m=4, n_p=8, top_frac=0.05)
    steps = 14
    recs = _lockstep(q0, cfg, steps)
    ref = arom.hdm_trajectory(q0, cfg.with_(precision=W.PREC_F64), steps)
    errs = [rel_err(r["state"], r["want"]) for r in recs]
    print("fp32 vs fp64 oracle (max rel) per step:", ["%.1e" % e for e in errs])
    assert max(errs[:5]) < 1e-6
    for r, q in zip(recs, ref):
        e32 = arom.rel_l1(r["state"], r["want"])
        ehyb = arom.rel_l1(r["want"], q.reshape(-1))
        if not r["oinfo"].was_full:
            print(f"k={r['k']}: fp32 dev {e32:.2e}  method error {ehyb:.2e}")
            assert e32 < ehyb


def test_all_cells_hybrid_equals_full_step_on_gpu():
    q0, cfg, _ = W.euler_vortex(n=40, seed=4)
    cfg = cfg.with_(nx=40, ny=40, w=4, m=2, n_p=4, top_frac=1.0, filt_orders=(),
                    precision=W.PREC_F64)
    with Ctx(cfg, q0) as (hy, ctx):
        q = torch.zeros(cfg.ndof, dtype=torch.float64, device="cuda")
        prev = torch.zeros_like(q)
        full = torch.zeros_like(q)
        seen = 0
        for _ in range(9):
            hy.hyrom_get_state(ctx, prev)
            info = hy.hyrom_step(ctx)
            if not info["was_full"] and info["n_s"] == cfg.ncell:
                hy.hyrom_get_state(ctx, q)
                hy.hyrom_stage_full_step(ctx, prev, full, info["k"])
                assert torch.equal(q, full)
                seen += 1
        assert seen >= 3


@pytest.mark.parametrize("prec", [W.PREC_F64, W.PREC_F32])
def test_graph_replayed_loops_match_direct_launches(prec):
    """On a created stream the rebuild's DEIM and oversampling loops are
    captured as CUDA graphs at the first rebuild and replayed at every later
    one; on the legacy default stream they are launched directly.  The two
    runs launch the same kernels in the same order, so states and sample
    masks are identical at every step (several rebuilds, both precisions)."""
    from paper_2301_01718_gb300 import hyrom as hy
    q0, cfg, _ = W.euler_oblique_shock(n=64, seed=3, k=4)
    cfg = cfg.with_(precision=prec, w=8, m=4, n_p=8)
    if prec == W.PREC_F64:
        cfg = cfg.with_(pod_tol=1e-10, pod_abs=1e-13)
    q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
    nw = (cfg.ncell + 31) // 32
    runs = []
    stream = torch.cuda.Stream()
    for st in (None, stream):
        ctx = hy.hyrom_init(cfg, q0d, stream=st.cuda_stream if st is not None else None)
        try:
            states, masks = [], []
            q = torch.zeros(cfg.ndof, dtype=tdtype(cfg), device="cuda")
            bm = torch.zeros(nw, dtype=torch.int32, device="cuda")
            for _ in range(cfg.w + 6):
                info = hy.hyrom_step(ctx)
                hy.hyrom_get_state(ctx, q)
                torch.cuda.synchronize()
                states.append(host(q).copy())
                if not info["was_full"]:
                    hy.hyrom_sample(ctx, bitmap_dev=bm)
                    torch.cuda.synchronize()
                    masks.append(host(bm).copy())
            runs.append((states, masks))
        finally:
            hy.hyrom_destroy(ctx)
    (s0, m0), (s1, m1) = runs
    assert len(m0) >= 5
    for a, b in zip(s0, s1):
        assert np.array_equal(a, b)
    for a, b in zip(m0, m1):
        assert np.array_equal(a, b)
