"""Checkpoint and resume (hyrom_save / hyrom_load) and the one-call batch
constructor hyrom_init_batch, through the C ABI.  A run saved after its first
rebuilds and loaded into a fresh context continues with the same bits
(states and sampled sets) as the run that was not interrupted; a file of
another layout is refused.  hyrom_init_batch's instances step to the same
bits as the same instances stepped alone."""
import os

import numpy as np
import pytest

import workloads as W
from tests.gpu_util import H, bits_of, dev, host, tdtype, torch

pytestmark = pytest.mark.gpu


def _cases():
    q, c, _ = W.euler_oblique_shock(n=48, seed=3, k=3)
    yield "shock_fp32", q, c
    q, c, _ = W.euler_vortex(n=40, seed=2)
    yield "vortex_fp64_sample_rows", q, c.with_(nx=40, ny=40, w=6, m=4, n_p=8,
                                                precision=W.PREC_F64, pod_tol=1e-10,
                                                pod_abs=1e-13, regress_rows=W.ROWS_SAMPLE)
    u, c, _ = W.burgers_sine(n=256, seed=1)
    yield "burgers_bdf1", u, c.with_(w=8, m=4, n_p=8)
    q, c = W.euler_riemann_x(n=60)
    yield "sod_muscl", q, c.with_(scheme=W.SCHEME_BDF2_MUSCL, w=6, m=3, n_p=6, top_frac=0.2,
                                  halo=2, pod_tol=1e-10, pod_abs=1e-13)


def _record(hy, ctx, cfg, steps):
    nw = (cfg.ncell + 31) // 32
    bm = torch.zeros(nw, dtype=torch.int32, device="cuda")
    q = torch.zeros(cfg.ndof, dtype=tdtype(cfg), device="cuda")
    out = []
    for _ in range(steps):
        info = hy.hyrom_step(ctx)
        hy.hyrom_get_state(ctx, q)
        hy.hyrom_sample(ctx, bitmap_dev=bm)
        out.append((info["k"], host(q).copy(), bits_of(bm, cfg.ncell)))
    return out


@pytest.mark.parametrize("name,q0,cfg", list(_cases()), ids=[c[0] for c in _cases()])
def test_resume_from_a_checkpoint_is_exact(name, q0, cfg, tmp_path):
    hy = H()
    path = str(tmp_path / "ck.bin")
    q0d = dev(np.asarray(q0).reshape(-1))
    a = hy.hyrom_init(cfg, q0d)
    try:
        for _ in range(cfg.w + 2):               # warm-up and two rebuilds
            hy.hyrom_step(a)
        hy.hyrom_save(a, path)
        want = _record(hy, a, cfg, 4)
    finally:
        hy.hyrom_destroy(a)
    assert os.path.getsize(path) > 0
    b = hy.hyrom_init(cfg, dev(np.zeros(cfg.ndof)))
    try:
        hy.hyrom_load(b, path)
        got = _record(hy, b, cfg, 4)
    finally:
        hy.hyrom_destroy(b)
    for (k1, s1, m1), (k2, s2, m2) in zip(got, want):
        assert k1 == k2
        assert np.array_equal(s1, s2), f"{name}: state differs at step {k1}"
        assert np.array_equal(m1, m2), f"{name}: sampled set differs at step {k1}"


def test_load_refuses_another_layout(tmp_path):
    hy = H()
    q0, cfg, _ = W.euler_oblique_shock(n=32, seed=3, k=3)
    path = str(tmp_path / "ck.bin")
    a = hy.hyrom_init(cfg, dev(q0.reshape(-1)))
    try:
        hy.hyrom_save(a, path)
    finally:
        hy.hyrom_destroy(a)
    q1, cfg1, _ = W.euler_oblique_shock(n=36, seed=3, k=3)
    b = hy.hyrom_init(cfg1, dev(q1.reshape(-1)))
    try:
        with pytest.raises(hy.HyromError) as e:
            hy.hyrom_load(b, path)
        assert e.value.status == hy.HYROM_EINVAL
        with pytest.raises(hy.HyromError):
            hy.hyrom_load(b, str(tmp_path / "missing.bin"))
    finally:
        hy.hyrom_destroy(b)


def test_init_batch_matches_instances_stepped_alone():
    hy = H()
    insts = [W.euler_vortex(n=n, seed=s)[:2] for n, s in ((36, 1), (44, 2), (52, 3))]
    insts = [(q, c.with_(nx=int(round(len(q[0]) ** 0.5)), ny=int(round(len(q[0]) ** 0.5)),
                         w=6, m=3, n_p=6)) for q, c in insts]
    steps = 10
    alone = []
    for q0, cfg in insts:
        ctx = hy.hyrom_init(cfg, dev(q0.reshape(-1)))
        try:
            for _ in range(steps):
                hy.hyrom_step(ctx)
            x = torch.zeros(cfg.ndof, dtype=tdtype(cfg), device="cuda")
            hy.hyrom_get_state(ctx, x)
            alone.append(host(x).copy())
        finally:
            hy.hyrom_destroy(ctx)
    q0s = [dev(q0.reshape(-1)) for q0, _ in insts]
    batch, ctxs = hy.hyrom_init_batch([c for _, c in insts], q0s, threads=2)
    try:
        status, _ = hy.hyrom_batch_step(batch, len(insts), nsteps=steps, ctxs=ctxs)
        assert status == [0] * len(insts)
        torch.cuda.synchronize()
        for ctx, (_, cfg), want in zip(ctxs, insts, alone):
            x = torch.zeros(cfg.ndof, dtype=tdtype(cfg), device="cuda")
            hy.hyrom_get_state(ctx, x)
            torch.cuda.synchronize()
            assert np.array_equal(host(x), want)
    finally:
        hy.hyrom_batch_destroy(batch)


def _run_with_set_state(hy, q0, cfg, steps, at, scale, flush_path=None):
    """Steps of an FP32 run in which, after every step, the state is read and
    written back through hyrom_get_state / hyrom_set_state (host buffers),
    scaled by `scale` after step `at`; with flush_path, hyrom_save right
    after each write forms the new state's Gram row at once."""
    nw = (cfg.ncell + 31) // 32
    bm = torch.zeros(nw, dtype=torch.int32, device="cuda")
    q = torch.zeros(cfg.ndof, dtype=tdtype(cfg), device="cuda")
    hq = torch.zeros(cfg.ndof, dtype=tdtype(cfg), pin_memory=True)
    ctx = hy.hyrom_init(cfg, dev(np.asarray(q0).reshape(-1)))
    out = []
    try:
        for i in range(steps):
            info = hy.hyrom_step(ctx)
            hy.hyrom_get_state(ctx, hq.data_ptr(), on_host=True)
            if i == at:
                hq.mul_(scale)
            hy.hyrom_set_state(ctx, hq.data_ptr(), on_host=True)
            if flush_path is not None:
                hy.hyrom_save(ctx, flush_path)
            if i < cfg.w:  # no sampled set before the first rebuild
                continue
            hy.hyrom_get_state(ctx, q)
            hy.hyrom_sample(ctx, bitmap_dev=bm)
            out.append((info["k"], host(q).copy(), bits_of(bm, cfg.ncell)))
    finally:
        hy.hyrom_destroy(ctx)
    return out


def test_set_state_gram_row_is_formed_with_the_same_bits(tmp_path):
    """hyrom_set_state leaves the new state's snapshot-Gram row to the next
    step's Gram pass (both rows in one pass over the window).  Writing back
    the state a step produced changes nothing: the run keeps the bits of a
    run without the round trips.  Writing a changed state gives the same bits
    whether its row is formed in the next step's pass or at once (here by the
    flush that hyrom_save makes)."""
    hy = H()
    q0, cfg, _ = W.euler_oblique_shock(n=48, seed=3, k=3)
    steps = cfg.w + 8
    ctx = hy.hyrom_init(cfg, dev(np.asarray(q0).reshape(-1)))
    try:
        for _ in range(cfg.w):
            hy.hyrom_step(ctx)
        plain = _record(hy, ctx, cfg, steps - cfg.w)
    finally:
        hy.hyrom_destroy(ctx)
    same = _run_with_set_state(hy, q0, cfg, steps, at=-1, scale=1.0)
    for a, b in zip(plain, same):
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]), a[0]
    at = cfg.w + 2
    late = _run_with_set_state(hy, q0, cfg, steps, at=at, scale=1.001)
    now = _run_with_set_state(hy, q0, cfg, steps, at=at, scale=1.001,
                              flush_path=str(tmp_path / "flush.ck"))
    j = at + 1 - cfg.w  # the first recorded step after the change
    assert not np.array_equal(late[j][1], plain[j][1])  # the change took effect
    for a, b in zip(late, now):
        assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2]), a[0]
