"""The batching form: instances stepped together by the library's thread
pool (each on its own stream), or in the fused form (every instance's
oversampling loop in one multi-instance launch per pass), give, instance by
instance and step by step, the same bits as the same instances stepped
alone; an FP64 instance of the batch also tracks the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import arom
from tests.gpu_util import H, host, rel_err, tdtype, torch

pytestmark = pytest.mark.gpu


def _instances():
    """Small uneven instances: grids 40..72 (ragged tails), k 3..6, sample
    fractions 3..20 %, FP32 and FP64."""
    out = []
    for i, b in enumerate(W.euler_batch(n_inst=5, seed=7, nmin=40, nmax=72, kmin=3, kmax=6,
                                        fmin=0.03, fmax=0.20)):
        q0, cfg = b
        if i == 0:
            cfg = cfg.with_(precision=W.PREC_F64, pod_tol=1e-10, pod_abs=1e-13)
        out.append((q0, cfg))
    return out


def _open(hy, insts):
    ctxs, streams = [], []
    for q0, cfg in insts:
        st = torch.cuda.Stream()
        q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
        ctxs.append(hy.hyrom_init(cfg, q0d, stream=st.cuda_stream))
        streams.append(st)
    torch.cuda.synchronize()
    return ctxs, streams


def _state(hy, ctx, cfg):
    q = torch.zeros(cfg.ndof, dtype=tdtype(cfg), device="cuda")
    hy.hyrom_get_state(ctx, q)
    torch.cuda.synchronize()
    return host(q).copy()


def _wide_instances():
    """Eight instances with windows of 72 to 96 snapshots: their eigensolver
    and pseudo-inverse kernels need different amounts of shared memory above
    the 48 KB default, set per kernel for the whole process."""
    return [b for b in W.euler_batch(n_inst=8, seed=9, nmin=40, nmax=80, kmin=36, kmax=48)]


@pytest.mark.parametrize("mode", ["streams", "fused"])
@pytest.mark.parametrize("kind", ["uneven", "wide"])
def test_batch_matches_instances_stepped_alone(kind, mode):
    hy = H()
    insts = _instances() if kind == "uneven" else _wide_instances()
    threads = 3 if kind == "uneven" else 8
    steps = max(c.w for _, c in insts) + 4          # warm-up and several rebuilds each
    # alone, one after another on the caller's thread
    ctxs, streams = _open(hy, insts)
    alone, alone_info = [], []
    try:
        for ctx, (_, cfg) in zip(ctxs, insts):
            infos = [hy.hyrom_step(ctx) for _ in range(steps)]
            infos[-1].pop("status")     # the batch reports statuses separately
            alone_info.append(infos[-1])
            alone.append(_state(hy, ctx, cfg))
    finally:
        for c in ctxs:
            hy.hyrom_destroy(c)
    # together: more instances than threads, in two calls (steps split unevenly)
    ctxs, streams = _open(hy, insts)
    try:
        b = hy.hyrom_batch_create(ctxs, threads=threads)
        try:
            assert hy.hyrom_batch_threads(b) == threads
            hy.hyrom_batch_set_mode(b, hy.HYROM_BATCH_FUSED if mode == "fused"
                                    else hy.HYROM_BATCH_STREAMS)
            st1, _ = hy.hyrom_batch_step(b, len(ctxs), nsteps=steps - 3, ctxs=ctxs)
            st2, infos = hy.hyrom_batch_step(b, len(ctxs), nsteps=3, ctxs=ctxs)
            assert st1 == [0] * len(ctxs) and st2 == [0] * len(ctxs)
            rows, ms = hy.hyrom_batch_tuning(b)
            if mode == "fused":
                # the autotuner timed its first candidates (each twice) on
                # these calls; the results above are the same whichever ran
                # each step
                assert rows in (0, 1024, 2048, 4096, 8192) and len(ms) == 4, (rows, ms)
                assert sum(x > 0 for x in ms) >= 2, ms
            else:
                assert rows == 0
        finally:
            hy.hyrom_batch_destroy(b)
        for i, (ctx, (_, cfg)) in enumerate(zip(ctxs, insts)):
            assert infos[i] == alone_info[i], f"instance {i}"
            assert np.array_equal(_state(hy, ctx, cfg), alone[i]), f"instance {i}"
            assert not infos[i]["was_full"] and infos[i]["rebuilt"]
    finally:
        for c in ctxs:
            hy.hyrom_destroy(c)


def test_batched_fp64_instance_tracks_oracle():
    hy = H()
    insts = _instances()
    q0, cfg = insts[0]
    steps = cfg.w + 4
    A = arom.Arom(q0, cfg)
    for _ in range(steps):
        A.step()
    ctxs, streams = _open(hy, insts[:3])
    try:
        b = hy.hyrom_batch_create(ctxs, threads=0)
        try:
            hy.hyrom_batch_step(b, len(ctxs), nsteps=steps)
        finally:
            hy.hyrom_batch_destroy(b)
        e = rel_err(_state(hy, ctxs[0], cfg), A.gamma.reshape(-1))
        print(f"batched FP64 instance after {steps} steps: rel err {e:.2e}")
        assert e < 1e-12, e
    finally:
        for c in ctxs:
            hy.hyrom_destroy(c)


def test_batch_rejects_bad_arguments():
    hy = H()
    insts = _instances()[:2]
    ctxs, streams = _open(hy, insts)
    try:
        for bad in ([], [ctxs[0], ctxs[0]], [ctxs[0], None]):
            with pytest.raises(hy.HyromError):
                hy.hyrom_batch_create(bad)
        with pytest.raises(hy.HyromError):
            hy.hyrom_batch_create(ctxs, threads=-1)
        b = hy.hyrom_batch_create(ctxs)
        try:
            with pytest.raises(hy.HyromError):
                hy.hyrom_batch_set_mode(b, 2)
        finally:
            hy.hyrom_batch_destroy(b)
    finally:
        for c in ctxs:
            hy.hyrom_destroy(c)
