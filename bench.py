#!/usr/bin/env python
"""Benchmark of the hybrid-snapshot adaptive ROM (Algorithm 1) on one GB300.

Workload (default): 2D Euler, 2048 x 2048 cells (16.8 M dofs), FP32 states,
a Mach-3 planar shock at a seeded angle with exact-state inflow and outflow
sides, SSP-RK2 HDM, k = 64 POD modes from w = 128 snapshots, n_p = 128
ODEIM points, top 5 % of cells by reconstruction error.  A "step" is one
hybrid step of Algorithm 1 (advance and basis update: partial HDM, gappy coordinates,
reconstruction, residual-gated filters, error indicator and selection,
POD, ODEIM, sampling sets).  The method's own w warm-up full steps and the
first rebuild run before the benchmark's warm-up steps.

Metric: hybrid steps per second (whole job: summed over replicas).  Also
reported: sampled cell-updates/s, per-stage milliseconds from CUDA events
on the library stream, the roofline of the dominant bandwidth kernel,
FP32-vs-FP64 error on a reduced grid, the end-to-end rate through host
buffers, the precision form (the sample-row normal matrix in each
precision), the batching form (64 uneven instances stepped one at a time
and by a pool of host threads), and the CPU oracle on a bounded sample.

--impl reference runs the CPU oracle instead (the only reference this
method has: the paper ships no code).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "hybrid steps/s (Algorithm 1, 2D Euler 2048^2, FP32 states)"
UNIT = "steps/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=2048)
    p.add_argument("--k", type=int, default=64)
    p.add_argument("--frac", type=float, default=0.05)
    p.add_argument("--seed", type=int, default=3)
    p.add_argument("--cpu-n", type=int, default=32, help="grid of the CPU oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-err", action="store_true")
    p.add_argument("--no-precision-form", action="store_true")
    p.add_argument("--no-odeim-batch", action="store_true",
                   help="skip the cheaper ODEIM variant's lines (b points per scoring pass)")
    p.add_argument("--precision-steps", type=int, default=4,
                   help="timed steps per variant of the precision form")
    p.add_argument("--no-batch-form", action="store_true")
    p.add_argument("--batch-n", type=int, default=64, help="instances of the batching form")
    p.add_argument("--batch-steps", type=int, default=3,
                   help="timed hybrid steps per instance in each batching-form arm")
    p.add_argument("--batch-fused-threads", default="8,16",
                   help="host threads of the fused batching arms (empty: none)")
    p.add_argument("--batch-threads", default="1,4,8,16",
                   help="host-thread counts timed in the batching form (1 = one at a time)")
    p.add_argument("--implicit-n", type=int, default=512,
                   help="grid of the implicit (paper's HDM) workload")
    p.add_argument("--no-implicit", action="store_true")
    p.add_argument("--adjoint-n", type=int, default=256, help="grid of the differentiation form")
    p.add_argument("--adjoint-steps", type=int, default=100)
    p.add_argument("--adjoint-k", type=int, default=16)
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--micro", choices=["sample_gram", "batch", "full_step", "np_sweep", "implicit",
                                       "adjoint",
                                       "vortex512", "rk2_vjp"], default=None,
                   help="instead of the step: time one stage on a synthetic input "
                        "(sample_gram: the sample-row normal matrix in each precision)")
    return p.parse_args()


def workload(a, n=None, prec=W.PREC_F32):
    q0, cfg, _ = W.euler_oblique_shock(n=n or a.n, seed=a.seed, k=a.k, frac=a.frac)
    return q0, cfg.with_(precision=prec)


def config_dict(a, cfg):
    return {"workload": f"euler2d_oblique_shock_{cfg.nx}x{cfg.ny}_k{cfg.m}_w{cfg.w}"
                        f"_np{cfg.n_p}_top{a.frac:g}",
            "cells": cfg.ncell, "dofs": cfg.ndof, "k": cfg.m, "w": cfg.w, "n_p": cfg.n_p,
            "sample_frac": a.frac, "scheme": "SSP-RK2 Rusanov", "filters": "Shapiro 2/4/6",
            "l2": "inputs larger than L2 (snapshot window %.1f GB)" % (4 * cfg.ndof * (cfg.w + 1) / 1e9)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------

def _oracle_step_time(a, n, steps, warmup):
    """Seconds per hybrid step of the oracle on an n^2 grid of the workload
    (after its untimed warm-up: the method's w full steps and first rebuild,
    then `warmup` hybrid steps), and the sampled cells per step."""
    from oracle import arom
    q0, cfg = workload(a, n=n, prec=W.PREC_F64)
    A = arom.Arom(q0, cfg)
    while True:
        info = A.step()
        if info.rebuilt and A.k >= cfg.w:
            break
    for _ in range(warmup):
        A.step()
    ns = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        ns += A.step().n_s
    return (time.perf_counter() - t0) / steps, ns / steps, cfg


def cpu_oracle_rate(a, steps=3, warmup=0, steps_large=None):
    """The oracle's hybrid steps/s at the benchmark grid, from timed samples of
    the same workload on two small grids (cpu_n^2 and (2 cpu_n)^2, `steps`
    hybrid steps each; steps_large on the larger one if given).  The
    oracle's time per step is not proportional to the
    cells at these sizes (a fixed part: the m x m eigenproblems and Python
    work of ODEIM's greedy steps), so it is fitted as t = t0 + t1 * cells
    through the two samples and evaluated at the benchmark's cells; the rate
    scaled by cells from the small grid alone is reported beside it."""
    n1, n2 = a.cpu_n, 2 * a.cpu_n
    t_1, ns1, cfg = _oracle_step_time(a, n1, steps, warmup)
    s2 = steps if steps_large is None else steps_large
    t_2, ns2, _ = _oracle_step_time(a, n2, s2, 0 if steps_large is not None else warmup)
    c1, c2, cb = n1 * n1, n2 * n2, a.n * a.n
    t1c = (t_2 - t_1) / (c2 - c1)
    t0c = t_1 - t1c * c1
    t_big = t0c + t1c * cb
    return {"value": 1.0 / t_big, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"{steps} and {s2} hybrid steps of the same workload (k={cfg.m}, "
                      f"w={cfg.w}) on {n1}x{n1} ({t_1:.2f} s/step) and {n2}x{n2} "
                      f"({t_2:.2f} s/step); "
                      f"time per step fitted as {t0c:.3g} s + {t1c:.3g} s/cell and "
                      f"evaluated at {a.n}x{a.n}",
            "s_per_step": {f"{n1}x{n1}": t_1, f"{n2}x{n2}": t_2},
            "fit_s_per_step": {"fixed": t0c, "per_cell": t1c},
            "scaled_by_cells_from_smallest": 1.0 / (t_1 * cb / c1),
            "sample_cell_updates_per_s": ns1 / t_1}


def _cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.strip().split(",") for r in self.out.read().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per launch (FP32 states, 4 bytes)
# ---------------------------------------------------------------------------

def stage_bytes(cfg, m_eff, n_s_avg, s=4):
    N, nc, w = cfg.ndof, cfg.ncell, cfg.w
    frac_breve = 1.0 - n_s_avg / nc
    return {
        # psi + Phi y on the S-breve dofs: read Phi rows and psi, write q
        "recon": s * N * frac_breve * (m_eff + 2),
        # window read, psi read, Phi write, next psi write
        "formphi": s * N * (w + 1 + m_eff + 1),
        # one new snapshot against w+1 ring slots (the new one stays in L2)
        "gram": s * N * (w + 1),
        # error indicator: read g, psi, Phi; write eps; keys and radix passes
        "select": s * N * (m_eff + 2) + s * nc + 8 * nc * 9,
    }


def fp64_peak_tflops():
    """This GPU's FP64 rate from the library's FMA loop (hyrom_probe_fp64),
    timed with CUDA events: the denominator of the FP64 stages' roofline."""
    import torch
    from paper_2301_01718_gb300 import hyrom
    blocks, iters, reps = 152 * 16, 2048, 5
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(2):
        hyrom.hyrom_probe_fp64(out, blocks, iters, st.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        hyrom.hyrom_probe_fp64(out, blocks, iters, st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize()
    flops = reps * blocks * 256 * 16 * iters
    return flops / (e0.elapsed_time(e1) * 1e-3) / 1e12


def stage_costs(cfg, m_eff, n_s_avg, n_p, sweeps_pod, s=4):
    """Work of the stages that stream no state-sized operand once, per step:
      partial  - the partial RK2 step on S-hat: read gamma_{k-1} on S-hat and
                 its 2-cell ring, write gamma_k on S-hat (c s (n_s + ring) 3)
      filter   - the first pass of each of the three orders over the grid:
                 read q and gamma_{k-1}, write g and the gate (~ s N 5)
      deim     - the greedy DEIM loop as written, one residual pass over Phi's
                 first l columns per point: s N (m^2/2 + 3m/2)  (naive)
      odeim    - the oversampling loop as written, one scoring pass over Phi
                 per point: s N m (n_p - m)  (naive)
      eig      - the POD eigensolve, one-sided Jacobi on the w x w factor:
                 ~12 w flops per column pair and sweep, 6 w^3 per sweep, plus
                 w^3/3 for the pivoted Cholesky (FP64 flops)
    The two ODEIM stages prune rows with certified bounds, so their naive
    bytes over time exceed the HBM rate: the ratio is the pruning's gain."""
    N, nc, w, m = cfg.ndof, cfg.ncell, cfg.w, m_eff
    ring = 4 * (n_s_avg ** 0.5) * 2 if cfg.ny > 1 else 4
    return {
        "partial": ("bytes", s * cfg.nvar * (n_s_avg + ring) * 3),
        "filter": ("bytes", 3 * s * N * 5),
        "deim": ("bytes_naive", s * N * (m * m / 2 + 1.5 * m)),
        "odeim": ("bytes_naive", s * N * m * max(n_p - m, 0)),
        "eig": ("fp64_flops", sweeps_pod * 6.0 * w ** 3 + w ** 3 / 3.0),
    }


def max_over_ranks(ms, world, device):
    """The slowest rank's time (ms): all ranks time the same number of steps
    between barriers, so the job's time is the maximum."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    return float(t.item())


def whole_job_rate(steps, world, ms_max):
    """Steps per second of the whole job: every replica did `steps` steps."""
    return world * steps / (ms_max / 1e3)


def run_ours(a):
    import torch
    import torch.distributed as dist
    from paper_2301_01718_gb300 import build, hyrom

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    q0, cfg = workload(a)
    stream = torch.cuda.Stream()
    q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = hyrom.hyrom_init(cfg, q0d, stream=stream.cuda_stream)
    del q0d
    try:
        # the method's own warm-up: w full steps and the first rebuild
        while True:
            info = hyrom.hyrom_step(ctx)
            if not info["was_full"]:
                break
        for _ in range(a.warmup):
            hyrom.hyrom_step(ctx)
        hyrom.hyrom_profile(ctx, True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        l0 = hyrom.hyrom_kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        ns_sum, infos = 0, []
        for _ in range(a.steps):
            info = hyrom.hyrom_step(ctx)
            ns_sum += info["n_s"]
            infos.append(info)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        launches = hyrom.hyrom_kernel_launches() - l0
        ck = clocks.stop()
        ms = e0.elapsed_time(e1)
        stages = hyrom.hyrom_stage_times(ctx)
        odc = hyrom.hyrom_odeim_counters(ctx)
        eig_sw = hyrom.hyrom_eig_sweeps(ctx)
        hyrom.hyrom_profile(ctx, False)
        ms_max = max_over_ranks(ms, world, "cuda")
        value = whole_job_rate(a.steps, world, ms_max)

        # end to end through host buffers (pinned): upload gamma_k, step,
        # download gamma_k+1, every step
        e2e = None
        if not a.no_e2e:
            hbuf = torch.empty(cfg.ndof, dtype=torch.float32, pin_memory=True)
            hyrom.hyrom_get_state(ctx, hbuf.data_ptr(), on_host=True)
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            ke = max(2, a.steps // 2)
            for _ in range(ke):
                hyrom.hyrom_set_state(ctx, hbuf.data_ptr(), on_host=True)
                hyrom.hyrom_step(ctx)
                hyrom.hyrom_get_state(ctx, hbuf.data_ptr(), on_host=True)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            el_max = max_over_ranks(el * 1e3, world, "cuda")
            e2e = {"value": whole_job_rate(ke, world, el_max), "unit": UNIT,
                   "h2d_bytes_per_step": 4 * cfg.ndof, "d2h_bytes_per_step": 4 * cfg.ndof,
                   "path": "hyrom_set_state(host) + hyrom_step + hyrom_get_state(host)"}
        m_eff = infos[-1]["m_eff"]
    finally:
        hyrom.hyrom_destroy(ctx)

    n_s_avg = ns_sum / a.steps
    per = {}
    byts = stage_bytes(cfg, m_eff, n_s_avg)
    peaks = _peaks()
    fp64 = fp64_peak_tflops() if rank == 0 else None
    costs = stage_costs(cfg, m_eff, n_s_avg, infos[-1]["n_p"], eig_sw["pod"])
    for name, (tot, cnt) in stages.items():
        if cnt == 0:
            continue
        d = {"ms_per_step": tot / a.steps, "launches": cnt, "ms_per_launch": tot / cnt,
             "share_of_step": (tot / a.steps) / (ms_max / a.steps)}
        if name in byts:
            d["gbs"] = byts[name] / (tot / cnt * 1e-3) / 1e9
            d["frac_of_hbm"] = d["gbs"] / peaks["hbm"]
        elif name in costs:
            kind, amount = costs[name]
            rate = amount / (tot / a.steps * 1e-3)
            if kind == "fp64_flops":
                d["fp64_tflops"] = rate / 1e12
                if fp64:
                    d["frac_of_fp64"] = rate / 1e12 / fp64
            else:
                d["gbs" if kind == "bytes" else "naive_gbs"] = rate / 1e9
                d["frac_of_hbm" if kind == "bytes" else "naive_over_hbm"] = rate / 1e9 / peaks["hbm"]
        per[name] = d
    # roofline of the dominant kernel with an algorithmic byte count
    cand = [(per[n]["ms_per_step"], n) for n in byts if n in per]
    roof = None
    if cand:
        _, dom = max(cand)
        ach = per[dom]["gbs"]
        traffic = None
        if dom == "formphi" and FORMPHI_TRAFFIC_PER_DOF is not None and cfg.w == 128 \
                and m_eff == 64:
            traffic = FORMPHI_TRAFFIC_PER_DOF * cfg.ndof
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm"],
                "unit": "GB/s", "frac": ach / peaks["hbm"], "traffic": traffic,
                "bytes_per_launch": byts[dom], "peak_source": peaks["src"]}
    # the step without ODEIM (a7): the step time less the DEIM and ODEIM stage
    # times (the method's own step recomputes the points every step)
    a7 = sum(per[n]["ms_per_step"] for n in ("odeim", "deim") if n in per)
    no_a7 = {"ms_per_step": ms_max / a.steps - a7, "steps_per_s": 1e3 / (ms_max / a.steps - a7),
             "odeim_ms_per_step": a7,
             "note": "derived: step time minus the DEIM and ODEIM stage times"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": config_dict(a, cfg),
           "sampled_cell_updates_per_s": (world * ns_sum / (stages["partial"][0] / 1e3)
                                          if stages.get("partial", (0, 0))[0] > 0 else None),
           "sampled_cells_per_s_of_step": world * ns_sum / (ms_max / 1e3),
           "fp64_peak_tflops_measured": fp64,
           "n_s_avg": n_s_avg, "m_eff": m_eff, "stages": per,
           "roofline": roof, "gpu_launches": int(launches), "clocks": ck, "e2e": e2e,
           "odeim_counters_last_step": odc, "eig_sweeps_last_step": eig_sw,
           "without_odeim": no_a7}
    if rank == 0 and not a.no_odeim_batch:   # (timed before the oracle runs load the host)
        out["odeim_batch_form"] = odeim_batch_form(a)
    if rank == 0 and not a.no_err:
        out["err_vs_oracle"] = err_vs_oracle(a)
    if rank == 0 and not a.no_precision_form:
        out["precision_form"] = precision_form(a)
    if rank == 0:
        out["full_step"] = full_step(a)
    if rank == 0 and not a.no_batch_form:
        out["batch_form"] = batch_form(a)
    if rank == 0 and not a.no_implicit:
        out["implicit_form"] = implicit_form(a)
    if rank == 0 and not a.no_adjoint:
        out["adjoint_form"] = adjoint_form(a)
    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_rate(a)
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


# DRAM bytes per launch of the roofline kernel per dof, from the ncu capture
# summarised in profiles/form_phi_tc_euler_1024.md (k_form_phi_tc, w = 128,
# m = 64, 1024 x 1024 cells), scaled by dofs; set to None when the kernel
# changes until it is captured again.
FORMPHI_TRAFFIC_PER_DOF = (2164398000 + 1078423000) / 4194304  # 773.2 B per dof


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm": float(d["hbm_gbs"]), "src": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    except (OSError, KeyError, ValueError):
        return {"hbm": 6800.0, "src": "fallback 6.8 TB/s"}


_ORACLE_RUNS = {}


def _oracle_run(q0, cfg, steps_hyb):
    """The oracle's states and sampled sets for the first `steps_hyb` hybrid
    steps of Algorithm 1 (cached per configuration)."""
    from oracle import arom
    key = repr(cfg)
    if key not in _ORACLE_RUNS:
        A = arom.Arom(q0, cfg)
        recs, hyb = [], 0
        while hyb < steps_hyb:
            info = A.step()
            if not info.was_full:
                hyb += 1
            recs.append((info.was_full, info.rebuilt, A.gamma.reshape(-1).copy(),
                         None if A.s_hat is None else A.s_hat.reshape(-1).copy()))
        _ORACLE_RUNS[key] = recs
    return _ORACLE_RUNS[key]


def err_vs_oracle(a, n=128, k=16, steps=12, **kw):
    """The FP32 GPU run against the FP64 oracle on an n^2 grid of the same
    workload with k modes (w = n_p = 2k): per hybrid step the relative L1 and
    max errors of the state and, at every rebuild, the Hamming distance
    between the two sampled sets S-hat (cells in one and not the other).  The
    two runs take their decisions (filter gates, selection, ODEIM points)
    each in its own arithmetic, so the sets can part where an FP32 value sits
    at a tie.  kw: further config fields of both runs."""
    import torch
    from paper_2301_01718_gb300 import hyrom
    q0, cfg = workload(a, n=n, prec=W.PREC_F32)
    cfg = cfg.with_(w=2 * k, m=k, n_p=2 * k, **kw)
    ocfg = cfg.with_(precision=W.PREC_F64, reduced_prec=W.RED_F32)
    want = _oracle_run(q0, ocfg, steps)
    q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = hyrom.hyrom_init(cfg, q0d)
    per = []
    try:
        q = torch.zeros(cfg.ndof, dtype=torch.float32, device="cuda")
        bm = torch.zeros((cfg.ncell + 31) // 32, dtype=torch.int32, device="cuda")
        for was_full, rebuilt, g_o, sh_o in want:
            info = hyrom.hyrom_step(ctx)
            if bool(info["was_full"]) != was_full:
                raise RuntimeError("full/hybrid schedules differ")
            if was_full:
                continue
            hyrom.hyrom_get_state(ctx, q)
            g = q.double().cpu().numpy()
            rec = {"k": int(info["k"]), "rel_l1": float(np.abs(g - g_o).sum() / np.abs(g_o).sum()),
                   "rel_max": float(np.abs(g - g_o).max() / np.abs(g_o).max())}
            if rebuilt:
                hyrom.hyrom_sample(ctx, bitmap_dev=bm)
                w = bm.cpu().numpy().view(np.uint32).astype(np.uint64)
                bits = ((w[:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1))
                sh = bits.reshape(-1)[: cfg.ncell].astype(bool)
                rec["hamming"] = int(np.count_nonzero(sh != sh_o))
                rec["n_s"] = int(sh_o.sum())
            per.append(rec)
    finally:
        hyrom.hyrom_destroy(ctx)
    ham = [r["hamming"] for r in per if "hamming" in r]
    return {"grid": f"{n}x{n}", "k": k, "w": 2 * k, "n_p": 2 * k, "hybrid_steps": len(per),
            "max_rel_l1": max(r["rel_l1"] for r in per),
            "max_rel_max": max(r["rel_max"] for r in per),
            "max_hamming": max(ham) if ham else None,
            "steps_with_identical_masks": sum(1 for h in ham if h == 0),
            "per_step": per}


def _err_summary(e):
    return {k: v for k, v in e.items() if k != "per_step"}


PRECISIONS = {"f32_cuda_cores": W.RED_F32, "tf32": W.RED_TF32, "bf16": W.RED_BF16,
              "tf32_split": W.RED_TF32_SPLIT}


def odeim_batch_form(a, values=(2, 4), steps=4):
    """The cheaper oversampling variant (odeim_batch = b: the b best rows of
    each scoring pass, not the paper's greedy) on the benchmark workload: ms
    per hybrid step and the DEIM + ODEIM stage times, beside the faithful
    method of the headline; and, for the largest b, the FP32 run's error
    against the FP64 oracle running the same variant (err_vs_oracle)."""
    out = {}
    for b in values:
        q0, cfg = workload(a)
        ms, st, ns = time_hybrid_steps(q0, cfg.with_(odeim_batch=b), steps)
        out[str(b)] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms,
                       "odeim_ms": st.get("odeim", 0.0), "deim_ms": st.get("deim", 0.0),
                       "odeim_counters_last_step": time_hybrid_steps.odeim_counters}
    if not a.no_err:
        e = err_vs_oracle(a, odeim_batch=max(values))
        out[str(max(values))]["err_vs_oracle"] = {k: v for k, v in e.items() if k != "per_step"}
    return {"workload": "the benchmark's, with b oversampling points per scoring pass",
            "steps": steps, "b": out}


def precision_form(a):
    """The reduced solve in its sample-row form (every dof row of S-hat) with
    the normal matrix Phi_S^T Phi_S in each precision: FP32 on the CUDA cores,
    TF32 and BF16 on the tensor cores (FP32 accumulation), and the TF32 hi/lo
    split; states, flux and right-hand side FP32, Cholesky and solve FP64.
    Per variant: the normal matrix's time per rebuild, steps/s of the whole
    step on the benchmark workload, and the state error against the FP64
    oracle's sample-row run (err_vs_oracle)."""
    import torch
    from paper_2301_01718_gb300 import hyrom
    out = {}
    for name, red in PRECISIONS.items():
        q0, cfg = workload(a)
        cfg = cfg.with_(regress_rows=W.ROWS_SAMPLE, reduced_prec=red)
        stream = torch.cuda.Stream()
        q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
        ctx = hyrom.hyrom_init(cfg, q0d, stream=stream.cuda_stream)
        del q0d
        try:
            while hyrom.hyrom_step(ctx)["was_full"]:
                pass
            for _ in range(3):
                hyrom.hyrom_step(ctx)
            hyrom.hyrom_profile(ctx, True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.precision_steps):
                hyrom.hyrom_step(ctx)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            st = hyrom.hyrom_stage_times(ctx)
            hyrom.hyrom_profile(ctx, False)
        finally:
            hyrom.hyrom_destroy(ctx)
        tot, cnt = st["snormal"]
        gt, gc = st["gappy"]
        out[name] = {"snormal_ms_per_rebuild": tot / max(cnt, 1), "rebuilds": cnt,
                     "gappy_ms_per_step": gt / a.precision_steps,
                     "steps_per_s": a.precision_steps / (ms / 1e3),
                     "err_vs_oracle": None if a.no_err else _err_summary(err_vs_oracle(
                         a, regress_rows=W.ROWS_SAMPLE, reduced_prec=red))}
    return {"workload": "same grid and method, reduced coordinates fitted on every dof row "
                        "of S-hat (normal equations)", "steps": a.precision_steps,
            "variants": out}


def micro_sample_gram(a, m=64, calls=10):
    """The sample-row normal matrix (hyrom_stage_gappy_rows) on an n^2 Euler
    grid with a random FP32 basis of m columns and every other cell sampled:
    CUDA-event time of the normal matrix per call in each precision, and its
    algorithmic bytes (4 B x rows x m) per second."""
    import torch
    from paper_2301_01718_gb300 import build, hyrom
    build.build()
    n = a.n
    out = {}
    for name, red in PRECISIONS.items():
        cfg = W.ArConfig(pde=W.PDE_EULER, scheme=W.SCHEME_RK2, nx=n, ny=n, dx=1.0 / n,
                         dy=1.0 / n, dt=1e-4, w=m, m=m, n_p=2 * m, precision=W.PREC_F32,
                         regress_rows=W.ROWS_SAMPLE, reduced_prec=red)
        N, nc = cfg.ndof, cfg.ncell
        g = torch.Generator(device="cuda").manual_seed(a.seed)
        phi = torch.randn(m * N, device="cuda", generator=g) / N ** 0.5
        cells = torch.arange(0, nc, 2, dtype=torch.int32, device="cuda")
        v = torch.randn(N, device="cuda", generator=g)
        psi = torch.randn(N, device="cuda", generator=g)
        ctx = hyrom.hyrom_init(cfg, torch.zeros(N, dtype=torch.float64, device="cuda"))
        try:
            y = torch.zeros(m, dtype=torch.float64, device="cuda")
            for _ in range(3):
                hyrom.hyrom_stage_gappy_rows(ctx, phi, m, cells, len(cells), v, psi, y)
            hyrom.hyrom_profile(ctx, True)
            for _ in range(calls):
                hyrom.hyrom_stage_gappy_rows(ctx, phi, m, cells, len(cells), v, psi, y)
            st = hyrom.hyrom_stage_times(ctx)
            hyrom.hyrom_profile(ctx, False)
        finally:
            hyrom.hyrom_destroy(ctx)
        rows = 4 * len(cells)
        ms = st["snormal"][0] / max(st["snormal"][1], 1)
        out[name] = {"ms": ms, "gbs": 4.0 * rows * m / (ms * 1e-3) / 1e9,
                     "solve_ms": st["gappy"][0] / max(st["gappy"][1], 1)}
    return {"micro": "sample_gram", "grid": f"{n}x{n}", "m": m,
            "rows": rows, "sample": "every other cell", "calls": calls, "variants": out}


def batch_form(a):
    """The batching form: a.batch_n independent Euler instances
    (workloads.euler_batch: grids log-uniform 128^2..1024^2, Mach 0.3..2,
    own basis k 8..48 and sample fraction 2..20 % each), every context on its
    own stream, stepped by hyrom_batch_step with 1 host thread (the instances
    one at a time) and with more threads (up to that many instances on the
    GPU at once), then in the fused form (HYROM_BATCH_FUSED: every
    instance's oversampling loop in one launch per pass, after the
    autotuner's nine untimed steps).  Each arm times a.batch_steps hybrid
    steps of every instance, host clock around the synchronised call; rates
    are instance hybrid steps/s and dof-steps/s (dofs advanced per second)."""
    import torch
    from paper_2301_01718_gb300 import build, hyrom
    build.build()
    insts = W.euler_batch(n_inst=a.batch_n, seed=5)
    ctxs, streams = [], []
    dofs = sum(c.ndof for _, c in insts)
    try:
        for q0, cfg in insts:
            st = torch.cuda.Stream()
            q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
            ctxs.append(hyrom.hyrom_init(cfg, q0d, stream=st.cuda_stream))
            streams.append(st)
            del q0d
        dev_bytes = sum(hyrom.hyrom_device_bytes(c) for c in ctxs)
        # each instance's own warm-up (w full steps and the first rebuild)
        for c in ctxs:
            while hyrom.hyrom_step(c)["was_full"]:
                pass
        arms, fused = {}, {}
        runs = [(int(x), False) for x in str(a.batch_threads).split(",") if x]
        runs += [(int(x), True) for x in str(a.batch_fused_threads).split(",") if x]
        for t, is_fused in runs:
            b = hyrom.hyrom_batch_create(ctxs, threads=t)
            try:
                if is_fused:
                    # the autotuner times its four candidates twice each
                    hyrom.hyrom_batch_set_mode(b, hyrom.HYROM_BATCH_FUSED)
                    hyrom.hyrom_batch_step(b, len(ctxs), nsteps=9, ctxs=ctxs)
                else:
                    hyrom.hyrom_batch_set_mode(b, hyrom.HYROM_BATCH_STREAMS)
                    hyrom.hyrom_batch_step(b, len(ctxs), nsteps=1, ctxs=ctxs)     # warm-up
                torch.cuda.synchronize()
                l0 = hyrom.hyrom_kernel_launches()
                t0 = time.perf_counter()
                _, infos = hyrom.hyrom_batch_step(b, len(ctxs), nsteps=a.batch_steps, ctxs=ctxs)
                torch.cuda.synchronize()
                el = time.perf_counter() - t0
                launches = hyrom.hyrom_kernel_launches() - l0
                threads = hyrom.hyrom_batch_threads(b)
                tuning = hyrom.hyrom_batch_tuning(b)
            finally:
                hyrom.hyrom_batch_destroy(b)
            assert all(not i["was_full"] for i in infos)
            steps = a.batch_steps * len(ctxs)
            arm = {"ms": el * 1e3, "instance_steps_per_s": steps / el,
                   "dof_steps_per_s": dofs * a.batch_steps / el,
                   "gpu_launches": int(launches)}
            if is_fused:
                arm["rows_per_cta"] = tuning[0]
                arm["tuning_ms_per_greedy_step"] = dict(zip(["1024", "2048", "4096", "8192"],
                                                            tuning[1]))
                fused[str(threads)] = arm
            else:
                arms[str(threads)] = arm
    finally:
        for c in ctxs:
            hyrom.hyrom_destroy(c)
    one = arms.get("1")
    best = max(list(arms.values()) + list(fused.values()),
               key=lambda r: r["instance_steps_per_s"])
    return {"workload": f"{len(insts)} Euler vortex instances, grids 128^2..1024^2 "
                        "log-uniform, Mach 0.3..2, k 8..48 (w = n_p = 2k), sample 2..20 %, FP32",
            "instances": len(insts), "dofs": dofs, "device_bytes": dev_bytes,
            "steps_per_instance": a.batch_steps, "unit": "instance hybrid steps/s",
            "threads": arms,
            "fused": {"form": "each step in two phases around one launch per pass of every "
                              "instance's oversampling loop (CUDA graph, autotuned rows per CTA)",
                      "threads": fused},
            "speedup_vs_one_at_a_time": (best["instance_steps_per_s"] /
                                         one["instance_steps_per_s"]) if one else None}


def full_step(a, calls=20, pairs=4):
    """The full SSP-RK2 HDM step (hyrom_stage_full_step: the fused flux
    kernel over every tile) on the benchmark grid: CUDA-event time of the
    kernel per launch (stage timer around the launch), and its algorithmic
    bytes (the state read once and written once: 2 x 4 x 4 B per cell) per
    second against the measured HBM peak.  `pairs` input/output pairs are
    used in turn, so that the bytes of consecutive launches (pairs x 134 MB
    at 2048^2) exceed L2."""
    import torch
    from paper_2301_01718_gb300 import build, hyrom
    build.build()
    q0, cfg = workload(a)
    q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = hyrom.hyrom_init(cfg, q0d)
    try:
        bufs = [(q0d.to(torch.float32).clone(), torch.empty(cfg.ndof, device="cuda"))
                for _ in range(pairs)]
        del q0d
        for i in range(3):
            hyrom.hyrom_stage_full_step(ctx, bufs[i % pairs][0], bufs[i % pairs][1], 1)
        hyrom.hyrom_profile(ctx, True)
        for i in range(calls):
            hyrom.hyrom_stage_full_step(ctx, bufs[i % pairs][0], bufs[i % pairs][1], 1)
        tot, cnt = hyrom.hyrom_stage_times(ctx)["full"]
        hyrom.hyrom_profile(ctx, False)
    finally:
        hyrom.hyrom_destroy(ctx)
    ms = tot / max(cnt, 1)
    byts = 2.0 * 4 * 4 * cfg.ncell
    peaks = _peaks()
    gbs = byts / (ms * 1e-3) / 1e9
    return {"kernel": "k_rk2_euler_sweep", "grid": f"{cfg.nx}x{cfg.ny}", "ms_per_launch": ms,
            "launches": cnt, "bytes_per_launch": byts, "achieved_gbs": gbs,
            "peak_gbs": peaks["hbm"], "frac": gbs / peaks["hbm"], "peak_source": peaks["src"]}


def time_hybrid_steps(q0, cfg, steps=4, warmup=2):
    """ms per hybrid step (CUDA events on the context stream) and per-stage
    ms per step of one context, after the method's own warm-up."""
    import torch
    from paper_2301_01718_gb300 import hyrom
    stream = torch.cuda.Stream()
    q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = hyrom.hyrom_init(cfg, q0d, stream=stream.cuda_stream)
    del q0d
    try:
        while hyrom.hyrom_step(ctx)["was_full"]:
            pass
        for _ in range(warmup):
            hyrom.hyrom_step(ctx)
        hyrom.hyrom_profile(ctx, True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ns = 0
        for _ in range(steps):
            ns += hyrom.hyrom_step(ctx)["n_s"]
        e1.record(stream)
        torch.cuda.synchronize()
        st = hyrom.hyrom_stage_times(ctx)
        hyrom.hyrom_profile(ctx, False)
        time_hybrid_steps.odeim_counters = hyrom.hyrom_odeim_counters(ctx)
    finally:
        hyrom.hyrom_destroy(ctx)
    ms = e0.elapsed_time(e1) / steps
    return ms, {k: v[0] / steps for k, v in st.items() if v[1]}, ns / steps


def np_sweep(a, values=(64, 96, 128, 160, 192), steps=4):
    """n_p sensitivity: the benchmark workload with n_p ODEIM points (k = 64;
    n_p <= 194 keeps the sampled pseudo-inverse in one CTA's shared memory)."""
    from paper_2301_01718_gb300 import build
    build.build()
    out = {}
    for n_p in values:
        q0, cfg = workload(a)
        cfg = cfg.with_(n_p=n_p)
        ms, st, ns = time_hybrid_steps(q0, cfg, steps)
        out[str(n_p)] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "n_s_avg": ns,
                         "odeim_ms": st.get("odeim", 0.0), "deim_ms": st.get("deim", 0.0),
                         "odeim_counters_last_step": time_hybrid_steps.odeim_counters}
    return {"workload": config_dict(a, cfg)["workload"], "steps": steps, "n_p": out}


def vortex512(a, steps=10):
    """The isentropic-vortex configuration (512^2 periodic Euler, k = 20,
    w = 40, 5 % sample, FP32): hybrid steps/s and the stage times.  Its
    snapshot window (4 x 512^2 x 41 x 4 B = 172 MB) is about L2's size, so
    the window passes run partly from L2: compare their GB/s with the 2048^2
    run's."""
    from paper_2301_01718_gb300 import build
    build.build()
    q0, cfg, _ = W.euler_vortex(n=512, seed=2)
    ms, st, ns = time_hybrid_steps(q0, cfg, steps)
    byts = stage_bytes(cfg, cfg.m, ns)
    gbs = {n: byts[n] / (st[n] * 1e-3) / 1e9 for n in byts if n in st and st[n] > 0}
    return {"workload": f"euler2d_vortex_{cfg.nx}x{cfg.ny}_k{cfg.m}_w{cfg.w}_top0.05",
            "ms_per_step": ms, "steps_per_s": 1e3 / ms, "n_s_avg": ns,
            "stages_ms": st, "stage_gbs": gbs,
            "odeim_counters_last_step": time_hybrid_steps.odeim_counters,
            "window_bytes": 4 * cfg.ndof * (cfg.w + 1)}


def rk2_vjp(a, n=1024, calls=10):
    """The adjoint of the SSP-RK2 Euler step (hyrom_stage_rk2_vjp, FP64) on
    the n^2 vortex of the differentiation form: CUDA events on the legacy
    stream around each call (its stage-1 recomputation, two L'^T passes and
    the host synchronisation), ms per call and cells per second."""
    import torch
    from paper_2301_01718_gb300 import build, hyrom
    build.build()
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    cfg = cfg.with_(precision=W.PREC_F64, w=4, m=2, n_p=4)
    q = torch.as_tensor(W.euler_vortex_theta(n, W.VORTEX_THETA0).reshape(-1),
                        dtype=torch.float64, device="cuda")
    ctx = hyrom.hyrom_init(cfg, q)
    try:
        lam = torch.randn(cfg.ndof, dtype=torch.float64, device="cuda")
        out = torch.empty_like(lam)
        work = torch.empty(3 * cfg.ndof, dtype=torch.float64, device="cuda")
        for _ in range(2):
            hyrom.hyrom_stage_rk2_vjp(ctx, q, lam, out, None, 2, work)
        ms = []
        for _ in range(calls):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            hyrom.hyrom_stage_rk2_vjp(ctx, q, lam, out, None, 2, work)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    finally:
        hyrom.hyrom_destroy(ctx)
    best = min(ms)
    return {"grid": f"{n}x{n}", "dtype": "f64", "ms_per_call": best,
            "ms_median": statistics.median(ms), "cells_per_s": cfg.ncell / (best * 1e-3)}


def implicit_form(a, n=None, steps=14):
    """The paper's own HDM (Sec. 3.1: MUSCL-minmod-Roe, BDF2 by Newton-GMRES,
    FP64) on the oblique-shock workload with the parameters of the paper's
    implosion run (w = 6, m = 4, z = 7, RRE threshold delta = 0.9, filters of
    orders 2, 4, 6): host-clocked time of each step of Algorithm 1 after the
    warm-up, split into full-HDM steps (every z-th) and hybrid steps (partial
    Newton solves with subiterations, reconstruction, filter, and the basis
    update), and the paper's speedup S = time per snapshot of the full HDM /
    time per snapshot of the AROM (Sec. 2.4.2) over the measured cycle."""
    import torch
    from paper_2301_01718_gb300 import hyrom
    n = n or a.implicit_n
    q0, cfg, _ = W.euler_oblique_shock(n=n, seed=a.seed, k=4)
    cfg = cfg.with_(scheme=W.SCHEME_BDF2_MUSCL, precision=W.PREC_F64, w=6, m=4, n_p=8, z=7,
                    sel_mode=W.SEL_RRE, delta=0.9, newton_tol=1e-10, pod_tol=1e-10,
                    pod_abs=1e-13)
    q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    ctx = hyrom.hyrom_init(cfg, q0d, stream=stream.cuda_stream)
    del q0d
    full, hyb, ns, J, passes = [], [], [], [], []
    try:
        k = 0
        while k < cfg.w + 1:                      # the method's warm-up
            k = hyrom.hyrom_step(ctx)["k"]
        hyrom.hyrom_profile(ctx, True)
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = hyrom.hyrom_step(ctx)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) * 1e3
            (full if info["was_full"] else hyb).append(dt)
            if not info["was_full"]:
                ns.append(info["n_s"])
                J.append(info["J"])
                passes.append(info["filt_passes"])
        st = hyrom.hyrom_stage_times(ctx)
        hyrom.hyrom_profile(ctx, False)
    finally:
        hyrom.hyrom_destroy(ctx)
    tf = statistics.median(full) if full else None
    th = statistics.mean(hyb) if hyb else None
    z = cfg.z
    out = {"workload": f"euler2d_oblique_shock_{n}x{n}_muscl_roe_bdf2_w{cfg.w}_m{cfg.m}_z{z}"
                       f"_rre{cfg.delta:g}",
           "full_ms": tf, "hybrid_ms": th, "full_steps": len(full), "hybrid_steps": len(hyb),
           "n_s_frac_mean": float(np.mean(ns)) / cfg.ncell if ns else None,
           "J_mean": float(np.mean(J)) if J else None,
           "filter_passes_mean": float(np.mean(passes)) if passes else None,
           "stage_ms_per_hybrid_step": {k2: v[0] / max(len(hyb), 1) for k2, v in st.items()
                                        if v[1] and k2 != "full"},
           "newton_tol": cfg.newton_tol}
    if tf and th:
        out["speedup_S"] = z * tf / ((z - 1) * th + tf)
        out["hybrid_over_full"] = th / tf
    return out


def adjoint_form(a, n=None, steps=None, k=None):
    """The differentiation form: J = time integral over `steps` steps of the
    pressure over a fixed 64 x 64 box of the vortex-plus-pulse problem with
    the eight-parameter initial state (euler_vortex_theta), FP64; dJ/dq0 by
    hyrom_adjoint (the forward run taped, then one reverse sweep) and
    dJ/dtheta = (dq0/dtheta)^T dJ/dq0 (dq0/dtheta by the complex step of the
    analytic initial state).  Host-clocked: the plain forward run of the same
    steps, and the whole gradient call."""
    import torch
    from paper_2301_01718_gb300 import hyrom
    n = n or a.adjoint_n
    steps = steps or a.adjoint_steps
    k = k or a.adjoint_k
    th0 = np.array(W.VORTEX_THETA0)
    q0 = W.euler_vortex_theta(n, th0)
    _, cfg, _ = W.euler_vortex(n=n, seed=2)
    cfg = cfg.with_(precision=W.PREC_F64, w=2 * k, m=k, n_p=2 * k, pod_tol=1e-10, pod_abs=1e-13)
    b0 = (n - 64) // 2
    box = (b0, b0 + 64, b0, b0 + 64)
    q0d = torch.as_tensor(q0.reshape(-1), dtype=torch.float64, device="cuda")
    ctx = hyrom.hyrom_init(cfg, q0d)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            hyrom.hyrom_step(ctx)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
    finally:
        hyrom.hyrom_destroy(ctx)
    ctx = hyrom.hyrom_init(cfg, q0d)
    try:
        g = torch.zeros(cfg.ndof, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J = hyrom.hyrom_adjoint(ctx, steps, box, g)
        torch.cuda.synchronize()
        t_grad = time.perf_counter() - t0
        lam = g.cpu().numpy()
    finally:
        hyrom.hyrom_destroy(ctx)
    dtheta = []
    for i in range(8):
        th = th0.astype(complex)
        th[i] += 1e-30j
        dtheta.append(float(lam @ (W.euler_vortex_theta(n, th).imag.reshape(-1) / 1e-30)))
    return {"workload": f"euler2d_vortex_theta_{n}x{n}_k{k}_w{2 * k}_steps{steps}_box64",
            "J": J, "dJ_dtheta": dict(zip(W.VORTEX_THETA_NAMES, dtheta)),
            "forward_s": t_fwd, "gradient_s": t_grad,
            "gradient_over_forward": t_grad / t_fwd,
            "tape_bytes": 8 * cfg.ndof * 3 * (steps + 1)}


def run_reference(a):
    """The CPU oracle as the reference arm: --warmup untimed and --steps timed
    hybrid steps, each a bounded sample (the cpu_n^2 grid of the same
    workload; up to 3 more on the (2 cpu_n)^2 grid for the size fit of
    cpu_oracle_rate), steps/s extrapolated to the benchmark grid."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    _, cfg = workload(a)
    steps = max(1, a.steps)
    cb = cpu_oracle_rate(a, steps=steps, warmup=a.warmup, steps_large=min(steps, 3))
    return {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": a.gpus, "steps": steps, "warmup": a.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(a, cfg),
            "cpu_baseline": {"kind": "oracle", "cores": cb["cores"], "sample": cb["sample"],
                             "value": cb["value"], "unit": UNIT},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    if a.micro == "sample_gram":
        out = micro_sample_gram(a)
    elif a.micro == "batch":
        out = {"micro": "batch", **batch_form(a)}
    elif a.micro == "full_step":
        out = {"micro": "full_step", **full_step(a)}
    elif a.micro == "implicit":
        out = {"micro": "implicit", **implicit_form(a)}
    elif a.micro == "adjoint":
        out = {"micro": "adjoint", **adjoint_form(a)}
    elif a.micro == "np_sweep":
        out = {"micro": "np_sweep", **np_sweep(a)}
    elif a.micro == "vortex512":
        out = {"micro": "vortex512", **vortex512(a)}
    elif a.micro == "rk2_vjp":
        out = {"micro": "rk2_vjp", **rk2_vjp(a)}
    else:
        out = run_reference(a) if a.impl == "reference" else run_ours(a)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
