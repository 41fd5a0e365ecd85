"""The multi-GPU form of bench.py is N independent replicas: every rank times
the same number of steps, the job's time is the slowest rank's, and the
rate is the total over ranks.  Checked here with two gloo ranks on the CPU;
the reference arm does its work on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 if rank == 0 else 150.0            # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, world, "cpu")
    rate = bench.whole_job_rate(10, world, ms_max)
    dist.destroy_process_group()
    q.put((rank, ms_max, rate))


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_steps():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms_max, rate in out:
        assert ms_max == 150.0
        assert rate == pytest.approx(2 * 10 / 0.150)


def test_reference_arm_works_on_rank_zero_only(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference"])
    assert bench.run_reference(bench.parse()) is None


def test_single_rank_rate():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0, 1, "cpu") == 42.0
    assert bench.whole_job_rate(10, 1, 500.0) == pytest.approx(20.0)


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference on a tiny oracle sample prints one JSON line
    with the contract's keys, the reference arm's e2e and cpu_baseline, and
    the same metric and workload as the GPU arm."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--cpu-n", "8"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    for key in ("value", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["config"]["workload"].startswith("euler2d_oblique_shock_2048x2048")
