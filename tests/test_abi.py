"""The C ABI without a GPU: libhyrom.so builds (nvcc cross-compiles for
sm_103a), loads, exports every function include/hyrom.h declares, and the
binding's ctypes structures have the C layout (checked against a C program
compiled with the host compiler)."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hyrom.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hyrom_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2301_01718_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_2301_01718_gb300 import hyrom
    for n in _declared():
        assert hasattr(hyrom, n), n


def test_struct_layout_matches_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2301_01718_gb300 import hyrom
    fields_c = [f for f, _ in hyrom.HyromConfig._fields_]
    fields_i = [f for f, _ in hyrom.HyromStepInfo._fields_]
    prog = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){",
            'printf("%zu %zu\\n", sizeof(hyrom_config), sizeof(hyrom_step_info));']
    prog += [f'printf("%zu\\n", offsetof(hyrom_config, {f}));' for f in fields_c]
    prog += [f'printf("%zu\\n", offsetof(hyrom_step_info, {f}));' for f in fields_i]
    prog += ["return 0;}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog))
    exe = tmp_path / "layout"
    subprocess.run([cc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    sz_c, sz_i = int(out[0]), int(out[1])
    assert sz_c == ctypes.sizeof(hyrom.HyromConfig)
    assert sz_i == ctypes.sizeof(hyrom.HyromStepInfo)
    offs = [int(x) for x in out[2:]]
    want = [getattr(hyrom.HyromConfig, f).offset for f in fields_c] + \
           [getattr(hyrom.HyromStepInfo, f).offset for f in fields_i]
    assert offs == want


def test_make_config_fills_every_field():
    import workloads as W
    from paper_2301_01718_gb300 import hyrom
    q0, cfg, _ = W.euler_oblique_shock(n=64, k=4)
    c = hyrom.make_config(cfg)
    assert (c.nx, c.ny, c.w, c.m, c.n_p) == (64, 64, 8, 4, 8)
    assert list(c.bc) == list(cfg.bc)
    assert list(c.shock_post) == list(cfg.shock_post)
    assert c.n_filt == 3 and list(c.filt_orders) == [1, 2, 3]
    assert c.pod_abs == cfg.pod_abs and c.tie_tol == cfg.tie_tol


def test_batch_argument_checks_need_no_gpu(lib):
    """The batch entry points reject bad arguments before any CUDA call."""
    from paper_2301_01718_gb300 import hyrom
    L = hyrom.lib()
    out = ctypes.c_void_p()
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.hyrom_batch_create(arr, 0, 0, ctypes.byref(out)) == hyrom.HYROM_EINVAL
    assert L.hyrom_batch_create(arr, 2, 0, ctypes.byref(out)) == hyrom.HYROM_EINVAL
    assert L.hyrom_batch_create(None, 1, 0, ctypes.byref(out)) == hyrom.HYROM_EINVAL
    first_null = (ctypes.c_void_p * 2)(None, 0x1000)      # rejected before any use
    assert L.hyrom_batch_create(first_null, 2, 0, ctypes.byref(out)) == hyrom.HYROM_EINVAL
    assert out.value is None
    assert L.hyrom_batch_step(None, 1, None, None) == hyrom.HYROM_EINVAL
    assert L.hyrom_batch_threads(None) == 0
    assert L.hyrom_batch_set_mode(None, hyrom.HYROM_BATCH_FUSED) == hyrom.HYROM_EINVAL
    assert L.hyrom_batch_tuning(None, None, None, 0) == -1
    L.hyrom_batch_destroy(None)


def test_batch_workload_recipe():
    """The batching form's instances: grids log-uniform in [128, 1024], k in
    [8, 48] with w = n_p = 2k, sample fractions in [2 %, 20 %], Mach in
    [0.3, 2.0]; reproducible from the seed."""
    import workloads as W
    a = W.euler_batch()
    b = W.euler_batch()
    assert len(a) == 64
    for (qa, ca), (qb, cb) in zip(a[:4], b[:4]):
        assert ca == cb and np.array_equal(qa, qb)
    n = np.array([c.nx for _, c in a])
    k = np.array([c.m for _, c in a])
    assert n.min() >= 128 and n.max() <= 1024 and len(set(n)) > 40
    assert k.min() >= 8 and k.max() <= 48 and len(set(k)) > 20
    assert all(c.w == 2 * c.m and c.n_p == 2 * c.m and c.nx == c.ny for _, c in a)
    assert all(0.02 <= c.top_frac <= 0.20 for _, c in a)
    # log-uniform sides: about half the instances below sqrt(128 * 1024)
    assert 20 <= (n < 362).sum() <= 44
