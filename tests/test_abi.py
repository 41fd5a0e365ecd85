"""The C ABI without a GPU: libhyrom.so builds (nvcc cross-compiles for
sm_103a), loads, exports every function include/hyrom.h declares, and the
binding's ctypes structures have the C layout (checked against a C program
compiled with the host compiler)."""
import ctypes
import os
import re
import shutil
import subprocess

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
