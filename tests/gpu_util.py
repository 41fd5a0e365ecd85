"""Helpers for the GPU parity tests: device arrays, bitmaps, a context
manager around hyrom_init/hyrom_destroy.  The CUDA library is built (or
found up to date) on first use."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402

_built = False


def H():
    """The binding, with the library built."""
    global _built
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01718_gb300 import build, hyrom
    if not _built:
        build.build()
        _built = True
    return hyrom


def tdtype(cfg):
    return torch.float32 if cfg.precision == W.PREC_F32 else torch.float64


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def to_bits(mask):
    """bool array over cells -> uint32 words (bit c%32 of word c/32)."""
    m = np.asarray(mask, bool).reshape(-1)
    n = m.size
    words = np.zeros((n + 31) // 32, dtype=np.uint64)
    idx = np.flatnonzero(m)
    np.bitwise_or.at(words, idx // 32, (np.uint64(1) << (idx % 32).astype(np.uint64)))
    return words.astype(np.uint32)


def from_bits(words, n):
    w = np.asarray(words).astype(np.uint64)
    bits = (w[:, None] >> np.arange(32, dtype=np.uint64)[None, :]) & np.uint64(1)
    return bits.reshape(-1)[:n].astype(bool)


def dev_bits(mask):
    return torch.as_tensor(to_bits(mask).view(np.int32), device="cuda")


def bits_of(t, n):
    return from_bits(host(t).view(np.uint32), n)


class Ctx:
    """with Ctx(cfg, q0) as (hy, ctx): ..."""

    def __init__(self, cfg, q0=None):
        self.cfg = cfg
        self.q0 = np.zeros(cfg.ndof) if q0 is None else np.asarray(q0, np.float64).reshape(-1)

    def __enter__(self):
        self.hy = H()
        self.q0d = dev(self.q0)
        self.ctx = self.hy.hyrom_init(self.cfg, self.q0d)
        return self.hy, self.ctx

    def __exit__(self, *a):
        self.hy.hyrom_destroy(self.ctx)
        return False


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)
