"""GB300 (sm_103a) implementation of the hybrid-snapshot adaptive ROM of
Zucatti & Zahr: CUDA kernels behind the C ABI in include/hyrom.h
(libhyrom.so), with a thin ctypes binding in `hyrom`.

    from paper_2301_01718_gb300 import hyrom
    ctx = hyrom.hyrom_init(cfg, q0_device_tensor)
    info = hyrom.hyrom_step(ctx)
"""
from . import hyrom  # noqa: F401

__all__ = ["hyrom"]
