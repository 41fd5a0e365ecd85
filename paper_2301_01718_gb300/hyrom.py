"""ctypes binding of libhyrom (include/hyrom.h): the same entry points, with
argument marshalling only.  Every computation runs in the CUDA library; if
the library is not built this module refuses to load.

Pointers may be given as ints (raw addresses), torch tensors (data_ptr())
or numpy arrays (host memory).  A non-OK status raises HyromError carrying
hyrom_last_error().
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhyrom.so")

HYROM_OK, HYROM_EINVAL, HYROM_ENOMEM, HYROM_ECUDA = 0, 1, 2, 3
HYROM_ENOTCONV, HYROM_ESTATE, HYROM_ECAP, HYROM_ETIMEOUT = 4, 5, 6, 7
HYROM_ERANK, HYROM_ENONPHYS = 8, 9
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ESTATE",
                6: "ECAP", 7: "ETIMEOUT", 8: "ERANK", 9: "ENONPHYS"}
PREC_F64, PREC_F32 = 0, 1


class HyromConfig(C.Structure):
    _fields_ = [
        ("pde", C.c_int32), ("scheme", C.c_int32), ("precision", C.c_int32),
        ("nx", C.c_int32), ("ny", C.c_int32), ("bc", C.c_int32 * 4),
        ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double), ("gamma", C.c_double),
        ("shock_n", C.c_double * 2), ("shock_d0", C.c_double), ("shock_speed", C.c_double),
        ("shock_pre", C.c_double * 4), ("shock_post", C.c_double * 4),
        ("w", C.c_int32), ("m", C.c_int32), ("z", C.c_int32), ("n_p", C.c_int32),
        ("sel_mode", C.c_int32), ("halo", C.c_int32), ("jmax", C.c_int32),
        ("jmax_f", C.c_int32), ("newton_max", C.c_int32), ("n_filt", C.c_int32),
        ("filt_orders", C.c_int32 * 3), ("regress_rows", C.c_int32),
        ("reduced_prec", C.c_int32), ("odeim_batch", C.c_int32),
        ("delta", C.c_double), ("top_frac", C.c_double), ("eps_y", C.c_double),
        ("eps_f", C.c_double), ("pod_tol", C.c_double), ("pod_abs", C.c_double),
        ("tie_tol", C.c_double), ("newton_tol", C.c_double),
        ("seed", C.c_uint64),
    ]


class HyromStepInfo(C.Structure):
    _fields_ = [
        ("k", C.c_int64), ("was_full", C.c_int32), ("rebuilt", C.c_int32), ("J", C.c_int32),
        ("n_s", C.c_int32), ("n_g", C.c_int32), ("n_p", C.c_int32), ("m_eff", C.c_int32),
        ("filt_passes", C.c_int32), ("newton_fail", C.c_int32), ("pad", C.c_int32),
        ("dy_last", C.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


class HyromError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hyrom {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def make_config(src) -> HyromConfig:
    """Fill a HyromConfig from any object (or dict) with fields of the same
    names, e.g. workloads.ArConfig."""
    get = src.get if isinstance(src, dict) else (lambda k, d=None: getattr(src, k, d))
    c = HyromConfig()
    for name, ctype in HyromConfig._fields_:
        if name == "n_filt":
            continue
        val = get(name, None)
        if val is None:
            continue
        if name == "filt_orders":
            orders = list(val)
            c.n_filt = len(orders)
            for i, o in enumerate(orders):
                c.filt_orders[i] = int(o)
        elif hasattr(ctype, "_length_"):
            arr = getattr(c, name)
            for i, v in enumerate(val):
                arr[i] = v
        else:
            setattr(c, name, val)
    return c


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return C.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"cannot pass {type(x)} as a pointer")


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhyrom.so is not built (run paper_2301_01718_gb300.build.build()); "
                           "there is no fallback implementation")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, st = C.c_void_p, C.c_int32, C.c_int64, C.c_int
    sigs = {
        "hyrom_init": (st, [C.POINTER(HyromConfig), vp, C.c_int, vp, C.POINTER(vp)]),
        "hyrom_destroy": (None, [vp]),
        "hyrom_last_error": (C.c_char_p, [vp]),
        "hyrom_device_bytes": (C.c_size_t, [vp]),
        "hyrom_kernel_launches": (C.c_uint64, []),
        "hyrom_profile": (st, [vp, C.c_int]),
        "hyrom_odeim_counters": (st, [vp, C.POINTER(i64)]),
        "hyrom_eig_sweeps": (st, [vp, C.POINTER(C.c_int32)]),
        "hyrom_stage_times": (st, [vp, C.POINTER(C.c_double), C.POINTER(i64)]),
        "hyrom_advance": (st, [vp, C.POINTER(HyromStepInfo)]),
        "hyrom_update_basis": (st, [vp, C.POINTER(HyromStepInfo)]),
        "hyrom_step": (st, [vp, C.POINTER(HyromStepInfo)]),
        "hyrom_sample": (st, [vp, vp, i64, C.POINTER(i64), vp]),
        "hyrom_get_state": (st, [vp, vp, C.c_int]),
        "hyrom_set_state": (st, [vp, vp, C.c_int]),
        "hyrom_get_basis": (st, [vp, vp, C.POINTER(i32), vp, vp, C.POINTER(i32)]),
        "hyrom_stage_full_step": (st, [vp, vp, vp, i64]),
        "hyrom_stage_partial_step": (st, [vp, vp, vp, vp, i64]),
        "hyrom_stage_gappy": (st, [vp, vp, i32, vp, i32, vp, vp, vp]),
        "hyrom_stage_reconstruct": (st, [vp, vp, i32, vp, vp, vp, vp]),
        "hyrom_stage_filter": (st, [vp, vp, vp, i64, C.POINTER(i32)]),
        "hyrom_stage_cell_error": (st, [vp, vp, vp, vp, i32, vp, vp]),
        "hyrom_stage_select": (st, [vp, vp, vp, C.POINTER(i32)]),
        "hyrom_stage_pod": (st, [vp, vp, i32, vp, vp, vp, C.POINTER(i32)]),
        "hyrom_stage_odeim": (st, [vp, vp, i32, i32, vp]),
        "hyrom_stage_masks": (st, [vp, vp, vp, i32, vp, vp, C.POINTER(i32)]),
        "hyrom_stage_gappy_rows": (st, [vp, vp, i32, vp, i32, vp, vp, vp]),
        "hyrom_gappy_static": (st, [vp, i64, i32, vp, i32, vp, vp, i32, vp, vp, C.c_char_p, i32]),
        "hyrom_selftest_math": (st, [i32, vp, vp, i64, vp]),
        "hyrom_probe_fp64": (st, [vp, i32, i32, vp]),
        "hyrom_stage_muscl_residual": (st, [vp, vp, vp, vp, i64, vp]),
        "hyrom_stage_muscl_jvp": (st, [vp, vp, vp, i64, i32, vp]),
        "hyrom_stage_muscl_step": (st, [vp, vp, vp, vp, vp, i64]),
        "hyrom_stage_muscl_filter": (st, [vp, vp, vp, vp, i64, C.POINTER(i32)]),
        "hyrom_stage_rk2_vjp": (st, [vp, vp, vp, vp, vp, i64, vp]),
        "hyrom_reduced_vjp_work_doubles": (C.c_size_t, [i32, i32]),
        "hyrom_stage_reduced_vjp": (st, [vp, vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp,
                                         vp]),
        "hyrom_batch_create": (st, [C.POINTER(vp), i32, i32, C.POINTER(vp)]),
        "hyrom_init_batch": (st, [C.POINTER(HyromConfig), C.POINTER(vp), i32, i32, i32,
                                  C.POINTER(vp), C.POINTER(vp)]),
        "hyrom_save": (st, [vp, C.c_char_p]),
        "hyrom_adjoint": (st, [vp, i32, C.POINTER(i32), C.POINTER(C.c_double), vp]),
        "hyrom_stage_pod_vjp": (st, [vp, vp, i32, vp, vp, i32, vp, vp]),
        "hyrom_stage_filter_vjp": (st, [vp, vp, vp, i64, vp]),
        "hyrom_load": (st, [vp, C.c_char_p]),
        "hyrom_batch_step": (st, [vp, i32, C.POINTER(HyromStepInfo), C.POINTER(i32)]),
        "hyrom_batch_threads": (i32, [vp]),
        "hyrom_batch_set_mode": (st, [vp, i32]),
        "hyrom_batch_tuning": (i32, [vp, C.POINTER(i32), C.POINTER(C.c_float), i32]),
        "hyrom_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("hyrom_")]


def _check(ctx, s):
    if s != HYROM_OK:
        msg = lib().hyrom_last_error(ctx).decode() if ctx else "invalid argument"
        raise HyromError(s, msg)


# ---- entry points (same names as the C ABI) ---------------------------------

def hyrom_init(cfg, q0, q0_on_host=False, stream=None):
    c = cfg if isinstance(cfg, HyromConfig) else make_config(cfg)
    out = C.c_void_p()
    s = lib().hyrom_init(C.byref(c), _ptr(q0), int(bool(q0_on_host)), _ptr(stream), C.byref(out))
    _check(None, s)
    return out.value


def hyrom_destroy(ctx):
    lib().hyrom_destroy(ctx)


def hyrom_last_error(ctx):
    return lib().hyrom_last_error(ctx).decode()


def hyrom_device_bytes(ctx):
    return lib().hyrom_device_bytes(ctx)


def hyrom_kernel_launches():
    return lib().hyrom_kernel_launches()


STAGES = ["full", "partial", "gappy", "recon", "filter", "select", "gram", "eig", "formphi",
          "odeim", "masks", "deim", "od_init", "od_probe", "od_screen", "od_exact",
          "od_update", "od_list", "snormal"]


def hyrom_profile(ctx, on=True):
    _check(ctx, lib().hyrom_profile(ctx, int(bool(on))))


def hyrom_odeim_counters(ctx):
    out = (C.c_int64 * 4)()
    _check(ctx, lib().hyrom_odeim_counters(ctx, out))
    return {"deim_rows": out[0], "odeim_full_bound": out[1], "odeim_exact": out[2],
            "odeim_steps": out[3]}


def hyrom_eig_sweeps(ctx):
    out = (C.c_int32 * 2)()
    _check(ctx, lib().hyrom_eig_sweeps(ctx, out))
    return {"pod": out[0], "odeim": out[1]}


def hyrom_stage_times(ctx):
    """{stage name: (total ms, intervals)}"""
    ms = (C.c_double * len(STAGES))()
    n = (C.c_int64 * len(STAGES))()
    _check(ctx, lib().hyrom_stage_times(ctx, ms, n))
    return {s: (ms[i], n[i]) for i, s in enumerate(STAGES)}


def _info_call(fn, ctx, allow=()):
    info = HyromStepInfo()
    s = fn(ctx, C.byref(info))
    if s not in allow:
        _check(ctx, s)
    d = info.as_dict()
    d["status"] = s
    return d


# HYROM_ERANK reports a completed step (fewer modes than m, or a
# rank-deficient sampled basis): returned in info["status"], not raised.
def hyrom_advance(ctx):
    return _info_call(lib().hyrom_advance, ctx, allow=(HYROM_OK,))


def hyrom_update_basis(ctx):
    return _info_call(lib().hyrom_update_basis, ctx, allow=(HYROM_OK, HYROM_ERANK))


def hyrom_step(ctx):
    return _info_call(lib().hyrom_step, ctx, allow=(HYROM_OK, HYROM_ERANK))


def hyrom_sample(ctx, idx_dev=None, cap=0, bitmap_dev=None):
    n = C.c_int64()
    _check(ctx, lib().hyrom_sample(ctx, _ptr(idx_dev), int(cap), C.byref(n), _ptr(bitmap_dev)))
    return n.value


def hyrom_get_state(ctx, q, on_host=False):
    _check(ctx, lib().hyrom_get_state(ctx, _ptr(q), int(bool(on_host))))


def hyrom_set_state(ctx, q, on_host=False):
    _check(ctx, lib().hyrom_set_state(ctx, _ptr(q), int(bool(on_host))))


def hyrom_get_basis(ctx, phi=None, psi=None, points=None):
    me, npp = C.c_int32(), C.c_int32()
    _check(ctx, lib().hyrom_get_basis(ctx, _ptr(phi), C.byref(me), _ptr(psi), _ptr(points),
                                      C.byref(npp)))
    return me.value, npp.value


def hyrom_stage_full_step(ctx, q_prev, q_out, k):
    _check(ctx, lib().hyrom_stage_full_step(ctx, _ptr(q_prev), _ptr(q_out), int(k)))


def hyrom_stage_partial_step(ctx, q_prev, q_io, s_hat, k):
    _check(ctx, lib().hyrom_stage_partial_step(ctx, _ptr(q_prev), _ptr(q_io), _ptr(s_hat), int(k)))


def hyrom_stage_gappy(ctx, phi, m, points, n_p, v, psi, y_out):
    _check(ctx, lib().hyrom_stage_gappy(ctx, _ptr(phi), int(m), _ptr(points), int(n_p), _ptr(v),
                                        _ptr(psi), _ptr(y_out)))


def hyrom_stage_reconstruct(ctx, phi, m, y, psi, s_hat, q_io):
    _check(ctx, lib().hyrom_stage_reconstruct(ctx, _ptr(phi), int(m), _ptr(y), _ptr(psi),
                                              _ptr(s_hat), _ptr(q_io)))


def hyrom_stage_filter(ctx, q_io, q_prev, k):
    p = C.c_int32()
    _check(ctx, lib().hyrom_stage_filter(ctx, _ptr(q_io), _ptr(q_prev), int(k), C.byref(p)))
    return p.value


def hyrom_stage_cell_error(ctx, g, psi, phi, m, y, eps_out):
    _check(ctx, lib().hyrom_stage_cell_error(ctx, _ptr(g), _ptr(psi), _ptr(phi), int(m), _ptr(y),
                                             _ptr(eps_out)))


def hyrom_stage_select(ctx, eps, g_bitmap):
    n = C.c_int32()
    _check(ctx, lib().hyrom_stage_select(ctx, _ptr(eps), _ptr(g_bitmap), C.byref(n)))
    return n.value


def hyrom_stage_pod(ctx, window, w, psi, phi_out, sigma_out=None):
    me = C.c_int32()
    _check(ctx, lib().hyrom_stage_pod(ctx, _ptr(window), int(w), _ptr(psi), _ptr(phi_out),
                                      _ptr(sigma_out), C.byref(me)))
    return me.value


def hyrom_stage_odeim(ctx, phi, m, n_p, points_out):
    _check(ctx, lib().hyrom_stage_odeim(ctx, _ptr(phi), int(m), int(n_p), _ptr(points_out)))


def hyrom_stage_gappy_rows(ctx, phi, m, cells, n_cells, v, psi, y_out):
    _check(ctx, lib().hyrom_stage_gappy_rows(ctx, _ptr(phi), int(m), _ptr(cells), int(n_cells),
                                             _ptr(v), _ptr(psi), _ptr(y_out)))


def hyrom_stage_masks(ctx, g_bitmap, points, n_p, s_hat, s_tilde):
    n = C.c_int32()
    _check(ctx, lib().hyrom_stage_masks(ctx, _ptr(g_bitmap), _ptr(points), int(n_p), _ptr(s_hat),
                                        _ptr(s_tilde), C.byref(n)))
    return n.value


def hyrom_stage_muscl_residual(ctx, q, q_prev, q_prev2, k, r_out):
    _check(ctx, lib().hyrom_stage_muscl_residual(ctx, _ptr(q), _ptr(q_prev), _ptr(q_prev2),
                                                 int(k), _ptr(r_out)))


def hyrom_stage_muscl_jvp(ctx, q, v, k, bdf2, jv_out):
    _check(ctx, lib().hyrom_stage_muscl_jvp(ctx, _ptr(q), _ptr(v), int(k), int(bool(bdf2)),
                                            _ptr(jv_out)))


def hyrom_stage_muscl_step(ctx, q_prev2, q_prev, q_io, s_hat, k):
    _check(ctx, lib().hyrom_stage_muscl_step(ctx, _ptr(q_prev2), _ptr(q_prev), _ptr(q_io),
                                             _ptr(s_hat), int(k)))


def hyrom_stage_muscl_filter(ctx, q_io, q_prev, q_prev2, k):
    p = C.c_int32()
    _check(ctx, lib().hyrom_stage_muscl_filter(ctx, _ptr(q_io), _ptr(q_prev), _ptr(q_prev2),
                                               int(k), C.byref(p)))
    return p.value


def hyrom_gappy_static(phi, ndof, m, points, n_p, v, psi, precision, y_out, stream=None):
    """Allocation-free gappy coordinates: no context, scratch in a static
    device array.  Raises HyromError with the library's reason on failure."""
    err = C.create_string_buffer(256)
    s = lib().hyrom_gappy_static(_ptr(phi), int(ndof), int(m), _ptr(points), int(n_p), _ptr(v),
                                 _ptr(psi), int(precision), _ptr(y_out), _ptr(stream), err,
                                 len(err))
    if s != HYROM_OK:
        raise HyromError(s, err.value.decode())


def hyrom_selftest_math(which, x, y, stream=None):
    """The library's FP64 reciprocal (which=0) or reciprocal square root
    (which=1) of the device doubles x into y, on `stream`."""
    s = lib().hyrom_selftest_math(int(which), _ptr(x), _ptr(y), int(x.numel()), _ptr(stream))
    if s != HYROM_OK:
        raise HyromError(s, "hyrom_selftest_math")


def hyrom_probe_fp64(out, blocks, iters, stream=None):
    """Enqueue the FP64 FMA loop (blocks * 256 * 16 * iters flops)."""
    s = lib().hyrom_probe_fp64(_ptr(out), int(blocks), int(iters), _ptr(stream))
    if s != HYROM_OK:
        raise HyromError(s, "hyrom_probe_fp64")


def hyrom_batch_create(ctxs, threads=0):
    """A batch over the contexts `ctxs` (kept by the caller) stepped by
    `threads` host threads (0: half the host's hardware threads, 1..8)."""
    n = len(ctxs)
    arr = (C.c_void_p * max(n, 1))(*ctxs)
    out = C.c_void_p()
    s = lib().hyrom_batch_create(arr, int(n), int(threads), C.byref(out))
    if s != HYROM_OK:
        raise HyromError(s, "hyrom_batch_create")
    return out.value


def hyrom_batch_step(batch, n, nsteps=1, ctxs=None):
    """nsteps hybrid steps of each of the n instances.  Returns (status per
    instance, info dict of each instance's last step); raises HyromError
    naming the failing instances (with their last error messages when the
    contexts `ctxs` are given) when any status is not OK."""
    infos = (HyromStepInfo * n)()
    st = (C.c_int32 * n)()
    s = lib().hyrom_batch_step(batch, int(nsteps), infos, st)
    status = list(st)
    if s != HYROM_OK:
        bad = [i for i, v in enumerate(status) if v]
        why = [f"{i}: {hyrom_last_error(ctxs[i])}" for i in bad] if ctxs else bad
        raise HyromError(s, f"instances failed: {why}")
    return status, [i.as_dict() for i in infos]


def hyrom_init_batch(cfgs, q0s, q0_on_host=False, threads=0):
    """Contexts (each on a stream of its own, owned by the batch) and a batch
    over them.  q0s: device tensors or addresses (host arrays with
    q0_on_host).  Returns (batch, [contexts])."""
    n = len(cfgs)
    carr = (HyromConfig * n)(*[c if isinstance(c, HyromConfig) else make_config(c) for c in cfgs])
    qarr = (C.c_void_p * n)(*[_ptr(q).value for q in q0s])
    ctxs = (C.c_void_p * n)()
    out = C.c_void_p()
    s = lib().hyrom_init_batch(carr, qarr, int(bool(q0_on_host)), n, int(threads), ctxs,
                               C.byref(out))
    if s != HYROM_OK:
        raise HyromError(s, "hyrom_init_batch")
    return out.value, [ctxs[i] for i in range(n)]


def hyrom_adjoint(ctx, steps, box, dJdq0):
    """J and dJ/dq0 (into the device array dJdq0) of the time-integrated box
    pressure over `steps` steps from the context's k = 0; returns J."""
    b = (C.c_int32 * 4)(*[int(v) for v in box])
    J = C.c_double()
    _check(ctx, lib().hyrom_adjoint(ctx, int(steps), b, C.byref(J), _ptr(dJdq0)))
    return J.value


def hyrom_stage_pod_vjp(ctx, window, w, psi, lphi, m, lam_window, lpsi_out):
    _check(ctx, lib().hyrom_stage_pod_vjp(ctx, _ptr(window), int(w), _ptr(psi), _ptr(lphi),
                                          int(m), _ptr(lam_window), _ptr(lpsi_out)))


def hyrom_stage_filter_vjp(ctx, q, q_prev, k, lam_io):
    _check(ctx, lib().hyrom_stage_filter_vjp(ctx, _ptr(q), _ptr(q_prev), int(k), _ptr(lam_io)))


def hyrom_save(ctx, path):
    _check(ctx, lib().hyrom_save(ctx, os.fsencode(path)))


def hyrom_load(ctx, path):
    _check(ctx, lib().hyrom_load(ctx, os.fsencode(path)))


def hyrom_batch_threads(batch):
    return lib().hyrom_batch_threads(batch)


HYROM_BATCH_STREAMS, HYROM_BATCH_FUSED = 0, 1


def hyrom_batch_set_mode(batch, mode):
    """HYROM_BATCH_STREAMS (each instance's steps whole on its own stream) or
    HYROM_BATCH_FUSED (all instances' oversampling loops as one launch per
    pass under a CUDA graph)."""
    s = lib().hyrom_batch_set_mode(batch, int(mode))
    if s != HYROM_OK:
        raise HyromError(s, "hyrom_batch_set_mode")


def hyrom_batch_tuning(batch):
    """The fused form's autotuner: (rows per CTA in use, 0 while timing;
    measured ms per greedy step of each candidate, -1 if untimed)."""
    r = C.c_int32()
    ms = (C.c_float * 8)()
    n = lib().hyrom_batch_tuning(batch, C.byref(r), ms, 8)
    return r.value, [ms[i] for i in range(max(n, 0))]


def hyrom_batch_destroy(batch):
    lib().hyrom_batch_destroy(batch)


def hyrom_stage_rk2_vjp(ctx, q_prev, lam_out, lam_in, s_hat, k, work):
    """lam_in = (d q_k / d q_prev)^T lam_out for the SSP-RK2 step k (partial on
    s_hat, or full when s_hat is None); work: 3 N doubles of device scratch."""
    _check(ctx, lib().hyrom_stage_rk2_vjp(ctx, _ptr(q_prev), _ptr(lam_out), _ptr(lam_in),
                                          _ptr(s_hat), int(k), _ptr(work)))


def hyrom_reduced_vjp_work_doubles(m, n_rows):
    return lib().hyrom_reduced_vjp_work_doubles(int(m), int(n_rows))


def hyrom_stage_reduced_vjp(ctx, phi, m, rows, n_rows, v, psi, y, s_hat, lam, lam_v, lam_psi,
                            lam_phi, work):
    """The reduced step's adjoint: lam_v, lam_psi, lam_phi from lam (FP64)."""
    _check(ctx, lib().hyrom_stage_reduced_vjp(ctx, _ptr(phi), int(m), _ptr(rows), int(n_rows),
                                              _ptr(v), _ptr(psi), _ptr(y), _ptr(s_hat),
                                              _ptr(lam), _ptr(lam_v), _ptr(lam_psi),
                                              _ptr(lam_phi), _ptr(work)))
