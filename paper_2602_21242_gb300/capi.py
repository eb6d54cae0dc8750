"""ctypes binding of liblbm.so -- the C ABI of include/lbm.h, same names.

Argument marshalling only: every computation runs in the library's CUDA
kernels. If the library cannot be found or built, loading raises
``RuntimeError``; there is no Python or CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LBM_LBGK, LBM_OREG, LBM_OREG_PARTIAL, LBM_OREG_COMPLETE, LBM_OREG_COMPLETE_NEQ, LBM_LBGK_POLY = 0, 1, 2, 3, 4, 5
LBM_F64, LBM_F32_SHIFT, LBM_F16_SHIFT, LBM_F64_DF = 0, 1, 2, 3
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6

STATUS_NAMES = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_ENONFINITE",
                -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE"}
MODELS = {"lbgk": LBM_LBGK, "oreg": LBM_OREG, "partial": LBM_OREG_PARTIAL, "complete": LBM_OREG_COMPLETE,
          "complete_neq": LBM_OREG_COMPLETE_NEQ, "lbgk_poly": LBM_LBGK_POLY}
PRECS = {"f64": LBM_F64, "f32": LBM_F32_SHIFT, "f16": LBM_F16_SHIFT, "f64df": LBM_F64_DF}

_lock = threading.Lock()
_lib = None

_i, _d, _p, _ll = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong
_pll = ctypes.POINTER(ctypes.c_longlong)
_pd = ctypes.POINTER(ctypes.c_double)
_SIGNATURES = {
    "lbm_version": ([], _i),
    "lbm_layout": ([_i, _i, _i, _pll, _pll, _pll], _i),
    "lbm_create": ([_i, _i, _d, _d, _i, ctypes.POINTER(_p)], _i),
    "lbm_create_ex": ([_i, _i, _d, _d, _i, _i, _p, _p, ctypes.POINTER(_p)], _i),
    "lbm_destroy": ([_p], _i),
    "lbm_set_stream": ([_p, _p], _i),
    "lbm_init": ([_p, _p, _p, _p], _i),
    "lbm_step": ([_p, _i], _i),
    "lbm_set_diagnostics_interval": ([_p, _i], _i),
    "lbm_set_walls": ([_p, _p, _pll], _i),
    "lbm_step_diagnostics": ([_p, _pd, _pll], _i),
    "lbm_moments": ([_p, _p, _p, _p], _i),
    "lbm_diagnostics": ([_p, _pd], _i),
    "lbm_get_state": ([_p, _p], _i),
    "lbm_set_state": ([_p, _p], _i),
    "lbm_halo_bytes": ([_p, _pll], _i),
    "lbm_halo_pack": ([_p, _p, _p], _i),
    "lbm_halo_unpack": ([_p, _p, _p], _i),
    "lbm_time": ([_p, _pll], _i),
    "lbm_run_host": ([_p, _p, _p, _p, _i, _p, _p, _p, _pd], _i),
    "lbm_sync": ([_p], _i),
    "lbm_measure_peak": ([_i, _pd], _i),
    "lbm_selftest_timeout": ([_i, _pd], _i),
    "lbm_selftest_fp64": ([_i, _pd, _ll, _pd], _i),
    "lbm_selftest_fp64_emu": ([_i, _pd, _pd, _ll, _pd, _pd], _i),
    "lbm_selftest_collide_f64": ([_i, _i, _d, _d, _pd, _ll, _pd, _pd], _i),
    "lbm_vjp": ([_p, _i, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p], _i),
    "lbm_vjp_forward": ([_p, _i, _i, _p, _p, _p], _i),
    "lbm_vjp_ex": ([_p, _i, _i, _p, _p, _p, _p, _p, _p, _p, _p, _p, _i], _i),
    "lbm_set_launch": ([_p, _i, _i, _i], _i),
    "lbm_set_launch_ex": ([_p, _i, _i, _i, _i], _i),
    "lbm_get_launch_ex": ([_p, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
    "lbm_step_noalloc": ([_i, _i, _d, _d, _i, _p, _p, _p, _p], _i),
    "lbm_get_launch": ([_p, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
    "lbm_last_error": ([_p], ctypes.c_char_p),
    "lbm_batch_create": ([_i, _p, _p, _p, _p, _i, _i, _p, ctypes.POINTER(_p)], _i),
    "lbm_batch_destroy": ([_p], _i),
    "lbm_batch_set_launch": ([_p, _i, _i, _i], _i),
    "lbm_batch_get_launch": ([_p, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
    "lbm_batch_set_launch_ex": ([_p, _i, _i, _i, _i], _i),
    "lbm_batch_get_launch_ex": ([_p] + [ctypes.POINTER(_i)] * 5, _i),
    "lbm_batch_set_mode": ([_p, _i], _i),
    "lbm_batch_set_diagnostics_interval": ([_p, _i], _i),
    "lbm_batch_init": ([_p, _p, _p, _p], _i),
    "lbm_batch_get_state": ([_p, _i, _p], _i),
    "lbm_batch_set_state": ([_p, _i, _p], _i),
    "lbm_batch_moments": ([_p, _p, _p, _p], _i),
    "lbm_batch_step": ([_p, _i], _i),
    "lbm_batch_step_diagnostics": ([_p, _pd, _pll], _i),
    "lbm_batch_diagnostics": ([_p, _pd], _i),
    "lbm_batch_info": ([_p, _pll, _pll, _pll], _i),
    "lbm_batch_sync": ([_p], _i),
    "lbm_batch_last_error": ([_p], ctypes.c_char_p),
}
LBM_BATCH_GRAPH, LBM_BATCH_PERSISTENT = 0, 1


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load liblbm.so (building it first if it is absent or stale and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            try:
                path = _build.build()
            except RuntimeError:
                if not os.path.exists(path):
                    raise
        if not os.path.exists(path):
            raise RuntimeError(f"liblbm.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def last_error(ctx=None) -> str:
    msg = load().lbm_last_error(ctx)
    return msg.decode() if msg else ""


def check(status: int, ctx=None) -> int:
    if status != LBM_OK:
        raise LBMError(status, last_error(ctx))
    return status


# ---------------------------------------------------------------- thin wrappers (same names as the ABI)

def lbm_version() -> int:
    return load().lbm_version()


def lbm_layout(nx: int, ny: int, prec: int):
    pitch, plane, nbytes = _ll(), _ll(), _ll()
    check(load().lbm_layout(nx, ny, prec, ctypes.byref(pitch), ctypes.byref(plane), ctypes.byref(nbytes)))
    return pitch.value, plane.value, nbytes.value


def lbm_create(nx: int, ny: int, theta: float, tau: float, model: int):
    ctx = _p()
    check(load().lbm_create(nx, ny, theta, tau, model, ctypes.byref(ctx)))
    return ctx


def lbm_create_ex(nx: int, ny: int, theta: float, tau: float, model: int, prec: int, stream: int = 0,
                  pop_buffers: int = 0):
    ctx = _p()
    check(load().lbm_create_ex(nx, ny, theta, tau, model, prec, stream or None, pop_buffers or None,
                               ctypes.byref(ctx)))
    return ctx


def lbm_destroy(ctx) -> None:
    check(load().lbm_destroy(ctx))


def lbm_set_stream(ctx, stream: int) -> None:
    check(load().lbm_set_stream(ctx, stream or None), ctx)


def lbm_init(ctx, d_rho: int, d_ux: int, d_uy: int) -> None:
    check(load().lbm_init(ctx, d_rho, d_ux, d_uy), ctx)


def lbm_step(ctx, n: int) -> None:
    check(load().lbm_step(ctx, n), ctx)


def lbm_set_diagnostics_interval(ctx, every: int) -> None:
    check(load().lbm_set_diagnostics_interval(ctx, every), ctx)


def lbm_set_walls(ctx, mask) -> int:
    """Fullway bounce-back wall nodes from a host (ny, nx) mask (nonzero = wall); None removes them.
    Returns the number of wall nodes."""
    n = _ll()
    if mask is None:
        check(load().lbm_set_walls(ctx, None, ctypes.byref(n)), ctx)
        return int(n.value)
    m = np.ascontiguousarray(np.asarray(mask) != 0, dtype=np.uint8)
    check(load().lbm_set_walls(ctx, m.ctypes.data, ctypes.byref(n)), ctx)
    return int(n.value)


def lbm_step_diagnostics(ctx, raise_nonfinite: bool = True):
    out = (ctypes.c_double * 5)()
    t = _ll()
    s = load().lbm_step_diagnostics(ctx, out, ctypes.byref(t))
    if s != LBM_OK and (raise_nonfinite or s != LBM_ENONFINITE):
        check(s, ctx)
    return list(out), t.value, s


def lbm_moments(ctx, d_rho: int, d_ux: int, d_uy: int) -> None:
    check(load().lbm_moments(ctx, d_rho, d_ux, d_uy), ctx)


def lbm_diagnostics(ctx, raise_nonfinite: bool = True):
    out = (ctypes.c_double * 5)()
    s = load().lbm_diagnostics(ctx, out)
    if s != LBM_OK and (raise_nonfinite or s != LBM_ENONFINITE):
        check(s, ctx)
    return list(out), s


def lbm_get_state(ctx, d_f: int) -> None:
    check(load().lbm_get_state(ctx, d_f), ctx)


def lbm_set_state(ctx, d_f: int) -> None:
    check(load().lbm_set_state(ctx, d_f), ctx)


def lbm_halo_bytes(ctx) -> int:
    n = _ll()
    check(load().lbm_halo_bytes(ctx, ctypes.byref(n)), ctx)
    return n.value


def lbm_halo_pack(ctx, d_up: int, d_down: int) -> None:
    check(load().lbm_halo_pack(ctx, d_up, d_down), ctx)


def lbm_halo_unpack(ctx, d_from_below: int, d_from_above: int) -> None:
    check(load().lbm_halo_unpack(ctx, d_from_below, d_from_above), ctx)


def lbm_time(ctx) -> int:
    t = _ll()
    check(load().lbm_time(ctx, ctypes.byref(t)), ctx)
    return t.value


def lbm_run_host(ctx, h_rho0: int, h_ux0: int, h_uy0: int, n: int, h_rho: int = 0, h_ux: int = 0, h_uy: int = 0,
                 want_diag: bool = False):
    diag = (ctypes.c_double * 5)() if want_diag else None
    check(load().lbm_run_host(ctx, h_rho0, h_ux0, h_uy0, n, h_rho or None, h_ux or None, h_uy or None, diag), ctx)
    return list(diag) if want_diag else None


def lbm_sync(ctx) -> None:
    check(load().lbm_sync(ctx), ctx)


def lbm_measure_peak(kind: int) -> float:
    """FLOP/s ceiling of the current device: kind 0 = FP64 FMA, 1 = FP32 FMA."""
    v = ctypes.c_double()
    check(load().lbm_measure_peak(kind, ctypes.byref(v)))
    return v.value


def lbm_set_launch(ctx, bx: int, by: int, rows: int) -> None:
    check(load().lbm_set_launch(ctx, bx, by, rows), ctx)


def lbm_get_launch(ctx):
    bx, by, rows = _i(), _i(), _i()
    check(load().lbm_get_launch(ctx, ctypes.byref(bx), ctypes.byref(by), ctypes.byref(rows)), ctx)
    return bx.value, by.value, rows.value


def lbm_step_noalloc(nx: int, ny: int, theta: float, tau: float, model: int, d_src: int, d_dst: int,
                     d_diag5: int, stream: int = 0) -> None:
    """One fused FP64 step + diagnostics on caller buffers, with no device allocation."""
    check(load().lbm_step_noalloc(nx, ny, theta, tau, model, d_src, d_dst, d_diag5, stream or None))


# ---------------------------------------------------------------- batched form

def batch_last_error(b) -> str:
    msg = load().lbm_batch_last_error(b)
    return msg.decode() if msg else ""


def bcheck(status: int, b=None) -> int:
    if status != LBM_OK:
        raise LBMError(status, batch_last_error(b) if b else last_error(None))
    return status


def lbm_batch_create(nx, ny, theta, tau, model: int, prec: int, stream: int = 0):
    n = len(nx)
    a_nx = (ctypes.c_int * n)(*[int(v) for v in nx])
    a_ny = (ctypes.c_int * n)(*[int(v) for v in ny])
    a_th = (ctypes.c_double * n)(*[float(v) for v in theta])
    a_tau = (ctypes.c_double * n)(*[float(v) for v in tau])
    b = _p()
    bcheck(load().lbm_batch_create(n, a_nx, a_ny, a_th, a_tau, model, prec, stream or None, ctypes.byref(b)))
    return b


def lbm_batch_destroy(b) -> None:
    bcheck(load().lbm_batch_destroy(b))


def lbm_batch_set_launch(b, bx: int, by: int, rows: int) -> None:
    bcheck(load().lbm_batch_set_launch(b, bx, by, rows), b)


def lbm_batch_get_launch(b):
    v = [_i() for _ in range(4)]
    bcheck(load().lbm_batch_get_launch(b, *[ctypes.byref(x) for x in v]), b)
    return tuple(x.value for x in v)


def lbm_batch_set_launch_ex(b, kind: int, bx: int, by: int, rows: int) -> None:
    bcheck(load().lbm_batch_set_launch_ex(b, kind, bx, by, rows), b)


def lbm_batch_get_launch_ex(b):
    """(kind, bx, by, rows, ntiles)."""
    v = [_i() for _ in range(5)]
    bcheck(load().lbm_batch_get_launch_ex(b, *[ctypes.byref(x) for x in v]), b)
    return tuple(x.value for x in v)


def lbm_batch_set_mode(b, mode: int) -> None:
    bcheck(load().lbm_batch_set_mode(b, mode), b)


def lbm_batch_set_diagnostics_interval(b, every: int) -> None:
    bcheck(load().lbm_batch_set_diagnostics_interval(b, every), b)


def lbm_batch_init(b, d_rho: int, d_ux: int, d_uy: int) -> None:
    bcheck(load().lbm_batch_init(b, d_rho, d_ux, d_uy), b)


def lbm_batch_get_state(b, k: int, d_f: int) -> None:
    bcheck(load().lbm_batch_get_state(b, k, d_f), b)


def lbm_batch_set_state(b, k: int, d_f: int) -> None:
    bcheck(load().lbm_batch_set_state(b, k, d_f), b)


def lbm_batch_moments(b, d_rho: int, d_ux: int, d_uy: int) -> None:
    bcheck(load().lbm_batch_moments(b, d_rho, d_ux, d_uy), b)


def lbm_batch_step(b, n: int) -> None:
    bcheck(load().lbm_batch_step(b, n), b)


def lbm_batch_step_diagnostics(b, n_domains: int, raise_nonfinite: bool = True):
    out = (ctypes.c_double * (5 * n_domains))()
    t = _ll()
    s = load().lbm_batch_step_diagnostics(b, out, ctypes.byref(t))
    if s != LBM_OK and (raise_nonfinite or s != LBM_ENONFINITE):
        bcheck(s, b)
    return [list(out[5 * k:5 * k + 5]) for k in range(n_domains)], t.value, s


def lbm_batch_diagnostics(b, n_domains: int, raise_nonfinite: bool = True):
    out = (ctypes.c_double * (5 * n_domains))()
    s = load().lbm_batch_diagnostics(b, out)
    if s != LBM_OK and (raise_nonfinite or s != LBM_ENONFINITE):
        bcheck(s, b)
    return [list(out[5 * k:5 * k + 5]) for k in range(n_domains)], s


def lbm_batch_info(b):
    v = [_ll() for _ in range(3)]
    bcheck(load().lbm_batch_info(b, *[ctypes.byref(x) for x in v]), b)
    return tuple(x.value for x in v)


def lbm_batch_sync(b) -> None:
    bcheck(load().lbm_batch_sync(b), b)


def lbm_vjp(ctx, n: int, ckpt_every: int, d_rho0: int, d_ux0: int, d_uy0: int, g_rho: int = 0, g_ux: int = 0,
            g_uy: int = 0, g_rho0: int = 0, g_ux0: int = 0, g_uy0: int = 0) -> None:
    """Cotangents of (rho0, u0) for cotangents of the moments after n steps (device pointers, 0 = NULL)."""
    check(load().lbm_vjp(ctx, n, ckpt_every, d_rho0, d_ux0, d_uy0, g_rho or None, g_ux or None, g_uy or None,
                         g_rho0 or None, g_ux0 or None, g_uy0 or None), ctx)


LBM_VJP_REUSE_FORWARD = 1


def lbm_vjp_forward(ctx, n: int, ckpt_every: int, d_rho0: int, d_ux0: int, d_uy0: int) -> None:
    """Forward pass of lbm_vjp on its own: init from (rho0, u0) and n checkpointed steps."""
    check(load().lbm_vjp_forward(ctx, n, ckpt_every, d_rho0, d_ux0, d_uy0), ctx)


def lbm_vjp_ex(ctx, n: int, ckpt_every: int, d_rho0: int, d_ux0: int, d_uy0: int, g_rho: int = 0, g_ux: int = 0,
               g_uy: int = 0, g_rho0: int = 0, g_ux0: int = 0, g_uy0: int = 0, flags: int = 0) -> None:
    """lbm_vjp with flags (LBM_VJP_REUSE_FORWARD: reuse the checkpoints of lbm_vjp_forward)."""
    check(load().lbm_vjp_ex(ctx, n, ckpt_every, d_rho0, d_ux0, d_uy0, g_rho or None, g_ux or None, g_uy or None,
                            g_rho0 or None, g_ux0 or None, g_uy0 or None, flags), ctx)


def lbm_set_launch_ex(ctx, kind: int, bx: int, by: int, rows: int) -> None:
    check(load().lbm_set_launch_ex(ctx, kind, bx, by, rows), ctx)


def lbm_get_launch_ex(ctx):
    v = [_i() for _ in range(4)]
    check(load().lbm_get_launch_ex(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return tuple(x.value for x in v)


def lbm_selftest_fp64(op: int, x):
    """Apply FP64 helper `op` (0-2: x/2, -x/2, x/4; 3: 1/x; 4: FP32 truncation) on the GPU."""
    import numpy as np
    xs = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    out = np.empty_like(xs)
    check(load().lbm_selftest_fp64(op, xs.ctypes.data_as(_pd), xs.size, out.ctypes.data_as(_pd)), None)
    return out


def lbm_selftest_fp64_emu(op: int, a, b):
    """Integer-pipe sum (op 0) or product (op 1) of the pairs (a, b) on the GPU, and the FP64
    instruction's; returns (emu, fp64)."""
    import numpy as np
    av = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    bv = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    if av.shape != bv.shape:
        raise ValueError("a and b must have the same shape")
    emu, ref = np.empty_like(av), np.empty_like(av)
    check(load().lbm_selftest_fp64_emu(op, av.ctypes.data_as(_pd), bv.ctypes.data_as(_pd), av.size,
                                       emu.ctypes.data_as(_pd), ref.ctypes.data_as(_pd)), None)
    return emu, ref


def lbm_selftest_collide_f64(model: int, theta: float, tau: float, f, mode: int = 0):
    """FP64 collision of the nodes f (n x 9) with the kernels' arithmetic (starting in product mode
    `mode`: 0 integer, 1 integer with zeros, 2 FP64 pipe) and with every product on the FP64 pipe;
    returns (emu, ref), each n x 14 (populations, m0, jx, jy, ux, uy)."""
    import numpy as np
    fv = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1, 9))
    n = fv.shape[0]
    emu, ref = np.empty((n, 14)), np.empty((n, 14))
    check(load().lbm_selftest_collide_f64(model, mode, theta, tau, fv.ctypes.data_as(_pd), n,
                                          emu.ctypes.data_as(_pd), ref.ctypes.data_as(_pd)), None)
    return emu, ref


def lbm_selftest_timeout(which: int):
    """Run a wait that must give up; returns (status, seconds)."""
    secs = ctypes.c_double()
    s = load().lbm_selftest_timeout(which, ctypes.byref(secs))
    return s, secs.value
