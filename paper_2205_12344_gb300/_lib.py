"""Thin ctypes binding of libewh.so (include/ewh.h): argument marshalling only.

Every computation runs in the CUDA library; there is no CPU fallback.  If the
library cannot be loaded the import fails loudly.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

EWH_OK, EWH_EINVAL, EWH_ENOMEM, EWH_ECUDA, EWH_ENOTCONV, EWH_EBREAKDOWN, EWH_ETIMEOUT = range(7)
EWH_BC_DIRICHLET, EWH_BC_FREE = 0, 1
EWH_FP64, EWH_FP32_STENCIL = 0, 1


class ewh_grid_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double),
                ("order", ctypes.c_int), ("bc", ctypes.c_int * 6), ("precision", ctypes.c_int),
                ("cfl", ctypes.c_double), ("periods", ctypes.c_int), ("corrected", ctypes.c_int),
                ("nt", ctypes.c_int), ("implicit", ctypes.c_int)]


class ewh_problem_info(ctypes.Structure):
    _fields_ = [("nt", ctypes.c_int), ("periods", ctypes.c_int), ("dt", ctypes.c_double),
                ("omega", ctypes.c_double), ("omega_tilde", ctypes.c_double), ("kt", ctypes.c_double),
                ("nodes", ctypes.c_longlong), ("n_unknowns", ctypes.c_longlong), ("nrhs", ctypes.c_int),
                ("nu", ctypes.c_int * 3), ("kernel_variant", ctypes.c_int * 2), ("resident", ctypes.c_int * 10)]


class ewh_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("s_applies", ctypes.c_int), ("s_applies_fp64", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int),
                ("minres_iters", ctypes.c_int)]


class ewh_stats(ctypes.Structure):
    _fields_ = [("wave_ms", ctypes.c_double * 2), ("steps", ctypes.c_longlong * 2),
                ("waves", ctypes.c_longlong * 2), ("launches", ctypes.c_longlong),
                ("grid_wait_timeouts", ctypes.c_longlong), ("loop_steps", ctypes.c_longlong * 2),
                ("loop_waves", ctypes.c_longlong * 2)]


class ewh_problem(ctypes.Structure):
    _fields_ = [("desc", ewh_grid_desc), ("rho", ctypes.c_void_p), ("lambda_", ctypes.c_void_p),
                ("mu", ctypes.c_void_p), ("omega", ctypes.c_double), ("forcing", ctypes.c_void_p),
                ("nrhs", ctypes.c_int)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes)
SIGNATURES = {
    "ewh_create": (ctypes.c_int, [ctypes.POINTER(ewh_grid_desc), _P, _P, _P, ctypes.c_double, _P, ctypes.c_int,
                                  _P, ctypes.POINTER(_P)]),
    "ewh_create_mapped": (ctypes.c_int, [ctypes.POINTER(ewh_grid_desc), _P, _P, _P, _P, _P, ctypes.c_double, _P,
                                         ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "ewh_get_info": (ctypes.c_int, [_P, ctypes.POINTER(ewh_problem_info)]),
    "ewh_apply_S": (ctypes.c_int, [_P, _P, _P]),
    "ewh_apply_S_fp64": (ctypes.c_int, [_P, _P, _P]),
    "ewh_apply_Pi0": (ctypes.c_int, [_P, _P]),
    "ewh_apply_minvK": (ctypes.c_int, [_P, _P, _P]),
    "ewh_mdot": (ctypes.c_int, [_P, _P, _P, _D]),
    "ewh_solve": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, _P, _P, ctypes.POINTER(ewh_solve_info)]),
    "ewh_solve_cr": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, _P, _P, ctypes.POINTER(ewh_solve_info)]),
    "ewh_solve_minres": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, _P, _P, ctypes.POINTER(ewh_solve_info)]),
    "ewh_residual_history": (ctypes.c_int, [_P, _D, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ewh_kernel_launches": (ctypes.c_longlong, [_P]),
    "ewh_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ewh_stats)]),
    "ewh_reset_stats": (ctypes.c_int, [_P]),
    "ewh_set_grid_wait": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "ewh_fma_rate": (ctypes.c_int, [ctypes.c_int, _D, _P]),
    "ewh_mdot_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _P, _P]),
    "ewh_batch_create": (ctypes.c_int, [ctypes.POINTER(ewh_problem), ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "ewh_batch_apply_S": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "ewh_batch_solve": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_P),
                                       ctypes.POINTER(ewh_solve_info)]),
    "ewh_batch_member": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "ewh_batch_kernel_launches": (ctypes.c_longlong, [_P]),
    "ewh_batch_last_error": (ctypes.c_char_p, [_P]),
    "ewh_batch_destroy": (None, [_P]),
    "ewh_conv3x3_fwd": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, _P]),
    "ewh_conv3x3_dgrad": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _P]),
    "ewh_conv3x3_wgrad": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _P]),
    "ewh_bias_grad": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.c_int, _P]),
    "ewh_leaky_relu_bwd": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_longlong, _P]),
    "ewh_avgpool2": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "ewh_avgpool2_bwd": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "ewh_upsample2": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _P]),
    "ewh_upsample2_bwd": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, _P]),
    "ewh_copy_channels": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "ewh_slice_channels": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _P]),
    "ewh_f32_to_bf16": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
    "ewh_scaled_l2_loss": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _P]),
    "ewh_adam_step": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_longlong, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, ctypes.c_int, _P]),
    "ewh_destroy": (None, [_P]),
    "ewh_last_error": (ctypes.c_char_p, [_P]),
    "ewh_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def load(path: str | None = None):
    """Load libewh.so (building it in-tree first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.LIB
        if not os.path.exists(path):
            _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class EwhError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (load().ewh_status_string(status).decode(), msg))
        self.status = status


def _check(status, ctx=None):
    if status != EWH_OK:
        raise EwhError(status, load().ewh_last_error(ctx).decode())
    return status


def _ptr(a):
    """Device or host address of a torch tensor / numpy array (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    if hasattr(a, "ctypes"):
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array")


# ---- same names as the C ABI -------------------------------------------------

def ewh_create(desc, rho, lam, mu, omega, forcing, nrhs, stream=None):
    lib = load()
    out = ctypes.c_void_p()
    st = ctypes.c_void_p(stream) if stream else None
    _check(lib.ewh_create(ctypes.byref(desc), _ptr(rho), _ptr(lam), _ptr(mu), float(omega), _ptr(forcing),
                          int(nrhs), st, ctypes.byref(out)))
    return out


def ewh_create_mapped(desc, x, y, rho, lam, mu, omega, forcing, nrhs, stream=None):
    lib = load()
    out = ctypes.c_void_p()
    st = ctypes.c_void_p(stream) if stream else None
    _check(lib.ewh_create_mapped(ctypes.byref(desc), _ptr(x), _ptr(y), _ptr(rho), _ptr(lam), _ptr(mu), float(omega),
                                 _ptr(forcing), int(nrhs), st, ctypes.byref(out)))
    return out


def ewh_get_info(ctx):
    info = ewh_problem_info()
    _check(load().ewh_get_info(ctx, ctypes.byref(info)), ctx)
    return info


def ewh_apply_S(ctx, v_in, v_out):
    return _check(load().ewh_apply_S(ctx, _ptr(v_in), _ptr(v_out)), ctx)


def ewh_apply_S_fp64(ctx, v_in, v_out):
    return _check(load().ewh_apply_S_fp64(ctx, _ptr(v_in), _ptr(v_out)), ctx)


def ewh_apply_Pi0(ctx, b_out):
    return _check(load().ewh_apply_Pi0(ctx, _ptr(b_out)), ctx)


def ewh_apply_minvK(ctx, u, out):
    return _check(load().ewh_apply_minvK(ctx, _ptr(u), _ptr(out)), ctx)


def ewh_mdot(ctx, x, y, nrhs):
    out = (ctypes.c_double * nrhs)()
    _check(load().ewh_mdot(ctx, _ptr(x), _ptr(y), out), ctx)
    return list(out)


def ewh_solve(ctx, tol, maxit, x0, v_out, raise_on_error=True):
    info = ewh_solve_info()
    s = load().ewh_solve(ctx, float(tol), int(maxit), _ptr(x0), _ptr(v_out), ctypes.byref(info))
    if raise_on_error and s not in (EWH_OK,):
        _check(s, ctx)
    return info


def ewh_solve_cr(ctx, tol, maxit, x0, v_out, raise_on_error=True):
    info = ewh_solve_info()
    s = load().ewh_solve_cr(ctx, float(tol), int(maxit), _ptr(x0), _ptr(v_out), ctypes.byref(info))
    if raise_on_error and s not in (EWH_OK,):
        _check(s, ctx)
    return info


def ewh_solve_minres(ctx, tol, maxit, x0, v_out, raise_on_error=True):
    info = ewh_solve_info()
    s = load().ewh_solve_minres(ctx, float(tol), int(maxit), _ptr(x0), _ptr(v_out), ctypes.byref(info))
    if raise_on_error and s not in (EWH_OK,):
        _check(s, ctx)
    return info


def ewh_residual_history(ctx):
    count = ctypes.c_int()
    load().ewh_residual_history(ctx, None, 0, ctypes.byref(count))
    buf = (ctypes.c_double * max(count.value, 1))()
    load().ewh_residual_history(ctx, buf, count.value, ctypes.byref(count))
    return list(buf)[:count.value]


def ewh_kernel_launches(ctx):
    return int(load().ewh_kernel_launches(ctx))


def ewh_get_stats(ctx):
    st = ewh_stats()
    _check(load().ewh_get_stats(ctx, ctypes.byref(st)), ctx)
    return st


def ewh_reset_stats(ctx):
    return _check(load().ewh_reset_stats(ctx), ctx)


def ewh_set_grid_wait(ctx, ns):
    return _check(load().ewh_set_grid_wait(ctx, int(ns)), ctx)


def ewh_fma_rate(precision, stream=None):
    """Measured FMA throughput (floating-point operations per second)."""
    out = ctypes.c_double()
    _check(load().ewh_fma_rate(int(precision), ctypes.byref(out), ctypes.c_void_p(stream) if stream else None))
    return out.value


def ewh_mdot_noalloc(x, y, w, nodes, ncomp, nbatch, out, stream=None):
    """Allocation-free weighted inner products into the device array ``out``."""
    st = ctypes.c_void_p(stream) if stream else None
    return _check(load().ewh_mdot_noalloc(_ptr(x), _ptr(y), _ptr(w), int(nodes), int(ncomp), int(nbatch),
                                          _ptr(out), st))


def ewh_batch_create(problems, stream=None):
    """problems: list of (desc, rho, lam, mu, omega, forcing, nrhs) with array arguments."""
    arr = (ewh_problem * len(problems))()
    for k, (desc, rho, lam, mu, omega, forcing, nrhs) in enumerate(problems):
        arr[k].desc = desc
        arr[k].rho = _ptr(rho)
        arr[k].lambda_ = _ptr(lam)
        arr[k].mu = _ptr(mu)
        arr[k].omega = float(omega)
        arr[k].forcing = _ptr(forcing)
        arr[k].nrhs = int(nrhs)
    out = ctypes.c_void_p()
    st = ctypes.c_void_p(stream) if stream else None
    _check(load().ewh_batch_create(arr, len(problems), st, ctypes.byref(out)))
    return out


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for k, t in enumerate(tensors):
        arr[k] = _ptr(t).value
    return arr


def _bcheck(status, b):
    if status != EWH_OK:
        raise EwhError(status, load().ewh_batch_last_error(b).decode())
    return status


def ewh_batch_apply_S(b, v_in, v_out):
    return _bcheck(load().ewh_batch_apply_S(b, _ptr_array(v_in), _ptr_array(v_out)), b)


def ewh_batch_solve(b, tol, maxit, v_out, raise_on_error=True):
    infos = (ewh_solve_info * len(v_out))()
    s = load().ewh_batch_solve(b, float(tol), int(maxit), _ptr_array(v_out), infos)
    if raise_on_error:
        _bcheck(s, b)
    return list(infos)


def ewh_batch_member(b, k):
    c = ctypes.c_void_p()
    _check(load().ewh_batch_member(b, int(k), ctypes.byref(c)))
    return c


def ewh_batch_kernel_launches(b):
    return int(load().ewh_batch_kernel_launches(b))


def ewh_batch_destroy(b):
    if b is not None:
        load().ewh_batch_destroy(b)


def ewh_destroy(ctx):
    if ctx is not None:
        load().ewh_destroy(ctx)


def ewh_last_error(ctx=None):
    return load().ewh_last_error(ctx).decode()


# ---- warm-start layers (device tensors; stream = torch stream handle or None)

def _s(stream):
    return ctypes.c_void_p(stream) if stream else None


def _net(name, *args):
    st = load()
    fn = getattr(st, name)
    conv = []
    for a in args:
        conv.append(_ptr(a) if (a is not None and hasattr(a, "data_ptr")) else a)
    return _check(fn(*conv))


def ewh_conv3x3_fwd(x, w, bias, y_pre, y_act, act, N, H, W, Ci, Co, stream=None):
    return _net("ewh_conv3x3_fwd", x, w, bias, y_pre, y_act, int(act), N, H, W, Ci, Co, _s(stream))


def ewh_conv3x3_dgrad(dy, w, w_scratch, dx, N, H, W, Ci, Co, stream=None):
    return _net("ewh_conv3x3_dgrad", dy, w, w_scratch, dx, N, H, W, Ci, Co, _s(stream))


def ewh_conv3x3_wgrad(x, dy, dw, N, H, W, Ci, Co, stream=None):
    return _net("ewh_conv3x3_wgrad", x, dy, dw, N, H, W, Ci, Co, _s(stream))


def ewh_bias_grad(dy, db, P, C, stream=None):
    return _net("ewh_bias_grad", dy, db, P, C, _s(stream))


def ewh_leaky_relu_bwd(pre, dy, dx, dx_bf16, n, stream=None):
    return _net("ewh_leaky_relu_bwd", pre, dy, dx, dx_bf16, n, _s(stream))


def ewh_avgpool2(x, y, N, H, W, C, stream=None):
    return _net("ewh_avgpool2", x, y, N, H, W, C, _s(stream))


def ewh_avgpool2_bwd(dy, dx, N, H, W, C, stream=None):
    return _net("ewh_avgpool2_bwd", dy, dx, N, H, W, C, _s(stream))


def ewh_upsample2(x, y, N, H, W, C, Cy, c_off, stream=None):
    return _net("ewh_upsample2", x, y, N, H, W, C, Cy, c_off, _s(stream))


def ewh_upsample2_bwd(dy, dx, N, H, W, C, Cy, c_off, stream=None):
    return _net("ewh_upsample2_bwd", dy, dx, N, H, W, C, Cy, c_off, _s(stream))


def ewh_copy_channels(x, y, P, C, Cy, c_off, stream=None):
    return _net("ewh_copy_channels", x, y, P, C, Cy, c_off, _s(stream))


def ewh_slice_channels(dy, dx, P, C, Cy, c_off, accumulate, stream=None):
    return _net("ewh_slice_channels", dy, dx, P, C, Cy, c_off, int(accumulate), _s(stream))


def ewh_f32_to_bf16(a, b, n, stream=None):
    return _net("ewh_f32_to_bf16", a, b, n, _s(stream))


def ewh_adam_step(param, grad, m, v, param_bf16, n, lr, beta1, beta2, eps, step, stream=None):
    return _net("ewh_adam_step", param, grad, m, v, param_bf16, n, float(lr), float(beta1), float(beta2),
                float(eps), int(step), _s(stream))


def ewh_scaled_l2_loss(y, t, grad, loss, P, C, Cu, N, stream=None):
    return _net("ewh_scaled_l2_loss", y, t, grad, loss, P, C, Cu, N, _s(stream))
