"""ctypes declarations of libsem's C ABI (include/sem.h), one wrapper per entry
point with the same name.  The wrappers only marshal arguments (tensor data
pointers, the current torch stream) and turn a negative status into an
exception; every step of the computation runs in libsem's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# SEM_LIBRARY selects another build of the library (the SEM_DEBUG one, for instance)
LIB_PATH = os.environ.get("SEM_LIBRARY") or os.path.join(HERE, "libsem.so")

SEM_OK = 0
SEM_ERR_ARG = -1
SEM_ERR_CUDA = -2
SEM_ERR_BAD_MESH = -3
SEM_ERR_NOT_CONVERGED = -4
SEM_ERR_NONFINITE = -5
SEM_ERR_UNSUPPORTED = -6
SEM_ERR_NOMEM = -7
SEM_ERR_TIMEOUT = -8

SEM_QUAD_LG = 0
SEM_QUAD_LGL = 1
SEM_PREC_FP64 = 0
SEM_PREC_FP32 = 1
SEM_PREC_FP32_BF16 = 2
SEM_PREC_DF64 = 3
SEM_PREC_BF16_TC = 4
SEM_PC_NONE = 0
SEM_PC_JACOBI = 1
SEM_PC_GMG = 2
SEM_REGION_BOX = 0
SEM_REGION_SPHERE = 1

ERROR_NAMES = {
    SEM_ERR_ARG: "SEM_ERR_ARG", SEM_ERR_CUDA: "SEM_ERR_CUDA", SEM_ERR_BAD_MESH: "SEM_ERR_BAD_MESH",
    SEM_ERR_NOT_CONVERGED: "SEM_ERR_NOT_CONVERGED", SEM_ERR_NONFINITE: "SEM_ERR_NONFINITE",
    SEM_ERR_UNSUPPORTED: "SEM_ERR_UNSUPPORTED", SEM_ERR_NOMEM: "SEM_ERR_NOMEM",
    SEM_ERR_TIMEOUT: "SEM_ERR_TIMEOUT",
}

# Every symbol include/sem.h declares.
EXPORTS = [
    "sem_version", "sem_create", "sem_destroy", "sem_last_error", "sem_num_dofs",
    "sem_num_elements", "sem_dof_coords", "sem_set_tissue", "sem_apply", "sem_diagonal",
    "sem_cg_solve", "sem_set_ionic", "sem_set_stimulus", "sem_state_create", "sem_state_destroy",
    "sem_state_set", "sem_state_get", "sem_state_restore", "sem_step", "sem_step_host", "sem_step_host_out",
    "sem_state_track_activation", "sem_state_get_activation",
    "sem_set_timing", "sem_apply_dot_static", "sem_set_gmg", "sem_vcycle", "sem_gmg_info",
    "sem_forward_record", "sem_adjoint_grad", "sem_set_operator_precision", "sem_set_deterministic",
    "sem_debug_set_map_entry", "sem_debug_hold_copy",
]


class SemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class sem_ionic_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("u_rest", "u_amp", "tau_in", "tau_out", "tau_open", "tau_close", "v_gate", "kappa")]


class sem_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("cg_iters", ctypes.c_int64),
                ("last_residual", ctypes.c_double), ("apply_ms", ctypes.c_double),
                ("n_apply", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("smoother_apply_ms", ctypes.c_double), ("n_smoother_apply", ctypes.c_int64),
                ("carried_solves", ctypes.c_int64)]


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    """The loaded libsem.so; raises if the library has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2205_05136_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "sem_version": (ctypes.c_char_p, []),
            "sem_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _DP, _I, _I, _I]),
            "sem_destroy": (_I, [_P]),
            "sem_last_error": (ctypes.c_char_p, [_P]),
            "sem_num_dofs": (_I, [_P, ctypes.POINTER(_I64)]),
            "sem_num_elements": (_I, [_P, ctypes.POINTER(_I64)]),
            "sem_dof_coords": (_I, [_P, _P, _P]),
            "sem_set_tissue": (_I, [_P, _P, _P, _P, _P]),
            "sem_apply": (_I, [_P, _D, _D, _P, _P, _I, _P]),
            "sem_diagonal": (_I, [_P, _D, _D, _P, _P]),
            "sem_cg_solve": (_I, [_P, _D, _P, _P, _D, _D, _I, _I, ctypes.POINTER(_I), _DP, _P]),
            "sem_set_ionic": (_I, [_P, ctypes.POINTER(sem_ionic_params)]),
            "sem_set_stimulus": (_I, [_P, _I, _DP, _D, _D, _D, _P]),
            "sem_state_create": (_I, [_P, ctypes.POINTER(_P)]),
            "sem_state_destroy": (_I, [_P]),
            "sem_state_set": (_I, [_P, _P, _P, _P]),
            "sem_state_get": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(_I64), _P]),
            "sem_state_restore": (_I, [_P, _P, _P, _P, _P, _I64, _P]),
            "sem_step": (_I, [_P, _P, _D, _I, _D, _D, _I, _I, ctypes.POINTER(sem_stats), _P]),
            "sem_step_host": (_I, [_P, _P, _P, _P, _P, _I64, _D, _D, _D, _I, _I,
                                   ctypes.POINTER(sem_stats), _P]),
            "sem_step_host_out": (_I, [_P, _P, _P, _P, _P, _P, _P, _I64, _D, _D, _D, _I, _I,
                                       ctypes.POINTER(sem_stats), _P]),
            "sem_state_track_activation": (_I, [_P, _I, _P]),
            "sem_state_get_activation": (_I, [_P, _P, _P, _P]),
            "sem_set_timing": (_I, [_P, _I]),
            "sem_apply_dot_static": (_I, [_P, _D, _D, _P, _P, _P, _P]),
            "sem_set_gmg": (_I, [_P, _I, _I, _I, _I]),
            "sem_set_operator_precision": (_I, [_P, _I]),
            "sem_set_deterministic": (_I, [_P, _I]),
            "sem_debug_set_map_entry": (_I, [_P, _I64, _I, ctypes.POINTER(_I)]),
            "sem_debug_hold_copy": (_I, [_P, _I]),
            "sem_forward_record": (_I, [_P, _P, _D, _I, _I, _P, _I, _P, _D, _D, _I, _I,
                                        ctypes.POINTER(sem_stats), _P]),
            "sem_adjoint_grad": (_I, [_P, _P, _P, _P, _P, _D, _D, _I, _I, ctypes.POINTER(sem_stats), _P]),
            "sem_vcycle": (_I, [_P, _D, _P, _P, _P]),
            "sem_gmg_info": (_I, [_P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                  ctypes.POINTER(_I), ctypes.POINTER(_I64), _DP, _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(rc: int, ctx=None):
    if rc != SEM_OK:
        msg = lib().sem_last_error(ctx)
        raise SemError(rc, msg.decode() if msg else "")
    return rc


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return _P(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, n=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} entries, has {t.numel()}")
    return _P(t.data_ptr())


# ---- same-name wrappers -------------------------------------------------

def sem_version() -> str:
    return lib().sem_version().decode()


def sem_create(nx, ny, nz, vertices, p, quad, device=0):
    import numpy as np
    v = np.ascontiguousarray(vertices, dtype=np.float64).reshape(-1)
    if v.size != (nx + 1) * (ny + 1) * (nz + 1) * 3:
        raise ValueError("vertices must hold (nx+1)(ny+1)(nz+1) points")
    out = _P()
    rc = lib().sem_create(ctypes.byref(out), nx, ny, nz, v.ctypes.data_as(_DP), p, quad, device)
    _check(rc, None)
    return out


def sem_destroy(ctx):
    return _check(lib().sem_destroy(ctx))


def sem_last_error(ctx) -> str:
    return lib().sem_last_error(ctx).decode()


def sem_num_dofs(ctx) -> int:
    n = _I64()
    _check(lib().sem_num_dofs(ctx, ctypes.byref(n)), ctx)
    return n.value


def sem_num_elements(ctx) -> int:
    n = _I64()
    _check(lib().sem_num_elements(ctx, ctypes.byref(n)), ctx)
    return n.value


def sem_dof_coords(ctx, xyz, stream=None):
    return _check(lib().sem_dof_coords(ctx, _P(xyz.data_ptr()), _stream(stream)), ctx)


def sem_set_tissue(ctx, sigma_l, sigma_t, theta, stream=None):
    ne = sem_num_elements(ctx)
    return _check(lib().sem_set_tissue(ctx, _dev(sigma_l, torch.float64, ne, "sigma_l"),
                                       _dev(sigma_t, torch.float64, ne, "sigma_t"),
                                       _dev(theta, torch.float64, ne, "theta"), _stream(stream)), ctx)


def sem_apply(ctx, alpha, beta, u, y, precision=SEM_PREC_FP64, stream=None):
    dt = torch.float64 if precision in (SEM_PREC_FP64, SEM_PREC_DF64) else torch.float32
    n = sem_num_dofs(ctx)
    return _check(lib().sem_apply(ctx, float(alpha), float(beta), _dev(u, dt, n, "u"),
                                  _dev(y, dt, n, "y"), int(precision), _stream(stream)), ctx)


def sem_diagonal(ctx, alpha, beta, d, stream=None):
    n = sem_num_dofs(ctx)
    return _check(lib().sem_diagonal(ctx, float(alpha), float(beta), _dev(d, torch.float64, n, "d"),
                                     _stream(stream)), ctx)


def sem_cg_solve(ctx, alpha, b, x, rtol, atol, maxit, precond=SEM_PC_JACOBI, stream=None,
                 raise_on_error=True):
    n = sem_num_dofs(ctx)
    it = _I()
    res = _D()
    rc = lib().sem_cg_solve(ctx, float(alpha), _dev(b, torch.float64, n, "b"),
                            _dev(x, torch.float64, n, "x"), float(rtol), float(atol), int(maxit),
                            int(precond), ctypes.byref(it), ctypes.byref(res), _stream(stream))
    if raise_on_error:
        _check(rc, ctx)
    return rc, it.value, res.value


def sem_set_ionic(ctx, params: dict):
    prm = sem_ionic_params(**{k: float(v) for k, v in params.items()})
    return _check(lib().sem_set_ionic(ctx, ctypes.byref(prm)), ctx)


def sem_set_stimulus(ctx, region, params, amplitude, t_on, t_off, stream=None):
    arr = (ctypes.c_double * len(params))(*[float(x) for x in params])
    return _check(lib().sem_set_stimulus(ctx, int(region), arr, float(amplitude), float(t_on),
                                         float(t_off), _stream(stream)), ctx)


def sem_state_create(ctx):
    out = _P()
    _check(lib().sem_state_create(ctx, ctypes.byref(out)), ctx)
    return out


def sem_state_destroy(st):
    return lib().sem_state_destroy(st)


def sem_state_set(ctx, st, u0, h0, stream=None):
    n = sem_num_dofs(ctx)
    return _check(lib().sem_state_set(st, _dev(u0, torch.float64, n, "u0"),
                                      _dev(h0, torch.float64, n, "h0"), _stream(stream)), ctx)


def sem_state_get(ctx, st, u=None, u_prev=None, h=None, h_prev=None, stream=None):
    n = sem_num_dofs(ctx)
    nout = _I64()
    ptrs = [_dev(t, torch.float64, n, nm) if t is not None else _P()
            for t, nm in ((u, "u"), (u_prev, "u_prev"), (h, "h"), (h_prev, "h_prev"))]
    _check(lib().sem_state_get(st, *ptrs, ctypes.byref(nout), _stream(stream)), ctx)
    return nout.value


def sem_state_restore(ctx, st, u, u_prev, h, h_prev, n, stream=None):
    nd = sem_num_dofs(ctx)
    return _check(lib().sem_state_restore(st, _dev(u, torch.float64, nd, "u"),
                                          _dev(u_prev, torch.float64, nd, "u_prev"),
                                          _dev(h, torch.float64, nd, "h"),
                                          _dev(h_prev, torch.float64, nd, "h_prev"), int(n),
                                          _stream(stream)), ctx)


def sem_step(ctx, st, dt, nsteps, rtol, atol, maxit, precond=SEM_PC_JACOBI, stream=None):
    stats = sem_stats()
    _check(lib().sem_step(ctx, st, float(dt), int(nsteps), float(rtol), float(atol), int(maxit),
                          int(precond), ctypes.byref(stats), _stream(stream)), ctx)
    return stats


def sem_step_host(ctx, u, u_prev, h, h_prev, n, dt, rtol, atol, maxit, precond=SEM_PC_JACOBI,
                  stream=None):
    """u, u_prev, h, h_prev: contiguous float64 CPU tensors (pinned for async copies)."""
    nd = sem_num_dofs(ctx)
    for t, name in ((u, "u"), (u_prev, "u_prev"), (h, "h"), (h_prev, "h_prev")):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != nd:
            raise TypeError(f"{name} must be a contiguous float64 CPU tensor of {nd} entries")
    stats = sem_stats()
    _check(lib().sem_step_host(ctx, _P(u.data_ptr()), _P(u_prev.data_ptr()), _P(h.data_ptr()),
                               _P(h_prev.data_ptr()), int(n), float(dt), float(rtol), float(atol),
                               int(maxit), int(precond), ctypes.byref(stats), _stream(stream)), ctx)
    return stats


def sem_step_host_out(ctx, u, u_prev, h, h_prev, u_next, h_next, n, dt, rtol, atol, maxit,
                      precond=SEM_PC_JACOBI, stream=None):
    """Inputs u, u_prev, h, h_prev and outputs u_next, h_next: contiguous float64
    CPU tensors (page-locked inputs are read by the device in place)."""
    nd = sem_num_dofs(ctx)
    for t, name in ((u, "u"), (u_prev, "u_prev"), (h, "h"), (h_prev, "h_prev"),
                    (u_next, "u_next"), (h_next, "h_next")):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != nd:
            raise TypeError(f"{name} must be a contiguous float64 CPU tensor of {nd} entries")
    stats = sem_stats()
    _check(lib().sem_step_host_out(ctx, _P(u.data_ptr()), _P(u_prev.data_ptr()), _P(h.data_ptr()),
                                   _P(h_prev.data_ptr()), _P(u_next.data_ptr()), _P(h_next.data_ptr()),
                                   int(n), float(dt), float(rtol), float(atol), int(maxit), int(precond),
                                   ctypes.byref(stats), _stream(stream)), ctx)
    return stats


def sem_state_track_activation(ctx, st, enable=True, stream=None):
    return _check(lib().sem_state_track_activation(st, 1 if enable else 0, _stream(stream)), ctx)


def sem_state_get_activation(ctx, st, tau, dudt_max, stream=None):
    """tau, dudt_max: float64 CUDA tensors of ndofs entries (or None)."""
    n = sem_num_dofs(ctx)
    t = _dev(tau, torch.float64, n, "tau") if tau is not None else None
    d = _dev(dudt_max, torch.float64, n, "dudt_max") if dudt_max is not None else None
    return _check(lib().sem_state_get_activation(st, t, d, _stream(stream)), ctx)


def sem_set_timing(ctx, enable: bool):
    return _check(lib().sem_set_timing(ctx, 1 if enable else 0), ctx)


def sem_apply_dot_static(ctx, alpha, beta, u, y, dot, stream=None):
    """y = alpha M u + beta K u and dot[0] = u . y with no allocation inside libsem
    (static device scratch; see include/sem.h)."""
    n = sem_num_dofs(ctx)
    return _check(lib().sem_apply_dot_static(ctx, float(alpha), float(beta),
                                             _dev(u, torch.float64, n, "u"),
                                             _dev(y, torch.float64, n, "y"),
                                             _dev(dot, torch.float64, 1, "dot"),
                                             _stream(stream)), ctx)


def sem_debug_set_map_entry(ctx, entry: int, value: int) -> int:
    """Plants `value` at map entry `entry` (SEM_DEBUG build only); returns the old value."""
    old = _I()
    _check(lib().sem_debug_set_map_entry(ctx, int(entry), int(value), ctypes.byref(old)), ctx)
    return old.value


def sem_debug_hold_copy(ctx, group: int):
    """SEM_DEBUG build only: the pipelined FP32 apply leaves out the metric copy of
    element group `group` (-1: none), so that its bounded wait runs out."""
    return _check(lib().sem_debug_hold_copy(ctx, int(group)), ctx)


def sem_set_deterministic(ctx, enable: bool):
    return _check(lib().sem_set_deterministic(ctx, 1 if enable else 0), ctx)


def sem_set_gmg(ctx, degree=3, coarse_degree=10, min_coarse_dofs=2000, precision=SEM_PREC_FP32):
    return _check(lib().sem_set_gmg(ctx, int(degree), int(coarse_degree), int(min_coarse_dofs),
                                    int(precision)), ctx)


def sem_vcycle(ctx, alpha, r, z, stream=None):
    n = sem_num_dofs(ctx)
    return _check(lib().sem_vcycle(ctx, float(alpha), _dev(r, torch.float64, n, "r"),
                                   _dev(z, torch.float64, n, "z"), _stream(stream)), ctx)


def sem_gmg_info(ctx, alpha, max_levels=32, stream=None):
    """dict(nlevels, p, dims, ndofs, lambda_max) of the multigrid hierarchy for alpha."""
    nl = _I()
    p = (_I * max_levels)()
    dims = (_I * (3 * max_levels))()
    nd = (_I64 * max_levels)()
    lam = (_D * max_levels)()
    _check(lib().sem_gmg_info(ctx, float(alpha), int(max_levels), ctypes.byref(nl), p, dims, nd,
                              lam, _stream(stream)), ctx)
    k = min(nl.value, max_levels)
    return dict(nlevels=nl.value, p=list(p[:k]), dims=[tuple(dims[3 * i:3 * i + 3]) for i in range(k)],
                ndofs=list(nd[:k]), lambda_max=list(lam[:k]))


def sem_forward_record(ctx, st, dt, nsteps, checkpoint_every, sensors, traces, rtol, atol, maxit,
                       precond=SEM_PC_JACOBI, stream=None):
    """sensors: CUDA int32 tensor; traces: CUDA float64 tensor of nsteps * len(sensors)."""
    ns = sensors.numel()
    stats = sem_stats()
    _check(lib().sem_forward_record(ctx, st, float(dt), int(nsteps), int(checkpoint_every),
                                    _dev(sensors, torch.int32, ns, "sensors"), int(ns),
                                    _dev(traces, torch.float64, nsteps * ns, "traces"), float(rtol),
                                    float(atol), int(maxit), int(precond), ctypes.byref(stats),
                                    _stream(stream)), ctx)
    return stats


def sem_adjoint_grad(ctx, trace_bar, g_sigma_l, g_sigma_t, g_theta, rtol, atol, maxit,
                     precond=SEM_PC_JACOBI, stream=None):
    ne = sem_num_elements(ctx)
    stats = sem_stats()
    _check(lib().sem_adjoint_grad(ctx, _dev(trace_bar, torch.float64, trace_bar.numel(), "trace_bar"),
                                  _dev(g_sigma_l, torch.float64, ne, "g_sigma_l"),
                                  _dev(g_sigma_t, torch.float64, ne, "g_sigma_t"),
                                  _dev(g_theta, torch.float64, ne, "g_theta"), float(rtol), float(atol),
                                  int(maxit), int(precond), ctypes.byref(stats), _stream(stream)), ctx)
    return stats


def sem_set_operator_precision(ctx, precision):
    return _check(lib().sem_set_operator_precision(ctx, int(precision)), ctx)
