"""Python binding of the C ABI in include/lbm.h (ctypes, marshalling only).

Every function here has the name of the C entry point it wraps and does
nothing but convert arguments; all computation runs in libmrtlbm.so's CUDA
kernels.  Loading fails loudly if the library has not been built: there is no
CPU fallback.

`Solver` is a thin convenience object over the same calls (it owns one
context and raises `LBMError` on a non-zero status).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the library (the bounds-checked one)
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(PKG, "_build", "libmrtlbm.so")

LBM_OK = 0
LBM_ERR_INVALID_ARG = 1
LBM_ERR_STATE = 2
LBM_ERR_CUDA = 3
LBM_ERR_OUT_OF_MEMORY = 4
LBM_ERR_NOT_CONVERGED = 5
LBM_ERR_DIVERGED = 6
LBM_ERR_STALLED = 7
LBM_ERR_TIMEOUT = 8
LBM_ERR_INTERNAL = 9
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "STATE", 3: "CUDA", 4: "OUT_OF_MEMORY",
                5: "NOT_CONVERGED", 6: "DIVERGED", 7: "STALLED", 8: "TIMEOUT", 9: "INTERNAL"}

LBM_AXIS_X, LBM_AXIS_Y, LBM_AXIS_Z = 0, 1, 2
LBM_LATERAL_PERIODIC, LBM_LATERAL_ADIABATIC = 0, 1
LBM_STORE_F32, LBM_STORE_BF16, LBM_STORE_F16 = 0, 1, 2


class lbm_solve_opts(ctypes.Structure):
    _fields_ = [("t_hot", ctypes.c_double), ("t_cold", ctypes.c_double),
                ("tau_max", ctypes.c_double), ("lattice_scale", ctypes.c_double),
                ("tol", ctypes.c_double), ("max_iters", ctypes.c_int64),
                ("check_every", ctypes.c_int32), ("stall_checks", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("host_loop", ctypes.c_int32),
                ("fuse", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_init", ctypes.POINTER(ctypes.c_float)), ("stream", ctypes.c_void_p)]


class lbm_batch_info(ctypes.Structure):
    _fields_ = [("n_solves", ctypes.c_int32), ("n_converged", ctypes.c_int32),
                ("total_updates", ctypes.c_int64), ("elapsed_ms", ctypes.c_double),
                ("block_threads", ctypes.c_int32), ("status", ctypes.c_int32),
                ("steps_per_launch", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lbm_launch_plan(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("pitch", ctypes.c_int32), ("steps_per_launch", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32), ("zchunk", ctypes.c_int32),
                ("block_threads", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lbm_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("k_eff", ctypes.c_double),
                ("residual_T", ctypes.c_double), ("residual_Q", ctypes.c_double),
                ("elapsed_ms", ctypes.c_double), ("lattice_scale", ctypes.c_double),
                ("status", ctypes.c_int32), ("checks", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_ctx_p = ctypes.c_void_p
_PROTOS = {
    "lbm_default_opts": (None, [ctypes.POINTER(lbm_solve_opts)]),
    "lbm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(_ctx_p)]),
    "lbm_set_geometry": (ctypes.c_int, [_ctx_p, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int]),
    "lbm_set_tensors": (ctypes.c_int, [_ctx_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "lbm_start": (ctypes.c_int, [_ctx_p, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(lbm_solve_opts)]),
    "lbm_advance": (ctypes.c_int, [_ctx_p, ctypes.c_int64]),
    "lbm_check": (ctypes.c_int, [_ctx_p, ctypes.POINTER(lbm_solve_info)]),
    "lbm_run": (ctypes.c_int, [_ctx_p, ctypes.POINTER(lbm_solve_info)]),
    "lbm_solve": (ctypes.c_int, [_ctx_p, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(lbm_solve_opts), ctypes.POINTER(lbm_solve_info)]),
    "lbm_k_eff": (ctypes.c_int, [_ctx_p, ctypes.POINTER(ctypes.c_double)]),
    "lbm_get_temperature": (ctypes.c_int, [_ctx_p, ctypes.POINTER(ctypes.c_float)]),
    "lbm_get_plane_flux": (ctypes.c_int, [_ctx_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "lbm_get_history": (ctypes.c_int, [_ctx_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "lbm_set_geometry_braid": (ctypes.c_int, [_ctx_p, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                              ctypes.c_int, ctypes.c_double,
                                              ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_double)]),
    "lbm_get_geometry": (ctypes.c_int, [_ctx_p, ctypes.POINTER(ctypes.c_uint8)]),
    "lbm_braid_voxelize_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.c_double, ctypes.c_void_p,
                                                  ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(ctypes.c_double),
                                                  ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]),
    "lbm_yarn_conductivity": (ctypes.c_int, [ctypes.c_double] * 4 +
                              [ctypes.POINTER(ctypes.c_double)] * 2),
    "lbm_braid_unit_cell": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double] + [ctypes.POINTER(ctypes.c_double)] * 5),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_ctx_p)]),
    "lbm_batch_add": (ctypes.c_int, [_ctx_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_uint8), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_solve": (ctypes.c_int, [_ctx_p, ctypes.c_int, ctypes.POINTER(lbm_solve_opts),
                                       ctypes.POINTER(lbm_batch_info)]),
    "lbm_batch_result": (ctypes.c_int, [_ctx_p, ctypes.c_int, ctypes.POINTER(lbm_solve_info)]),
    "lbm_batch_get_temperature": (ctypes.c_int, [_ctx_p, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_float)]),
    "lbm_batch_set_initial": (ctypes.c_int, [_ctx_p, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "lbm_batch_get_history": (ctypes.c_int, [_ctx_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_ctx_p]),
    "lbm_batch_destroy": (None, [_ctx_p]),
    "lbm_nn_conv3d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_conv3d_tc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_conv3d_tc_supported": (ctypes.c_int, [ctypes.c_int] * 6),
    "lbm_nn_conv3d_tc_cfg": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_conv3d_wgrad_tc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_conv3d_wgrad_tc_supported": (ctypes.c_int, [ctypes.c_int] * 6),
    "lbm_nn_weights_kmajor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_tc_error": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "lbm_nn_conv3d_wgrad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_flip_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_bias_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]),
    "lbm_nn_relu_mask": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]),
    "lbm_nn_pool2": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_void_p]),
    "lbm_nn_upsample2": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_void_p]),
    "lbm_nn_concat": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]),
    "lbm_nn_slice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_head": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]),
    "lbm_nn_input": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "lbm_nn_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_void_p]),
    "lbm_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbm_create_with_workspace": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(_ctx_p)]),
    "lbm_get_launch_plan": (ctypes.c_int, [_ctx_p, ctypes.POINTER(lbm_launch_plan)]),
    "lbm_debug_build": (ctypes.c_int, []),
    "lbm_debug_error": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint), ctypes.c_int]),
    "lbm_state_bytes": (ctypes.c_size_t, [_ctx_p]),
    "lbm_get_state": (ctypes.c_int, [_ctx_p, ctypes.c_void_p, ctypes.c_size_t]),
    "lbm_set_state": (ctypes.c_int, [_ctx_p, ctypes.c_void_p, ctypes.c_size_t]),
    "lbm_last_error": (ctypes.c_char_p, [_ctx_p]),
    "lbm_destroy": (None, [_ctx_p]),
}


def load(path: str = LIB_PATH):
    """Loads libmrtlbm.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run paper_1503_08718_gb300.build.build())")
        L = ctypes.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _f64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- one function per C entry point -------------------------------------

def lbm_default_opts() -> lbm_solve_opts:
    o = lbm_solve_opts()
    load().lbm_default_opts(ctypes.byref(o))
    return o


def lbm_create(nx: int, ny: int, nz: int, cuda_device: int = 0):
    h = _ctx_p()
    st = load().lbm_create(nx, ny, nz, cuda_device, ctypes.byref(h))
    return st, h


def lbm_workspace_bytes(nx: int, ny: int, nz: int, storage: int = 0) -> int:
    return int(load().lbm_workspace_bytes(nx, ny, nz, storage))


def lbm_create_with_workspace(nx: int, ny: int, nz: int, cuda_device: int, dev_ptr: int, nbytes: int):
    h = _ctx_p()
    st = load().lbm_create_with_workspace(nx, ny, nz, cuda_device, ctypes.c_void_p(dev_ptr), nbytes,
                                          ctypes.byref(h))
    return st, h


def lbm_set_geometry(ctx, phase: np.ndarray, n_phases: int) -> int:
    phase = np.ascontiguousarray(phase, dtype=np.uint8)
    return load().lbm_set_geometry(ctx, phase.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                   int(n_phases))


def lbm_set_tensors(ctx, lam: np.ndarray, n_phases: int) -> int:
    lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
    return load().lbm_set_tensors(ctx, _f64(lam), int(n_phases))


def lbm_start(ctx, axis: int, lateral: int, opts: lbm_solve_opts | None = None) -> int:
    return load().lbm_start(ctx, axis, lateral, ctypes.byref(opts) if opts is not None else None)


def lbm_advance(ctx, n_steps: int) -> int:
    return load().lbm_advance(ctx, int(n_steps))


def lbm_check(ctx, info: lbm_solve_info | None = None) -> int:
    return load().lbm_check(ctx, ctypes.byref(info) if info is not None else None)


def lbm_run(ctx, info: lbm_solve_info | None = None) -> int:
    return load().lbm_run(ctx, ctypes.byref(info) if info is not None else None)


def lbm_solve(ctx, axis: int, lateral: int, opts: lbm_solve_opts | None = None,
              info: lbm_solve_info | None = None) -> int:
    return load().lbm_solve(ctx, axis, lateral,
                            ctypes.byref(opts) if opts is not None else None,
                            ctypes.byref(info) if info is not None else None)


def lbm_k_eff(ctx):
    out = ctypes.c_double(0.0)
    st = load().lbm_k_eff(ctx, ctypes.byref(out))
    return st, out.value


def lbm_get_temperature(ctx, out: np.ndarray) -> int:
    assert out.dtype == np.float32 and out.flags.c_contiguous
    return load().lbm_get_temperature(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))


def lbm_get_plane_flux(ctx, out: np.ndarray) -> int:
    assert out.dtype == np.float64 and out.flags.c_contiguous
    return load().lbm_get_plane_flux(ctx, _f64(out), out.size)


def lbm_get_history(ctx, max_entries: int = 1 << 16):
    """Returns (status, array (n, 4) of iteration, k_eff, R_T, R_Q)."""
    out = np.zeros((max_entries, 4), np.float64)
    n = ctypes.c_int(0)
    st = load().lbm_get_history(ctx, _f64(out), max_entries, ctypes.byref(n))
    return st, out[: n.value]


def lbm_set_geometry_braid(ctx, g_rad: float, A: float, B: float, anchors: np.ndarray,
                           phi: float):
    anchors = np.ascontiguousarray(anchors, dtype=np.float64).reshape(-1, 2)
    used = ctypes.c_int(0)
    frac = ctypes.c_double(0.0)
    st = load().lbm_set_geometry_braid(ctx, g_rad, A, B, _f64(anchors.reshape(-1)),
                                       anchors.shape[0], phi, ctypes.byref(used),
                                       ctypes.byref(frac))
    return st, used.value, frac.value


def lbm_get_geometry(ctx, out: np.ndarray) -> int:
    assert out.dtype == np.uint8 and out.flags.c_contiguous
    return load().lbm_get_geometry(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))


def lbm_yarn_conductivity(lam_fL: float, lam_fT: float, lam_m: float, phi_fy: float):
    """Returns (status, lam_L, lam_T) of Eq. 36-37."""
    L, T = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().lbm_yarn_conductivity(lam_fL, lam_fT, lam_m, phi_fy, ctypes.byref(L), ctypes.byref(T))
    return st, L.value, T.value


def lbm_braid_unit_cell(phi_f: float, n_f: int, d_f: float, gamma_rad: float):
    """Returns (status, a, h, c, d, phi_fy) of Eq. 32-35."""
    out = [ctypes.c_double(0.0) for _ in range(5)]
    st = load().lbm_braid_unit_cell(phi_f, n_f, d_f, gamma_rad, *[ctypes.byref(o) for o in out])
    return (st,) + tuple(o.value for o in out)


LBM_NOALLOC_MAX_YARNS = 1024


def lbm_braid_voxelize_noalloc(nx: int, ny: int, nz: int, g_rad: float, A: float, B: float,
                               d_anchors: int, n_max: int, phi: float, d_phase: int,
                               stream: int | None = None):
    """Allocation-free voxeliser: d_anchors and d_phase are device
    addresses the caller owns.  Returns (status, n_used, fraction, message)."""
    used = ctypes.c_int(0)
    frac = ctypes.c_double(0.0)
    msg = ctypes.create_string_buffer(256)
    st = load().lbm_braid_voxelize_noalloc(nx, ny, nz, g_rad, A, B, d_anchors, n_max, phi,
                                           d_phase, ctypes.byref(used), ctypes.byref(frac),
                                           stream, msg, len(msg))
    return st, used.value, frac.value, msg.value.decode()


def lbm_debug_build() -> int:
    return int(load().lbm_debug_build())


def lbm_debug_error(clear: bool = True):
    """Returns (status, recorded bounds-check code)."""
    v = ctypes.c_uint(0)
    st = load().lbm_debug_error(ctypes.byref(v), int(clear))
    return st, v.value


def lbm_get_launch_plan(ctx):
    p = lbm_launch_plan()
    st = load().lbm_get_launch_plan(ctx, ctypes.byref(p))
    return st, p


def lbm_state_bytes(ctx) -> int:
    return int(load().lbm_state_bytes(ctx))


def lbm_get_state(ctx, out: np.ndarray) -> int:
    assert out.dtype == np.uint8 and out.flags.c_contiguous
    return load().lbm_get_state(ctx, out.ctypes.data, out.nbytes)


def lbm_set_state(ctx, state: np.ndarray) -> int:
    state = np.ascontiguousarray(state, dtype=np.uint8)
    return load().lbm_set_state(ctx, state.ctypes.data, state.nbytes)


def lbm_last_error(ctx) -> str:
    s = load().lbm_last_error(ctx)
    return s.decode() if s else ""


def lbm_destroy(ctx) -> None:
    load().lbm_destroy(ctx)


def lbm_batch_create(cuda_device: int = 0):
    h = _ctx_p()
    st = load().lbm_batch_create(cuda_device, ctypes.byref(h))
    return st, h


def lbm_batch_add(b, phase: np.ndarray, n_phases: int, lam: np.ndarray, axis: int):
    phase = np.ascontiguousarray(phase, dtype=np.uint8)
    lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
    nz, ny, nx = phase.shape
    i = ctypes.c_int(-1)
    st = load().lbm_batch_add(b, nx, ny, nz, phase.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              int(n_phases), _f64(lam), int(axis), ctypes.byref(i))
    return st, i.value


def lbm_batch_solve(b, lateral: int, opts: lbm_solve_opts | None = None,
                    info: lbm_batch_info | None = None) -> int:
    return load().lbm_batch_solve(b, lateral, ctypes.byref(opts) if opts is not None else None,
                                  ctypes.byref(info) if info is not None else None)


def lbm_batch_result(b, i: int, info: lbm_solve_info) -> int:
    return load().lbm_batch_result(b, i, ctypes.byref(info))


def lbm_batch_get_temperature(b, i: int, out: np.ndarray) -> int:
    assert out.dtype == np.float32 and out.flags.c_contiguous
    return load().lbm_batch_get_temperature(b, i, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))


def lbm_batch_set_initial(b, i: int, t_init) -> int:
    if t_init is None:
        return load().lbm_batch_set_initial(b, i, None)
    t_init = np.ascontiguousarray(t_init, dtype=np.float32)
    return load().lbm_batch_set_initial(b, i, t_init.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))


def lbm_batch_get_history(b, i: int, max_entries: int = 4096):
    """Returns (status, array (n, 5) of iteration, k_eff, R_T, R_Q, ms)."""
    out = np.zeros((max_entries, 5), np.float64)
    n = ctypes.c_int(0)
    st = load().lbm_batch_get_history(b, i, _f64(out), max_entries, ctypes.byref(n))
    return st, out[: n.value]


def lbm_batch_last_error(b) -> str:
    s = load().lbm_batch_last_error(b)
    return s.decode() if s else ""


def lbm_batch_destroy(b) -> None:
    load().lbm_batch_destroy(b)


# ---- network layers (device pointers as ints, cudaStream_t as int) -------

def _nn(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    call.__doc__ = f"{name}: see include/lbm.h; arguments are device addresses and sizes."
    return call


lbm_nn_conv3d = _nn("lbm_nn_conv3d")
lbm_nn_conv3d_wgrad = _nn("lbm_nn_conv3d_wgrad")
lbm_nn_conv3d_tc = _nn("lbm_nn_conv3d_tc")
lbm_nn_conv3d_tc_supported = _nn("lbm_nn_conv3d_tc_supported")
lbm_nn_conv3d_tc_cfg = _nn("lbm_nn_conv3d_tc_cfg")
lbm_nn_conv3d_wgrad_tc = _nn("lbm_nn_conv3d_wgrad_tc")
lbm_nn_conv3d_wgrad_tc_supported = _nn("lbm_nn_conv3d_wgrad_tc_supported")
lbm_nn_weights_kmajor = _nn("lbm_nn_weights_kmajor")


def lbm_nn_tc_error(clear: bool = True) -> int:
    """Error word of the tensor-core convolution (0: none); raises on a CUDA error."""
    v = ctypes.c_int(0)
    st = load().lbm_nn_tc_error(ctypes.byref(v), int(clear))
    if st != LBM_OK:
        raise LBMError(st, "reading the tensor-core convolution's error word failed")
    return v.value
lbm_nn_flip_weights = _nn("lbm_nn_flip_weights")
lbm_nn_bias_grad = _nn("lbm_nn_bias_grad")
lbm_nn_relu_mask = _nn("lbm_nn_relu_mask")
lbm_nn_pool2 = _nn("lbm_nn_pool2")
lbm_nn_upsample2 = _nn("lbm_nn_upsample2")
lbm_nn_concat = _nn("lbm_nn_concat")
lbm_nn_slice = _nn("lbm_nn_slice")
lbm_nn_head = _nn("lbm_nn_head")
lbm_nn_input = _nn("lbm_nn_input")
lbm_nn_adam = _nn("lbm_nn_adam")


# ---- convenience object ---------------------------------------------------

class LBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Solver:
    """One solver context for an (nz, ny, nx) cell on one CUDA device."""

    def __init__(self, nx: int, ny: int, nz: int, device: int = 0, workspace=None):
        """workspace: optional (device pointer, bytes) from which all of the
        context's device memory is carved (lbm_create_with_workspace); the
        caller keeps it alive until close()."""
        if workspace is None:
            st, h = lbm_create(nx, ny, nz, device)
        else:
            st, h = lbm_create_with_workspace(nx, ny, nz, device, int(workspace[0]), int(workspace[1]))
        if st != LBM_OK:
            raise LBMError(st, f"creating the context for {nx}x{ny}x{nz} on device {device} failed")
        self.h = h
        self.shape = (nz, ny, nx)

    def _ok(self, st: int, allow=()) -> int:
        if st != LBM_OK and st not in allow:
            raise LBMError(st, lbm_last_error(self.h))
        return st

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_geometry(self, phase, n_phases):
        self._ok(lbm_set_geometry(self.h, phase, n_phases))

    def set_tensors(self, lam):
        lam = np.asarray(lam, dtype=np.float64).reshape(-1, 6)
        self._ok(lbm_set_tensors(self.h, lam, lam.shape[0]))

    def set_geometry_braid(self, g_rad, anchors, phi, A=10.0, B=6.0):
        st, used, frac = lbm_set_geometry_braid(self.h, g_rad, A, B, anchors, phi)
        self._ok(st)
        return used, frac

    def geometry(self):
        out = np.empty(self.shape, np.uint8)
        self._ok(lbm_get_geometry(self.h, out))
        return out

    @staticmethod
    def opts(**kw) -> lbm_solve_opts:
        o = lbm_default_opts()
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def start(self, axis=2, lateral=0, opts=None):
        self._ok(lbm_start(self.h, axis, lateral, opts))

    def advance(self, n):
        self._ok(lbm_advance(self.h, n))

    def check(self) -> lbm_solve_info:
        info = lbm_solve_info()
        self._ok(lbm_check(self.h, info))
        return info

    def run(self, allow=(LBM_ERR_NOT_CONVERGED,)) -> lbm_solve_info:
        info = lbm_solve_info()
        self._ok(lbm_run(self.h, info), allow)
        return info

    def solve(self, axis=2, lateral=0, opts=None, allow=(LBM_ERR_NOT_CONVERGED,)):
        info = lbm_solve_info()
        self._ok(lbm_solve(self.h, axis, lateral, opts, info), allow)
        return info

    def k_eff(self) -> float:
        st, k = lbm_k_eff(self.h)
        self._ok(st)
        return k

    def temperature(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape, np.float32)
        self._ok(lbm_get_temperature(self.h, out))
        return out

    def history(self) -> np.ndarray:
        st, h = lbm_get_history(self.h)
        self._ok(st)
        return h

    def launch_plan(self) -> dict:
        st, p = lbm_get_launch_plan(self.h)
        self._ok(st)
        return p.as_dict()

    def get_state(self) -> np.ndarray:
        out = np.empty(lbm_state_bytes(self.h), np.uint8)
        self._ok(lbm_get_state(self.h, out))
        return out

    def set_state(self, state: np.ndarray):
        self._ok(lbm_set_state(self.h, state))

    def plane_flux(self, n_axis: int) -> np.ndarray:
        out = np.empty(n_axis, np.float64)
        self._ok(lbm_get_plane_flux(self.h, out))
        return out


class Batch:
    """Many independent solves advanced together by one graph launch."""

    def __init__(self, device: int = 0):
        st, h = lbm_batch_create(device)
        if st != LBM_OK:
            raise LBMError(st, "lbm_batch_create failed")
        self.h = h
        self.shapes = []

    def _ok(self, st, allow=()):
        if st != LBM_OK and st not in allow:
            raise LBMError(st, lbm_batch_last_error(self.h))
        return st

    def add(self, phase, lam, axis) -> int:
        lam = np.asarray(lam, dtype=np.float64).reshape(-1, 6)
        st, i = lbm_batch_add(self.h, phase, lam.shape[0], lam, axis)
        self._ok(st)
        self.shapes.append(np.asarray(phase).shape)
        return i

    def solve(self, lateral=0, opts=None) -> lbm_batch_info:
        info = lbm_batch_info()
        self._ok(lbm_batch_solve(self.h, lateral, opts, info))
        return info

    def result(self, i) -> lbm_solve_info:
        info = lbm_solve_info()
        self._ok(lbm_batch_result(self.h, i, info))
        return info

    def temperature(self, i) -> np.ndarray:
        out = np.empty(self.shapes[i], np.float32)
        self._ok(lbm_batch_get_temperature(self.h, i, out))
        return out

    def set_initial(self, i, t_init):
        if t_init is not None:
            assert tuple(np.shape(t_init)) == tuple(self.shapes[i])
        self._ok(lbm_batch_set_initial(self.h, i, t_init))

    def history(self, i) -> np.ndarray:
        st, h = lbm_batch_get_history(self.h, i)
        self._ok(st)
        return h

    def close(self):
        if getattr(self, "h", None):
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
