"""Python access to the FP64 CPU oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg use this module; the product package never
imports it.  The oracle is built from C with gcc (-O2, -ffp-contract=off,
OpenMP over planes); `build()` compiles it in place.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "_build", "liblbmoracle.so")

_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_u8 = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no CUDA)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [_i64, _i64, _i64, _u8, ctypes.c_int, _d,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_init_linear.argtypes = [ctypes.c_void_p]
            L.orc_init_field.argtypes = [ctypes.c_void_p, _d]
            L.orc_set_f.argtypes = [ctypes.c_void_p, _d]
            L.orc_get_f.argtypes = [ctypes.c_void_p, _d]
            L.orc_iter.restype = _i64
            L.orc_iter.argtypes = [ctypes.c_void_p]
            L.orc_step.argtypes = [ctypes.c_void_p, _i64]
            L.orc_temperature.argtypes = [ctypes.c_void_p, _d]
            L.orc_flux_field.restype = ctypes.c_int
            L.orc_flux_field.argtypes = [ctypes.c_void_p, _d]
            L.orc_plane_flux.restype = ctypes.c_int
            L.orc_plane_flux.argtypes = [ctypes.c_void_p, _d]
            L.orc_k_eff.restype = ctypes.c_int
            L.orc_k_eff.argtypes = [ctypes.c_void_p, _d, _d]
            L.orc_solve.restype = ctypes.c_int
            L.orc_solve.argtypes = [ctypes.c_void_p, ctypes.c_double, _i64, _i64, _d]
            L.orc_moment_matrix.argtypes = [_d]
            L.orc_tau.argtypes = [_d, ctypes.c_double, _d]
            L.orc_collision_matrix.restype = ctypes.c_int
            L.orc_collision_matrix.argtypes = [_d, ctypes.c_double, _d]
            L.orc_collide_node.argtypes = [_d, _d, _d]
            L.orc_lattice_scale.restype = ctypes.c_double
            L.orc_lattice_scale.argtypes = [_d, ctypes.c_int, ctypes.c_double]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_max_threads.restype = ctypes.c_int
            L.orc_braid_phase.restype = ctypes.c_int
            L.orc_braid_phase.argtypes = [_i64, _i64, _i64, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, _d,
                                          ctypes.c_int, ctypes.c_double, _u8,
                                          ctypes.POINTER(ctypes.c_int), _d]
            _lib = L
        return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_d)


def moment_matrix() -> np.ndarray:
    M = np.zeros(49)
    lib().orc_moment_matrix(_dp(M))
    return M.reshape(7, 7)


def tau_matrix(lam6, s: float) -> np.ndarray:
    lam6 = np.ascontiguousarray(lam6, dtype=np.float64)
    t = np.zeros(9)
    lib().orc_tau(_dp(lam6), s, _dp(t))
    return t.reshape(3, 3)


def collision_matrix(lam6, s: float) -> np.ndarray:
    lam6 = np.ascontiguousarray(lam6, dtype=np.float64)
    om = np.zeros(49)
    if lib().orc_collision_matrix(_dp(lam6), s, _dp(om)):
        raise ValueError("singular relaxation matrix")
    return om.reshape(7, 7)


def collide_node(omega: np.ndarray, f) -> np.ndarray:
    om = np.ascontiguousarray(omega, dtype=np.float64).reshape(49)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(7)
    lib().orc_collide_node(_dp(om), _dp(f), _dp(out))
    return out


def lattice_scale(lam, tau_max: float = 1.5) -> float:
    lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1, 6)
    return lib().orc_lattice_scale(_dp(lam), lam.shape[0], tau_max)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


class Lattice:
    """One FP64 oracle lattice.  phase has shape (nz, ny, nx), x fastest;
    lam has shape (n_phases, 6) in (xx, yy, zz, yz, xz, xy) order."""

    def __init__(self, phase, lam, s: float, axis: int = 2, lateral: int = 0,
                 t_hot: float = 1.0, t_cold: float = 0.0):
        self.phase = np.ascontiguousarray(phase, dtype=np.uint8)
        self.lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1, 6)
        nz, ny, nx = self.phase.shape
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.axis, self.lateral, self.s = axis, lateral, s
        self.t_hot, self.t_cold = t_hot, t_cold
        self._h = lib().orc_create(nx, ny, nz, self.phase.ctypes.data_as(_u8),
                                   self.lam.shape[0], _dp(self.lam), s, axis,
                                   lateral, t_hot, t_cold)
        if not self._h:
            raise ValueError("oracle rejected the lattice description")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init_linear(self):
        lib().orc_init_linear(self._h)

    def init_field(self, T):
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
        lib().orc_init_field(self._h, _dp(T))

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        assert f.size == 7 * self.N
        lib().orc_set_f(self._h, _dp(f))

    def get_f(self) -> np.ndarray:
        f = np.zeros(7 * self.N)
        lib().orc_get_f(self._h, _dp(f))
        return f.reshape((7,) + self.shape)

    @property
    def iter(self) -> int:
        return int(lib().orc_iter(self._h))

    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    def temperature(self) -> np.ndarray:
        T = np.zeros(self.N)
        lib().orc_temperature(self._h, _dp(T))
        return T.reshape(self.shape)

    def flux(self) -> np.ndarray:
        q = np.zeros(3 * self.N)
        if lib().orc_flux_field(self._h, _dp(q)):
            raise ValueError("singular tau block")
        return q.reshape((3,) + self.shape)

    def plane_flux(self) -> np.ndarray:
        n_a = self.shape[2 - self.axis]
        Qk = np.zeros(n_a)
        if lib().orc_plane_flux(self._h, _dp(Qk)):
            raise ValueError("plane flux failed")
        return Qk

    def k_eff(self):
        k = np.zeros(1)
        rq = np.zeros(1)
        if lib().orc_k_eff(self._h, _dp(k), _dp(rq)):
            raise ValueError("k_eff failed")
        return float(k[0]), float(rq[0])

    def solve(self, tol: float = 1e-8, check_every: int = 100,
              max_iters: int = 10_000_000):
        rt = np.zeros(1)
        rc = lib().orc_solve(self._h, tol, int(check_every), int(max_iters), _dp(rt))
        return rc, float(rt[0])


def braid_phase(nx: int, ny: int, nz: int, g_rad: float, anchors, phi: float,
                A: float = 10.0, B: float = 6.0):
    """The oracle's own voxelisation of the synthetic braided cell.
    Returns (phase (nz, ny, nx) uint8, yarns used, achieved fraction)."""
    anchors = np.ascontiguousarray(anchors, dtype=np.float64).reshape(-1, 2)
    phase = np.zeros((nz, ny, nx), dtype=np.uint8)
    used = ctypes.c_int(0)
    frac = np.zeros(1)
    rc = lib().orc_braid_phase(nx, ny, nz, g_rad, A, B, _dp(anchors.reshape(-1)),
                               anchors.shape[0], phi, phase.ctypes.data_as(_u8),
                               ctypes.byref(used), _dp(frac))
    if rc:
        raise ValueError(f"oracle voxeliser failed ({rc})")
    return phase, used.value, float(frac[0])
