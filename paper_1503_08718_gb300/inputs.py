"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module only *draws and lays out* inputs: voxel phase maps built from
integer rules, conductivity tensors of the material model, yarn anchor points
and sweep parameters.  It contains none of the lattice Boltzmann arithmetic,
so the CUDA path and the FP64 oracle can both consume its output without
sharing any of the method's code.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), a counter-based generator
whose published definition is reproduced here from that description.

Tensor layout everywhere: six components per phase in the order
(xx, yy, zz, yz, xz, xy).
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """splitmix64: state advances by the golden-ratio increment, output is
    the state passed through the 'variant 13' 64-bit finaliser."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1): top 53 bits times 2**-53."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# Conductivity tensors (material model of the paper's Eq. 26, written in 3D)
# --------------------------------------------------------------------------

def sym6(m) -> np.ndarray:
    """3x3 symmetric matrix -> (xx, yy, zz, yz, xz, xy)."""
    m = np.asarray(m, dtype=np.float64)
    return np.array([m[0, 0], m[1, 1], m[2, 2], m[1, 2], m[0, 2], m[0, 1]])


def full3(t6) -> np.ndarray:
    """(xx, yy, zz, yz, xz, xy) -> 3x3 symmetric matrix."""
    xx, yy, zz, yz, xz, xy = [float(v) for v in t6]
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def isotropic(k: float) -> np.ndarray:
    return sym6(np.eye(3) * k)


def transversely_isotropic(k_axial: float, k_trans: float, d) -> np.ndarray:
    """Tensor with conductivity k_axial along the unit axis d and k_trans
    across it: k_trans * I + (k_axial - k_trans) * d d^T (Eq. 26 rotated
    into xyz for a yarn whose principal axis is d)."""
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return sym6(k_trans * np.eye(3) + (k_axial - k_trans) * np.outer(d, d))


def axis_in_xz_from_z(angle_deg: float) -> np.ndarray:
    """Unit vector in the xz-plane at angle_deg from +z toward +x."""
    a = math.radians(angle_deg)
    return np.array([math.sin(a), 0.0, math.cos(a)])


def slab_tensor_2d_rotated(lam_eta: float, lam_zeta: float, beta_deg: float) -> np.ndarray:
    """Section 3.1 slab: principal values (eta, zeta) rotated by beta in the
    plane spanned by the lateral axis x and the flux axis z (Eq. 26 with the
    paper's y read as z).  Returns the 3D tensor with k_yy = lam_zeta."""
    b = math.radians(beta_deg)
    r = np.array([[math.cos(b), math.sin(b)], [-math.sin(b), math.cos(b)]])
    m2 = r @ np.diag([lam_eta, lam_zeta]) @ r.T
    m = np.zeros((3, 3))
    m[0, 0], m[0, 2], m[2, 0], m[2, 2] = m2[0, 0], m2[0, 1], m2[1, 0], m2[1, 1]
    m[1, 1] = lam_zeta
    return sym6(m)


def random_spd(rng: np.random.Generator, lo: float = 0.2, hi: float = 6.0) -> np.ndarray:
    """Random symmetric positive-definite tensor with eigenvalues in [lo, hi]."""
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    ev = rng.uniform(lo, hi, size=3)
    return sym6(q @ np.diag(ev) @ q.T)


# --------------------------------------------------------------------------
# Phase maps (uint8, shape (nz, ny, nx), x fastest)
# --------------------------------------------------------------------------

def layered_phase(nx: int, ny: int, nz: int, layer: int = 8, axis: int = 2,
                  first: int = 0) -> np.ndarray:
    """Alternating layers of `layer` voxels stacked along `axis`
    (0 = x, 1 = y, 2 = z); phase = first ^ ((coord // layer) & 1)."""
    idx = np.indices((nz, ny, nx))
    coord = idx[2 - axis]
    return (((coord // layer) & 1) ^ first).astype(np.uint8)


def random_phase(rng: np.random.Generator, nx: int, ny: int, nz: int,
                 n_phases: int) -> np.ndarray:
    return rng.integers(0, n_phases, size=(nz, ny, nx), dtype=np.uint8)


# --------------------------------------------------------------------------
# Synthetic four-directional braided cell parameters
# --------------------------------------------------------------------------

BRAID_SEMI_MAJOR = 10.0  # voxels
BRAID_SEMI_MINOR = 6.0   # voxels
BRAID_K_AXIAL = 6.0
BRAID_K_TRANS = 0.8
BRAID_K_MATRIX = 0.2
BRAID_FAMILY_SIGNS = ((1, 1), (-1, 1), (-1, -1), (1, -1))


def braid_anchors(nx: int, ny: int, seed: int, n_max: int = 256) -> np.ndarray:
    """Yarn anchor points (x0, y0) at z = 0, drawn in order from
    splitmix64(seed): x0 = nx * U, y0 = ny * U.  Shape (n_max, 2)."""
    g = SplitMix64(seed)
    out = np.empty((n_max, 2), dtype=np.float64)
    for i in range(n_max):
        out[i, 0] = nx * g.uniform()
        out[i, 1] = ny * g.uniform()
    return out


def braid_family_axes(g_deg: float) -> np.ndarray:
    """Unit yarn axes of the four families at interior braiding angle g
    (measured from +z): (sx sin g / sqrt2, sy sin g / sqrt2, cos g)."""
    g = math.radians(g_deg)
    s = math.sin(g) / math.sqrt(2.0)
    return np.array([[sx * s, sy * s, math.cos(g)] for sx, sy in BRAID_FAMILY_SIGNS])


def braid_tensors(g_deg: float, k_axial: float = BRAID_K_AXIAL,
                  k_trans: float = BRAID_K_TRANS,
                  k_matrix: float = BRAID_K_MATRIX) -> np.ndarray:
    """Five phases: matrix (isotropic) then the four yarn families."""
    rows = [isotropic(k_matrix)]
    for d in braid_family_axes(g_deg):
        rows.append(transversely_isotropic(k_axial, k_trans, d))
    return np.stack(rows)


def braid_sweep_cells(n_cells: int = 64, seed0: int = 1000):
    """Uneven-size cells of the batched sweep: per cell c, splitmix64(seed0+c)
    draws N_xy in {64, 80, ..., 160}, N_z in {N_xy, 2 N_xy} capped at 320,
    yarn fraction in U(0.30, 0.60) and braiding angle in U(20, 45) deg."""
    cells = []
    for c in range(n_cells):
        g = SplitMix64(seed0 + c)
        nxy = 64 + 16 * (g.next_u64() % 7)
        nz = min(nxy * (1 + int(g.next_u64() % 2)), 320)
        phi = 0.30 + 0.30 * g.uniform()
        ang = 20.0 + 25.0 * g.uniform()
        cells.append(dict(nx=int(nxy), ny=int(nxy), nz=int(nz), phi=phi,
                          g_deg=ang, seed=seed0 + c))
    return cells



def warm_cell_params(seed: int, g_range=(20.0, 45.0), phi_range=(0.30, 0.60)):
    """Braiding angle and yarn fraction of the seeded braided cells of the
    learned warm start (training, evaluation and the combined-form batch):
    splitmix64(10000 + seed) draws g in U(20, 45) deg, then phi in
    U(0.30, 0.60); the yarn anchors come from braid_anchors(..., seed)."""
    r = SplitMix64(10_000 + int(seed))
    g = g_range[0] + (g_range[1] - g_range[0]) * r.uniform()
    phi = phi_range[0] + (phi_range[1] - phi_range[0]) * r.uniform()
    return g, phi
