"""Test-side helpers built on the oracle's public step function.

`direct_fixed_point` solves the steady lattice Boltzmann problem as one dense
linear system instead of iterating: one oracle step is an affine map
f -> A f + b, so the fixed point solves (I - A) f = b.  A is assembled column
by column by stepping unit vectors on a copy of the lattice whose wall
temperatures are zero (the linear part), and b is one step of the zero state
with the real wall temperatures.  This pins the iteration's end point without
trusting the iteration loop or its stopping rule.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O


def direct_fixed_point(phase, lam, s, axis, lateral, t_hot=1.0, t_cold=0.0):
    lin = O.Lattice(phase, lam, s, axis, lateral, 0.0, 0.0)
    aff = O.Lattice(phase, lam, s, axis, lateral, t_hot, t_cold)
    n = 7 * lin.N
    A = np.empty((n, n))
    e = np.zeros(n)
    for k in range(n):
        e[k] = 1.0
        lin.set_f(e)
        lin.step(1)
        A[:, k] = lin.get_f().reshape(-1)
        e[k] = 0.0
    aff.set_f(np.zeros(n))
    aff.step(1)
    b = aff.get_f().reshape(-1)
    f = np.linalg.solve(np.eye(n) - A, b)
    aff.set_f(f)
    return aff, f


def mirror_doubled(phase, lam, axis):
    """Doubles the cell across both lateral faces (mirror images) and gives
    each mirrored copy the reflected tensors.  Reflecting coordinate b flips
    the sign of every off-diagonal component that carries b once."""
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, 6)
    n_ph = lam.shape[0]
    lats = [b for b in range(3) if b != axis]
    # off-diagonal components (yz, xz, xy) -> the pair of axes they couple
    pairs = {3: (1, 2), 4: (0, 2), 5: (0, 1)}
    new_lam = []
    for code in range(4):
        flips = [lats[0]] * (code & 1) + [lats[1]] * ((code >> 1) & 1)
        t = lam.copy()
        for b in flips:
            for comp, (p, q) in pairs.items():
                if b in (p, q):
                    t[:, comp] = -t[:, comp]
        new_lam.append(t)
    new_lam = np.concatenate(new_lam, axis=0)

    ph = np.asarray(phase)
    out = ph
    codes = np.zeros_like(ph, dtype=np.int64)
    for bit, b in enumerate(lats):
        arr_axis = 2 - b  # array axis of coordinate b
        out = np.concatenate([out, np.flip(out, axis=arr_axis)], axis=arr_axis)
        codes = np.concatenate([codes, np.flip(codes, axis=arr_axis) + (1 << bit)],
                               axis=arr_axis)
    new_phase = (out.astype(np.int64) + n_ph * codes).astype(np.uint8)
    return new_phase, new_lam


def harmonic_series(lams_aa, thicknesses):
    t = np.asarray(thicknesses, dtype=np.float64)
    return t.sum() / np.sum(t / np.asarray(lams_aa, dtype=np.float64))
