"""Pins of the oracle's synthetic braided-cell voxeliser (step-wise yarn
boundaries, Section 3.2; yarns at interior braiding angle g from z,
Section 4.1) against an independent numpy construction of the same cell."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1503_08718_gb300 import inputs as I


def _numpy_membership(nx, ny, nz, g_deg, anchors, A=10.0, B=6.0):
    """ellipse coordinate rho^2 = (w.u/A)^2 + (w.v/B)^2 of every voxel centre
    for every yarn, using the 3D offset from the anchor and all periodic
    images instead of the oracle's horizontal minimum-image offset."""
    axes = I.braid_family_axes(g_deg)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5,
                          np.arange(nx) + 0.5, indexing="ij")
    c = np.stack([x, y, z], -1)
    rho = np.full((len(anchors), nz, ny, nx), np.inf)
    for i, (x0, y0) in enumerate(anchors):
        d = axes[i % 4]
        u = np.cross([0.0, 0.0, 1.0], d)
        u /= np.linalg.norm(u)
        v = np.cross(d, u)
        for mx in (-1, 0, 1):
            for my in (-1, 0, 1):
                r = c - np.array([x0 + mx * nx, y0 + my * ny, 0.0])
                w = r - (r @ d)[..., None] * d
                val = (w @ u / A) ** 2 + (w @ v / B) ** 2
                rho[i] = np.minimum(rho[i], val)
    return rho


@pytest.mark.parametrize("g_deg,phi,seed", [(30.0, 0.30, 42), (22.5, 0.45, 3)])
def test_braid_voxeliser_matches_independent_geometry(g_deg, phi, seed):
    nx, ny, nz = 48, 48, 24
    anchors = I.braid_anchors(nx, ny, seed, n_max=64)
    phase, used, frac = O.braid_phase(nx, ny, nz, math.radians(g_deg), anchors, phi)
    assert phase.dtype == np.uint8 and phase.max() <= 4
    assert frac >= phi
    assert frac == pytest.approx(np.count_nonzero(phase) / phase.size)

    rho = _numpy_membership(nx, ny, nz, g_deg, anchors[:used])
    inside = rho <= 1.0
    # first containing yarn decides the family; matrix where none contains it
    first = np.where(inside.any(0), inside.argmax(0), -1)
    expect = np.where(first >= 0, 1 + first % 4, 0).astype(np.uint8)
    margin = np.abs(rho - 1.0).min(0)
    sure = margin > 1e-9
    assert np.count_nonzero(~sure) < 0.001 * phase.size
    assert np.array_equal(phase[sure], expect[sure])

    # the yarn count is the smallest that reaches phi
    prev = np.count_nonzero(inside[: used - 1].any(0)) / phase.size
    assert prev < phi


def test_braid_voxeliser_rejects_unreachable_fraction():
    anchors = I.braid_anchors(32, 32, 1, n_max=2)
    with pytest.raises(ValueError):
        O.braid_phase(32, 32, 8, math.radians(30.0), anchors, 0.9)


def test_braid_yarn_cross_section_area():
    """An isolated yarn cuts each horizontal plane in an ellipse of area
    pi A B / cos g (oblique cylinder), so its voxel count per plane is close."""
    nx = ny = 64
    g = 30.0
    anchors = np.array([[32.0, 32.0]])
    phase, used, frac = O.braid_phase(nx, ny, 4, math.radians(g), anchors, 1e-6)
    per_plane = np.count_nonzero(phase) / 4
    assert per_plane == pytest.approx(math.pi * 10 * 6 / math.cos(math.radians(g)), rel=0.03)
