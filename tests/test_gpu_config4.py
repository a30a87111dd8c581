"""The largest cell, 256x256x512 (braid angle 35 deg, yarn fraction 0.50,
seed 7): voxelisation, and 20 iterations along every axis with FP32, BF16 and
FP16 storage, compared with the FP64 oracle on every voxel.

This is the precision workload (2 x 0.94 GB of FP32 distributions, far
beyond L2) run in the launch configuration the solver uses for it: FP32
plain steps as fused pairs (rows of 256 nodes), 16-bit storage as single
steps.  Tolerances are those of the smaller parity cases: FP32 max|dT| and
k_eff relative 1e-5; 16-bit storage 0.5 u and 0.02 u (u the unit roundoff
of the format), the bounds of the storage tests.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1503_08718_gb300 import inputs as I
from paper_1503_08718_gb300 import lbm

pytestmark = pytest.mark.gpu

NX, NY, NZ = 256, 256, 512
G_DEG, PHI, SEED, NMAX = 35.0, 0.50, 7, 1024
N_ITER = 20
U = {lbm.LBM_STORE_BF16: 2.0 ** -8, lbm.LBM_STORE_F16: 2.0 ** -11}
T_TOL = {lbm.LBM_STORE_F32: 1e-5, **{k: 0.5 * u for k, u in U.items()}}
K_TOL = {lbm.LBM_STORE_F32: 1e-5, **{k: 0.02 * u for k, u in U.items()}}


@pytest.fixture(scope="module")
def cell():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_08718_gb300 import build
    build.build()
    lbm.load()
    anchors = I.braid_anchors(NX, NY, SEED, n_max=NMAX)
    g = math.radians(G_DEG)
    S = lbm.Solver(NX, NY, NZ)
    used, frac = S.set_geometry_braid(g, anchors, PHI)
    S.set_tensors(I.braid_tensors(G_DEG))
    ph_ref, used_ref, frac_ref = O.braid_phase(NX, NY, NZ, g, anchors, PHI)
    yield S, (used, frac), ph_ref, (used_ref, frac_ref)
    S.close()


def test_voxeliser_bit_exact_256x256x512(cell):
    S, got, ph_ref, want = cell
    assert got == want
    assert np.array_equal(S.geometry(), ph_ref)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_20_iterations_every_axis_and_storage(cell, axis):
    S, _, ph_ref, _ = cell
    lam = I.braid_tensors(G_DEG)
    ref = None
    for storage in (lbm.LBM_STORE_F32, lbm.LBM_STORE_BF16, lbm.LBM_STORE_F16):
        S.start(axis, 0, S.opts(storage=storage))
        S.advance(N_ITER - 1)
        info = S.check()
        if ref is None:
            L = O.Lattice(ph_ref, lam, info.lattice_scale, axis, 0)
            L.init_linear()
            L.step(N_ITER)
            ref = (L.temperature().astype(np.float64), L.k_eff()[0])
            del L
        dT = float(np.max(np.abs(S.temperature().astype(np.float64) - ref[0])))
        assert dT <= T_TOL[storage], (storage, dT)
        assert info.k_eff == pytest.approx(ref[1], rel=K_TOL[storage]), storage
