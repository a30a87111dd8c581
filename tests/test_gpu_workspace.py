"""Contexts whose device memory is a caller's workspace (here a torch tensor):
the same solves as an ordinary context, bit for bit, and no device memory of
their own."""
import math

import numpy as np
import pytest

from paper_1503_08718_gb300 import inputs as I
from paper_1503_08718_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_08718_gb300 import build
    build.build()
    lbm.load()
    return t


def _workspace(torch, nbytes):
    ws = torch.full((nbytes,), 0x7F, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    return ws


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_F32, lbm.LBM_STORE_BF16])
def test_workspace_context_equals_ordinary_context(torch, storage):
    rng = np.random.default_rng(5 + storage)
    shape = (40, 24, 20)
    lam = np.stack([I.random_spd(rng) for _ in range(3)])
    phase = I.random_phase(rng, *shape, 3)
    nbytes = lbm.lbm_workspace_bytes(*shape, storage)
    ws = _workspace(torch, nbytes)
    A = lbm.Solver(*shape, workspace=(ws.data_ptr(), nbytes))
    B = lbm.Solver(*shape)
    for S in (A, B):
        S.set_geometry(phase, 3)
        S.set_tensors(lam)
    for axis in (0, 1, 2):
        for lateral in (0, 1):
            o = lbm.Solver.opts(tol=0.0, max_iters=300, storage=storage)
            ia, ib = A.solve(axis, lateral, o), B.solve(axis, lateral, o)
            assert ia.k_eff == ib.k_eff and ia.iters == ib.iters
            assert np.array_equal(A.temperature(), B.temperature())
            assert np.array_equal(A.plane_flux(shape[axis]), B.plane_flux(shape[axis]))
    # the state lives in the caller's tensor
    assert int((ws != 0x7F).sum().item()) > 7 * shape[0] * shape[1] * shape[2]
    A.close()
    B.close()


def test_workspace_braid_geometry_and_memory(torch):
    """The voxeliser keeps its scratch in the workspace too; a context on a
    workspace takes no device memory of its own for its buffers."""
    nx, ny, nz = 128, 64, 96
    nbytes = lbm.lbm_workspace_bytes(nx, ny, nz, lbm.LBM_STORE_F32)
    ws = _workspace(torch, nbytes)
    anchors = I.braid_anchors(nx, ny, 3, n_max=256)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    A = lbm.Solver(nx, ny, nz, workspace=(ws.data_ptr(), nbytes))
    used_a = A.set_geometry_braid(math.radians(30.0), anchors, 0.4)
    A.set_tensors(I.braid_tensors(30.0))
    ia = A.solve(2, 0, lbm.Solver.opts(tol=0.0, max_iters=200))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # streams, events and graphs take a little; the buffers (~nbytes) do not
    assert free0 - free1 < nbytes // 2
    B = lbm.Solver(nx, ny, nz)
    used_b = B.set_geometry_braid(math.radians(30.0), anchors, 0.4)
    B.set_tensors(I.braid_tensors(30.0))
    ib = B.solve(2, 0, lbm.Solver.opts(tol=0.0, max_iters=200))
    assert used_a == used_b
    assert np.array_equal(A.geometry(), B.geometry())
    assert ia.k_eff == ib.k_eff
    A.close()
    B.close()


def test_workspace_errors(torch):
    shape = (32, 16, 24)
    f32 = lbm.lbm_workspace_bytes(*shape, lbm.LBM_STORE_F32)
    b16 = lbm.lbm_workspace_bytes(*shape, lbm.LBM_STORE_BF16)
    ws = _workspace(torch, f32)
    p = ws.data_ptr()
    # misaligned, host memory, too small for the cell's own buffers
    for ptr, n in ((p + 16, f32 - 16), (np.zeros(f32, np.uint8).ctypes.data, f32), (p, 4096)):
        st, h = lbm.lbm_create_with_workspace(*shape, 0, ptr, n)
        assert st == lbm.LBM_ERR_INVALID_ARG and not h.value
    # sized for 16-bit storage: 16-bit solves run, an FP32 solve does not fit
    rng = np.random.default_rng(9)
    S = lbm.Solver(*shape, workspace=(p, b16))
    S.set_geometry(I.random_phase(rng, *shape, 2), 2)
    S.set_tensors(np.stack([I.random_spd(rng) for _ in range(2)]))
    S.solve(2, 0, lbm.Solver.opts(tol=0.0, max_iters=100, storage=lbm.LBM_STORE_BF16))
    with pytest.raises(lbm.LBMError) as e:
        S.solve(2, 0, lbm.Solver.opts(tol=0.0, max_iters=100))
    assert e.value.status == lbm.LBM_ERR_OUT_OF_MEMORY
    assert "lbm_workspace_bytes" in lbm.lbm_last_error(S.h)
    S.close()
