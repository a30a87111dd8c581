"""The allocation-free voxeliser entry point (lbm_braid_voxelize_noalloc).

It serves callers that cannot allocate device memory themselves, such as a
process whose GPU memory is owned by a framework's caching allocator or a
service with a fixed memory budget: its scratch histogram is a fixed device
array inside the library.  The test allocates the inputs and outputs with
torch (the caller's memory), calls the entry point twice in a row with
different cells through the C ABI, and requires each phase map to equal the
one the allocating entry point (lbm_set_geometry_braid) produces, bit for
bit, as all integer outputs in this suite are compared.  This file is
collected last so that a stop at the first failure has run every other test.
"""
import math

import numpy as np
import pytest

from paper_1503_08718_gb300 import inputs as I
from paper_1503_08718_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_08718_gb300 import build
    build.build()
    lbm.load()
    torch.cuda.set_device(0)
    return torch


def _reference(nx, ny, nz, g_rad, anchors, phi):
    with lbm.Solver(nx, ny, nz) as S:
        used, frac = S.set_geometry_braid(g_rad, anchors, phi)
        return S.geometry(), used, frac


CELLS = [
    # (nx, ny, nz, braiding angle deg, yarn fraction, seed); the second cell
    # needs fewer yarns, so stale counts from the first call would show
    (96, 96, 64, 30.0, 0.45, 42),
    (80, 64, 50, 40.0, 0.30, 7),
]


def test_noalloc_voxeliser_matches_allocating_entry_point_twice(torch_cuda):
    torch = torch_cuda
    stream = torch.cuda.current_stream().cuda_stream
    for nx, ny, nz, g_deg, phi, seed in CELLS:
        anchors = I.braid_anchors(nx, ny, seed, n_max=128)
        d_anchors = torch.from_numpy(anchors).to("cuda")
        d_phase = torch.full((nz, ny, nx), 255, dtype=torch.uint8, device="cuda")
        g = math.radians(g_deg)
        st, used, frac, msg = lbm.lbm_braid_voxelize_noalloc(
            nx, ny, nz, g, 10.0, 6.0, d_anchors.data_ptr(), anchors.shape[0], phi,
            d_phase.data_ptr(), stream)
        assert st == lbm.LBM_OK, msg
        torch.cuda.synchronize()
        ref, used_ref, frac_ref = _reference(nx, ny, nz, g, anchors, phi)
        assert (used, frac) == (used_ref, frac_ref)
        assert np.array_equal(d_phase.cpu().numpy(), ref)


def test_noalloc_voxeliser_rejects_too_many_yarns(torch_cuda):
    torch = torch_cuda
    n = lbm.LBM_NOALLOC_MAX_YARNS + 1
    d_anchors = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    d_phase = torch.empty((4, 8, 8), dtype=torch.uint8, device="cuda")
    st, _, _, msg = lbm.lbm_braid_voxelize_noalloc(
        8, 8, 4, 0.5, 10.0, 6.0, d_anchors.data_ptr(), n, 0.1, d_phase.data_ptr(), None)
    assert st == lbm.LBM_ERR_INVALID_ARG
    assert "1024" in msg


def test_noalloc_voxeliser_rejects_host_pointers(torch_cuda):
    """A host buffer passed where device memory is expected is refused on
    the host (LBM_ERR_INVALID_ARG) before any kernel could touch it."""
    torch = torch_cuda
    anchors = np.ascontiguousarray(I.braid_anchors(8, 8, 3, n_max=16))
    host_phase = np.zeros((4, 8, 8), np.uint8)
    d_anchors = torch.from_numpy(anchors).to("cuda")
    d_phase = torch.empty((4, 8, 8), dtype=torch.uint8, device="cuda")
    for a_ptr, p_ptr in ((anchors.ctypes.data, d_phase.data_ptr()),
                         (d_anchors.data_ptr(), host_phase.ctypes.data)):
        st, _, _, msg = lbm.lbm_braid_voxelize_noalloc(
            8, 8, 4, 0.5, 10.0, 6.0, a_ptr, 16, 0.1, p_ptr, None)
        assert st == lbm.LBM_ERR_INVALID_ARG
        assert "device" in msg
