"""Failure exits of the solve and checkpoint / resume, through the C ABI.

Failures are injected on the host only (a non-finite start field, a stop
rule that must trip, an iteration cap); nothing here can fault the GPU.
A resumed solve must reproduce the uninterrupted one bit for bit: the
iteration is deterministic and the snapshot holds all of its state.
"""
import numpy as np
import pytest

from paper_1503_08718_gb300 import inputs as I
from paper_1503_08718_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_08718_gb300 import build
    build.build()
    lbm.load()


def _cell(nx=20, ny=16, nz=24, seed=5):
    rng = np.random.default_rng(seed)
    lam = np.stack([I.random_spd(rng) for _ in range(3)])
    phase = I.random_phase(rng, nx, ny, nz, 3)
    S = lbm.Solver(nx, ny, nz)
    S.set_geometry(phase, 3)
    S.set_tensors(lam)
    return S, phase, lam


def test_nonfinite_start_field_ends_diverged():
    S, phase, _ = _cell()
    T0 = np.full(phase.shape, 0.5, np.float32)
    T0[3, 4, 5] = np.nan
    o = S.opts(tol=1e-12, max_iters=1000)
    o.t_init = T0.ctypes.data_as(lbm.ctypes.POINTER(lbm.ctypes.c_float))
    S.start(2, 0, o)
    info = lbm.lbm_solve_info()
    st = lbm.lbm_run(S.h, info)
    assert st == lbm.LBM_ERR_DIVERGED, lbm.lbm_last_error(S.h)
    assert info.status == lbm.LBM_ERR_DIVERGED
    assert info.checks == 1                     # the first check stops the loop
    assert "non-finite" in lbm.lbm_last_error(S.h)
    # the context stays usable: a clean solve afterwards converges normally
    S.start(2, 0, S.opts(tol=1e-6))
    ok = S.run()
    assert ok.status == lbm.LBM_OK and np.isfinite(ok.k_eff)
    S.close()


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_BF16, lbm.LBM_STORE_F16])
def test_residual_floor_of_16bit_storage_ends_stalled(storage):
    """16-bit storage has a stochastic-rounding floor on R_T; with tol = 0
    and stall_checks = 2 the stop rule must report a stall, not run on."""
    S, _, _ = _cell(16, 16, 16)
    S.start(2, 0, S.opts(tol=0.0, max_iters=2_000_000, stall_checks=2, storage=storage))
    info = lbm.lbm_solve_info()
    st = lbm.lbm_run(S.h, info)
    assert st == lbm.LBM_ERR_STALLED, lbm.lbm_last_error(S.h)
    assert info.status == lbm.LBM_ERR_STALLED and info.iters < 2_000_000
    assert np.isfinite(info.k_eff) and S.k_eff() == info.k_eff
    S.close()


def test_iteration_cap_ends_not_converged_with_results_readable():
    S, _, _ = _cell()
    S.start(0, 1, S.opts(tol=1e-30, max_iters=600))
    info = lbm.lbm_solve_info()
    st = lbm.lbm_run(S.h, info)
    assert st == lbm.LBM_ERR_NOT_CONVERGED
    assert info.iters == 600 and info.checks == 6
    assert np.isfinite(S.k_eff())
    S.close()


@pytest.mark.parametrize("storage,lateral,axis", [
    (lbm.LBM_STORE_F32, 0, 2), (lbm.LBM_STORE_F32, 1, 0), (lbm.LBM_STORE_BF16, 0, 1)])
def test_resume_from_snapshot_is_bit_exact(storage, lateral, axis):
    S, phase, lam = _cell(32, 16, 20)
    opts = dict(tol=0.0, storage=storage)
    S.start(axis, lateral, S.opts(max_iters=2000, **opts))
    S.run()
    T_ref, k_ref, h_ref = S.temperature(), S.k_eff(), S.history()
    S.start(axis, lateral, S.opts(max_iters=1000, **opts))
    S.run()
    snap = S.get_state()
    assert snap.nbytes == lbm.lbm_state_bytes(S.h) > 0
    S.close()
    # a fresh context: same cell, same solve, the snapshot in place of the start
    R = lbm.Solver(*phase.shape[::-1])
    R.set_geometry(phase, lam.shape[0])
    R.set_tensors(lam)
    R.start(axis, lateral, R.opts(max_iters=2000, **opts))
    R.set_state(snap)
    info = R.run()
    assert info.iters == 2000
    assert np.array_equal(R.temperature(), T_ref)
    assert R.k_eff() == k_ref
    assert np.array_equal(R.history(), h_ref)
    # a snapshot of another solve is refused
    R.start((axis + 1) % 3, lateral, R.opts(max_iters=2000, **opts))
    st = lbm.lbm_set_state(R.h, snap)
    assert st == lbm.LBM_ERR_INVALID_ARG and "another solve" in lbm.lbm_last_error(R.h)
    st = lbm.lbm_set_state(R.h, snap[:100])
    assert st == lbm.LBM_ERR_INVALID_ARG
    R.close()
