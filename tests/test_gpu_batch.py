"""The batched solver (many uneven cells in one graph launch) against the
single-solve path and the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as O
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


def _cells(seed=0):
    """Uneven cells: ragged rows, odd sizes, every axis, 2 to 4 phases."""
    rng = np.random.default_rng(seed)
    spec = [((37, 30, 20), 2), ((21, 18, 26), 0), ((16, 9, 12), 1), ((40, 24, 18), 2),
            ((13, 10, 8), 0), ((32, 32, 32), 1)]
    out = []
    for (nx, ny, nz), axis in spec:
        n_ph = int(rng.integers(2, 5))
        lam = np.stack([I.random_spd(rng) for _ in range(n_ph)])
        out.append((I.random_phase(rng, nx, ny, nz, n_ph), lam, axis))
    return out


def _single(phase, lam, axis, lateral, opts):
    nz, ny, nx = phase.shape
    S = lbm.Solver(nx, ny, nz)
    S.set_geometry(phase, lam.shape[0])
    S.set_tensors(lam)
    info = S.solve(axis, lateral, opts)
    return info, S.temperature()


@pytest.mark.parametrize("lateral", [0, 1])
def test_batch_matches_single_solves_and_oracle(lateral):
    cells = _cells(lateral)
    B = lbm.Batch()
    for ph, lam, axis in cells:
        B.add(ph, lam, axis)
    opts = lbm.Solver.opts(tol=0.0, max_iters=600, check_every=100)
    binfo = B.solve(lateral, opts)
    assert binfo.n_solves == len(cells) and binfo.block_threads in (128, 256, 512)
    assert binfo.steps_per_launch == 1          # ragged rows: single steps only
    assert binfo.total_updates == 600 * sum(ph.size for ph, _, _ in cells)
    for i, (ph, lam, axis) in enumerate(cells):
        r = B.result(i)
        assert r.iters == 600 and r.checks == 6
        s_info, T_single = _single(ph, lam, axis, lateral, opts)
        T = B.temperature(i)
        assert np.max(np.abs(T - T_single)) <= 1e-6
        assert r.k_eff == pytest.approx(s_info.k_eff, rel=1e-6)
        ref = O.Lattice(ph, lam, r.lattice_scale, axis, lateral)
        ref.init_linear()
        ref.step(600)
        assert np.max(np.abs(T - ref.temperature())) <= 1e-5
        assert r.k_eff == pytest.approx(ref.k_eff()[0], rel=1e-5)


def test_batch_solves_converge_independently():
    """Cells converge after different iteration counts; each stops on its
    own and gives the single-solve result."""
    yarn = I.transversely_isotropic(6.0, 0.8, I.axis_in_xz_from_z(30.0))
    lam = np.stack([I.isotropic(0.2), yarn])
    B = lbm.Batch()
    sizes = [(8, 8, 16), (8, 8, 32), (12, 12, 24)]
    for nx, ny, nz in sizes:
        B.add(I.layered_phase(nx, ny, nz, layer=nz // 4), lam, 2)
    opts = lbm.Solver.opts(tol=1e-8, max_iters=2_000_000)
    binfo = B.solve(0, opts)
    assert binfo.n_converged == len(sizes) and binfo.status == lbm.LBM_OK
    iters = []
    for i, (nx, ny, nz) in enumerate(sizes):
        r = B.result(i)
        s_info, _ = _single(I.layered_phase(nx, ny, nz, layer=nz // 4), lam, 2, 0, opts)
        assert r.status == lbm.LBM_OK and r.residual_T <= 1e-8
        assert r.iters == s_info.iters
        assert r.k_eff == pytest.approx(s_info.k_eff, rel=1e-6)
        assert r.k_eff == pytest.approx(94.0 / 245.0, rel=2e-3)
        iters.append(r.iters)
    assert len(set(iters)) > 1


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_BF16, lbm.LBM_STORE_F16])
def test_batch_16bit_storage(storage):
    cells = _cells(7)[:4]
    B = lbm.Batch()
    for ph, lam, axis in cells:
        B.add(ph, lam, axis)
    opts = lbm.Solver.opts(tol=0.0, max_iters=400, storage=storage)
    B.solve(0, opts)
    for i, (ph, lam, axis) in enumerate(cells):
        r = B.result(i)
        s_info, T_single = _single(ph, lam, axis, 0, opts)
        assert r.k_eff == pytest.approx(s_info.k_eff, rel=1e-4)
        assert np.max(np.abs(B.temperature(i) - T_single)) <= 2e-3


def _cells4(seed=3):
    """Uneven cells whose canonical rows hold a multiple of 4 nodes (the
    batched two-step kernel takes them): every axis, tiles with a shorter
    last tile, rows of 20 to 160 nodes."""
    rng = np.random.default_rng(seed)
    spec = [((64, 40, 30), 2), ((24, 80, 20), 0), ((36, 44, 28), 1), ((16, 16, 48), 2),
            ((160, 14, 18), 2), ((52, 28, 16), 1)]
    out = []
    for (nx, ny, nz), axis in spec:
        n_ph = int(rng.integers(2, 5))
        lam = np.stack([I.random_spd(rng) for _ in range(n_ph)])
        out.append((I.random_phase(rng, nx, ny, nz, n_ph), lam, axis))
    return out


@pytest.mark.parametrize("lateral", [0, 1])
def test_batched_two_step_launches_equal_single_steps_bit_for_bit(lateral):
    """The batch with two-step launches forced (fuse = 2) against the same
    batch with single steps only (fuse = 0): identical iterates, bit for bit,
    and both within the parity bars of the oracle."""
    cells = _cells4(lateral)
    res = []
    for fuse in (2, 0):
        B = lbm.Batch()
        for ph, lam, axis in cells:
            B.add(ph, lam, axis)
        binfo = B.solve(lateral, lbm.Solver.opts(tol=0.0, max_iters=400, fuse=fuse))
        assert binfo.steps_per_launch == (2 if fuse else 1)
        res.append([(B.temperature(i), B.result(i).k_eff, B.result(i).residual_T)
                     for i in range(len(cells))])
        B.close()
    for i, (ph, lam, axis) in enumerate(cells):
        (T2, k2, r2), (T1, k1, r1) = res[0][i], res[1][i]
        assert np.array_equal(T2, T1) and k2 == k1 and r2 == r1
        ref = O.Lattice(ph, lam, O.lattice_scale(lam), axis, lateral)
        ref.init_linear()
        ref.step(400)
        assert np.max(np.abs(T2 - ref.temperature())) <= 1e-5
        assert k2 == pytest.approx(ref.k_eff()[0], rel=1e-5)


def test_batch_start_fields_and_timed_history():
    """Per-solve start fields (lbm_batch_set_initial) give the single-solve
    warm start's iterates, and the batch history records every check with
    its iteration, k_eff and a device time that grows with the iteration."""
    cells = _cells4(9)[:3]
    rng = np.random.default_rng(5)
    B = lbm.Batch()
    starts = []
    for i, (ph, lam, axis) in enumerate(cells):
        B.add(ph, lam, axis)
        # a smooth start field different from the linear profile
        T0 = (0.5 + 0.1 * rng.standard_normal(ph.shape)).astype(np.float32)
        starts.append(T0)
        B.set_initial(i, T0)
    opts = lbm.Solver.opts(tol=0.0, max_iters=800, check_every=100)
    B.solve(0, opts)
    for i, (ph, lam, axis) in enumerate(cells):
        nz, ny, nx = ph.shape
        S = lbm.Solver(nx, ny, nz)
        S.set_geometry(ph, lam.shape[0])
        S.set_tensors(lam)
        o = S.opts(tol=0.0, max_iters=800, check_every=100)
        o.t_init = starts[i].ctypes.data_as(lbm.ctypes.POINTER(lbm.ctypes.c_float))
        info = S.solve(axis, 0, o)
        assert np.max(np.abs(B.temperature(i) - S.temperature())) <= 1e-6
        assert B.result(i).k_eff == pytest.approx(info.k_eff, rel=1e-6)
        h = B.history(i)
        assert h.shape == (8, 5)
        assert np.array_equal(h[:, 0], np.arange(100, 801, 100))
        assert h[-1, 1] == B.result(i).k_eff
        assert np.all(np.diff(h[:, 4]) > 0) and h[0, 4] > 0
        S.close()
    B.set_initial(0, None)                      # back to the linear profile
    B.solve(0, opts)
    ph, lam, axis = cells[0]
    s_info, T_lin = _single(ph, lam, axis, 0, opts)
    assert np.max(np.abs(B.temperature(0) - T_lin)) <= 1e-6
    B.close()


def test_batch_errors():
    B = lbm.Batch()
    with pytest.raises(lbm.LBMError) as e:
        B.solve(0)
    assert e.value.status == lbm.LBM_ERR_STATE
    bad = np.zeros((4, 4, 4), np.uint8)
    bad[0, 0, 0] = 3
    with pytest.raises(lbm.LBMError):
        B.add(bad, np.stack([I.isotropic(1.0)] * 2), 2)
    with pytest.raises(lbm.LBMError):
        B.add(np.zeros((4, 4, 4), np.uint8), I.sym6(np.diag([1.0, -2.0, 1.0]))[None], 2)
    B.add(np.zeros((4, 4, 4), np.uint8), I.isotropic(1.0)[None], 2)
    with pytest.raises(lbm.LBMError):
        B.solve(0, lbm.Solver.opts(check_every=5))


def test_sweep_cells_batched_at_full_size_match_oracle():
    """Config 3 in the launch configuration the bench times: the first four
    cells of the seeded sweep (uneven sizes between 64^3 and 160x160x320)
    along x, y and z in one batch with the autotuned plan, 20 iterations from
    the linear start, every solve against the FP64 oracle on every voxel."""
    import math

    cells = I.braid_sweep_cells(4)
    B = lbm.Batch()
    solves = []
    for c in cells:
        with lbm.Solver(c["nx"], c["ny"], c["nz"]) as V:
            V.set_geometry_braid(math.radians(c["g_deg"]),
                                 I.braid_anchors(c["nx"], c["ny"], c["seed"], n_max=256), c["phi"])
            ph = V.geometry()
        lam = I.braid_tensors(c["g_deg"])
        for axis in (0, 1, 2):
            B.add(ph, lam, axis)
            solves.append((ph, lam, axis))
    info = B.solve(0, lbm.Solver.opts(tol=0.0, max_iters=20, check_every=20))
    assert info.n_solves == 12
    for i, (ph, lam, axis) in enumerate(solves):
        r = B.result(i)
        ref = O.Lattice(ph, lam, r.lattice_scale, axis, 0)
        ref.init_linear()
        ref.step(20)
        assert np.max(np.abs(B.temperature(i) - ref.temperature())) <= 1e-5
        assert r.k_eff == pytest.approx(ref.k_eff()[0], rel=1e-5)
    B.close()
