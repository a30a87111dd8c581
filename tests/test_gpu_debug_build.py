"""The bounds-checked build (LBM_DEBUG) in place of a memory checker.

The library is rebuilt with every global and ring access of the step
kernels checked against its buffer; a subprocess that loads that build (the
LBM_LIBRARY variable) runs single-step, two-step and batched solves on the
layouts most likely to expose an indexing error (ragged rows, rows that
straddle warps, short last tiles, one-quad rows, odd cells, every axis, both
lateral types, 16-bit storage) and requires a clean bounds word on every
call plus the oracle's temperature and k_eff."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
sys.path.insert(0, ROOT)
from oracle import oracle as O
from paper_1503_08718_gb300 import inputs as I
from paper_1503_08718_gb300 import lbm

lbm.load()
assert lbm.lbm_debug_build() == 1
cases = [((37, 30, 9), 2, 0, 0, 1), ((37, 30, 9), 2, 1, 0, 1), ((13, 10, 22), 0, 1, 0, 1),
         ((64, 40, 30), 2, 0, 0, 2), ((80, 24, 20), 2, 1, 0, 2), ((96, 13, 22), 2, 0, 0, 2),
         ((4, 3, 7), 2, 1, 0, 2), ((20, 36, 44), 1, 0, 0, 2), ((128, 16, 40), 2, 1, 0, 1),
         ((256, 8, 24), 2, 0, 0, 1), ((2, 2, 2), 2, 1, 0, 1),
         ((37, 30, 20), 2, 1, 1, 0), ((21, 18, 26), 0, 0, 2, 0)]
for shape, axis, lateral, storage, fuse in cases:
    rng = np.random.default_rng(sum(shape) + axis)
    lam = np.stack([I.random_spd(rng) for _ in range(3)])
    phase = I.random_phase(rng, *shape, 3)
    with lbm.Solver(*shape) as S:
        S.set_geometry(phase, 3)
        S.set_tensors(lam)
        info = S.solve(axis, lateral, S.opts(tol=0.0, max_iters=200, storage=storage, fuse=fuse))
        st, code = lbm.lbm_debug_error(True)
        assert st == 0 and code == 0, (shape, code)
        T = S.temperature()
    ref = O.Lattice(phase, lam, info.lattice_scale, axis, lateral)
    ref.init_linear()
    ref.step(200)
    tol = 1e-5 if storage == 0 else 2e-3
    dT = float(np.max(np.abs(T - ref.temperature())))
    assert dT <= tol, (shape, storage, dT)
# batched two-step launches and batched 16-bit single steps
for storage, fuse in ((0, 2), (1, 0)):
    B = lbm.Batch()
    cells = []
    for k, (shape, axis) in enumerate([((64, 40, 30), 2), ((24, 80, 20), 0), ((36, 44, 28), 1)]):
        rng = np.random.default_rng(100 + k)
        lam = np.stack([I.random_spd(rng) for _ in range(2)])
        phase = I.random_phase(rng, *shape, 2)
        B.add(phase, lam, axis)
        cells.append((phase, lam, axis))
    B.solve(1, lbm.Solver.opts(tol=0.0, max_iters=200, storage=storage, fuse=fuse))
    for i, (phase, lam, axis) in enumerate(cells):
        ref = O.Lattice(phase, lam, O.lattice_scale(lam), axis, 1)
        ref.init_linear()
        ref.step(200)
        tol = 1e-5 if storage == 0 else 2e-3
        assert float(np.max(np.abs(B.temperature(i) - ref.temperature()))) <= tol
    B.close()
print("bounds-checked build clean")
"""


def test_bounds_checked_build_is_clean_on_every_layout():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_08718_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, LBM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT), 1)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "bounds-checked build clean" in r.stdout
