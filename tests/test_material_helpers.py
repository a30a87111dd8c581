"""The material and unit-cell helpers of the C ABI (Eq. 32-37), pinned by the
paper's Table II and its Section 5 worked example.  Host-only calls."""
import math
import os

import pytest

from paper_1503_08718_gb300 import build, lbm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PHI_Y = math.pi * math.sqrt(3.0) / 8.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbm.load()


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [l.split() for l in fh if l.strip() and not l.startswith("#")]


@pytest.mark.parametrize("phi_f,lam_L,lam_T", [tuple(map(float, r)) for r in
                                                _rows("table2_yarn_conductivity.txt")])
def test_table2_yarn_conductivities(phi_f, lam_L, lam_T):
    """Table II divides by the rounded phi_y = 0.68 that Eq. 35 prints; its
    three decimals are rounded for lambda_L and cut for lambda_T = 0.3636."""
    st, L, T = lbm.lbm_yarn_conductivity(7.81, 0.675, 0.178, phi_f / 0.68)
    assert st == lbm.LBM_OK
    assert abs(L - lam_L) <= 5e-4
    assert abs(T - lam_T) <= 1e-3
    # with the exact phi_y the values move by less than the printed digits
    st, L2, T2 = lbm.lbm_yarn_conductivity(7.81, 0.675, 0.178, phi_f / PHI_Y)
    assert abs(L2 - lam_L) <= 2.5e-3 and abs(T2 - lam_T) <= 1e-3


def test_eq37_printed_numerator_contradicts_table2():
    """With the numerator 1 - phi_fy as printed, phi_f = 0.4 would give 0.308,
    not the tabulated 0.363: the reading phi_fy is the one Table II uses."""
    pfy = 0.4 / PHI_Y
    printed = 0.178 + (1 - pfy) / (1 / (0.675 - 0.178) + (1 - pfy) / (2 * 0.178))
    assert abs(printed - 0.363) > 0.05


def test_section5_worked_example_unit_cell():
    g = {r[0]: float(r[1]) for r in _rows("section5_unit_cell.txt")}
    st, a, h, c, d, pfy = lbm.lbm_braid_unit_cell(g["phi_f"], int(g["n_f"]), g["d_f_mm"],
                                                 math.radians(g["gamma_deg"]))
    assert st == lbm.LBM_OK
    for got, key in ((a, "a"), (h, "h"), (c, "c"), (d, "d")):
        assert got == pytest.approx(g[key], rel=1.5e-3), key
    # the 56 x 56 x 120 grid: the same spacing along x (a / 56) and z (h / 120)
    assert a / g["grid_x"] == pytest.approx(h / g["grid_z"], rel=5e-3)
    # Eq. 35: the yarn fraction of the cell is pi sqrt(3) / 8 for any angle
    assert pfy == pytest.approx(g["phi_f"] / PHI_Y)
    area = math.pi * c * d
    assert 8 * area * (h / math.cos(math.radians(g["gamma_deg"]))) / (a * a * h) == \
        pytest.approx(PHI_Y, rel=1e-12)


def test_helpers_reject_invalid_input():
    assert lbm.lbm_yarn_conductivity(7.81, 0.178, 0.178, 0.5)[0] == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lbm_yarn_conductivity(7.81, 0.675, 0.178, 1.0)[0] == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lbm_braid_unit_cell(0.7, 9000, 0.0069, 0.4)[0] == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lbm_braid_unit_cell(0.4, 9000, 0.0069, 0.0)[0] == lbm.LBM_ERR_INVALID_ARG
