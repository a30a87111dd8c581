"""Pins of the oracle's collision operator (Eq. 5-13) against facts the paper
and the algebra fix, none of which re-use the oracle's own construction."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1503_08718_gb300 import inputs as I

# D3Q7 velocities of Eq. 7 written as vectors, independently of the oracle.
E = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])
GAMMA = 1.0 / 8.0
EPS = 2 * GAMMA


def test_moment_matrix_rows_are_orthogonal_polynomials_of_the_velocities():
    M = O.moment_matrix()
    # Eq. 9-11: orthogonal basis vectors; squared norms follow from the rows.
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.allclose(np.diag(G), [7, 2, 2, 2, 42, 12, 4])
    # row 0 is the zeroth moment (T = sum f, Eq. 14), rows 1-3 the velocities
    assert np.array_equal(M[0], np.ones(7))
    for a in range(3):
        assert np.array_equal(M[1 + a], E[:, a])
    # higher rows are polynomials of |e|^2 and e_a^2 (6 - 7|e|^2, 3e_x^2 - |e|^2, e_y^2 - e_z^2)
    e2 = (E ** 2).sum(1)
    assert np.array_equal(M[4], 6 - 7 * e2)
    assert np.array_equal(M[5], 3 * E[:, 0] ** 2 - e2)
    assert np.array_equal(M[6], E[:, 1] ** 2 - E[:, 2] ** 2)


def test_tau_and_lattice_scale():
    lam = I.transversely_isotropic(6.0, 0.8, I.axis_in_xz_from_z(30.0))
    s = O.lattice_scale(lam[None], tau_max=1.5)
    tau = O.tau_matrix(lam, s)
    assert np.isclose(tau.diagonal().max(), 1.5, rtol=0, atol=1e-15)
    assert np.allclose(tau, tau.T)
    # off-diagonal entries carry the anisotropy, scaled the same way
    assert np.isclose(tau[0, 2], s * lam[4] / EPS)


@pytest.mark.parametrize("seed", range(6))
def test_collision_conserves_temperature_and_fixes_equilibrium(seed):
    rng = np.random.default_rng(seed)
    lam = I.random_spd(rng)
    s = rng.uniform(0.01, 0.05)
    om = O.collision_matrix(lam, s)
    f = rng.uniform(-1, 1, 7)
    fh = O.collide_node(om, f)
    assert abs(fh.sum() - f.sum()) <= 1e-14 * max(1.0, np.abs(f).sum())
    T = rng.uniform(-2, 2)
    feq = np.array([1 - 6 * GAMMA] + [GAMMA] * 6) * T
    assert np.allclose(O.collide_node(om, feq), feq, rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_collision_equals_reduced_flux_relaxation(seed):
    """With tau_0 = tau_4..6 = 1 the moments 0, 4, 5, 6 land on equilibrium and
    the flux moment j relaxes to (I - tau^-1) j; orthogonality of M then puts
    +-jhat/2 on each opposite pair.  Derived by hand, not from the oracle."""
    rng = np.random.default_rng(100 + seed)
    lam = I.random_spd(rng)
    s = rng.uniform(0.01, 0.08)
    tau = 0.5 * np.eye(3) + s * I.full3(lam) / EPS
    f = rng.uniform(-1, 1, 7)
    T = f.sum()
    j = np.array([f[1] - f[2], f[3] - f[4], f[5] - f[6]])
    jh = j - np.linalg.solve(tau, j)
    expect = np.array([(1 - 6 * GAMMA) * T,
                       GAMMA * T + jh[0] / 2, GAMMA * T - jh[0] / 2,
                       GAMMA * T + jh[1] / 2, GAMMA * T - jh[1] / 2,
                       GAMMA * T + jh[2] / 2, GAMMA * T - jh[2] / 2])
    got = O.collide_node(O.collision_matrix(lam, s), f)
    assert np.allclose(got, expect, rtol=0, atol=1e-14)


def test_isotropic_collision_is_single_relaxation_of_the_flux():
    lam = I.isotropic(1.0)
    s = 0.1
    tau = 0.5 + s / EPS
    f = np.arange(7, dtype=float) / 10
    fh = O.collide_node(O.collision_matrix(lam, s), f)
    j = np.array([f[1] - f[2], f[3] - f[4], f[5] - f[6]])
    jh = np.array([fh[1] - fh[2], fh[3] - fh[4], fh[5] - fh[6]])
    assert np.allclose(jh, (1 - 1 / tau) * j, atol=1e-15)
