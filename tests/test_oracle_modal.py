"""Pins of the modal oracle (Eq. 3.4 and the readings in oracle/modal.py)."""
import numpy as np
import pytest

from oracle import fe, modal
from synthetic import clamp_face_x0, sphere_voids


def _fixed_all_but_last_node():
    """One cube element with every node fixed but local node 7 (1, 1, 1)."""
    fixed = np.ones(3 * 8, np.uint8)
    fixed[21:24] = 0
    return fixed


def test_lumped_mass_closed_forms():
    nx, ny, nz = 5, 4, 3
    rng = np.random.default_rng(0)
    E = rng.uniform(0.1, 1.0, nx * ny * nz)
    m = modal.lumped_mass(nx, ny, nz, E, rho=2.5, h=0.5)
    # total: every element's rho_e h^3 in each of the three directions
    assert np.isclose(m.sum(), 3 * 2.5 * 0.5 ** 3 * E.sum(), rtol=1e-13)
    # an interior node of a uniform mesh collects one eighth of each of its eight elements
    mu = modal.lumped_mass(nx, ny, nz, np.ones(nx * ny * nz), rho=1.0, h=1.0)
    n = 2 + 6 * (2 + 5 * 1)
    assert np.allclose(mu[3 * n:3 * n + 3], 1.0)
    # a corner node: one eighth of one element
    assert np.allclose(mu[0:3], 1.0 / 8.0)


@pytest.mark.parametrize("h,rho,E", [(1.0, 1.0, 1.0), (0.5, 3.0, 2.0)])
def test_single_free_node_closed_form(h, rho, E):
    """K_ff is the node's 3x3 self block E h (d I + s (J - I)) with the Q1 cube
    integrals d = (lam + 4 mu)/9 and s = (lam + mu)/12, M_ff = rho E h^3 / 8 I:
    eigenvalues 8 (d - s) / (rho h^2) (twice) and 8 (d + 2 s) / (rho h^2)."""
    lam_l, mu_l = fe.lame(1.0, 0.3)
    d, s = (lam_l + 4 * mu_l) / 9.0, (lam_l + mu_l) / 12.0
    expect = np.sort([8 * (d - s) / (rho * h * h)] * 2 + [8 * (d + 2 * s) / (rho * h * h)])
    lam, phi = modal.modes_dense(1, 1, 1, np.array([E]), _fixed_all_but_last_node(), 3, rho=rho, h=h)
    assert np.allclose(lam, expect, rtol=1e-12)
    # the stiffest mode moves the node along (1, 1, 1)
    v = phi[2, 21:24]
    assert np.allclose(np.abs(v) / np.linalg.norm(v), np.full(3, 3 ** -0.5), atol=1e-12)


def _voided(nx, ny, nz, seed):
    return sphere_voids(nx, ny, nz, 3, 1.0, 2.0, seed, 1e-3)


def test_lanczos_matches_dense_eigensolver():
    nx, ny, nz = 6, 3, 2
    E = _voided(nx, ny, nz, 4)
    fixed = clamp_face_x0(nx, ny, nz)
    lam_a, phi_a = modal.modes(nx, ny, nz, E, fixed, 5)
    lam_b, phi_b = modal.modes_dense(nx, ny, nz, E, fixed, 5)
    assert np.allclose(lam_a, lam_b, rtol=1e-10)
    m = modal.lumped_mass(nx, ny, nz, E)
    for i in range(5):
        assert abs(abs(phi_a[i] @ (m * phi_b[i])) - 1.0) < 1e-8


def test_eigenpairs_satisfy_the_definition():
    nx, ny, nz = 8, 3, 4
    E = _voided(nx, ny, nz, 7)
    fixed = clamp_face_x0(nx, ny, nz)
    lam, phi = modal.modes(nx, ny, nz, E, fixed, 4)
    K = fe.assemble(nx, ny, nz, E)
    m = modal.lumped_mass(nx, ny, nz, E)
    fr = fe.free_dofs(fixed)
    G = phi @ (m[:, None] * phi.T)
    assert np.allclose(G, np.eye(4), atol=1e-10)                 # M-orthonormal
    assert np.all(phi[:, fixed == 1] == 0.0)
    assert np.all(np.diff(lam) > 0) and lam[0] > 0
    for i in range(4):
        r = (K @ phi[i] - lam[i] * m * phi[i])[fr]
        assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm((K @ phi[i])[fr])
        assert np.isclose(phi[i] @ (K @ phi[i]), lam[i], rtol=1e-10)   # Rayleigh quotient


def test_scaling_laws():
    """rho_e follows E_e, so a common factor on E leaves lambda unchanged;
    lambda scales as 1/rho and, with K ~ h and M ~ h^3, as 1/h^2."""
    nx, ny, nz = 6, 2, 2
    E = _voided(nx, ny, nz, 2)
    fixed = clamp_face_x0(nx, ny, nz)
    lam0, _ = modal.modes_dense(nx, ny, nz, E, fixed, 3)
    lam1, _ = modal.modes_dense(nx, ny, nz, 7.0 * E, fixed, 3)
    lam2, _ = modal.modes_dense(nx, ny, nz, E, fixed, 3, rho=4.0)
    lam3, _ = modal.modes_dense(nx, ny, nz, E, fixed, 3, h=0.25)
    assert np.allclose(lam1, lam0, rtol=1e-10)
    assert np.allclose(lam2, lam0 / 4.0, rtol=1e-10)
    assert np.allclose(lam3, lam0 * 16.0, rtol=1e-10)


def test_eigen_sensitivity_closed_forms():
    nx, ny, nz = 4, 3, 2
    rng = np.random.default_rng(3)
    E = rng.uniform(0.2, 1.0, nx * ny * nz)
    lam, rho, nu = 2.7, 1.3, 0.3
    X = fe.node_coordinates(nx, ny, nz)
    # uniform strain u = eps0 x: sigma:eps is E_e eps0:C:eps0 in every element, and
    # u at the centroid is eps0 x_c
    A = rng.standard_normal((3, 3))
    eps0 = 0.5 * (A + A.T)
    u = (X @ eps0.T).reshape(-1)
    lam_l, mu_l = fe.lame(1.0, nu)
    sig0 = 2 * mu_l * eps0 + lam_l * np.trace(eps0) * np.eye(3)
    xc = X[fe.element_nodes(nx, ny, nz)].mean(axis=1)
    uc = xc @ eps0.T
    expect = E * np.sum(sig0 * eps0) - lam * rho * E * np.sum(uc * uc, axis=1)
    assert np.allclose(modal.eigen_sensitivity(nx, ny, nz, E, u, lam, rho, nu), expect, rtol=1e-12, atol=1e-12)
    # rigid translation t: no strain, -lambda rho_e |t|^2 everywhere
    t = np.array([0.3, -1.1, 0.7])
    ut = np.tile(t, X.shape[0])
    assert np.allclose(modal.eigen_sensitivity(nx, ny, nz, E, ut, lam, rho, nu), -lam * rho * E * (t @ t),
                       rtol=1e-12)


def test_slender_cantilever_approaches_euler_bernoulli_frequencies():
    """A clamped-free beam of length L = 20 and unit square section (E = 1,
    rho = 1, lumped mass), refined through the thickness (h = 1/n): the first
    bending eigenvalue omega^2 falls monotonically onto Euler-Bernoulli's
    beta_1^4 E I / (rho A L^4) with the trilinear element's O(h^2) error
    (Richardson on n = 3, 4 within 1 %); bending pairs are equal (square
    section); the second bending eigenvalue extrapolates to within 3 % below
    its Euler-Bernoulli value (shear and rotary inertia lower it)."""
    L = 20
    b1, b2 = 1.8751040687119611, 4.6940911329741745          # roots of cos b cosh b = -1
    lam_eb1 = b1 ** 4 * (1.0 / 12.0) / L ** 4
    lam_eb2 = b2 ** 4 * (1.0 / 12.0) / L ** 4
    r1, r2 = [], []
    for n in (1, 2, 3, 4):
        nx = L * n
        lam, _ = modal.modes(nx, n, n, np.ones(nx * n * n), clamp_face_x0(nx, n, n), 4, rho=1.0, h=1.0 / n)
        assert abs(lam[1] - lam[0]) <= 1e-8 * lam[0] and abs(lam[3] - lam[2]) <= 1e-8 * lam[2]
        r1.append(lam[0] / lam_eb1)
        r2.append(lam[2] / lam_eb2)
    assert all(a > b > 1.0 for a, b in zip(r1, r1[1:]))
    e = [r - 1.0 for r in r1]
    assert 3.5 < e[0] / e[1] < 4.5 and 1.9 < e[1] / e[2] < 2.6
    assert abs((16.0 * r1[3] - 9.0 * r1[2]) / 7.0 - 1.0) < 1e-2
    x2 = (16.0 * r2[3] - 9.0 * r2[2]) / 7.0
    assert 0.97 < x2 < 1.0
