"""Pins of the oracle's element and global stiffness and of its solvers
(Eq. 1.1, Sec. 3.5) against exact integration, mechanics closed forms and
invariants."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact, fe
from synthetic import clamp_face_x0, edge_load


@pytest.mark.parametrize("nu", [Fraction(3, 10), Fraction(1, 4), Fraction(9, 20)])
def test_ke_matches_exact_rational_integration(nu):
    K = fe.ke_hex8(float(nu))
    Kx = np.array(exact.ke_exact(nu), dtype=np.float64)
    assert np.max(np.abs(K - Kx)) <= 1e-15 * np.max(np.abs(Kx)) * 10


def test_ke_symmetric_psd_six_zero_modes():
    K = fe.ke_hex8(0.3)
    assert np.array_equal(K, K.T)
    w = np.linalg.eigvalsh(K)
    tiny = 1e-12 * w.max()
    assert np.sum(np.abs(w) < tiny) == 6
    assert np.all(w > -tiny)


def test_ke_null_space_is_rigid_motion():
    K = fe.ke_hex8(0.3)
    X = fe.LOCAL_OFFSETS.astype(float) - 0.5
    rng = np.random.default_rng(0)
    for _ in range(5):
        t = rng.standard_normal(3)
        w = rng.standard_normal(3)
        u = (t[None, :] + np.cross(w[None, :], X)).reshape(-1)
        assert np.max(np.abs(K @ u)) < 1e-14 * np.max(np.abs(K)) * np.max(np.abs(u))


def test_ke_diagonal_closed_form_and_h_scaling():
    lam, mu = fe.lame(1.0, 0.3)
    K = fe.ke_hex8(0.3)
    # K_aa^{cc} = (lam + 2mu) * Int (dN/dx_c)^2 + mu * sum_{j!=c} Int (dN/dx_j)^2 = (lam + 4 mu)/9
    assert np.allclose(np.diag(K), (lam + 4 * mu) / 9.0, rtol=1e-15, atol=0)
    assert abs(K[0, 0] - 0.2350427350427350) < 1e-15
    assert np.allclose(fe.ke_hex8(0.3, h=2.0), 2.0 * K, rtol=1e-14, atol=0)
    assert np.allclose(fe.ke_hex8(0.3, E=3.0), 3.0 * K, rtol=1e-14, atol=0)


def test_assembled_matches_matrix_free_and_is_symmetric():
    nx, ny, nz = 3, 2, 2
    rng = np.random.default_rng(1)
    E = rng.uniform(1e-3, 1.0, nx * ny * nz)
    K = fe.assemble(nx, ny, nz, E)
    assert abs(K - K.T).max() <= 1e-15 * abs(K).max()
    u = rng.standard_normal(K.shape[0])
    assert np.allclose(K @ u, fe.matvec_free(nx, ny, nz, E, u), rtol=0, atol=1e-13)


def test_patch_test_uniform_strain():
    """A linear displacement field is reproduced exactly: K u vanishes at every
    interior node, and 1/2 u^T K u equals the continuum energy of the uniform
    strain over the mesh volume."""
    nx, ny, nz = 4, 3, 3
    K = fe.assemble(nx, ny, nz, np.ones(nx * ny * nz), 0.3)
    X = fe.node_coordinates(nx, ny, nz)
    rng = np.random.default_rng(2)
    A = rng.standard_normal((3, 3))
    u = (X @ A.T).reshape(-1)
    y = (K @ u).reshape(-1, 3)
    inner = (X[:, 0] > 0) & (X[:, 0] < nx) & (X[:, 1] > 0) & (X[:, 1] < ny) & (X[:, 2] > 0) & (X[:, 2] < nz)
    assert np.max(np.abs(y[inner])) < 1e-13
    eps = 0.5 * (A + A.T)
    lam, mu = fe.lame(1.0, 0.3)
    w = 0.5 * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)) * nx * ny * nz
    assert abs(0.5 * u @ (K @ u) - w) < 1e-12 * abs(w)


def _uniaxial_problem(nx, ny, nz, s, E0):
    """Symmetry supports u_x = 0 on x = 0, u_y = 0 on y = 0, u_z = 0 on z = 0,
    uniform traction s on x = nx applied as consistent nodal forces."""
    fixed = np.zeros((nz + 1, ny + 1, nx + 1, 3), np.uint8)
    fixed[:, :, 0, 0] = 1
    fixed[:, 0, :, 1] = 1
    fixed[0, :, :, 2] = 1
    f = np.zeros((nz + 1, ny + 1, nx + 1, 3))
    wy = np.ones(ny + 1)
    wy[[0, -1]] = 0.5
    wz = np.ones(nz + 1)
    wz[[0, -1]] = 0.5
    f[:, :, nx, 0] = s * np.outer(wz, wy)
    return fixed.reshape(-1), f.reshape(-1)


@pytest.mark.parametrize("solver", ["direct", "pcg"])
def test_uniaxial_tension_exact_solution(solver):
    nx, ny, nz, s, E0, nu = 5, 3, 2, 2.5, 3.0, 0.3
    K = fe.assemble(nx, ny, nz, np.full(nx * ny * nz, E0), nu)
    fixed, f = _uniaxial_problem(nx, ny, nz, s, E0)
    if solver == "direct":
        u = fe.solve_direct(K, f, fixed)
    else:
        u, it = fe.solve_pcg(K, f, fixed, rtol=1e-14)
        assert it > 0
    X = fe.node_coordinates(nx, ny, nz)
    exact_u = np.stack([s / E0 * X[:, 0], -nu * s / E0 * X[:, 1], -nu * s / E0 * X[:, 2]], 1).reshape(-1)
    assert np.max(np.abs(u - exact_u)) < 1e-12 * np.max(np.abs(exact_u))
    # compliance of a bar under uniform stress: s^2 / E0 * volume
    assert abs(fe.compliance(f, u) - s * s / E0 * nx * ny * nz) < 1e-12 * s * s / E0 * nx * ny * nz


def test_cantilever_tip_deflection_tends_to_timoshenko():
    """Slender cantilever L/H = 16, section 1 x 1, unit shear load at the tip:
    refinement through the thickness (1, 2, 4 elements) must increase the tip
    deflection monotonically toward P L^3/(3EI) + P L/(kappa G A)."""
    L, E0, nu = 16, 1.0, 0.3
    G = E0 / (2 * (1 + nu))
    dT = L ** 3 / (3 * E0 / 12.0) + L / (5.0 / 6.0 * G)
    d = []
    for n in (1, 2, 4):
        nx, ny, nz, h = L * n, n, n, 1.0 / n
        K = fe.assemble(nx, ny, nz, np.ones(nx * ny * nz), nu, h)
        fixed = clamp_face_x0(nx, ny, nz)
        w1 = np.ones(n + 1)
        w1[[0, -1]] = 0.5
        w1 *= h
        f = np.zeros((nz + 1, ny + 1, nx + 1, 3))
        f[:, :, nx, 2] = -np.outer(w1, w1)
        u = fe.solve_direct(K, f.reshape(-1), fixed)
        uz = u.reshape(nz + 1, ny + 1, nx + 1, 3)[:, :, nx, 2]
        d.append(-np.sum(np.outer(w1, w1) * uz))
    assert d[0] < d[1] < d[2] < dT
    assert d[2] > 0.95 * dT
    richardson = d[2] + (d[2] - d[1]) / 3.0
    assert abs(richardson - dT) < 0.02 * dT


def test_pcg_matches_direct_and_energy_identities():
    nx, ny, nz = 6, 3, 3
    rng = np.random.default_rng(3)
    E = np.where(rng.random(nx * ny * nz) < 0.3, 1e-3, 1.0)
    K = fe.assemble(nx, ny, nz, E)
    fixed = clamp_face_x0(nx, ny, nz)
    f = edge_load(nx, ny, nz)
    u1 = fe.solve_direct(K, f, fixed)
    u2, _ = fe.solve_pcg(K, f, fixed, rtol=1e-13)
    assert np.linalg.norm(u1 - u2) < 1e-9 * np.linalg.norm(u1)
    assert fe.relative_residual(K, u1, f, fixed) < 1e-12
    assert np.all(u1[fixed != 0] == 0)
    J = fe.compliance(f, u1)
    assert abs(J - u1 @ (K @ u1)) < 1e-12 * abs(J)
    # dense solve of the reduced system as a third route
    fr = fe.free_dofs(fixed)
    ud = np.linalg.solve(K.toarray()[np.ix_(fr, fr)], f[fr])
    assert np.linalg.norm(ud - u1[fr]) < 1e-10 * np.linalg.norm(ud)


def test_jacobi_diagonal_is_ke_diagonal_times_adjacent_moduli():
    nx, ny, nz = 3, 3, 2
    rng = np.random.default_rng(4)
    E = rng.uniform(0.1, 1.0, nx * ny * nz)
    d = fe.jacobi_diagonal(nx, ny, nz, E).reshape(-1, 3)
    en = fe.element_nodes(nx, ny, nz)
    s = np.zeros(d.shape[0])
    np.add.at(s, en.reshape(-1), np.repeat(E, 8))
    lam, mu = fe.lame(1.0, 0.3)
    assert np.allclose(d, ((lam + 4 * mu) / 9.0 * s)[:, None], rtol=1e-14)
