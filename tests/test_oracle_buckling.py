"""Pins of the buckling oracle (Eq. 3.5 and the readings in oracle/buckling.py)."""
import numpy as np

from oracle import buckling, fe
from synthetic import axial_face_load, clamp_face_x0


def test_geometric_element_of_the_identity_stress_is_the_q1_laplacian():
    """With S = I, G is the trilinear Laplace element of the cube: h/3 on the
    diagonal, 0 for nodes along an edge, -h/12 across a face or the body."""
    for h in (1.0, 0.4):
        G = buckling.geometric_element(np.eye(3), h)
        for a in range(8):
            for b in range(8):
                diff = bin(a ^ b).count("1")
                expect = {0: 1.0 / 3.0, 1: 0.0, 2: -1.0 / 12.0, 3: -1.0 / 12.0}[diff] * h
                assert abs(G[a, b] - expect) < 1e-14


def test_geometric_stiffness_annihilates_translations_and_integrates_linear_fields():
    nx, ny, nz = 4, 3, 2
    rng = np.random.default_rng(1)
    A = rng.standard_normal((nx * ny * nz, 3, 3))
    S = 0.5 * (A + np.swapaxes(A, 1, 2))                       # a symmetric stress per element
    h = 0.7
    Kg = buckling.assemble_geometric(nx, ny, nz, S, h)
    t = np.tile(rng.standard_normal(3), (nx + 1) * (ny + 1) * (nz + 1))
    assert np.abs(Kg @ t).max() < 1e-12
    # phi = B x has constant gradient: phi^T K_G phi = sum_e h^3 tr(B S_e B^T)
    B = rng.standard_normal((3, 3))
    X = fe.node_coordinates(nx, ny, nz, h)
    phi = (X @ B.T).reshape(-1)
    expect = sum(h ** 3 * np.trace(B @ S[e] @ B.T) for e in range(S.shape[0]))
    assert np.isclose(phi @ (Kg @ phi), expect, rtol=1e-12)


def _column(nx=10, ny=3, nz=2):
    return nx, ny, nz, np.ones(nx * ny * nz), axial_face_load(nx, ny, nz, -1.0), clamp_face_x0(nx, ny, nz)


def test_lanczos_matches_dense_and_the_definition():
    nx, ny, nz, E, f, fixed = _column()
    lam_a, phi_a, S = buckling.buckling(nx, ny, nz, E, f, fixed, 3)
    lam_b, phi_b, _ = buckling.buckling_dense(nx, ny, nz, E, f, fixed, 3)
    assert np.all(lam_a > 0) and np.all(np.diff(lam_a) > 0)
    assert np.allclose(lam_a, lam_b, rtol=1e-10)
    K = fe.assemble(nx, ny, nz, E)
    Kg = buckling.assemble_geometric(nx, ny, nz, S)
    fr = fe.free_dofs(fixed)
    for i in range(3):
        assert abs(abs(phi_a[i] @ (K @ phi_b[i])) - 1.0) < 1e-8
        r = ((K + lam_a[i] * Kg) @ phi_a[i])[fr]
        assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm((K @ phi_a[i])[fr])
        assert np.isclose(phi_a[i] @ (K @ phi_a[i]), 1.0, rtol=1e-12)
    # the compressed column: the state stress is compressive along x in every element
    assert np.all(S[:, 0, 0] < 0)


def test_scaling_laws():
    """lambda is the factor on f: f * c gives lambda / c; a common factor c on
    E leaves the state stress unchanged and gives lambda * c."""
    nx, ny, nz, E, f, fixed = _column(8, 2, 2)
    lam0, _, _ = buckling.buckling_dense(nx, ny, nz, E, f, fixed, 2)
    lam1, _, _ = buckling.buckling_dense(nx, ny, nz, E, 3.0 * f, fixed, 2)
    lam2, _, _ = buckling.buckling_dense(nx, ny, nz, 5.0 * E, f, fixed, 2)
    assert np.allclose(lam1, lam0 / 3.0, rtol=1e-10)
    assert np.allclose(lam2, lam0 * 5.0, rtol=1e-10)


def test_buckling_sensitivity_of_an_exact_mode_sums_to_zero():
    """Eq. 3.5's element terms split phi^T (K + lambda K_G) phi, which vanishes
    for an exact mode; each term is the element's own quadratic form."""
    nx, ny, nz, E, f, fixed = _column(8, 3, 2)
    E = E.copy()
    E[::5] = 0.3
    lam, phi, S = buckling.buckling(nx, ny, nz, E, f, fixed, 2)
    for i in range(2):
        T = buckling.buckling_sensitivity(nx, ny, nz, E, S, phi[i], lam[i])
        assert abs(T.sum()) <= 1e-9 * np.abs(T).sum()
        e = 7
        K0 = fe.ke_hex8(0.3)
        pe = phi[i][fe.element_dofs(nx, ny, nz)[e]]
        G = buckling.geometric_element(S[e])
        assert np.isclose(T[e], E[e] * pe @ K0 @ pe + lam[i] * pe @ np.kron(G, np.eye(3)) @ pe, rtol=1e-12)



def test_slender_column_approaches_the_euler_load():
    """A clamped-free column of length L = 20 and unit square section (E = 1,
    unit compressive end load), refined through the thickness (n elements,
    h = 1/n): the critical factor falls monotonically onto Euler's
    pi^2 E I / (4 L^2), I = 1/12, with the trilinear element's O(h^2) error
    (Richardson on n = 3, 4 within 0.5 %); the square section gives two equal
    factors; the centre line of the mode is the planar profile
    1 - cos(pi x / 2L) with no axial motion."""
    L = 20
    PE = np.pi ** 2 * (1.0 / 12.0) / (4.0 * L ** 2)
    ratios = []
    for n in (1, 2, 3, 4):
        nx, ny, nz = L * n, n, n
        lam, phi, _ = buckling.buckling(nx, ny, nz, np.ones(nx * ny * nz), axial_face_load(nx, ny, nz, -1.0),
                                        clamp_face_x0(nx, ny, nz), 2, h=1.0 / n)
        assert abs(lam[1] - lam[0]) <= 1e-8 * lam[0]
        ratios.append(lam[0] / PE)
    assert all(a > b > 1.0 for a, b in zip(ratios, ratios[1:]))
    err = [r - 1.0 for r in ratios]
    assert 3.5 < err[0] / err[1] < 4.5 and 1.9 < err[1] / err[2] < 2.6      # O(h^2): (2/1)^2, (3/2)^2
    assert abs((16.0 * ratios[3] - 9.0 * ratios[2]) / 7.0 - 1.0) < 5e-3
    n = 4
    nx = L * n
    U = phi[0].reshape(n + 1, n + 1, nx + 1, 3)[n // 2, n // 2]                # centre line, x = 0..L
    d = U[-1, 1:] / np.linalg.norm(U[-1, 1:])
    w = U[:, 1:] @ d
    x = np.arange(nx + 1) / n
    assert np.abs(w / w[-1] - (1.0 - np.cos(np.pi * x / (2.0 * L)))).max() < 2e-3
    assert np.abs(U[:, 1:] @ np.array([-d[1], d[0]])).max() < 1e-9 * abs(w[-1])
    assert np.abs(U[:, 0]).max() < 1e-9 * abs(w[-1])
