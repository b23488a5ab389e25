"""Pins of the oracle's sensitivity fields (Eqs. 3.2, 3.3 and the
element-sensitivity form of Sec. 3.1)."""
import numpy as np
import pytest

from oracle import fe, sensitivity
from synthetic import clamp_face_x0, edge_load


def _linear_field(nx, ny, nz, A):
    return (fe.node_coordinates(nx, ny, nz) @ A.T).reshape(-1)


def test_uniform_strain_gives_closed_form_fields():
    nx, ny, nz, nu, E0 = 3, 2, 2, 0.3, 2.0
    A = np.zeros((3, 3))
    A[0, 0] = 1.0                          # eps = diag(1, 0, 0)
    u = _linear_field(nx, ny, nz, A)
    E = np.full(nx * ny * nz, E0)
    T = sensitivity.topological_compliance(nx, ny, nz, E, u, nu)
    # lam + 2 mu = E (1-nu)/((1+nu)(1-2nu)), 3 lam + 2 mu = E/(1-2nu)
    closed = 4 * E0 * (1 - nu) / ((1 + nu) ** 2 * (1 - 2 * nu)) - (1 - 3 * nu) * E0 / ((1 - nu ** 2) * (1 - 2 * nu))
    assert np.allclose(T, closed, rtol=1e-13)
    s = sensitivity.strain_energy(nx, ny, nz, E, u, nu)
    assert np.allclose(s, E0 * (1 - nu) / ((1 + nu) * (1 - 2 * nu)), rtol=1e-13)


def test_von_mises_uniaxial_and_shear():
    nu, E0, s = 0.3, 1.0, -1.7
    eps = np.diag([s / E0, -nu * s / E0, -nu * s / E0])[None]
    sig = sensitivity.centroid_stress(eps, np.array([E0]), nu)
    assert np.allclose(sig[0], np.diag([s, 0, 0]), atol=1e-15)
    assert abs(sensitivity.von_mises(sig)[0] - abs(s)) < 1e-14
    tau = 0.4
    sig = np.zeros((1, 3, 3))
    sig[0, 0, 1] = sig[0, 1, 0] = tau
    assert abs(sensitivity.von_mises(sig)[0] - np.sqrt(3) * tau) < 1e-15


def test_fields_invariant_under_rotation_of_the_strain():
    rng = np.random.default_rng(5)
    nu = 0.3
    eps = rng.standard_normal((3, 3))
    eps = 0.5 * (eps + eps.T)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    nx = ny = nz = 1
    for A in (eps, Q @ eps @ Q.T):
        u = _linear_field(nx, ny, nz, A)
        E = np.ones(1)
        vals = (sensitivity.topological_compliance(nx, ny, nz, E, u, nu)[0],
                sensitivity.element_von_mises(nx, ny, nz, E, u, nu)[0])
        if A is eps:
            ref = vals
    assert np.allclose(vals, ref, rtol=1e-12)


def test_strain_energy_sums_to_compliance():
    nx, ny, nz = 6, 3, 3
    rng = np.random.default_rng(6)
    E = np.where(rng.random(nx * ny * nz) < 0.25, 1e-3, 1.0)
    K = fe.assemble(nx, ny, nz, E)
    fixed = clamp_face_x0(nx, ny, nz)
    f = edge_load(nx, ny, nz)
    u = fe.solve_direct(K, f, fixed)
    s = sensitivity.strain_energy(nx, ny, nz, E, u)
    assert abs(s.sum() - fe.compliance(f, u)) < 1e-11 * abs(fe.compliance(f, u))
    assert np.all(s >= -1e-15)


def test_pnorm_limits():
    v = np.array([1.0, 2.0, 3.0])
    assert abs(sensitivity.pnorm(v, 1) - 6.0) < 1e-15
    assert abs(sensitivity.pnorm(v, 2) - np.sqrt(14.0)) < 1e-14
    assert abs(sensitivity.pnorm(v, 200) - 3.0) < 0.02
    assert sensitivity.pnorm(np.zeros(3), 8) == 0.0


def test_centroid_strain_of_a_bilinear_field():
    """u_x = x y on the unit element: at the centroid d u_x/dx = y = 1/2 and
    d u_x/dy = x = 1/2, so eps_xx = 1/2, eps_xy = 1/4 (the trilinear
    interpolant of x y is exact)."""
    X = fe.node_coordinates(1, 1, 1)
    u = np.zeros((8, 3))
    u[:, 0] = X[:, 0] * X[:, 1]
    eps = sensitivity.centroid_strain(1, 1, 1, u.reshape(-1))[0]
    ref = np.zeros((3, 3))
    ref[0, 0] = 0.5
    ref[0, 1] = ref[1, 0] = 0.25
    assert np.allclose(eps, ref, atol=1e-15)


def _voided_problem():
    from synthetic import small_cantilever
    w = small_cantilever(8, 4, 4, seed=2, n_spheres=2, rmin=1.0, rmax=1.8, group=2)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    u = fe.solve_direct(K, w.f[0], w.fixed)
    return w, K, u


@pytest.mark.parametrize("p", [2.0, 8.0])
def test_pnorm_gradient_matches_central_differences(p):
    w, K, u = _voided_problem()
    g = sensitivity.pnorm_stress_gradient(w.nx, w.ny, w.nz, w.E, u, p)
    PN = lambda v: sensitivity.pnorm(sensitivity.element_von_mises(w.nx, w.ny, w.nz, w.E, v), p)
    rng = np.random.default_rng(5)
    for _ in range(4):
        d = rng.standard_normal(u.size)
        d *= np.linalg.norm(u) / np.linalg.norm(d)
        eps = 1e-5
        fd = (PN(u + eps * d) - PN(u - eps * d)) / (2 * eps)
        assert abs(g @ d - fd) <= 1e-6 * abs(fd) + 1e-12 * abs(PN(u))


def test_stress_sensitivity_with_lambda_equal_u_is_eq32():
    w, K, u = _voided_problem()
    a = sensitivity.stress_topological_sensitivity(w.nx, w.ny, w.nz, w.E, u, u)
    b = sensitivity.topological_compliance(w.nx, w.ny, w.nz, w.E, u)
    assert np.allclose(a, b, rtol=1e-14, atol=1e-14 * np.abs(b).max())


def test_adjoint_gives_the_load_derivative_of_the_pnorm_stress():
    """With K lambda = -d sigma_PN/du (free DOFs), d sigma_PN / d f = -lambda:
    checked by central differences of sigma_PN(u(f)) through direct solves."""
    w, K, u = _voided_problem()
    p = 6.0
    free = w.fixed == 0
    g = sensitivity.pnorm_stress_gradient(w.nx, w.ny, w.nz, w.E, u, p)
    lam = fe.solve_direct(K, -g * free, w.fixed)
    PN = lambda v: sensitivity.pnorm(sensitivity.element_von_mises(w.nx, w.ny, w.nz, w.E, v), p)
    rng = np.random.default_rng(9)
    for _ in range(3):
        df = rng.standard_normal(u.size) * free
        df *= np.linalg.norm(w.f[0]) / np.linalg.norm(df)
        h = 1e-5
        up = fe.solve_direct(K, w.f[0] + h * df, w.fixed)
        um = fe.solve_direct(K, w.f[0] - h * df, w.fixed)
        fd = (PN(up) - PN(um)) / (2 * h)
        assert abs(-lam @ df - fd) <= 1e-6 * abs(fd) + 1e-12 * abs(PN(u))
