"""Parity of the mixed-precision solve at the workloads' own tolerance
(relative residual 1e-6; Eq. 1.1, Sec. 3.5) on voided cantilevers, against
the oracle's FP64 solution, through the C ABI.

With void moduli of 1e-3 a relative residual of 1e-6 does not by itself bound
the displacement error by 1e-5, so both are checked: the FP64 true residual of
the returned u against the tolerance (the oracle's own matrix-free product),
and the errors against the oracle's solution:
  relative L2(u) <= 1e-5, relative J <= 1e-6,
  relative L2 over elements of s_e, Eq. 3.2 T_J and von Mises <= 1e-5.
The oracle solution is its plain Jacobi-PCG converged to a relative residual
of 1e-13 (a sparse direct factorisation of these 3-D meshes takes minutes);
its own error is checked against the direct solve on the smaller mesh."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2203_15115_gb300 as afd  # noqa: E402
from oracle import fe, sensitivity  # noqa: E402
from synthetic import small_cantilever  # noqa: E402

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    afd.lib()


def _oracle(w, K, r):
    u, _ = fe.solve_pcg(K, w.f[r], w.fixed, rtol=1e-13, maxiter=200000)
    return u


def _check_case(w, n_rhs):
    m = afd.Mesh(w.nx, w.ny, w.nz, precision=afd.AFD_MIXED, group=w.group)
    m.set_element_moduli(w.E)
    m.set_loads_bcs(w.f, w.fixed)
    u = np.zeros_like(w.f)
    stats = m.solve(TOL, u_out=u)
    J = m.compliance()
    fields = {}
    for kind in (afd.AFD_SENS_STRAIN_ENERGY, afd.AFD_SENS_TJ, afd.AFD_SENS_VON_MISES):
        out = np.zeros((n_rhs, m.nelem), np.float32)
        m.sensitivity(kind, out)
        fields[kind] = out
    m.close()
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    report = []
    for r in range(n_rhs):
        assert stats[r]["rel_residual"] <= TOL
        apply = lambda v: fe.matvec_free(w.nx, w.ny, w.nz, w.E, v)
        assert fe.relative_residual(apply, u[r], w.f[r], w.fixed) <= TOL
        uref = _oracle(w, K, r)
        eu = np.linalg.norm(u[r] - uref) / np.linalg.norm(uref)
        Jref = fe.compliance(w.f[r], uref)
        eJ = abs(J[r] - Jref) / abs(Jref)
        refs = {afd.AFD_SENS_STRAIN_ENERGY: sensitivity.strain_energy(w.nx, w.ny, w.nz, w.E, uref),
                afd.AFD_SENS_TJ: sensitivity.topological_compliance(w.nx, w.ny, w.nz, w.E, uref),
                afd.AFD_SENS_VON_MISES: sensitivity.element_von_mises(w.nx, w.ny, w.nz, w.E, uref)}
        es = {k: float(np.linalg.norm(fields[k][r] - ref) / np.linalg.norm(ref)) for k, ref in refs.items()}
        report.append((r, eu, eJ, es, stats[r]["iters"]))
        assert eu <= 1e-5, report[-1]
        assert eJ <= 1e-6, report[-1]
        for k, e in es.items():
            assert e <= 1e-5, (k, report[-1])
    print(report)


def test_oracle_reference_is_the_direct_solution():
    """The reference the checks below use (PCG to 1e-13) equals the sparse
    direct solution far inside the tested bounds (small voided mesh)."""
    w = small_cantilever(24, 12, 12, seed=31, n_spheres=5, rmin=2.0, rmax=4.0, group=4)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    ud = fe.solve_direct(K, w.f[0], w.fixed)
    up = _oracle(w, K, 0)
    assert np.linalg.norm(up - ud) <= 1e-9 * np.linalg.norm(ud)


def test_mixed_solve_at_1e6_voided_48x24x24():
    w = small_cantilever(48, 24, 24, seed=21, n_spheres=8, rmin=2.0, rmax=5.0, group=8)
    _check_case(w, 1)


def test_mixed_solve_at_1e6_voided_64x32x32():
    w = small_cantilever(64, 32, 32, seed=22, n_spheres=12, rmin=2.0, rmax=6.0, group=8)
    _check_case(w, 1)


def test_mixed_solve_at_1e6_voided_48x24x24_eight_load_cases():
    w = small_cantilever(48, 24, 24, seed=23, n_spheres=8, rmin=2.0, rmax=5.0, group=8, n_rhs=8)
    _check_case(w, 8)
