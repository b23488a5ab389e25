"""The double-float stiffness apply (AFD_F64_DF) and the mixed solve's
double-float refinement residual, against the oracle (Sec. 3.5: K u without
assembling K; the FP64 residual of the iterative refinement).

A double-float value is the unevaluated sum of two floats; the stencil reads
FP64 u and f, splits each value into such a pair by its bits (the leading 24
and the next 23 significand bits, |d| in [2^-103, 2^128)) or by FP64 casts
outside that range, and runs the modal element operator in pair arithmetic.
Every rounding is a few units of 2^-44 of the magnitudes it combines, so the
bound checked here is, per DOF,
    |y - (K u)_oracle| <= 2^-36 (|K| |u|)_oracle,
where |K| |u| bounds the sizes of the products summed into that DOF and the
factor 2^8 over 2^-44 covers the modal form's intermediate sums (up to eight
node values of an element) and the few roundings per stage.  An FP32 product
misses this bound by a factor of about 10^4; the FP64 product meets it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2203_15115_gb300 as afd  # noqa: E402
from oracle import fe  # noqa: E402
from synthetic import small_cantilever  # noqa: E402

BOUND = 2.0 ** -36


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    afd.lib()


def _masked(K, u, fixed):
    uu = u.copy()
    uu[fixed != 0] = 0.0
    y = K @ uu
    y[fixed != 0] = 0.0
    return y


def _mesh_case(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    E = rng.uniform(1e-3, 1.0, nx * ny * nz)
    E[rng.random(E.size) < 0.2] = 1e-3          # void elements
    ndof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    fixed = (rng.random(ndof) < 0.05).astype(np.uint8)
    fixed[: 3 * (nx + 1)] = 1
    m = afd.Mesh(nx, ny, nz, group=4)
    m.set_element_moduli(E)
    m.set_loads_bcs(np.zeros((1, ndof)), fixed)
    return m, fe.assemble(nx, ny, nz, E), fixed, rng


def _apply(m, arith, u):
    ud = torch.from_numpy(np.ascontiguousarray(u[None, :])).cuda()
    y = torch.zeros_like(ud)
    afd.afd_apply_stiffness(m.h, arith, 1, ud, y)
    return y.cpu().numpy()[0]


@pytest.mark.parametrize("dims", [(70, 40, 30), (33, 31, 9), (3, 2, 50)])
def test_double_float_apply_matches_the_oracle_to_its_bound(dims):
    """K u in double-float arithmetic on several x/y tiles with ragged edges
    and several z chunks, moduli 1e-3..1 with voids, scattered supports."""
    m, K, fixed, rng = _mesh_case(*dims, seed=sum(dims))
    u = rng.standard_normal(K.shape[0]) * np.exp(rng.uniform(-3, 3, K.shape[0]))
    y = _apply(m, afd.AFD_F64_DF, u)
    y64 = _apply(m, afd.AFD_F64, u)
    y32 = _apply(m, afd.AFD_F32, u.astype(np.float32)).astype(np.float64)
    m.close()
    yref = _masked(K, u, fixed)
    s = _masked(abs(K), np.abs(u), fixed)
    free = fixed == 0
    assert np.all(y[~free] == 0.0)
    assert np.all(np.abs(y - yref)[free] <= BOUND * s[free])
    assert np.all(np.abs(y64 - yref)[free] <= BOUND * s[free])
    # the bound is tight enough to tell FP32 arithmetic apart
    assert np.any(np.abs(y32 - yref)[free] > BOUND * s[free])


def test_every_value_class_of_the_bitwise_split():
    """u holds zeros of both signs, values at the edges of the bitwise split's
    range (2^-103, 2^127) and outside it (2^-104, 1e-35, 1e-300, an FP64
    subnormal), and values whose 24th..47th significand bits are set: each
    DOF meets the bound of the FP64 oracle.  (Values near FP32's largest
    overflow the pair arithmetic: the solver keeps its refinement residual in
    FP64 for loads outside 1e-20..1e20.)"""
    m, K, fixed, rng = _mesh_case(20, 9, 7, seed=4)
    n = K.shape[0]
    u = rng.standard_normal(n)
    special = np.array([0.0, -0.0, 2.0 ** -103, -(2.0 ** -103), 2.0 ** -104, 1e-35, -1e-300, 5e-324,
                        1.0 + 2.0 ** -23 + 2.0 ** -40, -(1.0 + 2.0 ** -30), 2.0 ** 100 * (1 + 2.0 ** -45)])
    idx = rng.choice(np.flatnonzero(fixed == 0), size=special.size, replace=False)
    u[idx] = special
    y = _apply(m, afd.AFD_F64_DF, u)
    m.close()
    yref = _masked(K, u, fixed)
    s = _masked(abs(K), np.abs(u), fixed)
    free = fixed == 0
    assert np.all(np.abs(y - yref)[free] <= BOUND * s[free])
    assert np.all(y[~free] == 0.0)


@pytest.mark.parametrize("tol", [1e-6, 1e-9])
def test_mixed_solve_with_the_double_float_residual(tol):
    """Mixed solves with the double-float refinement residual (the default at
    tolerances >= 1e-10) and with the FP64 one: both meet the tolerance in the
    oracle's FP64 residual, the reported residual agrees with the oracle's to
    1e-11 of ||f|| (its rounding is about 2^-44 of the element forces), and
    the displacements agree with the oracle's direct solution."""
    w = small_cantilever(36, 16, 12, seed=21, n_spheres=6, rmin=1.5, rmax=3.5, group=4)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    uref = fe.solve_direct(K, w.f[0], w.fixed)
    free = w.fixed == 0
    fn = np.linalg.norm(w.f[0][free])
    out = {}
    for rf in (0, 1):
        m = afd.Mesh(w.nx, w.ny, w.nz, group=w.group, residual_fp64=rf)
        m.set_element_moduli(w.E)
        m.set_loads_bcs(w.f, w.fixed)
        u = np.zeros_like(w.f)
        st = m.solve(tol, u_out=u)[0]
        m.close()
        r = w.f[0] - _masked(K, u[0], w.fixed)
        rel = np.linalg.norm(r[free]) / fn
        assert rel <= tol, (rf, rel, st)
        assert abs(st["rel_residual"] - rel) <= 1e-11, (rf, st["rel_residual"], rel)
        out[rf] = (u[0], st)
    for rf in (0, 1):
        e = np.linalg.norm(out[rf][0] - uref) / np.linalg.norm(uref)
        assert e <= 1e3 * tol, (rf, e)
