"""The inverse of the coarse matrix E = W^T K W (Sec. 3.5's deflation) as
the solver forms it, through afd_coarse_inverse, against the oracle's E
inverted by LAPACK in FP64.

The solver sweeps the unit-diagonal scaled matrix S = D^-1/2 E D^-1/2 by
blocked Gauss-Jordan without pivoting (E is SPD).  Bound, relative to
max |S^-1|:
    |inv - E_oracle^-1| <= 8 sqrt(n_c) kappa(S) u,
u the unit roundoff of the working type, kappa the 2-norm condition number
of S: the forward error of a backward-stable inversion of an SPD matrix,
with a factor for the n_c-term sums.  Meshes: n_c a multiple of 32 and not
(a ragged last tile), a single block column, FP32 and FP64 paths."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2203_15115_gb300 as afd  # noqa: E402
from oracle import deflation, fe  # noqa: E402
from synthetic import clamp_face_x0  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    afd.lib()


def _case(nx, ny, nz, g, seed):
    rng = np.random.default_rng(seed)
    E = rng.uniform(0.2, 1.0, nx * ny * nz)
    E[rng.random(E.size) < 0.25] = 1e-3
    fixed = clamp_face_x0(nx, ny, nz)
    fixed[rng.random(fixed.size) < 0.01] = 1
    K = fe.assemble(nx, ny, nz, E)
    W = deflation.deflation_matrix(nx, ny, nz, g, fixed)
    Ec = deflation.coarse_matrix(K, W, fixed)
    return E, fixed, Ec


@pytest.mark.parametrize("dims,g", [((24, 16, 8), 4),     # n_c = 6 x 6 x 4 x 2 = 288 (9 tiles)
                                    ((40, 20, 12), 4),    # n_c = 6 x 10 x 5 x 3 = 900 (ragged)
                                    ((8, 8, 8), 4)])      # n_c = 48 (two tiles, ragged)
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_coarse_inverse_matches_the_oracle(dims, g, precision):
    nx, ny, nz = dims
    E, fixed, Ec = _case(nx, ny, nz, g, seed=nx + ny + nz)
    prec = afd.AFD_MIXED if precision == "mixed" else afd.AFD_FP64
    m = afd.Mesh(nx, ny, nz, group=g, precision=prec)
    m.set_element_moduli(E)
    m.set_loads_bcs(np.zeros((1, 3 * (nx + 1) * (ny + 1) * (nz + 1))), fixed)
    inv = afd.afd_coarse_inverse(m.h)
    m.close()
    d = 1.0 / np.sqrt(np.diag(Ec))
    S = Ec * d[:, None] * d[None, :]
    kappa = np.linalg.cond(S)
    ref = np.linalg.inv(Ec)
    u = 2.0 ** -24 if precision == "mixed" else 2.0 ** -53
    n = Ec.shape[0]
    # compare in the scaled variables, where the bound holds entry by entry
    ref_s = ref / (d[:, None] * d[None, :])
    bound = 8 * np.sqrt(n) * kappa * u * np.max(np.abs(ref_s))
    err = np.max(np.abs(inv / (d[:, None] * d[None, :]) - ref_s))
    assert err <= bound, (precision, dims, err, bound, kappa)


def test_a_singular_coarse_matrix_is_refused():
    """No supports: the rigid modes of the whole body are in the null space
    of E, whose last scaled pivots fall to FP64 rounding level (about 1e-14,
    under the 1e-12 threshold), and the inversion refuses it.  (In FP32 the
    rounding level of those pivots is near the 1e-6 threshold, so only the
    FP64 path is asserted.)"""
    nx, ny, nz, g = 12, 8, 8, 4
    m = afd.Mesh(nx, ny, nz, group=g, precision=afd.AFD_FP64)
    m.set_element_moduli(np.ones(nx * ny * nz))
    m.set_loads_bcs(np.zeros((1, 3 * (nx + 1) * (ny + 1) * (nz + 1))), np.zeros(3 * (nx + 1) * (ny + 1) * (nz + 1),
                                                                           np.uint8))
    with pytest.raises(afd.AFDError) as ei:
        afd.afd_coarse_inverse(m.h)
    assert ei.value.code == afd.AFD_ERR_COARSE_SINGULAR
    m.close()
