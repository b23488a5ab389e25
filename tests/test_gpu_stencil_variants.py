"""Every CTA shape and plane staging the FP32 stencil's autotuner can pick,
checked element by element against the oracle (Sec. 3.5: K u without
assembling K), through the C ABI:

* K u alone (afd_apply_stiffness) against the oracle's assembled K with the
  fixed rows and columns removed;
* the fused step of the inner deflated PCG iteration
  (afd_apply_search_direction): p = z + W mu + beta p_old on the free DOFs
  against the oracle's W mu, q = K p against the assembled K applied to the
  kernel's own p, and p.q against the float64 dot of the returned vectors.

The shape is pinned with afd_set_stencil_shape, so the variant the autotuner
would take on a large mesh (e.g. the cp.async ring, 16 warps, 24 planes) is
the one that runs here.  Meshes: several x and y tiles with ragged edges and
several z chunks at every depth, scattered supports, moduli spanning 1e-3..1.

Tolerances (max-norm relative to the largest entry, derived from FP32
rounding): K u 2e-6 (a sum of <= 27 x 24 products, about 10 ulp of the
cancelling sum); p 2e-6 of max(|z| + |W mu| + |beta p_old|) (three roundings
of terms of that size); p.q 1e-5 relative (per-thread FP32 partial sums).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2203_15115_gb300 as afd  # noqa: E402
from oracle import deflation, fe  # noqa: E402
from synthetic import clamp_face_x0  # noqa: E402

PLANES = [2, 3, 4, 5, 6, 8, 12, 16, 24, 32]
WARPS = [8, 16]
STAGING = [0, 1, 2]
# (nx, ny, nz, group, supports): "scattered" fixes random DOFs everywhere (every tile takes the fixed-DOF
# path); "clamp" fixes the face x = 0 only, so most tiles take the path without fixed DOFs
MESHES = {"70x40x30": (70, 40, 30, 10, "scattered"), "3x2x50": (3, 2, 50, 2, "scattered"),
          "33x31x9": (33, 31, 9, 4, "clamp"), "95x33x21": (95, 33, 21, 8, "clamp")}


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def masked_matvec(K, u, fixed):
    uu = u.copy()
    uu[fixed != 0] = 0.0
    y = K @ uu
    y[fixed != 0] = 0.0
    return y


class Case:
    def __init__(self, nx, ny, nz, g, supports):
        rng = np.random.default_rng(nx * 10000 + ny * 100 + nz)
        self.nx, self.ny, self.nz, self.g = nx, ny, nz, g
        self.E = rng.uniform(1e-3, 1.0, nx * ny * nz)
        ndof = 3 * (nx + 1) * (ny + 1) * (nz + 1)
        if supports == "scattered":
            self.fixed = (rng.random(ndof) < 0.08).astype(np.uint8)
            self.fixed[: 3 * (nx + 1)] = 1   # a fully clamped first node row as well
        else:
            self.fixed = clamp_face_x0(nx, ny, nz)
        self.K = fe.assemble(nx, ny, nz, self.E)
        self.m = afd.Mesh(nx, ny, nz, group=g, precision=afd.AFD_MIXED)
        self.m.set_element_moduli(self.E)
        self.m.set_loads_bcs(np.zeros((1, ndof)), self.fixed)
        self.nc = afd.afd_coarse_size(self.m.h)
        R = 2
        self.u = rng.standard_normal((R, ndof)).astype(np.float32)
        self.y_ref = np.stack([masked_matvec(self.K, self.u[r].astype(np.float64), self.fixed) for r in range(R)])
        self.z = rng.standard_normal((R, ndof)).astype(np.float32)
        self.p_old = rng.standard_normal((R, ndof)).astype(np.float32)
        self.mu = 0.3 * rng.standard_normal((R, self.nc))
        self.beta = [0.7, -1.3]
        self.p_ref, self.p_scale = [], []
        for r in range(R):
            wmu = deflation.apply_w(nx, ny, nz, g, self.fixed, self.mu[r])
            z64, p64 = self.z[r].astype(np.float64), self.p_old[r].astype(np.float64)
            p = z64 + wmu + self.beta[r] * p64
            p[self.fixed != 0] = 0.0
            self.p_ref.append(p)
            self.p_scale.append(np.max(np.abs(z64) + np.abs(wmu) + abs(self.beta[r]) * np.abs(p64)))


@pytest.fixture(scope="module")
def cases():
    assert torch.cuda.is_available()
    afd.lib()
    out = {k: Case(*v) for k, v in MESHES.items()}
    yield out
    for c in out.values():
        c.m.close()


@pytest.mark.parametrize("staging", STAGING)
@pytest.mark.parametrize("warps", WARPS)
@pytest.mark.parametrize("mesh", list(MESHES))
def test_every_stencil_shape_matches_the_oracle(cases, mesh, warps, staging):
    c = cases[mesh]
    R = c.u.shape[0]
    ndof = c.u.shape[1]
    u = cuda(c.u)
    for planes in PLANES:
        afd.afd_set_stencil_shape(c.m.h, warps, planes, staging)
        shape = (warps, planes, staging)
        y = torch.zeros((R, ndof), dtype=torch.float32, device="cuda")
        afd.afd_apply_stiffness(c.m.h, afd.AFD_F32, R, u, y)
        y = y.cpu().numpy().astype(np.float64)
        err = np.max(np.abs(y - c.y_ref)) / np.max(np.abs(c.y_ref))
        assert err <= 2e-6, ("K u", shape, err)

        p = torch.full((R, ndof), np.nan, dtype=torch.float32, device="cuda")
        q = torch.full((R, ndof), np.nan, dtype=torch.float32, device="cuda")
        pq = afd.afd_apply_search_direction(c.m.h, R, cuda(c.z), cuda(c.p_old), cuda(c.mu), c.beta, p, q)
        p = p.cpu().numpy().astype(np.float64)
        q = q.cpu().numpy().astype(np.float64)
        for r in range(R):
            ep = np.max(np.abs(p[r] - c.p_ref[r])) / c.p_scale[r]
            assert ep <= 2e-6, ("p", shape, r, ep)
            assert np.all(p[r][c.fixed != 0] == 0.0)
            qref = masked_matvec(c.K, p[r], c.fixed)
            eq = np.max(np.abs(q[r] - qref)) / np.max(np.abs(qref))
            assert eq <= 2e-6, ("q", shape, r, eq)
            dot = float(p[r] @ q[r])
            assert abs(pq[r] - dot) <= 1e-5 * abs(dot), ("p.q", shape, r, pq[r], dot)


@pytest.fixture(scope="module")
def voided_case():
    """A voided cantilever and its oracle solution (direct solve), shared by the pinned-variant solves."""
    from synthetic import small_cantilever

    w = small_cantilever(40, 18, 14, seed=9, n_spheres=6, rmin=1.5, rmax=4.0, group=4)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    uref = fe.solve_direct(K, w.f[0], w.fixed)
    return w, uref, fe.compliance(w.f[0], uref)


@pytest.mark.parametrize("staging", STAGING)
@pytest.mark.parametrize("warps,planes", [(8, 3), (16, 5)])
def test_mixed_solve_with_every_stencil_variant_pinned(voided_case, staging, warps, planes):
    """The whole mixed solve with the FP32 stencil pinned to one variant (its
    residual mode at the deflated start, its fused mode in every iteration):
    the displacement matches the oracle's direct solution to the benchmark spec's
    1e-5 and J to 1e-6 (Eq. 1.1; Sec. 3.5)."""
    w, uref, Jref = voided_case
    m = afd.Mesh(w.nx, w.ny, w.nz, group=w.group, stencil_warps=warps, stencil_planes=planes)
    m.set_element_moduli(w.E)
    m.set_loads_bcs(w.f, w.fixed)
    afd.afd_set_stencil_shape(m.h, warps, planes, staging)
    u = np.zeros_like(w.f)
    st = m.solve(1e-8, u_out=u)
    J = m.compliance()[0]
    assert afd.afd_stencil_async(m.h) == staging
    m.close()
    assert np.linalg.norm(u[0] - uref) <= 1e-5 * np.linalg.norm(uref), st
    assert abs(J - Jref) <= 1e-6 * abs(Jref)


@pytest.mark.parametrize("staging", [2, 3])
def test_batched_solve_with_load_case_pairs(staging):
    """Three load cases solved at once with the packed-band stencil, its load
    cases in pairs (variant 3: the second pair holds one case, and the cases
    converge at different iterations, so a pair runs with one lane finished)
    or one case per launch lane set (variant 2): every displacement matches the
    oracle's direct solution to 1e-5 and J to 1e-6 (Eq. 1.1; Sec. 4.5's
    multiple loads)."""
    from synthetic import small_cantilever

    w = small_cantilever(32, 14, 10, seed=12, n_spheres=5, rmin=1.5, rmax=3.5, group=4, n_rhs=3)
    m = afd.Mesh(w.nx, w.ny, w.nz, group=w.group, stencil_warps=8, stencil_planes=4)
    m.set_element_moduli(w.E)
    m.set_loads_bcs(w.f, w.fixed)
    afd.afd_set_stencil_shape(m.h, 8, 4, staging)
    u = np.zeros_like(w.f)
    st = m.solve(1e-8, u_out=u)
    J = m.compliance()
    assert afd.afd_stencil_async(m.h) == staging
    m.close()
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    for r in range(3):
        uref = fe.solve_direct(K, w.f[r], w.fixed)
        assert np.linalg.norm(u[r] - uref) <= 1e-5 * np.linalg.norm(uref), (r, st[r])
        Jref = fe.compliance(w.f[r], uref)
        assert abs(J[r] - Jref) <= 1e-6 * abs(Jref), r
    assert len({s["iters"] for s in st}) > 1   # the cases stop at different iterations
