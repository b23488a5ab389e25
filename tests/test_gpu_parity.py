"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances (written here, derived from the arithmetic of each kernel):
stencil FP64 1e-13 and FP32 2e-6 relative (max-norm against max |y|);
coarse matrix 1e-12; FP64 solve
relative L2(u) <= 1e-9 and J <= 1e-10; mixed solve L2(u) <= 1e-5 and
J <= 1e-6; sensitivities 1e-5 (mixed) and 2e-7 (FP64, float32 output);
selection bit exact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2203_15115_gb300 as afd  # noqa: E402
from oracle import deflation, fe, levelset, sensitivity  # noqa: E402
from synthetic import (clamp_face_x0, cantilever_24x12x12_solid, edge_load, small_cantilever,  # noqa: E402
                       sphere_voids, top_point_loads)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    afd.lib()


def rand_fixed(nx, ny, nz, rng, p=0.1):
    return (rng.random(3 * (nx + 1) * (ny + 1) * (nz + 1)) < p).astype(np.uint8)


def oracle_masked_matvec(K, u, fixed):
    uu = u.copy()
    uu[fixed != 0] = 0.0
    y = K @ uu
    y[fixed != 0] = 0.0
    return y


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 3, 2), (33, 9, 5), (40, 17, 11), (3, 31, 8)])
def test_stencil_matches_assembled_K(dims):
    nx, ny, nz = dims
    rng = np.random.default_rng(sum(dims))
    E = rng.uniform(1e-3, 1.0, nx * ny * nz)
    fixed = rand_fixed(nx, ny, nz, rng)
    K = fe.assemble(nx, ny, nz, E)
    R = 3
    u = rng.standard_normal((R, K.shape[0]))
    m = afd.Mesh(nx, ny, nz)
    m.set_element_moduli(E)
    m.set_loads_bcs(np.zeros((1, K.shape[0])), fixed)
    ref = np.stack([oracle_masked_matvec(K, u[r], fixed) for r in range(R)])
    y64 = torch.zeros((R, K.shape[0]), dtype=torch.float64, device="cuda")
    afd.afd_apply_stiffness(m.h, afd.AFD_F64, R, cuda(u), y64)
    y64 = y64.cpu().numpy()
    assert np.max(np.abs(y64 - ref)) <= 1e-13 * np.max(np.abs(ref))
    y32 = torch.zeros((R, K.shape[0]), dtype=torch.float32, device="cuda")
    afd.afd_apply_stiffness(m.h, afd.AFD_F32, R, cuda(u.astype(np.float32)), y32)
    y32 = y32.cpu().numpy().astype(np.float64)
    ref32 = np.stack([oracle_masked_matvec(K, u[r].astype(np.float32).astype(np.float64), fixed) for r in range(R)])
    assert np.max(np.abs(y32 - ref32)) <= 2e-6 * np.max(np.abs(ref32))
    m.close()


@pytest.mark.parametrize("precision,cfp64,ctol", [(afd.AFD_FP64, 1, 1e-12), (afd.AFD_MIXED, 1, 1e-12),
                                                  (afd.AFD_MIXED, 0, 1e-6)])
@pytest.mark.parametrize("dims,g", [((4, 2, 2), 2), ((9, 5, 7), 3), ((12, 6, 6), 4)])
def test_deflation_operators_and_coarse_matrix(dims, g, precision, cfp64, ctol):
    """W^T, W and E = W^T K W against the oracle's dense W.  The mixed path
    builds E from FP64 element products by default (coarse_fp64 = 1); with
    coarse_fp64 = 0 from FP32 element products summed in FP64 (the coarse
    solve is a preconditioner component there), hence its looser bound."""
    nx, ny, nz = dims
    rng = np.random.default_rng(11)
    E = np.where(rng.random(nx * ny * nz) < 0.3, 1e-3, 1.0)
    fixed = clamp_face_x0(nx, ny, nz)
    fixed[rng.random(fixed.size) < 0.05] = 1
    m = afd.Mesh(nx, ny, nz, group=g, precision=precision, coarse_fp64=cfp64)
    m.set_element_moduli(E)
    m.set_loads_bcs(edge_load(nx, ny, nz)[None], fixed)
    W = deflation.deflation_matrix(nx, ny, nz, g, fixed)
    nc = W.shape[1]
    assert afd.afd_coarse_size(m.h) == nc
    v = rng.standard_normal((2, W.shape[0]))
    out = torch.zeros((2, nc), dtype=torch.float64, device="cuda")
    afd.afd_deflation_wt(m.h, 2, cuda(v), out)
    ref = v @ W
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    y = rng.standard_normal((2, nc))
    out2 = torch.zeros((2, W.shape[0]), dtype=torch.float64, device="cuda")
    afd.afd_deflation_w(m.h, 2, cuda(y), out2)
    ref2 = y @ W.T
    assert np.max(np.abs(out2.cpu().numpy() - ref2)) <= 1e-12 * np.max(np.abs(ref2))
    Ec = afd.afd_coarse_matrix(m.h)
    K = fe.assemble(nx, ny, nz, E)
    Eref = deflation.coarse_matrix(K, W, fixed)
    assert np.max(np.abs(Ec - Eref)) <= ctol * np.max(np.abs(Eref))
    m.close()


def _solve(w, precision, tol, group=None):
    m = afd.Mesh(w.nx, w.ny, w.nz, precision=precision, group=group or w.group)
    m.set_element_moduli(w.E)
    m.set_loads_bcs(w.f, w.fixed)
    u = np.zeros_like(w.f)
    stats = m.solve(tol, u_out=u)
    return m, u, stats


def test_fp64_solve_cantilever_24x12x12():
    w = cantilever_24x12x12_solid()
    m, u, stats = _solve(w, afd.AFD_FP64, 1e-10)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    uref = fe.solve_direct(K, w.f[0], w.fixed)
    assert np.linalg.norm(u[0] - uref) <= 1e-9 * np.linalg.norm(uref)
    assert fe.relative_residual(K, u[0], w.f[0], w.fixed) <= 1e-10
    J = m.compliance()[0]
    assert abs(J - fe.compliance(w.f[0], uref)) <= 1e-10 * abs(J)
    assert stats[0]["rel_residual"] <= 1e-10
    m.close()


@pytest.mark.parametrize("case", ["solid", "voids"])
def test_mixed_solve_matches_oracle(case):
    if case == "solid":
        w = cantilever_24x12x12_solid()
    else:
        w = small_cantilever(30, 14, 10, seed=3, n_spheres=6, rmin=1.5, rmax=4.0, group=4)
    m, u, stats = _solve(w, afd.AFD_MIXED, 1e-8)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    uref = fe.solve_direct(K, w.f[0], w.fixed)
    assert stats[0]["rel_residual"] <= 1e-8
    assert fe.relative_residual(K, u[0], w.f[0], w.fixed) <= 1.0001e-8
    assert np.linalg.norm(u[0] - uref) <= 1e-5 * np.linalg.norm(uref)
    J = m.compliance()[0]
    assert abs(J - fe.compliance(w.f[0], uref)) <= 1e-6 * abs(J)
    m.close()


@pytest.mark.parametrize("n_rhs", [1, 3])
def test_persistent_and_graph_inner_solvers_agree(n_rhs):
    """The cooperative persistent inner DPCG and the CUDA-graph chunks run the
    same iteration (Sec. 3.5): both reach the tolerance, agree with the direct
    solve, and take nearly the same number of iterations."""
    w = small_cantilever(40, 20, 12, seed=5, n_spheres=8, rmin=1.5, rmax=4.0, group=4, n_rhs=n_rhs)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    out = {}
    for pers in (1, 0):
        m = afd.Mesh(w.nx, w.ny, w.nz, group=w.group, persistent=pers)
        m.set_element_moduli(w.E)
        m.set_loads_bcs(w.f, w.fixed)
        u = np.zeros_like(w.f)
        st = m.solve(1e-9, u_out=u)
        out[pers] = (u, st)
        m.close()
    for r in range(n_rhs):
        uref = fe.solve_direct(K, w.f[r], w.fixed)
        for pers in (1, 0):
            u, st = out[pers]
            assert st[r]["rel_residual"] <= 1e-9
            assert np.linalg.norm(u[r] - uref) <= 1e-6 * np.linalg.norm(uref)
        i1, i0 = out[1][1][r]["iters"], out[0][1][r]["iters"]
        assert abs(i1 - i0) <= max(2, i0 // 50), (i1, i0)


def test_multi_rhs_batch_equals_single_solves():
    nx, ny, nz = 20, 10, 8
    E = sphere_voids(nx, ny, nz, 5, 1.5, 3.0, 4, 1e-3)
    fixed = clamp_face_x0(nx, ny, nz)
    f = np.concatenate([edge_load(nx, ny, nz)[None], top_point_loads(nx, ny, nz, 3, 9)])
    m = afd.Mesh(nx, ny, nz, group=4)
    m.set_element_moduli(E)
    m.set_loads_bcs(f, fixed)
    ub = np.zeros_like(f)
    m.solve(1e-9, u_out=ub)
    K = fe.assemble(nx, ny, nz, E)
    for r in range(f.shape[0]):
        ms = afd.Mesh(nx, ny, nz, group=4)
        ms.set_element_moduli(E)
        ms.set_loads_bcs(f[r:r + 1], fixed)
        us = np.zeros((1, f.shape[1]))
        ms.solve(1e-9, u_out=us)
        uref = fe.solve_direct(K, f[r], fixed)
        assert np.linalg.norm(ub[r] - uref) <= 1e-6 * np.linalg.norm(uref)
        assert np.linalg.norm(ub[r] - us[0]) <= 1e-6 * np.linalg.norm(uref)
        ms.close()
    m.close()


@pytest.mark.parametrize("precision,tol", [(afd.AFD_MIXED, 1e-5), (afd.AFD_FP64, 2e-7)])
def test_sensitivities_match_oracle(precision, tol):
    w = small_cantilever(24, 12, 8, seed=7, n_spheres=5, rmin=1.5, rmax=3.5, group=4)
    m, u, _ = _solve(w, precision, 1e-10 if precision == afd.AFD_FP64 else 1e-8)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    uref = fe.solve_direct(K, w.f[0], w.fixed)
    refs = {
        afd.AFD_SENS_STRAIN_ENERGY: sensitivity.strain_energy(w.nx, w.ny, w.nz, w.E, uref),
        afd.AFD_SENS_TJ: sensitivity.topological_compliance(w.nx, w.ny, w.nz, w.E, uref),
        afd.AFD_SENS_VON_MISES: sensitivity.element_von_mises(w.nx, w.ny, w.nz, w.E, uref),
    }
    for kind, ref in refs.items():
        out = np.zeros((1, m.nelem), np.float32)
        m.sensitivity(kind, out)
        assert np.linalg.norm(out[0] - ref) <= tol * np.linalg.norm(ref), kind
    p = 8.0
    pn = m.pnorm_stress(p)[0]
    assert abs(pn - sensitivity.pnorm(refs[afd.AFD_SENS_VON_MISES], p)) <= 10 * tol * pn
    s = np.zeros((1, m.nelem), np.float32)
    m.sensitivity(afd.AFD_SENS_STRAIN_ENERGY, s)
    assert abs(s.astype(np.float64).sum() - m.compliance()[0]) <= 1e-5 * m.compliance()[0]
    m.close()


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 4096, 4097, 100003])
def test_select_topk_bit_exact(n):
    rng = np.random.default_rng(n)
    keys = np.concatenate([rng.integers(-3, 4, n // 2).astype(np.float32),
                           rng.standard_normal(n - n // 2).astype(np.float32)])
    rng.shuffle(keys)
    if n > 3:
        keys[:3] = [0.0, -0.0, 0.0]
    dk = cuda(keys)
    for frac in (0.0, 0.01, 0.37, 0.5, 0.999, 1.0):
        k = levelset.keep_count(frac, n)
        kept = torch.zeros(n, dtype=torch.uint8, device="cuda")
        tau = afd.afd_select_topk(dk, k, kept)
        ref, tref = levelset.select_top(keys, k)
        assert np.array_equal(kept.cpu().numpy(), ref), (n, frac)
        if k:
            assert tau == np.float32(tref)


def test_levelset_update_keeps_the_oracle_set_up_to_rounding_ties():
    w = small_cantilever(24, 12, 8, seed=8, n_spheres=4, rmin=1.5, rmax=3.5, group=4, n_rhs=2)
    m, u, _ = _solve(w, afd.AFD_MIXED, 1e-9)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    fields = []
    for r in range(2):
        uref = fe.solve_direct(K, w.f[r], w.fixed)
        fields.append(sensitivity.strain_energy(w.nx, w.ny, w.nz, w.E, uref).astype(np.float32))
    weights = [1.0, 0.5]
    keys = levelset.combine(fields, weights)
    v = 0.8
    kref, tref = levelset.select_top(keys, levelset.keep_count(v, keys.size))
    kept = np.zeros(m.nelem, np.uint8)
    tau = m.levelset_update(afd.AFD_SENS_STRAIN_ENERGY, weights, v, kept)
    assert kept.sum() == kref.sum()
    diff = np.flatnonzero(kept != kref)
    # disagreements only where the oracle key sits within rounding of the cut
    assert np.all(np.abs(keys[diff] - tref) <= 1e-4 * abs(tref) + 1e-30)
    assert abs(tau - tref) <= 1e-4 * abs(tref)
    m.close()


def test_levelset_update_after_sensitivity_reuses_only_a_current_field():
    """afd_levelset_update reuses the field of an afd_sensitivity call of the
    same kind made just before it on the same mesh (Eq. 3.6's cut of Sec.
    3.1's field): the kept set and the cut value equal those of an update
    without the sensitivity call, bit for bit; after another call in between
    (new moduli and a new solve), or for another kind, the field is formed
    again from the current state."""
    w = small_cantilever(24, 12, 8, seed=8, n_spheres=4, rmin=1.5, rmax=3.5, group=4, n_rhs=2)
    weights = [1.0, 0.5]
    E2 = np.where(np.arange(w.E.size) % 7 == 0, 1e-3, w.E)

    def run(pre_kind, change):
        m = afd.Mesh(w.nx, w.ny, w.nz, precision=afd.AFD_MIXED, group=w.group, stencil_warps=8, stencil_planes=4)
        m.set_element_moduli(w.E)
        m.set_loads_bcs(w.f, w.fixed)
        m.solve(1e-9)
        out = np.zeros((2, m.nelem), np.float32)
        if pre_kind is not None:
            m.sensitivity(pre_kind, out)
        if change:
            m.set_element_moduli(E2)
            m.solve(1e-9)
        kept = np.zeros(m.nelem, np.uint8)
        tau = m.levelset_update(afd.AFD_SENS_STRAIN_ENERGY, weights, 0.8, kept)
        m.close()
        return kept, tau

    base = run(None, False)
    for pre in (afd.AFD_SENS_STRAIN_ENERGY, afd.AFD_SENS_VON_MISES):
        kept, tau = run(pre, False)
        assert np.array_equal(kept, base[0]) and tau == base[1], pre
    changed = run(None, True)
    kept, tau = run(afd.AFD_SENS_STRAIN_ENERGY, True)
    assert np.array_equal(kept, changed[0]) and tau == changed[1]
    assert not np.array_equal(changed[0], base[0])


def test_error_paths():
    nx, ny, nz = 6, 3, 3
    m = afd.Mesh(nx, ny, nz, group=2)
    with pytest.raises(afd.AFDError) as e:
        m.solve(1e-6)
    assert e.value.code == afd.AFD_ERR_STATE
    bad = np.ones(nx * ny * nz)
    bad[3] = np.nan
    with pytest.raises(afd.AFDError) as e:
        m.set_element_moduli(bad)
    assert e.value.code == afd.AFD_ERR_INVALID_ARG
    m.set_element_moduli(np.ones(nx * ny * nz))
    # no supports: the rigid motions of the whole body are in the coarse space
    m.set_loads_bcs(edge_load(nx, ny, nz)[None], np.zeros(3 * 7 * 4 * 4, np.uint8))
    with pytest.raises(afd.AFDError) as e:
        m.solve(1e-6)
    assert e.value.code == afd.AFD_ERR_COARSE_SINGULAR
    m.close()


@pytest.mark.parametrize("shape", [(7, 5, 6), (33, 17, 9), (64, 3, 40), (300, 7, 5), (5, 261, 3), (4, 3, 140)])
def test_casting_scan_bit_exact(shape):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx)
    T = rng.standard_normal(nx * ny * nz).astype(np.float32)
    T[::3] = T[1::3][: T[::3].size]         # ties and plateaus
    for axis in (0, 1, 2):
        n = shape[axis]
        for parting in sorted({0, 1, n // 2, n - 1, n} | {p for p in (127, 128, 129, 171) if p < n}):
            d = torch.from_numpy(T.copy()).cuda()
            afd.afd_casting_scan(d, nx, ny, nz, axis, parting)
            torch.cuda.synchronize()
            assert np.array_equal(d.cpu().numpy(), levelset.casting_scan(T, nx, ny, nz, axis, parting)), (axis, parting)
    with pytest.raises(afd.AFDError):
        afd.afd_casting_scan(torch.zeros(nx * ny * nz, device="cuda"), nx, ny, nz, 3, 0)
    with pytest.raises(afd.AFDError):
        afd.afd_casting_scan(torch.zeros(nx * ny * nz, device="cuda"), nx, ny, nz, 0, nx + 1)


@pytest.mark.parametrize("axis,parting", [(2, 0), (2, 4), (1, 6), (0, 10)])
def test_levelset_update_with_casting_matches_oracle(axis, parting):
    """Combine, casting scan and cut on the GPU's own fields give the oracle's
    kept set bit for bit, and the kept set has no undercut."""
    w = small_cantilever(24, 12, 8, seed=8, n_spheres=4, rmin=1.5, rmax=3.5, group=4, n_rhs=2)
    m, u, _ = _solve(w, afd.AFD_MIXED, 1e-9)
    s = np.zeros((2, m.nelem), np.float32)
    m.sensitivity(afd.AFD_SENS_STRAIN_ENERGY, s)
    weights = [1.0, 0.5]
    v = 0.7
    keys = levelset.casting_scan(levelset.combine([s[0], s[1]], weights), w.nx, w.ny, w.nz, axis, parting)
    kref, tref = levelset.select_top(keys, levelset.keep_count(v, keys.size))
    kept = np.zeros(m.nelem, np.uint8)
    tau = m.levelset_update(afd.AFD_SENS_STRAIN_ENERGY, weights, v, kept, casting=(axis, parting))
    assert np.array_equal(kept, kref)
    assert tau == np.float32(tref)
    kk = np.moveaxis(kept.reshape(w.nz, w.ny, w.nx), {0: 2, 1: 1, 2: 0}[axis], 0).astype(bool)
    for half in (kk[parting:], kk[:parting][::-1]):
        if half.shape[0] > 1:
            assert not np.any(~half[:-1] & half[1:])
    m.close()


@pytest.mark.parametrize("precision", [afd.AFD_MIXED, afd.AFD_FP64])
def test_stress_sensitivity_matches_oracle_adjoint(precision):
    """Eq. 3.3 with the adjoint state: lambda solves K lambda = -d sigma_PN/du and
    T_sigma follows from sigma(u) and eps(lambda), against the oracle's direct
    solves.  sigma_PN comes from the float32 von Mises field, whose rounding
    enters the adjoint right-hand side scaled by (p - 1): tolerance 2e-6."""
    w = small_cantilever(20, 10, 8, seed=6, n_spheres=4, rmin=1.5, rmax=3.0, group=4, n_rhs=2)
    m, u, _ = _solve(w, precision, 1e-10)
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    p = 6.0
    out = np.zeros((2, m.nelem), np.float32)
    lam = np.zeros_like(w.f)
    st = m.stress_sensitivity(p, 1e-10, out, lam)
    free = w.fixed == 0
    for r in range(2):
        assert st[r]["rel_residual"] <= 1e-10
        uref = fe.solve_direct(K, w.f[r], w.fixed)
        g = sensitivity.pnorm_stress_gradient(w.nx, w.ny, w.nz, w.E, uref, p)
        lref = fe.solve_direct(K, -g * free, w.fixed)
        assert np.linalg.norm(lam[r] - lref) <= 2e-6 * np.linalg.norm(lref)
        T = sensitivity.stress_topological_sensitivity(w.nx, w.ny, w.nz, w.E, uref, lref)
        assert np.max(np.abs(out[r] - T)) <= 2e-6 * np.max(np.abs(T))
    # the primal solution is untouched by the adjoint solve
    J = m.compliance()
    for r in range(2):
        assert abs(J[r] - float(w.f[r] @ u[r])) <= 1e-12 * abs(J[r])
    m.close()


def test_constrained_topology_driver_keeps_the_hard_constraints():
    """The Sec. 3.8 loop with hard compliance and stress constraints: the final
    feasible design meets both under the oracle's direct solve, its kept count
    matches its volume fraction, the volume steps follow the algorithm, and the
    AL scalars follow the oracle's Eqs. 3.11-3.12 on the recorded g."""
    nx, ny, nz = 24, 12, 12
    E0 = np.ones(nx * ny * nz)
    f, fixed = edge_load(nx, ny, nz), clamp_face_x0(nx, ny, nz)
    m = afd.Mesh(nx, ny, nz, group=4)
    m.set_loads_bcs(f[None], fixed)
    res = afd.run_constrained_topology(m, E0, compliance=1.5, stress=2.0, p=8.0, dv0=0.05, v_min=0.3, max_fea=50,
                                       tol=1e-8)
    m.close()
    hist = res["history"]
    assert res["stop"] in ("dv_min", "v_min", "max_fea")
    assert res["volume_fraction"] < 1.0
    K0 = fe.assemble(nx, ny, nz, E0)
    u0 = fe.solve_direct(K0, f, fixed)
    J0 = fe.compliance(f, u0)
    s0 = sensitivity.pnorm(sensitivity.element_von_mises(nx, ny, nz, E0, u0), 8.0)
    assert abs(res["reference"]["J"] - J0) <= 1e-6 * J0
    E = res["E"]
    u = fe.solve_direct(fe.assemble(nx, ny, nz, E), f, fixed)
    assert fe.compliance(f, u) <= 1.5 * J0 * (1 + 1e-6)
    assert sensitivity.pnorm(sensitivity.element_von_mises(nx, ny, nz, E, u), 8.0) <= 2.0 * s0 * (1 + 1e-5)
    assert int(res["kept"].sum()) == levelset.keep_count(res["volume_fraction"], E.size)
    mu = {"J": levelset.MU0, "sigma": levelset.MU0}
    gamma = {"J": levelset.GAMMA0, "sigma": levelset.GAMMA0}
    g_prev = {"J": 0.0, "sigma": 0.0}
    for k, h in enumerate(hist, start=1):
        for name in ("J", "sigma"):
            g = h["g"][name]
            mu[name] = levelset.multiplier_update(mu[name], gamma[name], g)
            gamma[name] = levelset.penalty_update(gamma[name], g, g_prev[name], k)
            g_prev[name] = g
            assert abs(h["mu"][name] - mu[name]) <= 1e-9 * max(1.0, abs(mu[name]))
            assert abs(h["gamma"][name] - gamma[name]) <= 1e-9 * gamma[name]
        assert h["violated"] == any(h["g"][n] > 0 for n in ("J", "sigma"))
        assert h["rel_residual"] <= 1e-8
    for a, b in zip(hist, hist[1:]):
        if a["violated"]:
            assert b["dv"] == a["dv"] / 2


def test_fp64_solve_with_a_coarse_problem_above_48kb_of_shared_memory():
    """n_c = 6144 (g = 4 on 64x32x32): the coarse step stages 48 KB of v in
    shared memory, above the default per-block limit.  The deflation space does
    not change the solution, so it must match the default grouping's."""
    w = small_cantilever(64, 32, 32, seed=5, n_spheres=8, rmin=2.0, rmax=5.0, group=4)
    m, u, stats = _solve(w, afd.AFD_FP64, 1e-10, group=4)
    assert afd.afd_coarse_size(m.h) == 6144
    assert stats[0]["rel_residual"] <= 1e-10
    m.close()
    m2, u2, _ = _solve(w, afd.AFD_FP64, 1e-10, group=16)
    m2.close()
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    assert fe.relative_residual(K, u[0], w.f[0], w.fixed) <= 1.0001e-10
    assert np.linalg.norm(u[0] - u2[0]) <= 1e-6 * np.linalg.norm(u2[0])


@pytest.mark.parametrize("precision", [afd.AFD_MIXED, afd.AFD_FP64])
def test_iteration_budget_stops_the_solve_with_not_converged(precision):
    """The stopping test at each iteration's start: with max_iter = 7 the loop
    stops after exactly 7 iterations and the solve reports NOT_CONVERGED,
    with the iterate it reached (residual below the initial one)."""
    w = small_cantilever(20, 10, 10, seed=4, n_spheres=4, rmin=1.5, rmax=3.0, group=4)
    m = afd.Mesh(w.nx, w.ny, w.nz, precision=precision, group=w.group, max_iter=7)
    m.set_element_moduli(w.E)
    m.set_loads_bcs(w.f, w.fixed)
    u = np.zeros_like(w.f)
    rc, stats = m.solve(1e-10, u_out=u, check=False)
    assert rc == afd.AFD_ERR_NOT_CONVERGED
    assert stats[0]["status"] == afd.AFD_ERR_NOT_CONVERGED
    assert stats[0]["iters"] == 7
    assert 0.0 < stats[0]["rel_residual"] < 1.0
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    assert abs(fe.relative_residual(K, u[0], w.f[0], w.fixed) - stats[0]["rel_residual"]) <= 1e-6
    with pytest.raises(afd.AFDError) as e:
        m.solve(1e-10)
    assert e.value.code == afd.AFD_ERR_NOT_CONVERGED
    m.close()


def test_iteration_kernel_timing_leaves_the_solution_and_the_solver_intact():
    """The measurement hook behind the bench's roofline: it runs the inner
    iteration's kernels after a mixed solve, reports a positive time for each,
    leaves u and J untouched, refuses a bad count, and the next solve (graphs
    recaptured) still meets its tolerance."""
    w = small_cantilever(20, 10, 10, seed=5, n_spheres=4, rmin=1.5, rmax=3.0, group=4)
    m, u, _ = _solve(w, afd.AFD_MIXED, 1e-8)
    J = m.compliance()[0]
    t = afd.afd_time_dpcg_kernels(m.h, 64)
    for k in ("stencil_us", "update_us", "coarse_rhs_us", "coarse_step_us"):
        assert np.isfinite(t[k]) and t[k] > 0.0
    with pytest.raises(afd.AFDError) as e:
        afd.afd_time_dpcg_kernels(m.h, 4097)
    assert e.value.code == afd.AFD_ERR_INVALID_ARG
    assert m.compliance()[0] == J
    u2 = np.zeros_like(w.f)
    stats = m.solve(1e-8, u_out=u2)
    assert stats[0]["rel_residual"] <= 1e-8
    assert np.linalg.norm(u2 - u) <= 1e-6 * np.linalg.norm(u)
    m.close()
