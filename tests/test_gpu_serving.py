"""Serving loop (continuous batching under an HBM budget): every result is the
same alone and in the mix, within the solve tolerance; admission respects the
budget; an oversize request is refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_2203_15115_gb300 as afd  # noqa: E402
from synthetic import clamp_face_x0, edge_load, sphere_voids  # noqa: E402

SIZES = [(12, 6, 6), (16, 8, 8), (20, 10, 10), (12, 6, 6), (24, 12, 12), (16, 8, 8), (20, 10, 10)]
TOL = 1e-9


def _inputs(nx, ny, nz, seed):
    E = sphere_voids(nx, ny, nz, 3, 1.5, 3.0, seed, 1e-3)
    return E, edge_load(nx, ny, nz), clamp_face_x0(nx, ny, nz)


def _alone(nx, ny, nz, E, f, fixed):
    m = afd.Mesh(nx, ny, nz)
    m.set_element_moduli(E)
    m.set_loads_bcs(f[None], fixed)
    u = np.zeros((1, f.size))
    m.solve(TOL, u_out=u)
    J = m.compliance()[0]
    m.close()
    return u[0], J


@pytest.mark.parametrize("slots,budget_factor", [(3, 100.0), (4, 1.3)])
def test_results_same_alone_and_in_the_mix(slots, budget_factor):
    assert torch.cuda.is_available()
    afd.lib()
    biggest = max(afd.afd_mesh_bytes(*d) for d in SIZES)
    srv = afd.Server(max_slots=slots, budget_bytes=budget_factor * biggest)
    inputs = [(d, *_inputs(*d, seed=i)) for i, d in enumerate(SIZES)]
    ids = [srv.submit(*d, E, f, fixed, TOL) for d, E, f, fixed in inputs]
    for rid, (d, E, f, fixed) in zip(ids, inputs):
        rc, st, J, lat, u = srv.wait(rid)
        assert rc == afd.AFD_OK, st
        assert st["rel_residual"] <= TOL
        assert lat > 0
        ua, Ja = _alone(*d, E, f, fixed)
        assert np.linalg.norm(u - ua) <= 1e-6 * np.linalg.norm(ua)
        assert abs(J - Ja) <= 1e-8 * abs(Ja)
    srv.close()


def test_oversize_request_is_refused():
    srv = afd.Server(max_slots=1, budget_bytes=1e6)
    E, f, fixed = _inputs(12, 6, 6, 0)
    with pytest.raises(afd.AFDError) as e:
        srv.submit(12, 6, 6, E, f, fixed, 1e-6)
    assert e.value.code == afd.AFD_ERR_OOM
    srv.close()


def test_pool_reuses_meshes_of_the_same_size():
    srv = afd.Server(max_slots=2, budget_bytes=100 * afd.afd_mesh_bytes(16, 8, 8))
    for rep in range(3):
        ids = [srv.submit(16, 8, 8, *_inputs(16, 8, 8, seed=rep * 2 + k), TOL) for k in range(2)]
        for rid in ids:
            rc, st, J, lat, u = srv.wait(rid, want_u=False)
            assert rc == afd.AFD_OK
    n, b = srv.resident()
    assert n <= 2 and b <= 2 * afd.afd_mesh_bytes(16, 8, 8)
    srv.close()


def test_budget_evicts_idle_meshes():
    big = afd.afd_mesh_bytes(24, 12, 12)
    srv = afd.Server(max_slots=1, budget_bytes=1.2 * big)
    for d in [(12, 6, 6), (16, 8, 8), (24, 12, 12), (12, 6, 6)]:
        rid = srv.submit(*d, *_inputs(*d, seed=1), TOL)
        rc, st, J, lat, u = srv.wait(rid, want_u=False)
        assert rc == afd.AFD_OK
        n, b = srv.resident()
        assert b <= 1.2 * big
    srv.close()


def test_session_warm_start_matches_a_cold_solve():
    """Successive solves of one session with the same loads start from the
    previous solution (fewer iterations) and agree with a cold solve."""
    nx, ny, nz = 24, 12, 12
    E0, f, fixed = _inputs(nx, ny, nz, seed=7)
    E1 = E0.copy()
    E1[: nx * ny * 2] *= 0.97          # a small design change, as between level-set iterations
    srv = afd.Server(max_slots=2, budget_bytes=100 * afd.afd_mesh_bytes(nx, ny, nz))
    rc, st0, J0, _, u0 = srv.wait(srv.submit(nx, ny, nz, E0, f, fixed, TOL, session=5))
    assert rc == afd.AFD_OK
    rc, st1, J1, _, u1 = srv.wait(srv.submit(nx, ny, nz, E1, f, fixed, TOL, session=5))
    assert rc == afd.AFD_OK
    rc, stc, Jc, _, uc = srv.wait(srv.submit(nx, ny, nz, E1, f, fixed, TOL))
    assert rc == afd.AFD_OK
    assert st1["iters"] < stc["iters"], (st1["iters"], stc["iters"])
    assert np.linalg.norm(u1 - uc) <= 1e-6 * np.linalg.norm(uc)
    assert abs(J1 - Jc) <= 1e-8 * abs(Jc)
    srv.end_session(5)
    srv.close()
