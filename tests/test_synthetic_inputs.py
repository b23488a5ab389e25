"""The seeded synthetic inputs follow their stated recipe: sizes, supports,
load totals and placement, void patterns reproducible from the seed, the
8-load-case batch and the serving stream's size, void-fraction and arrival
mix.  Both the oracle and the CUDA path take these inputs, so a drift here
would move both sides together; these checks pin the inputs themselves."""
import numpy as np
import pytest

import synthetic as S


def _node(nx, ny, i, j, k):
    return i + (nx + 1) * (j + (ny + 1) * k)


def test_clamp_and_edge_load_placement():
    nx, ny, nz = 6, 3, 2
    fixed = S.clamp_face_x0(nx, ny, nz).reshape(nz + 1, ny + 1, nx + 1, 3)
    assert fixed.dtype == np.uint8
    assert np.all(fixed[:, :, 0, :] == 1) and not np.any(fixed[:, :, 1:, :])
    f = S.edge_load(nx, ny, nz, -2.0).reshape(nz + 1, ny + 1, nx + 1, 3)
    assert np.isclose(f.sum(), -2.0)
    assert np.allclose(f[0, :, nx, 2], -2.0 / (ny + 1))
    f[0, :, nx, 2] = 0.0
    assert not np.any(f)
    a = S.axial_face_load(nx, ny, nz, -1.0).reshape(nz + 1, ny + 1, nx + 1, 3)
    assert np.isclose(a[:, :, nx, 0].sum(), -1.0) and np.count_nonzero(a) == (ny + 1) * (nz + 1)


def test_sphere_voids_are_seeded_and_follow_their_definition():
    nx, ny, nz = 20, 10, 8
    E1 = S.sphere_voids(nx, ny, nz, 6, 1.5, 3.0, seed=5)
    assert np.array_equal(E1, S.sphere_voids(nx, ny, nz, 6, 1.5, 3.0, seed=5))
    assert not np.array_equal(E1, S.sphere_voids(nx, ny, nz, 6, 1.5, 3.0, seed=6))
    assert set(np.unique(E1)) <= {1e-3, 1.0}
    # the same spheres drawn again from the same generator: an element is void iff its centroid is inside one
    rng = np.random.Generator(np.random.PCG64(5))
    centres = rng.uniform([0, 0, 0], [nx, ny, nz], size=(6, 3))
    radii = rng.uniform(1.5, 3.0, size=6)
    assert np.all(radii >= 1.5) and np.all(radii <= 3.0)
    for e in range(nx * ny * nz):
        i, j, k = e % nx, (e // nx) % ny, e // (nx * ny)
        c = np.array([i + 0.5, j + 0.5, k + 0.5])
        inside = np.any(np.sum((centres - c) ** 2, axis=1) < radii ** 2)
        assert (E1[e] == 1e-3) == inside


def test_void_fraction_spheres_reach_their_target():
    for target, seed in ((0.1, 1), (0.25, 2), (0.4, 3)):
        E = S.void_fraction_spheres(32, 16, 16, target, np.random.Generator(np.random.PCG64(seed)))
        frac = float(np.mean(E == 1e-3))
        assert target <= frac < target + 0.25        # the last sphere overshoots by at most its own volume


def test_top_point_loads_are_unit_forces_on_the_top_face():
    nx, ny, nz = 12, 6, 6
    f = S.top_point_loads(nx, ny, nz, 8, seed=11)
    assert f.shape == (8, 3 * S.node_count(nx, ny, nz))
    assert np.array_equal(f, S.top_point_loads(nx, ny, nz, 8, seed=11))
    for r in range(8):
        nz_idx = np.flatnonzero(f[r])
        n = nz_idx[0] // 3
        assert np.all(nz_idx // 3 == n)                # one node
        i, j, k = n % (nx + 1), (n // (nx + 1)) % (ny + 1), n // ((nx + 1) * (ny + 1))
        assert k == nz and i >= 1                      # top face, off the clamp
        assert np.isclose(np.linalg.norm(f[r, 3 * n:3 * n + 3]), 1.0)


def test_named_workloads_have_their_stated_shapes():
    w0 = S.cantilever_24x12x12_solid()
    assert (w0.nx, w0.ny, w0.nz, w0.n_rhs) == (24, 12, 12, 1) and np.all(w0.E == 1.0) and w0.tol == 1e-10
    assert w0.ndof == 12675
    w1 = S.cantilever_128x64x64_voids()
    assert (w1.nx, w1.ny, w1.nz, w1.n_rhs, w1.tol) == (128, 64, 64, 1, 1e-6)
    assert w1.ndof == 1635075
    assert np.array_equal(w1.E, S.sphere_voids(128, 64, 64, 40, 4.0, 10.0, 1, 1e-3))
    assert 0.0 < np.mean(w1.E == 1e-3) < 0.5
    w2 = S.multiload_96x48x48_voids()
    assert (w2.nx, w2.ny, w2.nz, w2.n_rhs) == (96, 48, 48, 8) and w2.ndof == 698691
    assert np.allclose(np.linalg.norm(w2.f, axis=1), 1.0)


@pytest.mark.parametrize("rate", [50.0, 0.0])
def test_serving_stream_mix(rate):
    reqs = S.serving_stream(256, seed=3, rate_per_s=rate)
    assert len(reqs) == 256 and [r["id"] for r in reqs] == list(range(256))
    assert reqs == S.serving_stream(256, seed=3, rate_per_s=rate)
    sizes = {r["nx"] for r in reqs}
    assert sizes <= {32, 48, 64, 96, 128, 160} and len(sizes) == 6
    assert all(r["ny"] == r["nx"] // 2 == r["nz"] for r in reqs)
    assert all(0.1 <= r["void_fraction"] <= 0.4 for r in reqs)
    t = [r["arrival_s"] for r in reqs]
    if rate > 0:
        assert all(b >= a for a, b in zip(t, t[1:]))
        gaps = np.diff([0.0] + t)
        assert abs(np.mean(gaps) * rate - 1.0) < 0.2      # Poisson arrivals at the given rate
    else:
        assert all(x == 0.0 for x in t)
    E, f, fixed = S.serving_request_inputs(reqs[0])
    n = reqs[0]["nx"] * reqs[0]["ny"] * reqs[0]["nz"]
    assert E.shape == (n,) and np.mean(E == 1e-3) >= reqs[0]["void_fraction"]
    assert f.shape == (1, fixed.size)
