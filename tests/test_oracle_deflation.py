"""Pins of the oracle's deflation space (rigid-body modes of agglomerated node
groups) and of its coarse matrix."""
import numpy as np

from oracle import deflation, fe
from synthetic import clamp_face_x0


def test_single_group_modes_are_rigid():
    nx, ny, nz, g = 3, 3, 3, 3
    K = fe.assemble(nx, ny, nz, np.ones(27))
    W = deflation.deflation_matrix(nx, ny, nz, g, np.zeros(3 * 64, np.uint8))
    assert W.shape == (3 * 64, 6)
    assert np.max(np.abs(K @ W)) < 1e-13
    assert np.linalg.matrix_rank(W) == 6


def test_group_map_folds_last_plane():
    gid = deflation.node_groups(4, 2, 2, 2).reshape(3, 3, 5)
    assert gid[0, 0].tolist() == [0, 0, 1, 1, 1]
    assert deflation.group_counts(4, 2, 2, 2) == (2, 1, 1)


def test_piecewise_rigid_energy_lives_on_group_boundaries():
    """W mu is rigid on each group, so only elements whose nodes span two
    groups carry strain energy."""
    nx, ny, nz, g = 4, 2, 2, 2
    rng = np.random.default_rng(8)
    E = rng.uniform(0.5, 1.0, nx * ny * nz)
    W = deflation.deflation_matrix(nx, ny, nz, g, np.zeros(3 * 5 * 3 * 3, np.uint8))
    u = W @ rng.standard_normal(W.shape[1])
    from oracle import sensitivity
    s = sensitivity.strain_energy(nx, ny, nz, E, u)
    gid = deflation.node_groups(nx, ny, nz, g)
    en = fe.element_nodes(nx, ny, nz)
    straddle = np.array([len(set(gid[row])) > 1 for row in en])
    assert np.all(np.abs(s[~straddle]) < 1e-12)
    assert np.all(s[straddle] > 1e-8)


def test_coarse_matrix_spd_with_clamp_and_six_zero_modes_without():
    nx, ny, nz, g = 4, 2, 2, 2
    E = np.ones(nx * ny * nz)
    K = fe.assemble(nx, ny, nz, E)
    fixed = clamp_face_x0(nx, ny, nz)
    W = deflation.deflation_matrix(nx, ny, nz, g, fixed)
    Ec = deflation.coarse_matrix(K, W, fixed)
    assert np.allclose(Ec, Ec.T, atol=1e-13)
    assert np.linalg.eigvalsh(Ec).min() > 1e-8
    free = np.zeros_like(fixed)
    W0 = deflation.deflation_matrix(nx, ny, nz, g, free)
    w = np.linalg.eigvalsh(deflation.coarse_matrix(K, W0, free))
    assert np.sum(np.abs(w) < 1e-10 * w.max()) == 6


def test_apply_w_equals_the_dense_deflation_matrix():
    """W mu without forming W agrees with the explicit columns (ragged group
    grid, last planes folded, scattered supports), and it is rigid on one
    unsupported group: K (W mu) = 0."""
    rng = np.random.default_rng(21)
    for (nx, ny, nz, g) in ((5, 3, 4, 2), (7, 4, 3, 3), (3, 3, 3, 3)):
        nn = (nx + 1) * (ny + 1) * (nz + 1)
        fixed = (rng.random(3 * nn) < 0.1).astype(np.uint8)
        W = deflation.deflation_matrix(nx, ny, nz, g, fixed)
        mu = rng.standard_normal(W.shape[1])
        assert np.max(np.abs(deflation.apply_w(nx, ny, nz, g, fixed, mu) - W @ mu)) < 1e-13
    K = fe.assemble(3, 3, 3, np.ones(27))
    v = deflation.apply_w(3, 3, 3, 3, np.zeros(3 * 64, np.uint8), rng.standard_normal(6))
    assert np.max(np.abs(K @ v)) < 1e-12 * np.max(np.abs(v))
