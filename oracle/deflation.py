"""Deflation space of the assembly-free deflated CG (Sec. 3.5).

The paper delegates the deflation space to its ref. [42] and prints no
definition.  Reading used here (the rigid-body modes of agglomerated node
groups):
  * nodes are agglomerated into boxes of g x g x g element widths:
    node (i, j, k) belongs to group (min(i // g, nx/g - 1), ...) per axis, so
    the last node plane folds into the last group;
  * each group G contributes 6 columns to W: the three translations and the
    three infinitesimal rotations about the group's node centroid c_G,
        T_c = e_c,   R_c(x) = e_c x (x - c_G),
    restricted to the group's nodes, with zero rows at fixed DOFs;
  * the coarse matrix is E = W^T K W (K with the fixed rows and columns
    removed), dense, FP64.

The oracle never uses W to solve (deflation does not change the solution of
K u = f); it is used to pin the CUDA coarse operators on tiny meshes.
Column order inside a group: (T_x, T_y, T_z, R_x, R_y, R_z); group order
G = Gx + NGx * (Gy + NGy * Gz).
"""
from __future__ import annotations

import numpy as np

from . import fe


def group_counts(nx, ny, nz, g):
    return max(nx // g, 1), max(ny // g, 1), max(nz // g, 1)


def node_groups(nx, ny, nz, g) -> np.ndarray:
    """Group index of every node."""
    ngx, ngy, ngz = group_counts(nx, ny, nz, g)
    X = fe.node_coordinates(nx, ny, nz).astype(np.int64)
    gx = np.minimum(X[:, 0] // g, ngx - 1)
    gy = np.minimum(X[:, 1] // g, ngy - 1)
    gz = np.minimum(X[:, 2] // g, ngz - 1)
    return gx + ngx * (gy + ngy * gz)


def group_centroids(nx, ny, nz, g) -> np.ndarray:
    """(N_g, 3) mean coordinate of each group's nodes."""
    X = fe.node_coordinates(nx, ny, nz)
    gid = node_groups(nx, ny, nz, g)
    ng = int(np.prod(group_counts(nx, ny, nz, g)))
    cnt = np.bincount(gid, minlength=ng).astype(np.float64)
    return np.stack([np.bincount(gid, weights=X[:, c], minlength=ng) / cnt for c in range(3)], axis=1)


def deflation_matrix(nx, ny, nz, g, fixed: np.ndarray) -> np.ndarray:
    """Dense W (ndof x 6 N_g) of rigid-body modes per group."""
    X = fe.node_coordinates(nx, ny, nz)
    gid = node_groups(nx, ny, nz, g)
    c = group_centroids(nx, ny, nz, g)
    nn = X.shape[0]
    ng = c.shape[0]
    W = np.zeros((3 * nn, 6 * ng))
    rel = X - c[gid]
    for n in range(nn):
        G = gid[n]
        for comp in range(3):
            W[3 * n + comp, 6 * G + comp] = 1.0
        for axis in range(3):
            e = np.zeros(3)
            e[axis] = 1.0
            W[3 * n:3 * n + 3, 6 * G + 3 + axis] = np.cross(e, rel[n])
    W[np.asarray(fixed) != 0, :] = 0.0
    return W


def coarse_matrix(K, W: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """E = W^T K W with fixed DOFs eliminated (their rows of W are zero, and
    the fixed rows/columns of K are dropped)."""
    fr = fe.free_dofs(fixed)
    Kff = K[fr][:, fr]
    Wf = W[fr]
    return Wf.T @ (Kff @ Wf)


def apply_w(nx, ny, nz, g, fixed: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """W mu without forming W: at node n of group G the rigid motion
    t_G + omega_G x (x_n - c_G), with mu = (t_x, t_y, t_z, omega_x, omega_y,
    omega_z) per group in the column order of ``deflation_matrix``; zero at
    fixed DOFs."""
    X = fe.node_coordinates(nx, ny, nz)
    gid = node_groups(nx, ny, nz, g)
    c = group_centroids(nx, ny, nz, g)
    m6 = np.asarray(mu, dtype=np.float64).reshape(-1, 6)
    rel = X - c[gid]
    out = m6[gid, :3] + np.cross(m6[gid, 3:], rel)
    out = out.reshape(-1)
    out[np.asarray(fixed) != 0] = 0.0
    return out
