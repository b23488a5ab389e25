"""Finite element definitions for K u = f on a voxel hex8 mesh (Eq. 1.1, Sec. 3.5).

The paper names the element stiffness matrix K^e (Eq. 3.5) and states that the
domain is discretised with hexahedral elements (Sec. 3.8, step 1) but prints no
formula for it.  Reading used here: 8-node trilinear hexahedron on a cube of
edge h, isotropic linear elasticity with Lame parameters from (E, nu), full
2x2x2 Gauss quadrature (exact for the cube, the integrand being at most
quadratic per axis), engineering shear strains in Voigt form.

Index conventions are those of ``synthetic`` (x fastest for elements, nodes and
the 8 local nodes of an element; DOF = 3 * node + component).

Per-element modulus: K = sum_e E_e P_e^T K0 P_e, where K0 is the element matrix
for E = 1 (the solid / weak-void material model of the workloads).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# local node a = ax + 2*ay + 4*az  ->  offset (ax, ay, az)
LOCAL_OFFSETS = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.int64)


def lame(E: float, nu: float):
    """Lame parameters (lambda, mu) of an isotropic material."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_voigt(E: float, nu: float) -> np.ndarray:
    """6x6 isotropic constitutive matrix, Voigt order (xx, yy, zz, xy, yz, zx),
    engineering shear strains."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def shape_gradients(xi: np.ndarray, h: float = 1.0) -> np.ndarray:
    """Physical gradients of the 8 trilinear shape functions at a point of the
    unit reference cube xi in [0,1]^3; returns (8, 3)."""
    g = np.zeros((8, 3))
    for a, (ax, ay, az) in enumerate(LOCAL_OFFSETS):
        fx = xi[0] if ax else 1.0 - xi[0]
        fy = xi[1] if ay else 1.0 - xi[1]
        fz = xi[2] if az else 1.0 - xi[2]
        dx = 1.0 if ax else -1.0
        dy = 1.0 if ay else -1.0
        dz = 1.0 if az else -1.0
        g[a] = [dx * fy * fz, fx * dy * fz, fx * fy * dz]
    return g / h


def strain_displacement(grad: np.ndarray) -> np.ndarray:
    """6x24 B matrix (Voigt, engineering shear) from (8,3) shape gradients."""
    B = np.zeros((6, 24))
    for a in range(8):
        gx, gy, gz = grad[a]
        c = 3 * a
        B[0, c + 0] = gx
        B[1, c + 1] = gy
        B[2, c + 2] = gz
        B[3, c + 0] = gy
        B[3, c + 1] = gx
        B[4, c + 1] = gz
        B[4, c + 2] = gy
        B[5, c + 0] = gz
        B[5, c + 2] = gx
    return B


def ke_hex8(nu: float, h: float = 1.0, E: float = 1.0) -> np.ndarray:
    """24x24 element stiffness K^e (Eq. 3.5 names it) of the trilinear hex on a
    cube of edge h: sum over the 2x2x2 Gauss points of w B^T D B."""
    D = elasticity_voigt(E, nu)
    g = 1.0 / np.sqrt(3.0)
    pts = [(1.0 - g) / 2.0, (1.0 + g) / 2.0]
    K = np.zeros((24, 24))
    w = (h / 2.0) ** 3  # weight 1/2 per axis on [0,1], times h per axis
    for x in pts:
        for y in pts:
            for z in pts:
                B = strain_displacement(shape_gradients(np.array([x, y, z]), h))
                K += w * B.T @ D @ B
    return 0.5 * (K + K.T)


def element_nodes(nx: int, ny: int, nz: int) -> np.ndarray:
    """(N_e, 8) global node indices of each element's local nodes."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.reshape(-1), j.reshape(-1), k.reshape(-1)
    nxn, nyn = nx + 1, ny + 1
    out = np.empty((i.size, 8), dtype=np.int64)
    for a, (ax, ay, az) in enumerate(LOCAL_OFFSETS):
        out[:, a] = (i + ax) + nxn * ((j + ay) + nyn * (k + az))
    return out


def element_dofs(nx: int, ny: int, nz: int) -> np.ndarray:
    """(N_e, 24) global DOF indices, local DOF 3a + c."""
    en = element_nodes(nx, ny, nz)
    return (3 * en[:, :, None] + np.arange(3)[None, None, :]).reshape(en.shape[0], 24)


def node_coordinates(nx: int, ny: int, nz: int, h: float = 1.0) -> np.ndarray:
    """(N_nodes, 3) coordinates."""
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return h * np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], axis=1).astype(np.float64)


def assemble(nx: int, ny: int, nz: int, E: np.ndarray, nu: float = 0.3, h: float = 1.0) -> sp.csr_matrix:
    """Global K = sum_e E_e P_e^T K0 P_e (Eq. 1.1), FP64 CSR, no boundary
    conditions applied."""
    K0 = ke_hex8(nu, h)
    dofs = element_dofs(nx, ny, nz)
    ne = dofs.shape[0]
    rows = np.repeat(dofs, 24, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, 24)).reshape(-1)
    vals = (np.asarray(E, dtype=np.float64)[:, None, None] * K0[None, :, :]).reshape(-1)
    n = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    K = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    K.sum_duplicates()
    assert K.shape == (n, n) and ne == nx * ny * nz
    return K


def matvec_free(nx: int, ny: int, nz: int, E: np.ndarray, u: np.ndarray, nu: float = 0.3,
                h: float = 1.0, chunk: int = 1 << 18) -> np.ndarray:
    """y = K u element by element without forming K (same definition as
    ``assemble``, for meshes too large to assemble).  No boundary conditions."""
    K0 = ke_hex8(nu, h)
    dofs = element_dofs(nx, ny, nz)
    y = np.zeros_like(u, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    for s in range(0, dofs.shape[0], chunk):
        d = dofs[s:s + chunk]
        ue = u[d]                                   # (c, 24)
        ye = (ue @ K0) * E[s:s + chunk, None]       # K0 symmetric
        y += np.bincount(d.reshape(-1), weights=ye.reshape(-1), minlength=u.size)
    return y


def free_dofs(fixed: np.ndarray) -> np.ndarray:
    return np.flatnonzero(np.asarray(fixed) == 0)


def solve_direct(K: sp.csr_matrix, f: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """Solve K_ff u_f = f_f with u = 0 on the fixed DOFs (sparse LU, FP64)."""
    fr = free_dofs(fixed)
    Kff = K[fr][:, fr].tocsc()
    u = np.zeros(K.shape[0])
    u[fr] = spla.spsolve(Kff, f[fr])
    return u


def solve_pcg(K: sp.csr_matrix, f: np.ndarray, fixed: np.ndarray, rtol: float = 1e-12,
              maxiter: int = 100000, x0=None):
    """Plain Jacobi-preconditioned CG on K_ff u_f = f_f, FP64, stopping when
    ||f_f - K_ff u_f||_2 <= rtol * ||f_f||_2.  Returns (u, iterations)."""
    fr = free_dofs(fixed)
    A = K[fr][:, fr].tocsr()
    b = f[fr]
    dinv = 1.0 / A.diagonal()
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, dtype=np.float64)[fr].copy()
    r = b - A @ x
    z = dinv * r
    p = z.copy()
    rz = r @ z
    bn = np.linalg.norm(b)
    it = 0
    while np.linalg.norm(r) > rtol * bn and it < maxiter:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    u = np.zeros(K.shape[0])
    u[fr] = x
    return u, it


def relative_residual(K_or_apply, u: np.ndarray, f: np.ndarray, fixed: np.ndarray) -> float:
    """||f - K u||_2 / ||f||_2 over the free DOFs."""
    Ku = K_or_apply(u) if callable(K_or_apply) else K_or_apply @ u
    fr = free_dofs(fixed)
    return float(np.linalg.norm((f - Ku)[fr]) / np.linalg.norm(f[fr]))


def compliance(f: np.ndarray, u: np.ndarray) -> float:
    """J = f^T u (the compliance of Eqs. 1.3-1.4)."""
    return float(np.dot(f, u))


def jacobi_diagonal(nx: int, ny: int, nz: int, E: np.ndarray, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """diag(K) per DOF (no boundary conditions), as the diagonal of the
    assembled matrix."""
    return assemble(nx, ny, nz, E, nu, h).diagonal()
