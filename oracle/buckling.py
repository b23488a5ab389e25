"""Linear buckling and the buckling-load sensitivity (Eq. 3.5).

Test infrastructure: only tests/, the smoke check and the benchmark's CPU
baseline import this module; the product path never does.

Eq. 3.5 gives the sensitivity of the buckling load factor as
u^T (K^e - lambda K_sigma^e) u with the element geometric stiffness K_sigma^e,
the critical load factor lambda and the buckling mode u.  The paper does not
define K_sigma^e or the pre-buckling state.  Readings used here:

  * Pre-buckling state: the static solution u0 of the load case f
    (K u0 = f on the free DOFs); its stress S_e = E_e C eps(u0) taken at the
    element centroid and held constant over the element (the sampling point of
    Eqs. 3.2 and 3.3).
  * Geometric stiffness of the state: K_G^e[(a, i), (b, j)] =
    delta_ij * integral over the element of grad N_a . S_e grad N_b, with the
    2x2x2 Gauss rule (exact for the cube).  Eq. 3.5's K_sigma is read with the
    sign that makes its buckling equation (K - lambda K_sigma) phi = 0, i.e.
    K_sigma = -K_G (positive where the state compresses).
  * Buckling: (K + lambda K_G) phi = 0 on the free DOFs (phi = 0 on fixed
    DOFs); lambda_cr is the smallest positive lambda, the factor on f at which
    the structure buckles.  It is computed as the largest mu of
    (-K_G) phi = mu K phi, lambda = 1 / mu; modes are K-normalised
    (phi^T K phi = 1).
  * Eq. 3.5 per element: phi_e^T (E_e K0 - lambda K_sigma^e) phi_e
    = phi_e^T (E_e K0 + lambda K_G^e) phi_e; the element terms of an exact
    mode sum to phi^T (K + lambda K_G) phi = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe, sensitivity


def centroid_stress_state(nx, ny, nz, E, u0, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """(N_e, 3, 3) stress of the pre-buckling state at each element centroid."""
    return sensitivity.centroid_stress(sensitivity.centroid_strain(nx, ny, nz, u0, h), E, nu)


def geometric_element(S: np.ndarray, h: float = 1.0) -> np.ndarray:
    """8 x 8 matrix G[a, b] = integral of grad N_a . S grad N_b over a cube of
    edge h (2x2x2 Gauss); the element geometric stiffness is G kron I_3."""
    g = 1.0 / np.sqrt(3.0)
    pts = [(1.0 - g) / 2.0, (1.0 + g) / 2.0]
    w = (h / 2.0) ** 3
    G = np.zeros((8, 8))
    for x in pts:
        for y in pts:
            for z in pts:
                D = fe.shape_gradients(np.array([x, y, z]), h)   # (8, 3)
                G += w * D @ S @ D.T
    return G


def assemble_geometric(nx, ny, nz, S: np.ndarray, h: float = 1.0) -> sp.csr_matrix:
    """Global K_G = sum_e P_e^T (G_e kron I_3) P_e, FP64 CSR."""
    en = fe.element_nodes(nx, ny, nz)
    rows, cols, vals = [], [], []
    for e in range(en.shape[0]):
        G = geometric_element(S[e], h)
        for c in range(3):
            d = 3 * en[e] + c
            rows.append(np.repeat(d, 8))
            cols.append(np.tile(d, 8))
            vals.append(G.reshape(-1))
    n = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    Kg = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    Kg.sum_duplicates()
    return Kg


def _pencil(nx, ny, nz, E, f, fixed, nu, h):
    K = fe.assemble(nx, ny, nz, E, nu, h)
    u0 = fe.solve_direct(K, f, fixed)
    S = centroid_stress_state(nx, ny, nz, E, u0, nu, h)
    Kg = assemble_geometric(nx, ny, nz, S, h)
    fr = fe.free_dofs(fixed)
    return K, Kg, S, fr


def _finish(mu, vec, fr, K, k):
    keep = np.argsort(-mu)[:k]
    mu = mu[keep]
    if not np.all(mu > 0):
        raise ValueError("fewer positive buckling factors than requested")
    phi = np.zeros((k, K.shape[0]))
    phi[:, fr] = vec[:, keep].T
    for i in range(k):
        phi[i] /= np.sqrt(phi[i] @ (K @ phi[i]))
        j = np.argmax(np.abs(phi[i]))
        if phi[i, j] < 0:
            phi[i] = -phi[i]
    return 1.0 / mu, phi


def buckling(nx, ny, nz, E, f, fixed, k: int, nu: float = 0.3, h: float = 1.0):
    """The k smallest positive load factors (ascending) and their K-normalised
    modes, by Lanczos on (-K_G, K) (scipy eigsh, largest algebraic mu).
    Also returns the pre-buckling stress state."""
    K, Kg, S, fr = _pencil(nx, ny, nz, E, f, fixed, nu, h)
    Kff, Kgff = K[fr][:, fr].tocsc(), Kg[fr][:, fr].tocsc()
    mu, vec = spla.eigsh(-Kgff, k=k, M=Kff, which="LA", tol=1e-13)
    lam, phi = _finish(mu, vec, fr, K, k)
    return lam, phi, S


def buckling_dense(nx, ny, nz, E, f, fixed, k: int, nu: float = 0.3, h: float = 1.0):
    """The same from the dense generalised symmetric eigensolver (LAPACK)."""
    K, Kg, S, fr = _pencil(nx, ny, nz, E, f, fixed, nu, h)
    mu, vec = sla.eigh(-Kg[fr][:, fr].toarray(), K[fr][:, fr].toarray())
    lam, phi = _finish(mu, vec, fr, K, k)
    return lam, phi, S


def buckling_sensitivity(nx, ny, nz, E, S, phi, lam: float, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """Eq. 3.5 per element: phi_e^T (E_e K0 - lambda K_sigma^e) phi_e with
    K_sigma^e = -K_G^e (reading above)."""
    se = sensitivity.strain_energy(nx, ny, nz, E, phi, nu, h)
    en = fe.element_nodes(nx, ny, nz)
    pe = phi.reshape(-1, 3)[en]                                  # (N_e, 8, 3)
    geo = np.array([np.einsum("ac,ab,bc->", pe[e], geometric_element(S[e], h), pe[e]) for e in range(en.shape[0])])
    return se + lam * geo
