"""Modal analysis and the eigenvalue topological sensitivity (Eq. 3.4).

Test infrastructure: only tests/, the smoke check and the benchmark's CPU
baseline import this module; the product path never does.

Eq. 3.4 gives the topological sensitivity of the n-th eigenvalue as
sigma:eps - omega_n^2 rho |u_n|^2, with u_n the n-th mode shape and rho the
material density.  The paper defines neither the mass matrix nor how the
void material's density is modelled.  Readings used here:

  * Lumped mass: every node of element e receives rho_e h^3 / 8 in each of
    its three directions (the row-sum lumping of the trilinear element's
    consistent mass, which for a cube gives each node exactly one eighth).
  * rho_e = rho * E_e: the density follows the modulus (solid 1, void e_void),
    so that void regions keep the solid's wave speed and produce no spurious
    low-frequency local modes.
  * The eigenproblem is K_ff phi = lambda M_ff phi on the free DOFs (phi = 0 on
    fixed DOFs), lambda = omega^2, the modes M-orthonormal (phi^T M phi = 1).
  * Eq. 3.4 is evaluated at the element centroid, like Eqs. 3.2 and 3.3:
    sigma(phi):eps(phi) - lambda rho_e |phi(centroid)|^2, phi(centroid) the
    mean of the element's eight nodal vectors.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe, sensitivity


def lumped_mass(nx: int, ny: int, nz: int, E: np.ndarray, rho: float = 1.0, h: float = 1.0) -> np.ndarray:
    """Diagonal of the lumped mass matrix per DOF (length 3 N_nodes)."""
    en = fe.element_nodes(nx, ny, nz)
    me = rho * np.asarray(E, dtype=np.float64) * h ** 3 / 8.0          # per element node
    mn = np.bincount(en.reshape(-1), weights=np.repeat(me, 8), minlength=(nx + 1) * (ny + 1) * (nz + 1))
    return np.repeat(mn, 3)


def _free_problem(nx, ny, nz, E, fixed, rho, nu, h):
    K = fe.assemble(nx, ny, nz, E, nu, h)
    m = lumped_mass(nx, ny, nz, E, rho, h)
    fr = fe.free_dofs(fixed)
    return K[fr][:, fr].tocsc(), m[fr], fr, K.shape[0], m


def _normalise(lam, vec_f, fr, n, m_full):
    order = np.argsort(lam)
    lam = lam[order]
    phi = np.zeros((lam.size, n))
    phi[:, fr] = vec_f[:, order].T
    for i in range(lam.size):
        phi[i] /= np.sqrt(phi[i] @ (m_full * phi[i]))
        j = np.argmax(np.abs(phi[i]))
        if phi[i, j] < 0:
            phi[i] = -phi[i]
    return lam, phi


def modes(nx: int, ny: int, nz: int, E: np.ndarray, fixed: np.ndarray, k: int, rho: float = 1.0,
          nu: float = 0.3, h: float = 1.0):
    """The k smallest eigenpairs of K_ff phi = lambda M_ff phi: shift-invert
    Lanczos (scipy eigsh around 0).  Returns (lambda ascending, phi (k, ndof)),
    phi M-orthonormal, zero on fixed DOFs, largest |component| positive."""
    Kff, mf, fr, n, m_full = _free_problem(nx, ny, nz, E, fixed, rho, nu, h)
    lam, vec = spla.eigsh(Kff, k=k, M=sp.diags(mf).tocsc(), sigma=0.0, which="LM", tol=1e-13)
    return _normalise(lam, vec, fr, n, m_full)


def modes_dense(nx: int, ny: int, nz: int, E: np.ndarray, fixed: np.ndarray, k: int, rho: float = 1.0,
                nu: float = 0.3, h: float = 1.0):
    """The same eigenpairs from the dense generalised symmetric eigensolver
    (LAPACK), for tiny meshes."""
    Kff, mf, fr, n, m_full = _free_problem(nx, ny, nz, E, fixed, rho, nu, h)
    lam, vec = sla.eigh(Kff.toarray(), np.diag(mf), subset_by_index=[0, k - 1])
    return _normalise(lam, vec, fr, n, m_full)


def eigen_sensitivity(nx: int, ny: int, nz: int, E: np.ndarray, phi: np.ndarray, lam: float, rho: float = 1.0,
                      nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """T_lambda of Eq. 3.4 at each element centroid for one mode (phi, lambda)."""
    eps = sensitivity.centroid_strain(nx, ny, nz, phi, h)
    sig = sensitivity.centroid_stress(eps, E, nu)
    se = np.einsum("eij,eij->e", sig, eps)
    uc = phi.reshape(-1, 3)[fe.element_nodes(nx, ny, nz)].mean(axis=1)     # (N_e, 3)
    rho_e = rho * np.asarray(E, dtype=np.float64)
    return se - lam * rho_e * np.einsum("ec,ec->e", uc, uc)
