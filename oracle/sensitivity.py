"""Per-element sensitivity fields (Sec. 3.1, Eqs. 3.2, 3.3, 3.5).

Readings of the paper:
  * Element strain energy s_e = u_e^T (E_e K0) u_e: the element-removal
    ("element-sensitivity") form that Sec. 3.1 falls back to when no closed
    form is available, with sum_e s_e = u^T K u = f^T u = J.
  * Eq. 3.2 is printed as the 2-D (plane) topological derivative of the
    compliance.  It is evaluated exactly as printed,
        T_J = 4/(1+nu) sigma:eps - (1-3 nu)/(1-nu^2) tr(sigma) tr(eps),
    with 3-D tensors eps = sym(grad u) and sigma = E_e (lam tr(eps) I + 2 mu eps)
    taken at the element centroid (the paper does not say where the field is
    sampled).
  * Von Mises stress at the element centroid; the p-norm stress of Eq. 3.3 is
    (sum_e sigma_vm,e^p)^(1/p), no volume weighting (p is not given in the
    paper; it is an argument).
  * Eq. 3.3 is garbled (tr(lambda) of a vector field, no adjoint equation).
    Read consistently with Eq. 3.2 as
        T_sigma = 4/(1+nu) sigma(u):eps(lambda) - (1-3 nu)/(1-nu^2) tr sigma(u) tr eps(lambda),
    at the element centroid, with the adjoint lambda solving
    K lambda = -d sigma_PN / d u on the free DOFs (zero on fixed DOFs).
"""
from __future__ import annotations

import numpy as np

from . import fe


def centroid_strain(nx, ny, nz, u: np.ndarray, h: float = 1.0) -> np.ndarray:
    """(N_e, 3, 3) small-strain tensor sym(grad u) at each element centroid."""
    grad = fe.shape_gradients(np.array([0.5, 0.5, 0.5]), h)   # (8, 3)
    en = fe.element_nodes(nx, ny, nz)
    ue = u.reshape(-1, 3)[en]                                  # (N_e, 8, 3): [e, a, component]
    F = np.einsum("eac,aj->ecj", ue, grad)                     # F[e, c, j] = d u_c / d x_j
    return 0.5 * (F + np.swapaxes(F, 1, 2))


def centroid_stress(eps: np.ndarray, E: np.ndarray, nu: float) -> np.ndarray:
    """sigma = E_e (lam tr(eps) I + 2 mu eps) with (lam, mu) of the unit modulus."""
    lam, mu = fe.lame(1.0, nu)
    tr = np.trace(eps, axis1=1, axis2=2)
    sig = 2.0 * mu * eps + lam * tr[:, None, None] * np.eye(3)[None]
    return np.asarray(E, dtype=np.float64)[:, None, None] * sig


def strain_energy(nx, ny, nz, E: np.ndarray, u: np.ndarray, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """s_e = u_e^T (E_e K0) u_e for every element."""
    K0 = fe.ke_hex8(nu, h)
    ue = u[fe.element_dofs(nx, ny, nz)]
    return np.asarray(E, dtype=np.float64) * np.einsum("ei,ij,ej->e", ue, K0, ue)


def topological_compliance(nx, ny, nz, E: np.ndarray, u: np.ndarray, nu: float = 0.3,
                           h: float = 1.0) -> np.ndarray:
    """T_J of Eq. 3.2 at each element centroid."""
    eps = centroid_strain(nx, ny, nz, u, h)
    sig = centroid_stress(eps, E, nu)
    s_e = np.einsum("eij,eij->e", sig, eps)
    return 4.0 / (1.0 + nu) * s_e - (1.0 - 3.0 * nu) / (1.0 - nu * nu) * \
        np.trace(sig, axis1=1, axis2=2) * np.trace(eps, axis1=1, axis2=2)


def von_mises(sig: np.ndarray) -> np.ndarray:
    """Von Mises equivalent stress of (N, 3, 3) stress tensors, through the
    deviatoric invariant: sqrt(3/2 s:s), s = sigma - tr(sigma)/3 I."""
    dev = sig - np.trace(sig, axis1=1, axis2=2)[:, None, None] / 3.0 * np.eye(3)[None]
    return np.sqrt(1.5 * np.einsum("eij,eij->e", dev, dev))


def element_von_mises(nx, ny, nz, E, u, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    return von_mises(centroid_stress(centroid_strain(nx, ny, nz, u, h), E, nu))


def pnorm(values: np.ndarray, p: float) -> float:
    """(sum_e v_e^p)^(1/p) (Eq. 3.3's p-norm stress measure)."""
    v = np.asarray(values, dtype=np.float64)
    m = v.max()
    if m == 0.0:
        return 0.0
    return float(m * np.sum((v / m) ** p) ** (1.0 / p))


def pnorm_stress_gradient(nx, ny, nz, E, u, p: float, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """d sigma_PN / d u, assembled over the nodes (FP64, no boundary conditions),
    by the chain rule through the definitions above:
      d sigma_PN / d s_e   = sigma_PN^(1-p) s_e^(p-1)           (s_e = von Mises of element e)
      d s_e / d sigma_e     = 3/2 dev(sigma_e) / s_e
      d s_e / d eps_e       = C : (d s_e / d sigma_e)          (C self-adjoint)
      d eps_e / d u_(a,c)   = sym(e_c (x) grad N_a) at the centroid.
    Elements with s_e = 0 contribute nothing."""
    eps = centroid_strain(nx, ny, nz, u, h)
    sig = centroid_stress(eps, E, nu)
    vm = von_mises(sig)
    PN = pnorm(vm, p)
    dev = sig - np.trace(sig, axis1=1, axis2=2)[:, None, None] / 3.0 * np.eye(3)[None]
    coef = np.zeros_like(vm)
    nzv = vm > 0
    coef[nzv] = PN ** (1.0 - p) * vm[nzv] ** (p - 1.0) * 1.5 / vm[nzv]
    X = coef[:, None, None] * dev                                   # d sigma_PN / d sigma_e
    lam, mu = fe.lame(1.0, nu)
    D = np.asarray(E, dtype=np.float64)[:, None, None] * (2.0 * mu * X + lam * np.trace(X, axis1=1, axis2=2)[:, None, None] * np.eye(3)[None])
    grad = fe.shape_gradients(np.array([0.5, 0.5, 0.5]), h)          # (8, 3)
    ge = np.einsum("ecj,aj->eac", D, grad)                          # (N_e, 8, 3)
    g = np.zeros(u.size, dtype=np.float64).reshape(-1, 3)
    np.add.at(g, fe.element_nodes(nx, ny, nz), ge)
    return g.reshape(-1)


def stress_topological_sensitivity(nx, ny, nz, E, u, lam_adj, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """T_sigma of Eq. 3.3 (reading above) at each element centroid."""
    eps = centroid_strain(nx, ny, nz, u, h)
    sig = centroid_stress(eps, E, nu)
    eps_l = centroid_strain(nx, ny, nz, lam_adj, h)
    return 4.0 / (1.0 + nu) * np.einsum("eij,eij->e", sig, eps_l) - (1.0 - 3.0 * nu) / (1.0 - nu * nu) * \
        np.trace(sig, axis1=1, axis2=2) * np.trace(eps_l, axis1=1, axis2=2)
