"""Exact rational element stiffness, used only to pin ``fe.ke_hex8``.

Computes K^e of the trilinear hex on the unit cube (h = 1) by exact polynomial
integration in rational arithmetic, from the elasticity tensor in index form

    K[(a,c),(b,d)] = sum_{i,j} C_{c i d j} * Int dN_a/dx_i dN_b/dx_j,
    C_{c i d j} = lam d_ci d_dj + mu (d_cd d_ij + d_cj d_id),

with each integral factorised into three 1-D integrals of the linear shape
functions phi_0 = 1 - t, phi_1 = t.  This route (tensor form, exact
integrals) shares nothing with the quadrature / Voigt B-matrix route of
``fe.ke_hex8`` beyond the element definition itself.
"""
from __future__ import annotations

from fractions import Fraction


def _one_d(s: int, t: int, ds: bool, dt: bool) -> Fraction:
    """Int_0^1 phi_s^(ds) phi_t^(dt) dt for the linear 1-D shape functions."""
    sign = lambda q: Fraction(1) if q == 1 else Fraction(-1)  # noqa: E731
    if ds and dt:
        return sign(s) * sign(t)
    if ds:
        return sign(s) * Fraction(1, 2)
    if dt:
        return sign(t) * Fraction(1, 2)
    return Fraction(1, 3) if s == t else Fraction(1, 6)


def ke_exact(nu: Fraction, E: Fraction = Fraction(1)):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    offs = [(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]

    def grad_int(a, b, i, j):
        val = Fraction(1)
        for axis in range(3):
            val *= _one_d(offs[a][axis], offs[b][axis], axis == i, axis == j)
        return val

    def C(c, i, d, j):
        v = Fraction(0)
        if c == i and d == j:
            v += lam
        if c == d and i == j:
            v += mu
        if c == j and i == d:
            v += mu
        return v

    K = [[Fraction(0)] * 24 for _ in range(24)]
    for a in range(8):
        for b in range(8):
            G = [[grad_int(a, b, i, j) for j in range(3)] for i in range(3)]
            for c in range(3):
                for d in range(3):
                    s = Fraction(0)
                    for i in range(3):
                        for j in range(3):
                            cc = C(c, i, d, j)
                            if cc:
                                s += cc * G[i][j]
                    K[3 * a + c][3 * b + d] = s
    return K
