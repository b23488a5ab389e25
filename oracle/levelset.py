"""Topological level-set extraction and augmented-Lagrangian updates
(Secs. 3.2-3.4, Eqs. 3.6, 3.11, 3.12, 3.17, 3.18; algorithm of Sec. 3.8).

Readings of the paper:
  * Eq. 3.6 keeps the points where the level-set exceeds a cut tau; the cut is
    chosen so that the target volume fraction v is met: the k = round(v N_e)
    elements with the largest level-set value are kept, ties broken toward the
    lower element index (a stable sort), tau is the k-th largest value.
  * Kept elements get modulus 1, the others the weak-void modulus.
  * Before combining, each constraint field is divided by its largest
    magnitude (the paper combines fields of different units, Eq. 3.17).
  * Eq. 3.18 is printed without parentheses; read as
    T_Lbar_i = (mu_i + gamma_i g_i) T_g_i when mu_i + gamma_i g_i > 0, else 0.
  * Eq. 3.12 is ambiguous in sign; read as: keep gamma when
    max(g^{k+1}, 0) <= varsigma * max(g^k, 0), else gamma <- max(eta gamma, k^2),
    with varsigma = 0.25, eta = 10 (the values of Sec. 3.3).
  * The normalised constraint is g = J / J_all - 1 (J_all = alpha J0).

The combination is done in float32 with one rounding per operation in a fixed
order (divide by the max magnitude, multiply by the weight, add), so that the
integer decision (which elements are kept) can be compared bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

MU0 = 100.0       # Sec. 3.8 step 1
GAMMA0 = 10.0     # Sec. 3.8 step 1
VARSIGMA = 0.25   # Sec. 3.3, after Eq. 3.12
ETA = 10.0        # Sec. 3.3, after Eq. 3.12


def constraint_value(J: float, J_all: float) -> float:
    """Normalised compliance constraint g = J / J_all - 1 (<= 0 when met)."""
    return J / J_all - 1.0


def multiplier_update(mu: float, gamma: float, g: float) -> float:
    """Eq. 3.11: mu <- max(mu + gamma g, 0)."""
    return max(mu + gamma * g, 0.0)


def penalty_update(gamma: float, g_new: float, g_old: float, k: int) -> float:
    """Eq. 3.12 (reading above)."""
    if max(g_new, 0.0) <= VARSIGMA * max(g_old, 0.0):
        return gamma
    return max(ETA * gamma, float(k * k))


def al_weight(mu: float, gamma: float, g: float) -> float:
    """Eq. 3.18 weight of a constraint field: mu + gamma g if positive, else 0."""
    w = mu + gamma * g
    return w if w > 0.0 else 0.0


def combine(fields, weights) -> np.ndarray:
    """T_L = sum_i w_i * (T_i / max|T_i|) (Eq. 3.17 with normalised fields),
    float32, fixed operation order."""
    out = None
    for T, w in zip(fields, weights):
        T = np.asarray(T, dtype=np.float32)
        m = np.float32(np.max(np.abs(T))) if T.size else np.float32(0)
        scaled = (T / m) if m > 0 else np.zeros_like(T)
        term = (np.float32(w) * scaled.astype(np.float32)).astype(np.float32)
        out = term if out is None else (out + term).astype(np.float32)
    return out


def keep_count(volume_fraction: float, n: int) -> int:
    """k = round(v N_e), clamped to [0, N_e] (round half up)."""
    return int(min(max(math.floor(volume_fraction * n + 0.5), 0), n))


def select_top(values: np.ndarray, k: int):
    """Eq. 3.6 at the cut that keeps k elements: a stable descending sort keeps
    the k largest values, equal values in ascending index order.  Returns
    (kept mask uint8, tau) with tau the k-th largest value (nan when k == 0)."""
    v = np.asarray(values)
    order = np.argsort(-v.astype(np.float64), kind="stable")
    kept = np.zeros(v.size, dtype=np.uint8)
    kept[order[:k]] = 1
    tau = float(v[order[k - 1]]) if k > 0 else float("nan")
    return kept, tau


def casting_scan(T: np.ndarray, nx: int, ny: int, nz: int, axis: int, parting: int) -> np.ndarray:
    """Casting constraint on the level-set field (Sec. 3.7), float32.

    Reading: along every line of elements parallel to `axis` (0 = x, 1 = y,
    2 = z), the elements with index >= `parting` form one half of the cast
    part and those below it the other; each half is drawn away from the
    parting plane.  On each half the field is replaced, from the far face
    toward the parting plane, by
        T'(k) = max(T(k), nextafter(T'(k_far_neighbour), +inf)),
    i.e. a running maximum raised by one float32 step per element, so that T'
    strictly increases toward the parting plane wherever it was propagated.
    The kept set of any cut then covers, on every line and half, a run of
    elements starting at the parting plane: no undercut for the draw.
    Element order e = i + nx (j + ny k); T has nx*ny*nz values."""
    a = np.asarray(T, dtype=np.float32).reshape(nz, ny, nx)
    ax = {0: 2, 1: 1, 2: 0}[axis]           # numpy axis of the element index along `axis`
    a = np.moveaxis(a, ax, 0).copy()         # (n_axis, ...)
    n = a.shape[0]
    up = np.float32(np.inf)
    for k in range(n - 2, parting - 1, -1):  # upper half: from the far face k = n-1 down to `parting`
        a[k] = np.maximum(a[k], np.nextafter(a[k + 1], up))
    for k in range(1, min(parting, n)):      # lower half: from k = 0 up to parting-1
        a[k] = np.maximum(a[k], np.nextafter(a[k - 1], up))
    return np.moveaxis(a, 0, ax).reshape(-1).astype(np.float32)


def apply_topology(kept: np.ndarray, e_void: float) -> np.ndarray:
    return np.where(np.asarray(kept) != 0, 1.0, e_void)
