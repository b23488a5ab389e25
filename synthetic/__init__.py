"""Seeded synthetic workloads for the voxel hex8 cantilever problems.

This module builds INPUTS only: mesh sizes, per-element Young's moduli from a
seeded void pattern, load vectors and Dirichlet masks.  It holds none of the
method's arithmetic (no stiffness, no solve, no sensitivity) and is the only
module shared by the CPU oracle and the CUDA path.

Index conventions (the paper is silent on them; these are the ones the whole
project uses):
  * element (i, j, k), 0 <= i < nx ...      e = i + nx * (j + ny * k)
  * node    (i, j, k), 0 <= i <= nx ...     n = i + (nx+1) * (j + (ny+1) * k)
  * degree of freedom                        d = 3 * n + c,  c in {x, y, z}
  * element edge h = 1, so element (i, j, k) spans [i, i+1] x [j, j+1] x [k, k+1]

Random numbers come from numpy ``Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

__all__ = [
    "Workload",
    "node_count",
    "element_count",
    "clamp_face_x0",
    "edge_load",
    "axial_face_load",
    "sphere_voids",
    "void_fraction_spheres",
    "top_point_loads",
    "cantilever_24x12x12_solid",
    "cantilever_128x64x64_voids",
    "multiload_96x48x48_voids",
    "serving_stream",
    "levelset_384x192x192",
    "small_cantilever",
]


def node_count(nx: int, ny: int, nz: int) -> int:
    return (nx + 1) * (ny + 1) * (nz + 1)


def element_count(nx: int, ny: int, nz: int) -> int:
    return nx * ny * nz


def clamp_face_x0(nx: int, ny: int, nz: int) -> np.ndarray:
    """uint8 mask over DOFs, 1 on every DOF of the nodes with i == 0."""
    mask = np.zeros((nz + 1, ny + 1, nx + 1, 3), dtype=np.uint8)
    mask[:, :, 0, :] = 1
    return mask.reshape(-1)


def edge_load(nx: int, ny: int, nz: int, total: float = -1.0) -> np.ndarray:
    """Load ``total`` in z spread evenly over the nodes of the bottom edge of
    the face x = nx (nodes i = nx, k = 0, j = 0..ny)."""
    f = np.zeros((nz + 1, ny + 1, nx + 1, 3), dtype=np.float64)
    f[0, :, nx, 2] = total / (ny + 1)
    return f.reshape(-1)


def axial_face_load(nx: int, ny: int, nz: int, total: float = -1.0) -> np.ndarray:
    """Load ``total`` in x spread evenly over the nodes of the face x = nx (a
    compressive end load for a column clamped at x = 0 when negative)."""
    f = np.zeros((nz + 1, ny + 1, nx + 1, 3), dtype=np.float64)
    f[:, :, nx, 0] = total / ((ny + 1) * (nz + 1))
    return f.reshape(-1)


def _centroids(nx: int, ny: int, nz: int):
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return (i + 0.5).reshape(-1), (j + 0.5).reshape(-1), (k + 0.5).reshape(-1)


def _apply_spheres(nx, ny, nz, centres, radii):
    cx, cy, cz = _centroids(nx, ny, nz)
    void = np.zeros(cx.shape, dtype=bool)
    for (x0, y0, z0), r in zip(centres, radii):
        void |= (cx - x0) ** 2 + (cy - y0) ** 2 + (cz - z0) ** 2 < r * r
    return void


def sphere_voids(nx: int, ny: int, nz: int, n_spheres: int = 40, rmin: float = 4.0,
                 rmax: float = 10.0, seed: int = 1, e_void: float = 1e-3,
                 e_solid: float = 1.0) -> np.ndarray:
    """Per-element moduli: ``n_spheres`` spheres with centres uniform in the box
    [0,nx]x[0,ny]x[0,nz] and radii uniform in [rmin, rmax]; an element whose
    centroid lies inside any sphere gets ``e_void``, every other ``e_solid``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform([0, 0, 0], [nx, ny, nz], size=(n_spheres, 3))
    radii = rng.uniform(rmin, rmax, size=n_spheres)
    void = _apply_spheres(nx, ny, nz, centres, radii)
    return np.where(void, e_void, e_solid).astype(np.float64)


def void_fraction_spheres(nx: int, ny: int, nz: int, target: float, rng: np.random.Generator,
                          rmin: float = 4.0, rmax: float = 10.0, e_void: float = 1e-3,
                          e_solid: float = 1.0, max_spheres: int = 10000) -> np.ndarray:
    """Add radius-U[rmin,rmax] spheres at uniform centres until the void volume
    fraction reaches ``target`` (each sphere marks the elements whose centroid
    lies inside it; only its bounding box is visited)."""
    void = np.zeros((nz, ny, nx), dtype=bool)
    n = void.size
    count = 0
    for _ in range(max_spheres):
        if count >= target * n:
            break
        x0, y0, z0 = rng.uniform([0, 0, 0], [nx, ny, nz])
        r = rng.uniform(rmin, rmax)
        i0, i1 = max(int(np.floor(x0 - r)), 0), min(int(np.ceil(x0 + r)) + 1, nx)
        j0, j1 = max(int(np.floor(y0 - r)), 0), min(int(np.ceil(y0 + r)) + 1, ny)
        k0, k1 = max(int(np.floor(z0 - r)), 0), min(int(np.ceil(z0 + r)) + 1, nz)
        if i0 >= i1 or j0 >= j1 or k0 >= k1:
            continue
        cz, cy, cx = np.meshgrid(np.arange(k0, k1) + 0.5, np.arange(j0, j1) + 0.5, np.arange(i0, i1) + 0.5,
                                 indexing="ij")
        inside = (cx - x0) ** 2 + (cy - y0) ** 2 + (cz - z0) ** 2 < r * r
        box = void[k0:k1, j0:j1, i0:i1]
        count += int(np.count_nonzero(inside & ~box))
        box |= inside
    return np.where(void.reshape(-1), e_void, e_solid).astype(np.float64)


def top_point_loads(nx: int, ny: int, nz: int, n_rhs: int, seed: int) -> np.ndarray:
    """``n_rhs`` load cases, each a unit force at a uniform-random node of the top
    face (k = nz, i >= 1) with a direction uniform on the unit sphere
    (normalised Gaussian).  Returns an array of shape (n_rhs, ndof)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ndof = 3 * node_count(nx, ny, nz)
    f = np.zeros((n_rhs, ndof), dtype=np.float64)
    for r in range(n_rhs):
        i = int(rng.integers(1, nx + 1))
        j = int(rng.integers(0, ny + 1))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        n = i + (nx + 1) * (j + (ny + 1) * nz)
        f[r, 3 * n:3 * n + 3] = d
    return f


@dataclasses.dataclass
class Workload:
    """One synthetic solve problem."""
    name: str
    nx: int
    ny: int
    nz: int
    E: np.ndarray            # (nx*ny*nz,) float64
    f: np.ndarray            # (n_rhs, ndof) float64
    fixed: np.ndarray        # (ndof,) uint8
    nu: float = 0.3
    group: int = 8           # deflation agglomeration: elements per group per axis
    tol: float = 1e-6        # relative residual target
    e_void: float = 1e-3

    @property
    def n_rhs(self) -> int:
        return self.f.shape[0]

    @property
    def ndof(self) -> int:
        return 3 * node_count(self.nx, self.ny, self.nz)


def small_cantilever(nx: int, ny: int, nz: int, seed: Optional[int] = None, n_spheres: int = 0,
                     rmin: float = 1.0, rmax: float = 2.5, group: int = 2, n_rhs: int = 1,
                     e_void: float = 1e-3) -> Workload:
    """A small clamped cantilever for parity tests: edge load in the first load
    case, optional seeded voids, optional extra random point-load cases."""
    if seed is not None and n_spheres > 0:
        E = sphere_voids(nx, ny, nz, n_spheres, rmin, rmax, seed, e_void)
    else:
        E = np.ones(element_count(nx, ny, nz))
    f = [edge_load(nx, ny, nz)]
    if n_rhs > 1:
        f.extend(top_point_loads(nx, ny, nz, n_rhs - 1, 1000 + (seed or 0)))
    return Workload(f"cantilever_{nx}x{ny}x{nz}", nx, ny, nz, E, np.stack(f),
                    clamp_face_x0(nx, ny, nz), group=group, e_void=e_void)


def cantilever_24x12x12_solid() -> Workload:
    """24x12x12 all-solid cantilever, face x=0 clamped, load -1 in z on the
    bottom edge of face x=24, 4x4x4-element groups, tolerance 1e-10."""
    nx, ny, nz = 24, 12, 12
    return Workload("cantilever_24x12x12_solid", nx, ny, nz, np.ones(nx * ny * nz),
                    edge_load(nx, ny, nz)[None, :], clamp_face_x0(nx, ny, nz), group=4, tol=1e-10)


def cantilever_128x64x64_voids(seed: int = 1, group: int = 16) -> Workload:
    """128x64x64 cantilever with 40 seeded spherical voids (radii U[4,10],
    void E = 1e-3), same clamp and edge load, tolerance 1e-6."""
    nx, ny, nz = 128, 64, 64
    E = sphere_voids(nx, ny, nz, 40, 4.0, 10.0, seed, 1e-3)
    return Workload("cantilever_128x64x64_voids", nx, ny, nz, E, edge_load(nx, ny, nz)[None, :],
                    clamp_face_x0(nx, ny, nz), group=group, tol=1e-6)


def multiload_96x48x48_voids(seed: int = 2, n_rhs: int = 8, group: int = 16) -> Workload:
    """96x48x48 cantilever with seeded voids and ``n_rhs`` unit point loads at
    random top-face nodes with random directions, solved as one batch."""
    nx, ny, nz = 96, 48, 48
    E = sphere_voids(nx, ny, nz, 40, 4.0, 10.0, seed, 1e-3)
    f = top_point_loads(nx, ny, nz, n_rhs, seed)
    return Workload("multiload_96x48x48_voids", nx, ny, nz, E, f, clamp_face_x0(nx, ny, nz),
                    group=group, tol=1e-6)


def levelset_384x192x192(group: int = 8) -> Workload:
    """384x192x192 all-solid cantilever (the start of the 20-iteration
    volume-minimisation run), edge load, tolerance 1e-6."""
    nx, ny, nz = 384, 192, 192
    return Workload("levelset_384x192x192", nx, ny, nz, np.ones(nx * ny * nz),
                    edge_load(nx, ny, nz)[None, :], clamp_face_x0(nx, ny, nz), group=group, tol=1e-6)


def serving_stream(n_requests: int = 256, seed: int = 3, sizes=(32, 48, 64, 96, 128, 160),
                   rate_per_s: float = 50.0) -> List[dict]:
    """A stream of solve requests: mesh nx x nx/2 x nx/2 with nx uniform in
    ``sizes``, a void fraction uniform in [0.1, 0.4] reached with seeded
    spheres, cantilever clamp and edge load, Poisson arrival times with the
    given rate (rate <= 0 gives a burst at t = 0).  Moduli are generated lazily
    from the per-request seed to keep the stream small."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for r in range(n_requests):
        nx = int(rng.choice(sizes))
        frac = float(rng.uniform(0.1, 0.4))
        if rate_per_s > 0:
            t += float(rng.exponential(1.0 / rate_per_s))
        out.append({"id": r, "nx": nx, "ny": nx // 2, "nz": nx // 2, "void_fraction": frac,
                    "seed": int(rng.integers(0, 2**31 - 1)), "arrival_s": t})
    return out


def serving_request_inputs(req: dict):
    """Moduli, load and mask of one serving request (see ``serving_stream``)."""
    nx, ny, nz = req["nx"], req["ny"], req["nz"]
    rng = np.random.Generator(np.random.PCG64(req["seed"]))
    E = void_fraction_spheres(nx, ny, nz, req["void_fraction"], rng)
    return E, edge_load(nx, ny, nz)[None, :], clamp_face_x0(nx, ny, nz)
