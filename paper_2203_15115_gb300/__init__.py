"""Python binding of the assembly-free deflated FE hot path (arXiv 2203.15115).

Argument marshalling only: every step of the path runs in the CUDA kernels of
``lib/libafdcg.so`` behind the C ABI of ``include/afd.h``; the functions here
carry the same names.  Host arrays are numpy arrays; device arrays are torch
CUDA tensors (PyTorch supplies device memory and the current stream).  There
is no CPU fallback: importing the binding without the built library raises.
"""
from __future__ import annotations

import ctypes
import time
import os
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libafdcg.so")

AFD_OK = 0
AFD_ERR_INVALID_ARG = -1
AFD_ERR_OOM = -2
AFD_ERR_NOT_CONVERGED = -3
AFD_ERR_COARSE_SINGULAR = -4
AFD_ERR_NAN = -5
AFD_ERR_CUDA = -6
AFD_ERR_STATE = -7
AFD_FP64 = 0
AFD_MIXED = 1
AFD_F32 = 0
AFD_F64 = 1
AFD_F64_DF = 2   # double data, double-float arithmetic
AFD_SENS_STRAIN_ENERGY = 0
AFD_SENS_TJ = 1
AFD_SENS_VON_MISES = 2

# every entry point of include/afd.h
EXPORTS = [
    "afd_default_options", "afd_create_mesh", "afd_set_element_moduli", "afd_set_loads_bcs", "afd_solve",
    "afd_compliance", "afd_sensitivity", "afd_pnorm_stress", "afd_levelset_update", "afd_apply_stiffness",
    "afd_deflation_wt", "afd_deflation_w", "afd_coarse_size", "afd_coarse_matrix", "afd_coarse_inverse",
    "afd_select_topk",
    "afd_ndof", "afd_nelem", "afd_destroy", "afd_last_error", "afd_al_init", "afd_al_update", "afd_al_weight",
    "afd_time_stiffness", "afd_kernel_launches", "afd_select_topk_noalloc", "afd_stencil_depth",
    "afd_stencil_warps", "afd_solver_phase_times", "afd_time_dpcg_kernels", "afd_set_stencil_shape",
    "afd_stencil_async",
    "afd_mesh_bytes", "afd_server_create", "afd_server_submit", "afd_server_wait", "afd_server_destroy",
    "afd_server_submit_session", "afd_server_end_session", "afd_server_resident", "afd_levelset_update_cast",
    "afd_casting_scan", "afd_stress_sensitivity", "afd_levelset_update_fields", "afd_modal",
    "afd_eigen_sensitivity", "afd_buckling", "afd_buckling_sensitivity", "afd_apply_search_direction",
    "afd_topology_run", "afd_constrained_topology", "afd_volume_minimisation",
]


class afd_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("group", ctypes.c_int), ("nu", ctypes.c_double),
                ("h", ctypes.c_double), ("e_void", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("max_refine", ctypes.c_int), ("inner_tol", ctypes.c_double), ("check_every", ctypes.c_int),
                ("autotune", ctypes.c_int), ("persistent", ctypes.c_int), ("stencil_warps", ctypes.c_int),
                ("stencil_planes", ctypes.c_int), ("pdl", ctypes.c_int), ("inner_aim", ctypes.c_double),
                ("coarse_fp64", ctypes.c_int),
                ("residual_fp64", ctypes.c_int)]


class afd_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refine_steps", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("ms", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class afd_server_config(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("budget_bytes", ctypes.c_double), ("opt", afd_options)]


class afd_al_state(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_double), ("gamma", ctypes.c_double), ("g", ctypes.c_double), ("k", ctypes.c_int)]


class AFDError(RuntimeError):
    def __init__(self, code: int, msg: str, stats=None):
        super().__init__(f"afd error {code}: {msg}")
        self.code = code
        self.stats = stats


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2203_15115_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        sig = {
            "afd_default_options": (None, [ctypes.POINTER(afd_options)]),
            "afd_create_mesh": (i, [i, i, i, ctypes.POINTER(afd_options), vp, ctypes.POINTER(vp)]),
            "afd_set_element_moduli": (i, [vp, vp, i]),
            "afd_set_loads_bcs": (i, [vp, i, vp, i, vp, i]),
            "afd_solve": (i, [vp, d, i, ctypes.POINTER(afd_stats), vp, i]),
            "afd_compliance": (i, [vp, ctypes.POINTER(d)]),
            "afd_sensitivity": (i, [vp, i, vp, i]),
            "afd_pnorm_stress": (i, [vp, d, ctypes.POINTER(d)]),
            "afd_levelset_update": (i, [vp, i, ctypes.POINTER(d), d, ctypes.POINTER(d), vp]),
            "afd_apply_stiffness": (i, [vp, i, i, vp, vp]),
            "afd_deflation_wt": (i, [vp, i, vp, vp]),
            "afd_deflation_w": (i, [vp, i, vp, vp]),
            "afd_coarse_size": (i, [vp]),
            "afd_coarse_inverse": (i, [vp, vp]),
            "afd_coarse_matrix": (i, [vp, vp]),
            "afd_select_topk": (i, [vp, i64, i64, vp, ctypes.POINTER(ctypes.c_float), vp]),
            "afd_ndof": (i64, [vp]),
            "afd_nelem": (i64, [vp]),
            "afd_destroy": (None, [vp]),
            "afd_last_error": (ctypes.c_char_p, []),
            "afd_al_init": (None, [ctypes.POINTER(afd_al_state)]),
            "afd_al_update": (None, [ctypes.POINTER(afd_al_state), d]),
            "afd_al_weight": (d, [ctypes.POINTER(afd_al_state)]),
            "afd_time_stiffness": (i, [vp, i, i, vp, vp, i, ctypes.POINTER(d)]),
            "afd_kernel_launches": (i64, [vp]),
            "afd_select_topk_noalloc": (i, [vp, i64, i64, vp, ctypes.POINTER(ctypes.c_float), vp]),
            "afd_stencil_depth": (i, [vp]),
            "afd_stencil_warps": (i, [vp]),
            "afd_set_stencil_shape": (i, [vp, i, i, i]),
            "afd_stencil_async": (i, [vp]),
            "afd_solver_phase_times": (i, [vp, ctypes.POINTER(ctypes.c_double), i]),
            "afd_time_dpcg_kernels": (i, [vp, i, i, i, ctypes.POINTER(ctypes.c_double)]),
            "afd_mesh_bytes": (ctypes.c_size_t, [i, i, i, i, ctypes.POINTER(afd_options)]),
            "afd_server_create": (i, [ctypes.POINTER(afd_server_config), ctypes.POINTER(vp)]),
            "afd_server_submit": (i, [vp, i, i, i, vp, vp, vp, d, ctypes.POINTER(i64)]),
            "afd_server_wait": (i, [vp, i64, ctypes.POINTER(afd_stats), ctypes.POINTER(d), ctypes.POINTER(d), vp]),
            "afd_server_destroy": (None, [vp]),
            "afd_server_submit_session": (i, [vp, i64, i, i, i, vp, vp, vp, d, ctypes.POINTER(i64)]),
            "afd_server_end_session": (i, [vp, i64]),
            "afd_server_resident": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(d)]),
            "afd_levelset_update_cast": (i, [vp, i, ctypes.POINTER(d), d, i, i, ctypes.POINTER(d), vp]),
            "afd_casting_scan": (i, [vp, i, i, i, i, i, vp]),
            "afd_stress_sensitivity": (i, [vp, d, d, vp, i, ctypes.POINTER(afd_stats), vp, i]),
            "afd_modal": (i, [vp, i, d, d, i, ctypes.POINTER(d), vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
            "afd_eigen_sensitivity": (i, [vp, vp, i]),
            "afd_buckling": (i, [vp, i, d, i, ctypes.POINTER(d), vp, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
            "afd_buckling_sensitivity": (i, [vp, vp, i]),
            "afd_levelset_update_fields": (i, [vp, vp, i, i, ctypes.POINTER(d), d, i, i, ctypes.POINTER(d), vp]),
            "afd_apply_search_direction": (i, [vp, i, vp, vp, vp, ctypes.POINTER(d), vp, vp, ctypes.POINTER(d)]),
            "afd_topology_run": (i, [vp, vp, vp, vp, i, vp]),
            "afd_constrained_topology": (i, [vp, vp, vp, i, vp, vp, vp]),
            "afd_volume_minimisation": (i, [vp, i, d, d, d, i, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def afd_last_error() -> str:
    return lib().afd_last_error().decode()


def _check(rc: int, stats=None):
    if rc != AFD_OK:
        raise AFDError(rc, afd_last_error(), stats)


def _arr(x, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if hasattr(x, "data_ptr"):  # torch tensor
        if x.dtype.itemsize != np.dtype(dtype).itemsize:
            raise TypeError(f"expected a tensor of {np.dtype(dtype)}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), 0, a


def current_stream():
    """cudaStream_t of torch's current stream (None when torch/CUDA is absent)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return None


def afd_default_options() -> afd_options:
    o = afd_options()
    lib().afd_default_options(ctypes.byref(o))
    return o


def afd_create_mesh(nx: int, ny: int, nz: int, options: Optional[afd_options] = None, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    s = stream if stream is not None else current_stream()
    _check(lib().afd_create_mesh(nx, ny, nz, ctypes.byref(options) if options is not None else None, s,
                                 ctypes.byref(h)))
    return h


def afd_destroy(mesh) -> None:
    if mesh:
        lib().afd_destroy(mesh)


def afd_ndof(mesh) -> int:
    return int(lib().afd_ndof(mesh))


def afd_nelem(mesh) -> int:
    return int(lib().afd_nelem(mesh))


def afd_set_element_moduli(mesh, E) -> None:
    p, dev, _k = _arr(E, np.float64)
    _check(lib().afd_set_element_moduli(mesh, p, dev))


def afd_set_loads_bcs(mesh, f, fixed) -> None:
    n_rhs = int(f.shape[0]) if len(f.shape) == 2 else 1
    pf, df, _k1 = _arr(f, np.float64)
    pm, dm, _k2 = _arr(fixed, np.uint8)
    _check(lib().afd_set_loads_bcs(mesh, n_rhs, pf, df, pm, dm))


def afd_solve(mesh, rel_tol: float, n_rhs: int, warm_start: bool = False, u_out=None, check: bool = True):
    """Returns the per-RHS stats as dicts; raises AFDError unless check=False."""
    st = (afd_stats * n_rhs)()
    if u_out is not None:
        pu, du, _k = _arr(u_out, np.float64)
    else:
        pu, du = None, 0
    rc = lib().afd_solve(mesh, rel_tol, int(warm_start), st, pu, du)
    stats = [s.as_dict() for s in st]
    if check:
        _check(rc, stats)
    return stats if check else (rc, stats)


def afd_compliance(mesh, n_rhs: int) -> np.ndarray:
    J = (ctypes.c_double * n_rhs)()
    _check(lib().afd_compliance(mesh, J))
    return np.array(J[:])


def afd_sensitivity(mesh, kind: int, out) -> None:
    p, dev, _k = _arr(out, np.float32)
    _check(lib().afd_sensitivity(mesh, kind, p, dev))


def afd_pnorm_stress(mesh, p: float, n_rhs: int) -> np.ndarray:
    out = (ctypes.c_double * n_rhs)()
    _check(lib().afd_pnorm_stress(mesh, p, out))
    return np.array(out[:])


def afd_levelset_update(mesh, kind: int, weights, volume_fraction: float, kept_out: Optional[np.ndarray] = None,
                        casting=None) -> float:
    """casting = (axis, parting) applies afd_levelset_update_cast."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    tau = ctypes.c_double()
    pk = None
    if kept_out is not None:
        assert kept_out.dtype == np.uint8 and kept_out.flags.c_contiguous
        pk = ctypes.c_void_p(kept_out.ctypes.data)
    pw = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if casting is None:
        _check(lib().afd_levelset_update(mesh, kind, pw, volume_fraction, ctypes.byref(tau), pk))
    else:
        axis, parting = casting
        _check(lib().afd_levelset_update_cast(mesh, kind, pw, volume_fraction, int(axis), int(parting),
                                              ctypes.byref(tau), pk))
    return tau.value


def afd_stress_sensitivity(mesh, n_rhs: int, p: float, rel_tol: float, out, lambda_out=None):
    """T_sigma of Eq. 3.3 into out (n_rhs x nelem float32); returns the adjoint
    solves' stats; lambda_out (n_rhs x ndof float64) receives the adjoint."""
    po, od, _k1 = _arr(out, np.float32)
    st = (afd_stats * n_rhs)()
    pl, ld = (None, 0)
    if lambda_out is not None:
        pl, ld, _k2 = _arr(lambda_out, np.float64)
    _check(lib().afd_stress_sensitivity(mesh, p, rel_tol, po, od, st, pl, ld), [s.as_dict() for s in st])
    return [s.as_dict() for s in st]


def afd_modal(mesh, n_modes: int, rho: float = 1.0, tol: float = 1e-6, max_iter: int = 100, modes_out=None,
              check: bool = True):
    """The n_modes smallest eigenpairs of K phi = lambda M phi (lumped mass,
    rho_e = rho E_e).  Returns (lambda (n_modes,), info dict); modes_out
    (n_modes x ndof float64, numpy or torch) receives the M-orthonormal modes.
    With check=False a stop at max_iter returns normally (info["rc"])."""
    lam = (ctypes.c_double * n_modes)()
    steps, solves = ctypes.c_int(0), ctypes.c_int(0)
    pm, md = (None, 0)
    if modes_out is not None:
        pm, md, _k = _arr(modes_out, np.float64)
    rc = lib().afd_modal(mesh, n_modes, rho, tol, max_iter, lam, pm, md, ctypes.byref(steps), ctypes.byref(solves))
    info = {"rc": rc, "steps": steps.value, "solve_iters": solves.value}
    if check or rc not in (AFD_OK, AFD_ERR_NOT_CONVERGED):
        _check(rc, info)
    return np.array(lam[:], dtype=np.float64), info


def afd_eigen_sensitivity(mesh, out) -> None:
    """T_lambda of Eq. 3.4 for the modes of the last afd_modal into out
    (n_modes x nelem float32, numpy or torch)."""
    po, od, _k = _arr(out, np.float32)
    _check(lib().afd_eigen_sensitivity(mesh, po, od))


def afd_buckling(mesh, n_modes: int, tol: float = 1e-6, max_iter: int = 100, modes_out=None, check: bool = True):
    """The n_modes smallest positive buckling load factors of load case 0's
    static state (afd_solve first).  Returns (lambda (n_modes,), info dict);
    modes_out (n_modes x ndof float64) receives the K-orthonormal modes."""
    lam = (ctypes.c_double * n_modes)()
    steps, solves = ctypes.c_int(0), ctypes.c_int(0)
    pm, md = (None, 0)
    if modes_out is not None:
        pm, md, _k = _arr(modes_out, np.float64)
    rc = lib().afd_buckling(mesh, n_modes, tol, max_iter, lam, pm, md, ctypes.byref(steps), ctypes.byref(solves))
    info = {"rc": rc, "steps": steps.value, "solve_iters": solves.value}
    if check or rc not in (AFD_OK, AFD_ERR_NOT_CONVERGED):
        _check(rc, info)
    return np.array(lam[:], dtype=np.float64), info


def afd_buckling_sensitivity(mesh, out) -> None:
    """Eq. 3.5 for the modes of the last afd_buckling into out (n_modes x
    nelem float32, numpy or torch)."""
    po, od, _k = _arr(out, np.float32)
    _check(lib().afd_buckling_sensitivity(mesh, po, od))


def afd_levelset_update_fields(mesh, fields, weights, volume_fraction: float, casting=None, kept_out=None) -> float:
    """Level-set cut of sum_i weights[i] * fields[i] / max|fields[i]| (fields: (nf, nelem)
    float32, numpy or torch); casting = (axis, parting) or None."""
    nf = int(fields.shape[0])
    pf, on_dev, _k = _arr(fields, np.float32)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    assert w.size == nf
    tau = ctypes.c_double()
    pk = None
    if kept_out is not None:
        assert kept_out.dtype == np.uint8 and kept_out.flags.c_contiguous
        pk = ctypes.c_void_p(kept_out.ctypes.data)
    axis, parting = casting if casting is not None else (-1, 0)
    _check(lib().afd_levelset_update_fields(mesh, pf, on_dev, nf, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            volume_fraction, int(axis), int(parting), ctypes.byref(tau), pk))
    return tau.value


def afd_casting_scan(keys, nx: int, ny: int, nz: int, axis: int, parting: int, stream=None) -> None:
    """In-place casting scan of a device float32 tensor (torch) of nx*ny*nz keys."""
    pk, on_dev, _k = _arr(keys, np.float32)
    if not on_dev:
        raise ValueError("afd_casting_scan takes a device tensor")
    _check(lib().afd_casting_scan(pk, nx, ny, nz, axis, parting, stream if stream is not None else current_stream()))


def afd_apply_stiffness(mesh, arith: int, n_rhs: int, u, y) -> None:
    dt = np.float32 if arith == AFD_F32 else np.float64
    pu, _, _k1 = _arr(u, dt)
    py, _, _k2 = _arr(y, dt)
    _check(lib().afd_apply_stiffness(mesh, arith, n_rhs, pu, py))


def afd_apply_search_direction(mesh, n_rhs: int, z, p_old, mu, beta, p_out, q_out) -> np.ndarray:
    """p = z + W mu + beta p_old (free DOFs) and q = K p by the solver's fused
    FP32 stencil; returns p.q per load case.  Device tensors only."""
    for name, x in (("z", z), ("p_old", p_old), ("mu", mu), ("p_out", p_out), ("q_out", q_out)):
        if not (hasattr(x, "data_ptr") and x.is_cuda):
            raise TypeError(f"{name} must be a CUDA tensor")
    pz, _, _k1 = _arr(z, np.float32)
    pp, _, _k2 = _arr(p_old, np.float32)
    pm, _, _k3 = _arr(mu, np.float64)
    po, _, _k4 = _arr(p_out, np.float32)
    pq, _, _k5 = _arr(q_out, np.float32)
    b = (ctypes.c_double * n_rhs)(*[float(x) for x in beta])
    out = (ctypes.c_double * n_rhs)()
    _check(lib().afd_apply_search_direction(mesh, n_rhs, pz, pp, pm, b, po, pq, out))
    return np.array(out[:])


def afd_deflation_wt(mesh, n_rhs: int, v, out) -> None:
    pv, _, _k1 = _arr(v, np.float64)
    po, _, _k2 = _arr(out, np.float64)
    _check(lib().afd_deflation_wt(mesh, n_rhs, pv, po))


def afd_deflation_w(mesh, n_rhs: int, y, out) -> None:
    py, _, _k1 = _arr(y, np.float64)
    po, _, _k2 = _arr(out, np.float64)
    _check(lib().afd_deflation_w(mesh, n_rhs, py, po))


def afd_coarse_size(mesh) -> int:
    return int(lib().afd_coarse_size(mesh))


def afd_coarse_matrix(mesh) -> np.ndarray:
    nc = afd_coarse_size(mesh)
    out = np.zeros((nc, nc))
    _check(lib().afd_coarse_matrix(mesh, ctypes.c_void_p(out.ctypes.data)))
    return out


def afd_coarse_inverse(mesh) -> np.ndarray:
    """The solver's inverse of W^T K W, as FP64 on the host."""
    nc = afd_coarse_size(mesh)
    out = np.zeros((nc, nc))
    _check(lib().afd_coarse_inverse(mesh, ctypes.c_void_p(out.ctypes.data)))
    return out


def _select_args(keys, kept):
    """Device pointers and the key count of a top-k selection; both arrays must
    be CUDA tensors, kept at least as long as keys."""
    for name, x in (("keys", keys), ("kept", kept)):
        if not (hasattr(x, "data_ptr") and x.is_cuda):
            raise TypeError(f"{name} must be a CUDA tensor")
    if keys.device != kept.device:
        raise ValueError("keys and kept must be on the same device")
    n = int(keys.numel())
    if int(kept.numel()) < n:
        raise ValueError(f"kept holds {kept.numel()} bytes for {n} keys")
    pk, _, _k1 = _arr(keys, np.float32)
    po, _, _k2 = _arr(kept, np.uint8)
    return pk, po, n, (_k1, _k2)


def afd_select_topk(keys, k: int, kept, stream=None) -> float:
    pk, po, n, _keep = _select_args(keys, kept)
    tau = ctypes.c_float()
    s = stream if stream is not None else current_stream()
    _check(lib().afd_select_topk(pk, n, int(k), po, ctypes.byref(tau), s))
    return tau.value


def afd_time_stiffness(mesh, arith: int, n_rhs: int, u, y, launches: int) -> float:
    """Mean device ms per stiffness apply, timed with CUDA events on the mesh's stream."""
    dt = np.float32 if arith == AFD_F32 else np.float64
    pu, _, _k1 = _arr(u, dt)
    py, _, _k2 = _arr(y, dt)
    ms = ctypes.c_double()
    _check(lib().afd_time_stiffness(mesh, arith, n_rhs, pu, py, launches, ctypes.byref(ms)))
    return ms.value


def afd_stencil_depth(mesh) -> int:
    return int(lib().afd_stencil_depth(mesh))


def afd_stencil_warps(mesh) -> int:
    return int(lib().afd_stencil_warps(mesh))


def afd_set_stencil_shape(mesh, warps: int, planes: int, async_staging: int = 0) -> None:
    _check(lib().afd_set_stencil_shape(mesh, warps, planes, async_staging))


def afd_stencil_async(mesh) -> int:
    return int(lib().afd_stencil_async(mesh))


def afd_time_dpcg_kernels(mesh, iters: int = 50, nsplit: int = 0, variant: int = 0) -> dict:
    out = (ctypes.c_double * 5)()
    _check(lib().afd_time_dpcg_kernels(mesh, iters, nsplit, variant, out))
    return {"stencil_us": out[0], "update_us": out[1], "coarse_rhs_us": out[2], "coarse_step_us": out[3],
            "prolong_us": out[4]}


def afd_solver_phase_times(mesh, reset: bool = True) -> dict:
    out = (ctypes.c_double * 10)()
    _check(lib().afd_solver_phase_times(mesh, out, int(reset)))
    names = ["stencil_ms", "update_ms", "coarse_rhs_ms", "coarse_apply_ms", "scalars_ms", "iterations",
             "stencil_wait_ms", "update_wait_ms", "coarse_rhs_wait_ms", "coarse_apply_wait_ms"]
    return {k: out[q] for q, k in enumerate(names)}


def afd_kernel_launches(mesh) -> int:
    return int(lib().afd_kernel_launches(mesh))


def afd_select_topk_noalloc(keys, k: int, kept, stream=None) -> float:
    """afd_select_topk without device allocation (file-scope device scratch,
    at most 16,777,216 keys; see include/afd.h)."""
    pk, po, n, _keep = _select_args(keys, kept)
    tau = ctypes.c_float()
    s = stream if stream is not None else current_stream()
    _check(lib().afd_select_topk_noalloc(pk, n, int(k), po, ctypes.byref(tau), s))
    return tau.value


def afd_mesh_bytes(nx: int, ny: int, nz: int, n_rhs: int = 1, options: Optional[afd_options] = None) -> int:
    return int(lib().afd_mesh_bytes(nx, ny, nz, n_rhs, ctypes.byref(options) if options is not None else None))


class Server:
    """Serving loop (afd_server_*): requests of different mesh sizes admitted
    continuously under a device-memory budget, solved concurrently in
    max_slots slots.  submit() copies the host inputs; wait() returns
    (status, stats, J, latency_ms, u)."""

    def __init__(self, max_slots: int = 4, budget_bytes: float = 60e9, precision: int = AFD_MIXED, **opts):
        cfg = afd_server_config()
        cfg.max_slots, cfg.budget_bytes = max_slots, float(budget_bytes)
        cfg.opt = afd_default_options()
        cfg.opt.precision = precision
        for k, v in opts.items():
            setattr(cfg.opt, k, v)
        self.cfg = cfg
        self.h = ctypes.c_void_p()
        _check(lib().afd_server_create(ctypes.byref(cfg), ctypes.byref(self.h)))
        self.sizes = {}

    def submit(self, nx: int, ny: int, nz: int, E, f, fixed, rel_tol: float, session: int = 0) -> int:
        pE, _, k1 = _arr(E, np.float64)
        pf, _, k2 = _arr(np.asarray(f).reshape(-1), np.float64)
        pm, _, k3 = _arr(fixed, np.uint8)
        rid = ctypes.c_int64()
        _check(lib().afd_server_submit_session(self.h, session, nx, ny, nz, pE, pf, pm, rel_tol, ctypes.byref(rid)))
        self.sizes[rid.value] = 3 * (nx + 1) * (ny + 1) * (nz + 1)
        return rid.value

    def wait(self, rid: int, want_u: bool = True):
        st = afd_stats()
        J = ctypes.c_double()
        lat = ctypes.c_double()
        n = self.sizes.pop(rid)
        u = np.zeros(n) if want_u else None
        rc = lib().afd_server_wait(self.h, rid, ctypes.byref(st), ctypes.byref(J), ctypes.byref(lat),
                                   ctypes.c_void_p(u.ctypes.data) if want_u else None)
        return rc, st.as_dict(), J.value, lat.value, u

    def end_session(self, session: int):
        _check(lib().afd_server_end_session(self.h, session))

    def resident(self):
        n = ctypes.c_int()
        b = ctypes.c_double()
        _check(lib().afd_server_resident(self.h, ctypes.byref(n), ctypes.byref(b)))
        return n.value, b.value

    def close(self):
        if self.h:
            lib().afd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def afd_al_init() -> afd_al_state:
    s = afd_al_state()
    lib().afd_al_init(ctypes.byref(s))
    return s


def afd_al_update(s: afd_al_state, g_new: float) -> None:
    lib().afd_al_update(ctypes.byref(s), g_new)


def afd_al_weight(s: afd_al_state) -> float:
    return float(lib().afd_al_weight(ctypes.byref(s)))


class afd_topology_spec(ctypes.Structure):
    _fields_ = [("bound", ctypes.c_double * 4), ("soft", ctypes.c_int * 4), ("p", ctypes.c_double),
                ("dv0", ctypes.c_double), ("dv_min", ctypes.c_double), ("v_min", ctypes.c_double),
                ("conv", ctypes.c_double), ("max_fea", ctypes.c_int), ("tol", ctypes.c_double),
                ("eig_tol", ctypes.c_double), ("rho", ctypes.c_double), ("casting_axis", ctypes.c_int),
                ("casting_parting", ctypes.c_int)]


class afd_topology_record(ctypes.Structure):
    _fields_ = [("fea", ctypes.c_int), ("v", ctypes.c_double), ("target", ctypes.c_double), ("dv", ctypes.c_double),
                ("value", ctypes.c_double * 4), ("g", ctypes.c_double * 4), ("violated", ctypes.c_int),
                ("iters", ctypes.c_int), ("rel_residual", ctypes.c_double), ("mu", ctypes.c_double * 4),
                ("gamma", ctypes.c_double * 4)]


class afd_topology_result(ctypes.Structure):
    _fields_ = [("stop", ctypes.c_int), ("fea", ctypes.c_int), ("n_records", ctypes.c_int),
                ("volume_fraction", ctypes.c_double), ("reference", ctypes.c_double * 4)]


TOPO_ANALYSE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double))
TOPO_STEP = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p)
TOPO_CUT = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_double)


class afd_topology_ops(ctypes.Structure):
    _fields_ = [("analyse", TOPO_ANALYSE), ("save_feasible", TOPO_STEP), ("restore_feasible", TOPO_STEP),
                ("cut", TOPO_CUT)]


class afd_volmin_record(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int), ("volume_fraction", ctypes.c_double), ("J", ctypes.c_double),
                ("J_over_J0", ctypes.c_double), ("g", ctypes.c_double), ("iters", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("ms", ctypes.c_double), ("tau", ctypes.c_double),
                ("al_weight", ctypes.c_double), ("mu", ctypes.c_double), ("gamma", ctypes.c_double),
                ("kept", ctypes.c_longlong)]


# constraint names in the order of AFD_CON_COMPLIANCE .. AFD_CON_BUCKLING
CONSTRAINTS = ("J", "sigma", "lambda", "P")
_STOPS = {0: "max_fea", 1: "dv_min", 2: "v_min"}


def topology_spec(compliance=None, stress=None, eigen=None, buckling=None, soft=(), p: float = 8.0,
                  dv0: float = 0.05, dv_min: Optional[float] = None, v_min: float = 0.05, conv: float = 0.01,
                  max_fea: int = 200, tol: float = 1e-6, eig_tol: float = 1e-6, rho: float = 1.0,
                  casting=None) -> afd_topology_spec:
    """The afd_topology_spec of the keyword arguments (None: constraint absent;
    soft names among "lambda", "P"; casting (axis, parting) or None)."""
    sp = afd_topology_spec()
    for c, b in enumerate((compliance, stress, eigen, buckling)):
        sp.bound[c] = 0.0 if b is None else float(b)
        sp.soft[c] = int(CONSTRAINTS[c] in set(soft))
    sp.p, sp.dv0, sp.dv_min, sp.v_min, sp.conv = p, dv0, (0.0 if dv_min is None else dv_min), v_min, conv
    sp.max_fea, sp.tol, sp.eig_tol, sp.rho = max_fea, tol, eig_tol, rho
    sp.casting_axis, sp.casting_parting = (-1, 0) if casting is None else (int(casting[0]), int(casting[1]))
    return sp


def _topology_output(sp, hist, res) -> dict:
    """Records and result of a Sec. 3.8 run as Python dicts (values of absent
    constraints are None)."""
    act = [sp.bound[c] > 0 for c in range(4)]

    def opt(x):
        return None if x != x else float(x)

    out = []
    for r in hist[:min(res.n_records, len(hist))]:
        rec = {"fea": r.fea, "v": r.v, "target": r.target, "dv": r.dv, "violated": bool(r.violated),
               "iters": r.iters, "rel_residual": r.rel_residual}
        for c, name in enumerate(CONSTRAINTS):
            rec[name] = opt(r.value[c])
        rec["g"] = {name: r.g[c] for c, name in enumerate(CONSTRAINTS) if act[c]}
        rec["mu"] = {name: r.mu[c] for c, name in enumerate(CONSTRAINTS) if act[c]}
        rec["gamma"] = {name: r.gamma[c] for c, name in enumerate(CONSTRAINTS) if act[c]}
        out.append(rec)
    return {"history": out, "volume_fraction": res.volume_fraction, "stop": _STOPS[res.stop], "fea": res.fea,
            "reference": {name: opt(res.reference[c]) for c, name in enumerate(CONSTRAINTS)}}


def afd_topology_run(spec: afd_topology_spec, analyse, save_feasible, restore_feasible, cut,
                     hist_cap: int = 1000) -> dict:
    """The Sec. 3.8 loop of the library (afd_topology_run) over Python
    analyses: analyse(warm) -> (values[4], iters, rel_residual) with None for
    constraints it does not evaluate; save_feasible(); restore_feasible();
    cut(weights[4], v_target).  An exception in a callback ends the run with
    AFD_ERR_STATE and is re-raised."""
    err = []

    def guard(fn):
        def wrapped(*a):
            try:
                return fn(*a)
            except BaseException as e:  # noqa: BLE001 - re-raised after the C call returns
                err.append(e)
                return AFD_ERR_STATE
        return wrapped

    @guard
    def _analyse(ctx, warm, val, it, rel):
        v, iters, r = analyse(bool(warm))
        for c in range(4):
            val[c] = float("nan") if v[c] is None else float(v[c])
        it[0], rel[0] = int(iters), float(r)
        return AFD_OK

    @guard
    def _save(ctx):
        save_feasible()
        return AFD_OK

    @guard
    def _restore(ctx):
        restore_feasible()
        return AFD_OK

    @guard
    def _cut(ctx, w, v):
        cut([w[c] for c in range(4)], float(v))
        return AFD_OK

    ops = afd_topology_ops(TOPO_ANALYSE(_analyse), TOPO_STEP(_save), TOPO_STEP(_restore), TOPO_CUT(_cut))
    hist = (afd_topology_record * hist_cap)()
    res = afd_topology_result()
    rc = lib().afd_topology_run(ctypes.byref(spec), ctypes.byref(ops), None, hist, hist_cap, ctypes.byref(res))
    if err:
        raise err[0]
    _check(rc)
    return _topology_output(spec, hist, res)


def run_volume_minimisation(mesh: "Mesh", steps: int = 20, dv: float = 0.02, j_factor: float = 1.6,
                            tol: float = 1e-6, kind: int = AFD_SENS_STRAIN_ENERGY, on_step=None,
                            kept_out=None, u_out=None) -> list:
    """Compliance-constrained volume minimisation with fixed volume steps
    (afd_volume_minimisation: Sec. 3.8 with v_k = 1 - k dv; Eqs. 3.6, 3.11,
    3.12, 3.17, 3.18), run by the library from the mesh's current moduli and
    loads.  Returns one dict per solve (step 0 is the initial design); on_step
    is called with each afterwards.  kept_out (host uint8, nelem) receives the
    last kept mask; u_out (host float64, ndof) the last displacement."""
    hist = (afd_volmin_record * (steps + 1))()
    pk, _, _k1 = _arr(kept_out, np.uint8) if kept_out is not None else (None, 0, None)
    pu, _, _k2 = _arr(u_out, np.float64) if u_out is not None else (None, 0, None)
    if kept_out is not None and not isinstance(kept_out, np.ndarray):
        raise TypeError("kept_out must be a host numpy array")
    _check(lib().afd_volume_minimisation(mesh.h, steps, dv, j_factor, tol, kind, hist, pk, pu))
    out = []
    for r in hist:
        rec = {k: getattr(r, k) for k, _ in afd_volmin_record._fields_}
        if r.step == 0:
            rec["tau"] = None
        out.append(rec)
        if on_step:
            on_step(rec)
    return out


def run_constrained_topology(mesh: "Mesh", E_init, compliance: Optional[float] = None, stress: Optional[float] = None,
                             p: float = 8.0, dv0: float = 0.05, dv_min: Optional[float] = None, v_min: float = 0.05,
                             max_fea: int = 200, conv: float = 0.01, tol: float = 1e-6, casting=None,
                             on_step=None, eigen: Optional[float] = None, rho: float = 1.0,
                             eig_tol: float = 1e-6, buckling: Optional[float] = None, soft=()) -> dict:
    """The algorithm of Sec. 3.8 with Eq. 3.21's constraints, run by the library
    on the mesh (afd_constrained_topology; every analysis, field and cut stays
    on the device): min |Omega| subject to J <= compliance J_0,
    sigma_PN <= stress sigma_0, lambda_1 >= eigen lambda_1,0 and
    P >= buckling P_0 (any may be None; "lambda" and "P" may be soft).  Starts
    from E_init.  Returns the history (one dict per analysis; on_step is called
    with each afterwards), the final feasible design's kept mask, moduli and
    volume fraction, why it stopped, the number of analyses and the reference
    values."""
    if not set(soft) <= {"lambda", "P"}:
        raise ValueError("only the eigenvalue and buckling constraints can be soft")
    sp = topology_spec(compliance, stress, eigen, buckling, soft, p, dv0, dv_min, v_min, conv, max_fea, tol,
                       eig_tol, rho, casting)
    mesh.set_element_moduli(np.asarray(E_init, dtype=np.float64))
    ne = mesh.nelem
    hist = (afd_topology_record * max(1, max_fea))()
    res = afd_topology_result()
    kept = np.zeros(ne, np.uint8)
    E = np.zeros(ne)
    _check(lib().afd_constrained_topology(mesh.h, ctypes.byref(sp), hist, max(1, max_fea), ctypes.byref(res),
                                          ctypes.c_void_p(kept.ctypes.data), ctypes.c_void_p(E.ctypes.data)))
    out = _topology_output(sp, hist, res)
    out["kept"], out["E"] = kept, E
    if on_step:
        for rec in out["history"]:
            on_step(rec)
    return out


class Mesh:
    """Owning handle around one afd_mesh (same calls, managed lifetime)."""

    def __init__(self, nx: int, ny: int, nz: int, precision: int = AFD_MIXED, group: int = 0, nu: float = 0.3,
                 e_void: float = 1e-3, **opts):
        o = afd_default_options()
        o.precision, o.group, o.nu, o.e_void = precision, group, nu, e_void
        for k, v in opts.items():
            setattr(o, k, v)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.options = o
        self.h = afd_create_mesh(nx, ny, nz, o)
        self.n_rhs = 0

    @property
    def ndof(self) -> int:
        return afd_ndof(self.h)

    @property
    def nelem(self) -> int:
        return afd_nelem(self.h)

    def set_element_moduli(self, E):
        afd_set_element_moduli(self.h, E)

    def set_loads_bcs(self, f, fixed):
        self.n_rhs = int(f.shape[0]) if len(f.shape) == 2 else 1
        afd_set_loads_bcs(self.h, f, fixed)

    def solve(self, rel_tol: float, warm_start: bool = False, u_out=None, check: bool = True):
        return afd_solve(self.h, rel_tol, self.n_rhs, warm_start, u_out, check)

    def compliance(self) -> np.ndarray:
        return afd_compliance(self.h, self.n_rhs)

    def sensitivity(self, kind: int, out):
        afd_sensitivity(self.h, kind, out)

    def pnorm_stress(self, p: float) -> np.ndarray:
        return afd_pnorm_stress(self.h, p, self.n_rhs)

    def stress_sensitivity(self, p: float, rel_tol: float, out, lambda_out=None):
        return afd_stress_sensitivity(self.h, self.n_rhs, p, rel_tol, out, lambda_out)

    def modal(self, n_modes: int, rho: float = 1.0, tol: float = 1e-6, max_iter: int = 100, modes_out=None,
              check: bool = True):
        return afd_modal(self.h, n_modes, rho, tol, max_iter, modes_out, check)

    def eigen_sensitivity(self, out) -> None:
        afd_eigen_sensitivity(self.h, out)

    def buckling(self, n_modes: int, tol: float = 1e-6, max_iter: int = 100, modes_out=None, check: bool = True):
        return afd_buckling(self.h, n_modes, tol, max_iter, modes_out, check)

    def buckling_sensitivity(self, out) -> None:
        afd_buckling_sensitivity(self.h, out)

    def levelset_update(self, kind: int, weights, volume_fraction: float, kept_out=None, casting=None) -> float:
        return afd_levelset_update(self.h, kind, weights, volume_fraction, kept_out, casting)

    def close(self):
        if self.h:
            afd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
