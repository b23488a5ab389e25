"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/afd.h; its host-only scalar routines (Eqs. 3.11, 3.12,
3.18) agree with the oracle's."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def afd():
    from paper_2203_15115_gb300 import build

    build.build()
    import paper_2203_15115_gb300 as afd

    afd.lib()
    return afd


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "afd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(afd_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(afd):
    names = declared_symbols()
    assert len(names) >= 20
    L = ctypes.CDLL(afd.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(afd.EXPORTS) == names


def test_default_options(afd):
    o = afd.afd_default_options()
    assert o.precision == afd.AFD_MIXED and abs(o.nu - 0.3) < 1e-15 and o.e_void == 1e-3


def test_al_scalars_match_oracle(afd):
    from oracle import levelset

    s = afd.afd_al_init()
    assert (s.mu, s.gamma, s.k) == (levelset.MU0, levelset.GAMMA0, 0)
    mu, gamma, g_old = levelset.MU0, levelset.GAMMA0, 0.0
    for k, g in enumerate([-0.4, -0.1, 0.3, 0.25, 0.05, 0.01, -0.2, 0.6], start=1):
        afd.afd_al_update(s, g)
        mu = levelset.multiplier_update(mu, gamma, g)
        gamma = levelset.penalty_update(gamma, g, g_old, k)
        g_old = g
        assert s.mu == mu and s.gamma == gamma and s.k == k
        assert afd.afd_al_weight(s) == levelset.al_weight(mu, gamma, g)


def test_mesh_bytes_estimate_grows_with_the_mesh(afd):
    a = afd.afd_mesh_bytes(32, 16, 16)
    b = afd.afd_mesh_bytes(64, 32, 32)
    c = afd.afd_mesh_bytes(64, 32, 32, 8)
    ndof = 3 * 65 * 33 * 33
    assert 0 < a < b < c
    assert b > ndof * (3 * 8 + 8 * 4)       # at least the FP64 and FP32 vectors
    assert afd.afd_mesh_bytes(0, 1, 1) == 0


def test_product_path_fails_loudly_without_its_library(afd, monkeypatch):
    """No CPU fallback: without the built library every call raises."""
    monkeypatch.setattr(afd, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libafdcg.so"))
    monkeypatch.setattr(afd, "_lib", None)
    with pytest.raises(RuntimeError):
        afd.lib()
    with pytest.raises(RuntimeError):
        afd.Mesh(4, 2, 2)


def test_options_are_validated_before_any_device_call(afd):
    """Bad options are refused with AFD_ERR_INVALID_ARG on any machine, GPU or
    not; the device is touched only by a valid request."""
    for bad in ({"stencil_warps": 12}, {"stencil_planes": -1}, {"inner_aim": 1.5}, {"nu": 0.5},
                {"max_iter": 0}, {"e_void": 0.0}, {"precision": 7}):
        with pytest.raises(afd.AFDError) as e:
            afd.Mesh(4, 2, 2, **bad)
        assert e.value.code == afd.AFD_ERR_INVALID_ARG, bad


def test_a_valid_request_without_a_gpu_is_an_error_not_a_crash(afd):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(afd.AFDError) as e:
        afd.Mesh(4, 2, 2)
    assert e.value.code == afd.AFD_ERR_CUDA
