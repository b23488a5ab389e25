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
