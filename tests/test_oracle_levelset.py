"""Pins of the level-set extraction (Eq. 3.6) and of the augmented-Lagrangian
scalar updates (Eqs. 3.11, 3.12, 3.18)."""
import os

import numpy as np
import pytest

from oracle import levelset

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_constants_are_the_papers():
    g = _golden()
    assert levelset.MU0 == g["mu0"] and levelset.GAMMA0 == g["gamma0"]
    assert levelset.VARSIGMA == g["varsigma"] and levelset.ETA == g["eta"]


def test_multiplier_and_penalty_sequences_by_hand():
    mu, gamma = 100.0, 10.0
    # g = -0.5: mu = max(100 - 5, 0) = 95
    assert levelset.multiplier_update(mu, gamma, -0.5) == 95.0
    # a large violation drives mu to 0 only when mu + gamma g < 0
    assert levelset.multiplier_update(3.0, 10.0, -0.5) == 0.0
    # constraint satisfied (g <= 0) both times: gamma kept
    assert levelset.penalty_update(10.0, -0.1, -0.3, 1) == 10.0
    # violation not reduced to a quarter: gamma -> max(10 * 10, k^2)
    assert levelset.penalty_update(10.0, 0.2, 0.4, 3) == 100.0
    assert levelset.penalty_update(10.0, 0.2, 0.4, 20) == 400.0
    # violation reduced below a quarter: gamma kept
    assert levelset.penalty_update(10.0, 0.05, 0.4, 3) == 10.0
    assert levelset.al_weight(100.0, 10.0, -0.5) == 95.0
    assert levelset.al_weight(1.0, 10.0, -0.5) == 0.0


def test_select_top_matches_brute_force_with_ties():
    rng = np.random.default_rng(7)
    for n in (1, 2, 7, 100, 1000):
        v = rng.integers(0, 5, n).astype(np.float32)     # many ties
        for frac in (0.0, 0.13, 0.5, 0.98, 1.0):
            k = levelset.keep_count(frac, n)
            kept, tau = levelset.select_top(v, k)
            order = sorted(range(n), key=lambda i: (-float(v[i]), i))
            ref = np.zeros(n, np.uint8)
            ref[order[:k]] = 1
            assert np.array_equal(kept, ref)
            assert kept.sum() == k
            if k:
                assert tau == float(v[order[k - 1]])


def test_keep_count_rounding():
    assert levelset.keep_count(0.5, 3) == 2       # 1.5 rounds up
    assert levelset.keep_count(0.98, 100) == 98
    assert levelset.keep_count(1.2, 10) == 10
    assert levelset.keep_count(-0.1, 10) == 0


def test_combine_normalises_each_field():
    a = np.array([2.0, -4.0, 1.0], np.float32)
    b = np.array([0.5, 0.25, 1.0], np.float32)
    out = levelset.combine([a, b], [1.0, 2.0])
    assert out.dtype == np.float32
    assert np.allclose(out, [0.5 + 1.0, -1.0 + 0.5, 0.25 + 2.0], rtol=0, atol=1e-7)
