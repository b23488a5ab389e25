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


def _cast_brute(T, nx, ny, nz, axis, parting):
    """Definition written per element: T'(e) = max over the elements f of its
    line and half at or beyond e (away from the parting plane) of T(f) raised
    by one float32 step per element between f and e."""
    a = np.asarray(T, np.float32).reshape(nz, ny, nx)
    out = np.empty_like(a)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                idx = [i, j, k]
                c = idx[axis]
                n = (nx, ny, nz)[axis]
                far = range(c, n) if c >= parting else range(c, -1, -1)
                best = None
                for f in far:
                    q = list(idx)
                    q[axis] = f
                    v = a[q[2], q[1], q[0]]
                    for _ in range(abs(f - c)):
                        v = np.nextafter(v, np.float32(np.inf))
                    best = v if best is None else max(best, v)
                out[k, j, i] = best
    return out.reshape(-1)


@pytest.mark.parametrize("axis,parting", [(0, 0), (1, 3), (2, 5), (0, 7), (2, 0)])
def test_casting_scan_matches_its_definition(axis, parting):
    rng = np.random.default_rng(3 + axis)
    nx, ny, nz = 7, 5, 6
    T = rng.standard_normal(nx * ny * nz).astype(np.float32)
    T[::4] = T[1::4][: T[::4].size]           # plateaus and ties
    got = levelset.casting_scan(T, nx, ny, nz, axis, parting)
    assert np.array_equal(got, _cast_brute(T, nx, ny, nz, axis, parting))


def test_casting_scan_properties_and_no_undercut():
    rng = np.random.default_rng(11)
    nx, ny, nz = 12, 8, 10
    T = rng.random(nx * ny * nz).astype(np.float32)
    for axis, parting in [(0, 4), (1, 0), (2, 10), (2, 3)]:
        S = levelset.casting_scan(T, nx, ny, nz, axis, parting)
        assert np.all(S >= T)
        assert np.array_equal(levelset.casting_scan(S, nx, ny, nz, axis, parting), S)   # idempotent
        n = (nx, ny, nz)[axis]
        a = np.moveaxis(S.reshape(nz, ny, nx), {0: 2, 1: 1, 2: 0}[axis], 0)
        # strictly increasing toward the parting plane on both halves
        assert np.all(a[parting:-1] > a[parting + 1:]) if parting < n - 1 else True
        assert np.all(a[1:parting] > a[:parting - 1]) if parting > 1 else True
        for v in (0.3, 0.5, 0.8):
            kept, _ = levelset.select_top(S, levelset.keep_count(v, S.size))
            kk = np.moveaxis(kept.reshape(nz, ny, nx), {0: 2, 1: 1, 2: 0}[axis], 0).astype(bool)
            # kept elements on each half are a run starting at the parting plane
            up, lo = kk[parting:], kk[:parting][::-1]
            for half in (up, lo):
                if half.shape[0] > 1:
                    assert not np.any(~half[:-1] & half[1:])
