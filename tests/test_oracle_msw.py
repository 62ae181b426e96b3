"""Pins of the oracle's max-sliced W2 over rotations (Eq.
max_sliced_wasserstein, with the level average 1/M per angle).

The maximum over angles of the per-angle W2^2 is pinned by: the uniform
case (every column equal: the max is that value and equals the sliced
mean); the shift of an isotropic Gaussian (per-angle W2^2 = <s, e_k>^2, so
the max is |s|^2 when an angle points along s, twice the sliced W2^2 of
1/2 |s|^2); exact quarter turns; the bound max >= mean (the sliced curve);
and the exact per-angle W2^2 of two histograms within Theorem E3's bound."""
import math

import numpy as np
import pytest

import oracle
from tests import analytic


def test_max_of_equal_columns_is_the_mean():
    rng = np.random.default_rng(0)
    n, M = 12, 7
    u = np.sort(rng.normal(size=M))
    v = np.sort(rng.normal(size=M))
    Qf = np.tile(u, (n, 1))
    Qg = np.tile(v, (n, 1))
    D = oracle.msw_curve(Qf, Qg)
    np.testing.assert_allclose(D, np.mean((u - v) ** 2), rtol=1e-14)
    np.testing.assert_allclose(D, oracle.rotation_curve(Qf, Qg), rtol=1e-14)


def test_max_dominates_the_sliced_mean_and_matches_brute_force():
    rng = np.random.default_rng(1)
    n, M = 10, 6
    Qf, Qg = np.sort(rng.normal(size=(2, n, M)), axis=2)
    D = oracle.msw_curve(Qf, Qg)
    S = oracle.rotation_curve(Qf, Qg)
    assert np.all(D >= S - 1e-15)
    for l in range(n):
        cols = [np.mean((Qf[k] - Qg[(k - l) % n]) ** 2) for k in range(n)]
        assert D[l] == pytest.approx(max(cols), rel=1e-14)


def test_shifted_gaussian_max_is_twice_the_sliced_value():
    """Per-angle W2^2 of a shifted density is <s, e_k>^2: the sliced mean is
    |s|^2 / 2 (Thm. shift at p = 2) and the max is |s|^2 (an angle of the
    grid along s)."""
    rng = np.random.default_rng(9)
    n, M, B, h = 64, 256, 364, 2 / 256
    th = 2 * np.pi * np.arange(n) / n
    mix = analytic.random_mixture(rng, 2)
    s = 0.1 * np.array([math.cos(th[5]), math.sin(th[5])])  # along grid angle 5
    Qf = oracle.quantiles(analytic.mixture_hist(*mix, th, B, h), h, M)
    Qg = oracle.quantiles(analytic.mixture_hist(*analytic.transform_mixture(mix, shift=s),
                                                th, B, h), h, M)
    D = oracle.msw_curve(Qf, Qg)
    assert D[0] == pytest.approx(s @ s, rel=2e-3)
    assert oracle.rotation_curve(Qf, Qg)[0] == pytest.approx(0.5 * (s @ s), rel=2e-3)


@pytest.mark.parametrize("translation", [1, 0])
def test_quarter_turn_is_exact(translation):
    rng = np.random.default_rng(21)
    L, n, M = 16, 16, 8
    F = rng.random((L, L)) ** 2
    G90 = np.array([[F[L - 1 - c, r] for c in range(L)] for r in range(L)])
    res, D, _ = oracle.align_pair_msw(F, G90, n, M, translation=translation)
    assert res["best_l"] == 3 * n // 4
    assert res["d2"] < 1e-26


def test_per_angle_value_within_the_exact_w2_bound():
    """Each column term is the sampled-level W2^2 of the two projections;
    it lies within Theorem E3's 8h + 16/M of the exact histogram W2^2."""
    rng = np.random.default_rng(3)
    L, n, M = 24, 8, 64
    f, g = rng.random((2, L, L)) ** 2
    h = 2.0 / L
    Uf = oracle.project(oracle.prepare(f)[0], n)
    Ug = oracle.project(oracle.prepare(g)[0], n)
    Qf, Qg = oracle.quantiles(Uf, h, M), oracle.quantiles(Ug, h, M)
    D = oracle.msw_curve(Qf, Qg)
    exact = max(oracle.w2_hist_exact(Uf[k], Ug[k], h) for k in range(n))
    assert abs(D[0] - exact) <= 8 * h + 16 / M
