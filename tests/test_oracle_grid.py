"""Pins of the oracle's explicit translation sampling (the translation of
the whole image restricted to a grid, searched by brute force).

The grid search is evaluated from its definition; these tests pin it to
independent facts: a one-point grid at 0 is the rotation-only distance; the
unbounded closed-form optimum D_T(l) is a lower bound; and, because J(l, s)
is a quadratic in s with curvature rho = 1/2 (sliced W2) or 1 (two parts,
ramp-filtered), the grid minimum equals D_T(l) + rho |g - c(l)|^2 at the grid
point g nearest the closed-form optimum c(l)."""
import numpy as np
import pytest

import oracle


def nearest(c, K, step):
    return np.clip(np.rint(c / step), -K, K) * step


@pytest.mark.parametrize("metric", [0, 1])
def test_one_point_grid_is_rotation_only(metric):
    rng = np.random.default_rng(2 + metric)
    f, g = rng.random((2, 16, 16)) ** 2
    n, M = 12, 8
    _, D, S = oracle.align_pair_grid(f, g, n, M, 0, 0.1, metric=metric)
    ref = oracle.align_pair_rfsw if metric else oracle.align_pair
    _, D0, _ = ref(f, g, n, M, translation=0)
    np.testing.assert_allclose(D, D0, rtol=1e-13, atol=1e-18)
    assert np.all(S == 0)


@pytest.mark.parametrize("metric,rho", [(0, 0.5), (1, 1.0)])
def test_grid_minimum_is_closed_form_plus_distance_to_nearest_point(metric, rho):
    rng = np.random.default_rng(7 + metric)
    L, n, M = 16, 12, 8
    f, g = rng.random((2, L, L)) ** 2
    step, K = (2.0 / L) / 4, 5
    _, DG, SG = oracle.align_pair_grid(f, g, n, M, K, step, metric=metric)
    ref = oracle.align_pair_rfsw if metric else oracle.align_pair
    _, DT, ST = ref(f, g, n, M, translation=1)
    assert np.all(DG >= DT - 1e-15)
    for l in range(n):
        gpt = nearest(ST[l], K, step)
        assert DG[l] == pytest.approx(DT[l] + rho * np.sum((gpt - ST[l]) ** 2), rel=1e-10, abs=1e-16)
        np.testing.assert_allclose(SG[l], gpt, atol=1e-12)
