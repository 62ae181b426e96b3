"""Golden fixtures (tests/golden/).

paper_constants.txt holds closed-form values the paper states (cited there);
the oracle is pinned to them.  golden_cases.json holds the oracle's outputs
for small formula-defined inputs, written by tests/golden/make_golden.py
(which calls only the oracle): the oracle must reproduce them (any change to
its arithmetic shows up here), and the GPU tests compare the CUDA path with
them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def paper_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, value = line.split()[:2]
                out[name] = float(value)
    return out


def golden_cases():
    with open(os.path.join(GOLDEN, "golden_cases.json")) as fh:
        return json.load(fh)["cases"]


def test_constants_follow_the_stated_formulas():
    c = paper_constants()
    g = math.gamma
    assert c["sw2_shift_factor"] == pytest.approx(g(1.5) / (math.sqrt(math.pi) * g(2.0)),
                                                  rel=1e-15)
    assert c["rfsw2_shift_factor"] == pytest.approx(2 * g(1.5) / (math.sqrt(math.pi) * g(2.0)),
                                                    rel=1e-15)
    assert c["sw2_view_constant"] == pytest.approx(math.sqrt(1 - 4 / (3 * math.pi)), rel=1e-15)


def _gauss_img(L, cx, cy, s):
    h = 2.0 / L
    x = -1 + (np.arange(L) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    img = np.exp(-0.5 * ((X - cx) ** 2 + (Y - cy) ** 2) / s ** 2)
    return img / img.sum()


def test_oracle_translation_factor_is_the_papers():
    """Thm. "Translation equivariance" at p = 2: SW2^2(f, T_s f) = 1/2 |s|^2.
    An isotropic Gaussian and a copy shifted by whole pixels (mass kept in
    the grid); rotation only (translation = 0), rotation l = 0."""
    c = paper_constants()["sw2_shift_factor"]
    L, n, M = 64, 64, 128
    h = 2.0 / L
    f = _gauss_img(L, 0.0, 0.0, 0.12)
    for dr, dc in [(3, 0), (0, -5), (4, 3)]:
        g = np.roll(np.roll(f, dr, axis=0), dc, axis=1)
        _, D, _ = oracle.align_pair(f, g, n, M, translation=0)
        s2 = (dr * h) ** 2 + (dc * h) ** 2
        assert D[0] == pytest.approx(c * s2, rel=2e-3), (dr, dc, D[0], c * s2)


def _views(L, theta, comps):
    """Two tomographic views (about the x axis, theta apart) of a 3-D Gaussian
    mixture: each component projects to the 2-D Gaussian with mean E mu and
    covariance E Sigma E^T, E = the 2 x 3 basis of the viewing plane."""
    h = 2.0 / L
    x = -1 + (np.arange(L) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    out = []
    for th in (0.0, theta):
        E = np.array([[1, 0, 0], [0, math.cos(th), math.sin(th)]])
        img = np.zeros((L, L))
        for w, mu, Sig in comps:
            m, C = E @ mu, E @ Sig @ E.T
            Ci = np.linalg.inv(C)
            dx, dy = X - m[0], Y - m[1]
            e = Ci[0, 0] * dx * dx + 2 * Ci[0, 1] * dx * dy + Ci[1, 1] * dy * dy
            img += w * np.exp(-0.5 * e) / (2 * math.pi * math.sqrt(np.linalg.det(C)))
        out.append(img / img.sum())
    return out


def test_oracle_view_stability_bound():
    """Table tab:view / Thm. view at p = 2: SW2 between two views theta
    apart of one density in the unit ball is at most sqrt(1 - 4/(3 pi))
    theta, and grows linearly in theta."""
    c = paper_constants()["sw2_view_constant"]
    rng = np.random.default_rng(3)
    comps = []
    for _ in range(4):
        mu = rng.uniform(-0.35, 0.35, 3)
        A = rng.standard_normal((3, 3))
        Q, _ = np.linalg.qr(A)
        s = rng.uniform(0.06, 0.16, 3)
        comps.append((rng.uniform(0.5, 1.0), mu, Q @ np.diag(s ** 2) @ Q.T))
    L, n, M = 64, 64, 64
    d = {}
    for th in (0.1, 0.2):
        I1, I2 = _views(L, th, comps)
        _, D, _ = oracle.align_pair(I1, I2, n, M, translation=0)
        d[th] = math.sqrt(D[0])
        assert d[th] <= c * th
    assert 1.7 <= d[0.2] / d[0.1] <= 2.3


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_oracle_reproduces_golden_cases(case):
    f = np.array(case["f"], dtype=np.float32).astype(np.float64)
    g = np.array(case["g"], dtype=np.float32).astype(np.float64)
    n, M = case["n"], case["M"]
    res, D, S = oracle.align_pair(f, g, n, M, level_rule=case["level_rule"],
                                  translation=case["translation"])
    np.testing.assert_allclose(D, case["D"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(S, case["shifts"], rtol=1e-12, atol=1e-15)
    assert res["best_l"] == case["best_l"]
    F, _ = oracle.prepare(f)
    Q = oracle.quantiles(oracle.project(F, n), 2.0 / F.shape[0], M, level_rule=case["level_rule"])
    np.testing.assert_allclose(Q, case["quantiles_f"], rtol=1e-12, atol=1e-15)
