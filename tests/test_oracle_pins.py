"""Pins for the FP64 oracle: closed forms, invariants and brute force.

Each test pins one routine of ``oracle/`` against something other than the
oracle itself: a value worked out by hand from the geometry, a closed form
(the 1-D Gaussian W2, Theorem 3.2 at p = 2), an exact invariant (mass, first
moment, mirror and quarter-turn symmetries, cyclic column shifts), a library
routine (numpy's FFT for the rotation search) or brute force on tiny inputs.
"""
import math

import numpy as np
import pytest

import oracle
from tests import analytic

pytest.importorskip("scipy")


def centroid(F):
    L = F.shape[0]
    h = 2.0 / L
    x = -1.0 + (np.arange(L) + 0.5) * h
    m = F.sum()
    return np.array([(F.sum(axis=0) * x).sum() / m, (F.sum(axis=1) * x).sum() / m])


# ---------------------------------------------------------------- projection

def test_default_bins_hold_every_pixel_with_half_bin_margin():
    for L in [1, 2, 3, 4, 16, 39, 64, 85, 96, 128, 192, 256, 512]:
        B = oracle.default_bins(L)
        reach = (L - 1) / math.sqrt(2.0)  # |s|/h for the corner pixel centres
        assert (B - 1) / 2 - reach >= 0.5 - 1e-12
        assert B % 2 == 0


def test_projection_single_pixel_by_hand():
    # L = 4, h = 1/2, B = 2*ceil(3/sqrt2)+2 = 8, bin centres s_b = (b-3.5)/2.
    # Pixel (row 0, column 3) has centre x = 0.75, y = -0.75.
    F = np.zeros((4, 4))
    F[0, 3] = 1.0
    U = oracle.project(F, n=8)
    assert U.shape == (8, 8)
    # theta = 0: s = x = 0.75 -> u = 1.5 + 3.5 = 5 -> all mass in bin 5
    np.testing.assert_allclose(U[0], np.eye(8)[5], atol=1e-15)
    # theta = pi/4: s = (0.75 - 0.75)/sqrt2 = 0 -> u = 3.5 -> bins 3, 4 half each
    np.testing.assert_allclose(U[1], 0.5 * (np.eye(8)[3] + np.eye(8)[4]), atol=1e-12)
    # theta = pi/2: s = y = -0.75 -> u = -1.5 + 3.5 = 2 -> bin 2
    np.testing.assert_allclose(U[2], np.eye(8)[2], atol=1e-12)
    # theta = pi: s = -x -> u = 2 -> bin 2
    np.testing.assert_allclose(U[4], np.eye(8)[2], atol=1e-12)
    # theta = 3pi/2: s = -y = 0.75 -> bin 5
    np.testing.assert_allclose(U[6], np.eye(8)[5], atol=1e-12)


@pytest.mark.parametrize("L,n", [(16, 12), (33, 20), (64, 36)])
def test_projection_keeps_mass_and_first_moment(L, n):
    rng = np.random.default_rng(L)
    F = rng.random((L, L)) ** 3  # asymmetric in x, y and along the diagonals
    F /= F.sum()
    U = oracle.project(F, n)
    B = U.shape[1]
    h = 2.0 / L
    s = (np.arange(B) - (B - 1) / 2) * h
    c = centroid(F)
    for k in range(n):
        t = 2 * np.pi * k / n
        assert abs(U[k].sum() - 1.0) < 1e-13
        assert abs((U[k] * s).sum() - (c[0] * np.cos(t) + c[1] * np.sin(t))) < 1e-13


def test_projection_mirror_and_quarter_turn():
    rng = np.random.default_rng(7)
    L, n = 24, 16
    F = rng.random((L, L))
    F /= F.sum()
    U = oracle.project(F, n)
    # P_{theta+pi} f(s) = P_theta f(-s); bin centres are symmetric about 0
    for k in range(n // 2):
        np.testing.assert_allclose(U[k + n // 2], U[k][::-1], atol=1e-14)
    # g = R_{90 deg} f on the cell grid: g(x, y) = f(y, -x)  =>  G[r][c] = F[L-1-c][r]
    G = np.empty_like(F)
    for r in range(L):
        for c in range(L):
            G[r, c] = F[L - 1 - c, r]
    V = oracle.project(G, n)
    for k in range(n):  # P_theta(R_alpha f) = P_{theta - alpha} f
        np.testing.assert_allclose(V[k], U[(k - n // 4) % n], atol=1e-14)


def test_projection_of_sampled_gaussian_matches_radon_transform():
    # A wide Gaussian sampled at cell centres.  At axis-aligned angles the
    # cell centres sit on bin centres and the splatted CDF matches the
    # analytic projection's CDF at the nodes.  At every angle the mean is
    # exact and the variance differs by at most the splat's own spread
    # (t(1-t) h^2 <= h^2/4) plus the histogram's h^2/12.  At 45 degrees the
    # pixel-driven splat shows the usual moire (centres on a lattice of pitch
    # h/sqrt 2), so no node-wise CDF pin is made there.
    L, n = 128, 8
    mix = ([1.0], [np.array([0.1, -0.05])], [np.array([[0.03, 0.01], [0.01, 0.02]])])
    F = analytic.pixel_image(mix, L)
    F /= F.sum()
    U = oracle.project(F, n)
    B = U.shape[1]
    h = 2.0 / L
    A = analytic.mixture_hist(*mix, 2 * np.pi * np.arange(n) / n, B, h)
    A /= A.sum(axis=1, keepdims=True)
    err = np.abs(np.cumsum(U, axis=1) - np.cumsum(A, axis=1))
    assert err[0::2].max() < 2e-4  # midpoint samples vs bin integrals: O(h^2)
    s = (np.arange(B) - (B - 1) / 2) * h
    var_u = (U * s * s).sum(1) - (U * s).sum(1) ** 2
    var_a = (A * s * s).sum(1) - (A * s).sum(1) ** 2
    assert np.all(np.abs(var_u - var_a) <= h * h / 4 + h * h / 12)


# ----------------------------------------------------------------- quantiles

def test_quantiles_of_uniform_histogram_closed_form():
    B, h, M = 40, 0.05, 16
    U = np.zeros((1, B))
    U[0, 11:18] = 3.0  # uniform on [e_11, e_18]
    Q = oracle.quantiles(U, h, M)
    e11 = (11 - B / 2) * h
    z = (np.arange(M) + 0.5) / M
    np.testing.assert_allclose(Q[0], e11 + 7 * h * z, atol=1e-14)
    Q1 = oracle.quantiles(U, h, M, level_rule=1)
    np.testing.assert_allclose(Q1[0, 1:], e11 + 7 * h * np.arange(1, M) / M, atol=1e-14)
    assert Q1[0, 0] == -B / 2 * h  # z = 0: the left end of the domain


@pytest.mark.parametrize("M", [1, 2, 7, 64, 257])
def test_quantiles_invert_the_piecewise_linear_cdf(M):
    """With every bin's mass positive, the CDF of Sec. 2.3 (cumulative sums at
    the bin edges, linear inside a bin) is strictly increasing, so Q(z) is its
    plain inverse: np.interp of z F_B over (F_j, e_j).  Both level rules; M = 1
    under the midpoint rule is the median."""
    rng = np.random.default_rng(M)
    B, h = 37, 0.13
    U = rng.uniform(0.05, 2.0, size=(5, B))
    e = (np.arange(B + 1) - B / 2) * h
    for rule, z in ((0, (np.arange(M) + 0.5) / M), (1, np.arange(M) / M)):
        Q = oracle.quantiles(U, h, M, level_rule=rule)
        for r in range(U.shape[0]):
            F = np.concatenate([[0.0], np.cumsum(U[r])])
            np.testing.assert_allclose(Q[r], np.interp(z * F[-1], F, e), rtol=0, atol=1e-12)


def test_sampled_w2_of_two_uniforms_closed_form():
    # Q_a(z) = e_5 + 4hz, Q_b(z) = e_20 + 8hz: the difference is D - 4hz, whose
    # midpoint mean square is D^2 - 4hD + 16h^2 (4M^2-1)/(12M^2) and whose
    # integral is D^2 - 4hD + 16h^2/3.
    B, h, M = 40, 0.05, 24
    Ua = np.zeros(B); Ua[5:9] = 1.0
    Ub = np.zeros(B); Ub[20:28] = 0.5
    Q = oracle.quantiles(np.stack([Ua, Ub]), h, M)
    D = (5 - 20) * h
    want = D * D - 4 * h * D + 16 * h * h * (4 * M * M - 1) / (12 * M * M)
    assert abs(np.mean((Q[0] - Q[1]) ** 2) - want) < 1e-14
    exact = oracle.w2_hist_exact(Ua, Ub, h)
    assert abs(exact - (D * D - 4 * h * D + 16 * h * h / 3)) < 1e-14


def test_quantile_takes_left_end_of_flat_cdf_and_domain_start_at_zero():
    # Masses 1,1,1 in bins 2..4, nothing in 5..6, masses 1,1,1 in 7..9.
    # level_rule 1 with M = 2: z = 0 and z = 1/2; tau = 3 = F_5 = F_6 = F_7.
    # inf{t : F(t) >= z} (App. A.1.1): at z = 0 every t of the domain
    # qualifies, so Q(0) = e_0; at z = 1/2 it is the left end of the flat part.
    B, h = 12, 0.25
    U = np.zeros((1, B))
    U[0, [2, 3, 4, 7, 8, 9]] = 1.0
    Q = oracle.quantiles(U, h, 2, level_rule=1)
    e = lambda j: (j - B / 2) * h
    assert Q[0, 0] == pytest.approx(e(0), abs=1e-15)
    assert Q[0, 1] == pytest.approx(e(5), abs=1e-15)


def test_w2_gaussian_closed_form_and_E3_bound():
    # 1-D W2 between Gaussians: (mu1-mu2)^2 + (s1-s2)^2.  The exact histogram
    # W2 converges to it as O(h^2); the sampled-level sum stays within the
    # E3 bound 8h + 16/M (App. A, Theorem E3) of the exact histogram value.
    from scipy.special import ndtr
    cf = 0.15 ** 2 + 0.04 ** 2
    for B, h, M in [(182, 2 / 128, 128), (364, 2 / 256, 256), (2048, 1 / 1024, 4096)]:
        e = (np.arange(B + 1) - B / 2) * h
        Ua = np.diff(ndtr((e - 0.10) / 0.08))
        Ub = np.diff(ndtr((e + 0.05) / 0.12))
        ex = oracle.w2_hist_exact(Ua, Ub, h)
        assert abs(ex - cf) < 0.05 * h * h
        for rule in (0, 1):
            Q = oracle.quantiles(np.stack([Ua, Ub]), h, M, level_rule=rule)
            assert abs(np.mean((Q[0] - Q[1]) ** 2) - ex) <= 8 * h + 16 / M
    Q = oracle.quantiles(np.stack([Ua, Ub]), h, M, level_rule=0)
    assert abs(np.mean((Q[0] - Q[1]) ** 2) - cf) < 2e-6  # midpoint levels, finest grid


def test_sampled_w2_within_E3_bound_on_random_histograms():
    rng = np.random.default_rng(3)
    B, h = 92, 2 / 64
    for M in (16, 64, 128):
        for _ in range(5):
            Ua = rng.random(B) * (rng.random(B) < 0.6)
            Ub = rng.random(B) * (rng.random(B) < 0.6)
            Q = oracle.quantiles(np.stack([Ua, Ub]), h, M)
            ex = oracle.w2_hist_exact(Ua, Ub, h)
            assert abs(np.mean((Q[0] - Q[1]) ** 2) - ex) <= 8 * h + 16 / M


# ------------------------------------------------------------ rotation search

def test_rotation_curve_equals_fft_cross_correlation():
    # Eq. discrete_rot_sw2: ||U - T_l V||^2 = ||U||^2 + ||V||^2 - 2 corr(l), with
    # corr(l) the per-row circular cross-correlation along angle (numpy FFT).
    rng = np.random.default_rng(11)
    n, M = 24, 7
    Qf, Qg = rng.normal(size=(n, M)), rng.normal(size=(n, M))
    D = oracle.rotation_curve(Qf, Qg)
    Ff, Fg = np.fft.fft(Qf, axis=0), np.fft.fft(Qg, axis=0)
    corr = np.fft.ifft((Ff * np.conj(Fg)).sum(axis=1)).real
    want = ((Qf ** 2).sum() + (Qg ** 2).sum() - 2 * corr) / (n * M)
    np.testing.assert_allclose(D, want, rtol=0, atol=1e-12)


def test_cyclic_column_shift_is_found_exactly():
    rng = np.random.default_rng(5)
    n, M, l0 = 36, 9, 13
    Qf = rng.normal(size=(n, M))
    Qg = np.roll(Qf, -l0, axis=0)  # Qg[(k - l0) mod n] = Qf[k]
    D = oracle.rotation_curve(Qf, Qg)
    assert int(np.argmin(D)) == l0
    assert D[l0] == 0.0
    assert np.all(np.delete(D, l0) > 1e-3)


@pytest.mark.parametrize("translation", [0, 1])
def test_quarter_and_half_turn_images_align_exactly(translation):
    rng = np.random.default_rng(21)
    L, n, M = 16, 16, 8
    F = rng.random((L, L)) ** 2
    G90 = np.empty_like(F)
    for r in range(L):
        for c in range(L):
            G90[r, c] = F[L - 1 - c, r]  # g = R_{+90 deg} f
    res, D, _ = oracle.align_pair(F, G90, n, M, translation=translation)
    assert res["best_l"] == 3 * n // 4  # rotate g by -90 deg
    assert res["d2"] < 1e-26
    res, D, _ = oracle.align_pair(F, F[::-1, ::-1], n, M, translation=translation)
    assert res["best_l"] == n // 2
    assert res["d2"] < 1e-26


def test_rotation_by_grid_multiple_on_analytic_projections():
    # Zero distance and the exact shift when an image is compared with itself
    # rotated by a multiple of 2 pi / n.  Done on analytic
    # projections, where rotating the mixture is exact.
    rng = np.random.default_rng(8)
    n, M, B, h = 40, 32, 182, 2 / 128
    th = 2 * np.pi * np.arange(n) / n
    mix = analytic.random_mixture(rng, 3)
    m = 7
    mix_g = analytic.transform_mixture(mix, beta=2 * np.pi * m / n)
    Qf = oracle.quantiles(analytic.mixture_hist(*mix, th, B, h), h, M)
    Qg = oracle.quantiles(analytic.mixture_hist(*mix_g, th, B, h), h, M)
    D = oracle.rotation_curve(Qf, Qg)
    assert int(np.argmin(D)) == (-m) % n
    assert D[(-m) % n] < 1e-24


# --------------------------------------------------------------- translation

def test_translation_identity_D0_minus_DT():
    # J(l, s) is quadratic in s with Hessian I (sum_k e_k e_k^T = n/2 I), so
    # the rotation-only distance exceeds the translated one by |s*(l)|^2 / 2.
    rng = np.random.default_rng(2)
    L, n, M = 20, 24, 10
    f, g = rng.random((L, L)) ** 3, rng.random((L, L)) ** 3
    _, D0, _ = oracle.align_pair(f, g, n, M, translation=0)
    _, DT, S = oracle.align_pair(f, g, n, M, translation=1)
    np.testing.assert_allclose(D0 - DT, 0.5 * (S ** 2).sum(axis=1), rtol=0, atol=1e-14)


def test_translation_closed_form_beats_brute_force_grid():
    # Brute force over s on a fine grid, with J(l, s) evaluated from the
    # uncentred quantiles: a translation by s adds <s, e_k> to column k.
    rng = np.random.default_rng(4)
    L, n, M = 16, 12, 8
    f, g = rng.random((L, L)) ** 2, rng.random((L, L)) ** 2
    res, DT, S = oracle.align_pair(f, g, n, M, translation=1)
    h = 2.0 / L
    Qf = oracle.quantiles(oracle.project(oracle.prepare(f)[0], n), h, M)
    Qg = oracle.quantiles(oracle.project(oracle.prepare(g)[0], n), h, M)
    th = 2 * np.pi * np.arange(n) / n
    E = np.stack([np.cos(th), np.sin(th)], axis=1)
    for l in (0, 5, res["best_l"]):
        Vl = np.roll(Qg, l, axis=0)  # Vl[k] = Qg[(k - l) mod n]
        grid = np.arange(-32, 33) * (h / 16)
        best = np.inf
        for sx in S[l, 0] + grid:
            for sy in S[l, 1] + grid:
                off = E @ np.array([sx, sy])
                J = np.mean((Qf - Vl - off[:, None]) ** 2)
                if J < best:
                    best, arg = J, (sx, sy)
        assert best >= DT[l] - 1e-15
        assert abs(best - DT[l]) < 1e-6
        assert np.hypot(arg[0] - S[l, 0], arg[1] - S[l, 1]) <= h / 16 * 1.5


def test_shift_theorem_p2_on_analytic_gaussians():
    # Theorem 3.2 at p = 2: d_SW2^2(f, T_s f) = Gamma(3/2)/(sqrt(pi) Gamma(2))
    # |s|^2 = |s|^2 / 2.  The uniform angle grid averages <s, e_k>^2 to
    # exactly |s|^2 / 2 for n >= 3, so the only error is the histogram's.
    rng = np.random.default_rng(9)
    n, M, B, h = 64, 256, 364, 2 / 256
    th = 2 * np.pi * np.arange(n) / n
    mix = analytic.random_mixture(rng, 2)
    s = np.array([0.11, -0.07])
    Qf = oracle.quantiles(analytic.mixture_hist(*mix, th, B, h), h, M)
    Qg = oracle.quantiles(analytic.mixture_hist(*analytic.transform_mixture(mix, shift=s),
                                                th, B, h), h, M)
    const = math.gamma(1.5) / (math.sqrt(math.pi) * math.gamma(2.0))
    assert const == pytest.approx(0.5)
    D0 = oracle.rotation_curve(Qf, Qg)
    assert D0[0] == pytest.approx(const * (s @ s), rel=2e-3)
    af, Qfc = oracle.center(Qf)
    ag, Qgc = oracle.center(Qg)
    np.testing.assert_allclose(af - ag, -s, atol=h / M)  # s* = a_f - a_g = -s
    DT = oracle.rotation_curve(Qfc, Qgc)
    assert DT[0] < 1e-6


def test_sw2_of_anisotropic_gaussians_matches_angle_average():
    # Per angle, W2^2 = (<dmu, e>)^2 + (sqrt(e^T S1 e) - sqrt(e^T S2 e))^2; the
    # discrete SW2 is the mean over the n grid angles (Eq. discrete_sw2).
    n, M, B, h = 48, 512, 364, 2 / 256
    th = 2 * np.pi * np.arange(n) / n
    R = analytic.rot(0.6)
    S1 = R @ np.diag([0.09 ** 2, 0.04 ** 2]) @ R.T
    S2 = np.diag([0.05 ** 2, 0.07 ** 2])
    mu1, mu2 = np.array([0.1, 0.05]), np.array([-0.08, 0.02])
    Qa = oracle.quantiles(analytic.mixture_hist([1.0], [mu1], [S1], th, B, h), h, M)
    Qb = oracle.quantiles(analytic.mixture_hist([1.0], [mu2], [S2], th, B, h), h, M)
    E = np.stack([np.cos(th), np.sin(th)], axis=1)
    per = (E @ (mu1 - mu2)) ** 2 + (np.sqrt(np.einsum("ki,ij,kj->k", E, S1, E))
                                    - np.sqrt(np.einsum("ki,ij,kj->k", E, S2, E))) ** 2
    D0 = oracle.rotation_curve(Qa, Qb)
    assert D0[0] == pytest.approx(per.mean(), rel=2e-3)


def test_fig2_distance_grows_with_shift_and_minimum_at_half_turn():
    # Fig. 2: an 85 x 85 Gaussian blob shifted right by 0..20 pixels; the
    # rotation-only distance grows in proportion to the shift (d = |s|/sqrt 2),
    # and the shifted copy turned by 180 degrees is found at 180 degrees.
    L, n, M = 85, 84, 64
    h = 2.0 / L
    blob = ([1.0], [np.array([-0.2, 0.05])], [np.diag([0.10 ** 2, 0.06 ** 2])])
    f = analytic.pixel_image(blob, L)
    ratios = []
    for px in (4, 8, 12, 16, 20):
        g = np.zeros_like(f)
        g[:, px:] = f[:, :-px]  # shift right by px cells
        res, D0, _ = oracle.align_pair(f, g, n, M, translation=0)
        ratios.append(math.sqrt(D0[0]) / (px * h))
    np.testing.assert_allclose(ratios, 1 / math.sqrt(2), rtol=1e-2)
    # A lone ellipse is symmetric under a half turn; add a second, smaller
    # blob so that the half turn is the unique optimum.
    f2 = f + analytic.pixel_image(([0.4], [np.array([-0.35, 0.3])],
                                   [np.diag([0.05 ** 2, 0.03 ** 2])]), L)
    g = np.zeros_like(f2)
    g[:, 20:] = f2[:, :-20]
    g = g[::-1, ::-1]
    res, DT, S = oracle.align_pair(f2, g, n, M, translation=1)
    # A pixel shift is a shift of the splatted projection only up to the
    # splat's interpolation, so D_T(n/2) is small but not zero.
    assert res["best_l"] == n // 2
    assert res["d2"] < 1e-3 * np.median(DT)
    np.testing.assert_allclose(res["shift"], [-20 * h, 0.0], atol=h / 20)


def test_unusable_images_get_status():
    L, n, M = 8, 8, 4
    good = np.ones((L, L))
    res, D, _ = oracle.align_pair(np.zeros((L, L)), good, n, M)
    assert res["status"] == 1 and np.isnan(res["d2"])
    bad = good.copy(); bad[2, 3] = np.nan
    res, D, _ = oracle.align_pair(good, bad, n, M)
    assert res["status"] == 2
    res, D, _ = oracle.align_pair(good, -good, n, M)  # all mass clipped away
    assert res["status"] == 2


def test_all_pairs_matches_single_pairs():
    rng = np.random.default_rng(12)
    L, n, M = 16, 12, 6
    q = rng.random((3, L, L)) ** 2
    t = rng.random((2, L, L)) ** 2
    out = oracle.align_all_pairs(q, t, n, M, nthreads=3)
    for i in range(3):
        for j in range(2):
            r, _, _ = oracle.align_pair(q[i], t[j], n, M)
            assert out[i, j]["best_l"] == r["best_l"]
            assert out[i, j]["d2"] == r["d2"]
            np.testing.assert_array_equal(out[i, j]["shift"], r["shift"])


@pytest.mark.parametrize("projector", [0, 1])  # linear splat, Fourier slice
def test_theorem_2_1_discrete_distance_converges_at_first_order(projector):
    """Theorem 2.1: the discrete sliced W2 of L x L cell averages with n
    angles is within C (1/n + 1/L + eps) of the continuous distance.  Two
    isotropic Gaussians well inside the unit disk have d_SW2^2 = |dmu|^2 / 2 +
    (s1 - s2)^2 (their projections are N(<mu, e>, s^2), and the angle grid
    averages <dmu, e>^2 to |dmu|^2 / 2 exactly).  Exact cell averages at
    L = 16 .. 128 with n = M = L (the paper's setting): the error falls at
    least like 1/L (error x L does not grow) and below 0.1% at L = 128."""
    from scipy.special import ndtr

    def cells(mu, s, L):
        e = -1.0 + np.arange(L + 1) * (2.0 / L)
        px = np.diff(ndtr((e - mu[0]) / s))
        py = np.diff(ndtr((e - mu[1]) / s))
        return np.outer(py, px) / (2.0 / L) ** 2  # rows follow y, columns x

    mu1, s1 = np.array([0.12, -0.05]), 0.14
    mu2, s2 = np.array([-0.06, 0.09]), 0.10
    d = mu1 - mu2
    exact = 0.5 * (d @ d) + (s1 - s2) ** 2
    sizes = (16, 32, 64, 128)
    errs = []
    for L in sizes:
        _, D, _ = oracle.align_pair(cells(mu1, s1, L), cells(mu2, s2, L), L, L, translation=0,
                                    projector=projector)
        errs.append(abs(D[0] - exact))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    scaled = [e * L for e, L in zip(errs, sizes)]
    assert max(scaled) <= 1.1 * scaled[0], scaled
    assert errs[-1] < 1e-3 * exact
