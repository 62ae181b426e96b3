"""Pins for the oracle's Fourier-slice projector (Sec. 2.1 Eq. 1d_ift,
Sec. 2.3 "Computation", Theorem proj_nufft in App. A).

``oracle.project_slice`` sums the slice samples of the cell image and the
band-limited projection straight from their definitions.  It is pinned
against things other than itself:
- exact invariants: mass, the theta + pi mirror, quarter turns of the cell
  grid;
- a special case that reduces to numpy's FFT: at theta = 0 and pi/2 the slice
  samples are the DFT of the column (row) sums times sinc(pi j / B);
- the paper's error bound (Theorem proj_nufft, exact samples) on a Gaussian
  whose projections are known in closed form, and the second-order
  convergence to them (a half-cell offset or a wrong sinc would leave first
  order);
- the whole pipeline with this projector: an exact quarter turn is found at
  distance zero.
"""
import numpy as np
import pytest

import oracle

scipy_special = pytest.importorskip("scipy.special")


def random_image(rng, L):
    F = rng.random((L, L)) ** 3
    return F / F.sum()


def cell_gaussian(L, mu, sig):
    """Cell masses of the isotropic Gaussian N(mu, sig^2 I): products of
    normal CDF differences over the cell edges (exact)."""
    h = 2.0 / L
    e = -1.0 + np.arange(L + 1) * h
    ndtr = scipy_special.ndtr
    px = np.diff(ndtr((e - mu[0]) / sig))
    py = np.diff(ndtr((e - mu[1]) / sig))
    return np.outer(py, px)  # [row r: y][column c: x]


@pytest.mark.parametrize("L,n", [(16, 12), (33, 20), (40, 8)])
def test_slice_rows_keep_the_mass_exactly(L, n):
    F = random_image(np.random.default_rng(L), L)
    U = oracle.project_slice(F, n)
    assert U.shape == (n, oracle.bins_for(L, projector=1))
    np.testing.assert_allclose(U.sum(axis=1), 1.0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("L,B", [(32, 32), (32, 48), (24, 40)])
def test_axis_angles_reduce_to_an_fft_filter(L, B):
    # At theta = 0 the slice sample at omega_j = 2 pi j / (B h) is
    # sinc(pi j / B) times the DFT of the column sums placed on the bin grid
    # (cell centre x_c is bin centre s_{c + (B-L)/2}), so
    #   U[0] = Re ifft( fft(z) * sinc(j / B) ),  j = -B/2 .. B/2-1 (np.sinc).
    # At theta = pi/2 the same holds with the row sums.
    F = random_image(np.random.default_rng(B + L), L)
    n = 8
    U = oracle.project_slice(F, n, B)
    j = np.fft.fftfreq(B, 1.0 / B)
    for k, sums in ((0, F.sum(axis=0)), (n // 4, F.sum(axis=1))):
        z = np.zeros(B)
        z[(B - L) // 2:(B - L) // 2 + L] = sums
        ref = np.fft.ifft(np.fft.fft(z) * np.sinc(j / B)).real
        np.testing.assert_allclose(U[k], ref, rtol=0, atol=1e-14)


def test_mirror_and_quarter_turn():
    rng = np.random.default_rng(5)
    L, n = 20, 16
    F = random_image(rng, L)
    U = oracle.project_slice(F, n)
    for k in range(n // 2):  # P_{theta+pi} f(s) = P_theta f(-s), computed independently
        np.testing.assert_allclose(U[k + n // 2], U[k][::-1], rtol=0, atol=1e-14)
    # g = R_{90 deg} f on the cell grid: G[r][c] = F[L-1-c][r]
    G = np.empty_like(F)
    for r in range(L):
        for c in range(L):
            G[r, c] = F[L - 1 - c, r]
    V = oracle.project_slice(G, n)
    for k in range(n):  # P_theta(R_alpha f) = P_{theta - alpha} f
        np.testing.assert_allclose(V[k], U[(k - n // 4) % n], rtol=0, atol=1e-14)


def test_theorem_bound_and_second_order_convergence_on_a_gaussian():
    # f = N(mu, sig^2 I): P_theta f = N(<mu, e>, sig^2); Lipschitz constant
    # K = max |grad f| = e^{-1/2} / (2 pi sig^3).  Theorem proj_nufft with
    # exact samples bounds the L2(-1, 1) error by 4 sqrt(2/pi) K / L.  The
    # norm is taken by the midpoint rule on the bin centres inside (-1, 1).
    mu, sig = np.array([0.1, -0.05]), 0.12
    K = np.exp(-0.5) / (2 * np.pi * sig ** 3)
    n = 8
    errs = []
    for L in (32, 64, 128):
        F = cell_gaussian(L, mu, sig)
        F /= F.sum()
        U = oracle.project_slice(F, n)
        B = U.shape[1]
        h = 2.0 / L
        s = (np.arange(B) - (B - 1) / 2) * h
        inside = np.abs(s) < 1.0
        worst = 0.0
        for k in range(n):
            t = 2 * np.pi * k / n
            m = mu @ np.array([np.cos(t), np.sin(t)])
            Pf = np.exp(-0.5 * ((s - m) / sig) ** 2) / (sig * np.sqrt(2 * np.pi))
            worst = max(worst, np.sqrt(h * np.sum((U[k] / h - Pf)[inside] ** 2)))
        assert worst <= 4 * np.sqrt(2 / np.pi) * K / L
        errs.append(worst)
    # halving h divides the error by ~4 (measured 3.93, 3.98); first order gives 2
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


@pytest.mark.parametrize("translation", [1, 0])
def test_quarter_turn_is_found_at_zero_distance(translation):
    rng = np.random.default_rng(11)
    L, n, M = 24, 16, 20
    F = random_image(rng, L)
    G = np.empty_like(F)
    for r in range(L):
        for c in range(L):
            G[r, c] = F[L - 1 - c, r]  # g = R_{90} f
    # g rotated by alpha aligns onto f at alpha = -90 degrees: l* = 3n/4
    res, D, S = oracle.align_pair(F, G, n, M, translation=translation, projector=1)
    assert res["status"] == 0
    assert res["best_l"] == 3 * n // 4
    assert abs(res["d2"]) < 1e-12
    assert D.min() == D[3 * n // 4]


def test_clipping_is_applied_for_sliced_w2_only():
    # A single bright cell rings: the band-limited rows go negative.  Sliced
    # W2 clips them (the quantiles see max(U, 0)); the ramp-filtered path
    # splits the signed rows itself.  Both pipelines accept the image.
    L, n, M = 16, 8, 12
    F = np.zeros((L, L))
    F[5, 9] = 1.0
    U = oracle.project_slice(F, n)
    assert U.min() < -1e-3
    G = np.roll(F, 1, axis=1)
    r0, _, _ = oracle.align_pair(F, G, n, M, projector=1)
    r1, _, _ = oracle.align_pair_rfsw(F, G, n, M, projector=1)
    assert r0["status"] == 0 and r1["status"] == 0
    Qp = oracle.quantiles(np.maximum(U, 0.0), 2.0 / L, M)
    assert np.all(np.isfinite(Qp))


@pytest.mark.parametrize("projector", [0, 1])
def test_transform_images_are_the_steps_of_align_pair(projector):
    # The batched per-image transform (used by the GPU tests to score many
    # pairs cheaply) is the same prepare / project / quantile / centre chain
    # as align_pair: its curve and shifts reproduce align_pair's exactly,
    # and an unusable image is reported.
    rng = np.random.default_rng(23 + projector)
    L, n, M = 20, 12, 9
    imgs = np.stack([random_image(rng, L) for _ in range(3)] + [np.zeros((L, L))])
    Q, A, ok = oracle.transform_images(imgs, n, M, projector=projector, nthreads=2)
    assert list(ok) == [True, True, True, False]
    for i, j in ((0, 1), (2, 0)):
        res, D, S = oracle.align_pair(imgs[i], imgs[j], n, M, projector=projector)
        _, Qci = oracle.center(Q[i])
        _, Qcj = oracle.center(Q[j])
        np.testing.assert_array_equal(oracle.rotation_curve(Qci, Qcj), D)
        np.testing.assert_allclose(oracle.shifts_of(A[i], A[j], n), S, rtol=0, atol=1e-15)
        res0, D0, _ = oracle.align_pair(imgs[i], imgs[j], n, M, translation=0,
                                        projector=projector)
        np.testing.assert_array_equal(oracle.rotation_curve(Q[i], Q[j]), D0)
