"""The seeded input recipes of the workloads (no GPU): every image is
nonnegative with unit mass; shifts, sizes and request mixes follow the stated
ranges and weights; the 2 x 2 upsampling is exact under the cell-average model;
the same seed gives the same inputs."""
import numpy as np

from paper_2503_13756_gb300 import synth


def unit_mass(imgs):
    imgs = np.asarray(imgs, dtype=np.float64)
    assert np.all(imgs >= 0)
    np.testing.assert_allclose(imgs.reshape(-1, imgs.shape[-1] ** 2).sum(axis=1), 1.0, rtol=1e-5)


def test_single_pair_recipe():
    d = synth.single_pair()
    assert d["f"].shape == d["g"].shape == (64, 64) and d["f"].dtype == np.float64
    unit_mass(np.stack([d["f"], d["g"]]))
    assert np.all(np.abs(d["shift"]) <= 4) and np.all(d["shift"] == np.rint(d["shift"]))
    assert 0.0 <= d["beta"] < 2 * np.pi
    # a rotated, shifted, warped and noisy copy: close to the reference but not equal
    assert 0 < np.abs(d["f"] - d["g"]).sum() < 2.0


def test_many_to_many_recipe():
    d = synth.many_to_many(n_queries=40, n_templates=8, L=64)
    assert d["queries"].shape == (40, 64, 64) and d["templates"].shape == (8, 64, 64)
    unit_mass(d["queries"])
    unit_mass(d["templates"])
    assert np.all((0 <= d["source"]) & (d["source"] < 8))
    assert np.all(np.abs(d["shift"]) <= 8)


def test_uneven_batch_size_mix_and_shift_scaling():
    d = synth.uneven_batch(n_queries=3000, n_templates_per_L=2)
    counts = np.array([len(d[L]["queries"]) for L in synth.UNEVEN_SIZES])
    assert counts.sum() == 3000
    p = np.array(synth.UNEVEN_WEIGHTS)
    sigma = np.sqrt(3000 * p * (1 - p))
    assert np.all(np.abs(counts - 3000 * p) <= 4 * sigma), counts
    for L in synth.UNEVEN_SIZES:
        b = d[L]
        assert b["queries"].shape[1:] == (L, L) and b["templates"].shape == (2, L, L)
        assert np.all(np.abs(b["shift"]) <= 8 * L // 128)
        unit_mass(b["templates"])
        if len(b["queries"]):
            unit_mass(b["queries"][:20])


def test_upsampling_is_exact_for_cell_averages():
    rng = np.random.default_rng(2)
    img = rng.random((2, 16, 16))
    up = synth.upsample2(img)
    assert up.shape == (2, 32, 32)
    # each coarse cell is the sum of its 4 fine cells (mass per cell kept)
    np.testing.assert_allclose(up.reshape(2, 16, 2, 16, 2).sum(axis=(2, 4)), img, rtol=1e-12)


def test_serving_schedule_is_poisson_with_log_uniform_counts():
    n = 4000
    t, counts, Ls, picks = synth.serving_schedule(n, rate_hz=200.0, max_images=512, Lb=256)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 200.0) < 4 * (1 / 200.0) / np.sqrt(n)  # exponential: std = mean
    assert counts.min() >= 1 and counts.max() <= 512
    # log-uniform on [1, 512]: the median is sqrt(512) ~ 22.6
    assert 18 <= np.median(counts) <= 28
    assert set(np.unique(Ls)) == {128, 256} and abs((Ls == 256).mean() - 0.5) < 0.05
    assert all(len(pk) == c for pk, c in zip(picks, counts))


def test_random_dense_is_uniform_with_unit_mass():
    x = synth.random_dense(32, count=3)
    unit_mass(x)
    # U[0, 1) pixels normalised by their sum: the mean pixel is 1 / L^2 and
    # the values spread over (0, 2 / L^2)
    assert x.max() < 2.2 / 32 ** 2 and x.min() >= 0


def test_same_seed_same_inputs():
    a = synth.many_to_many(n_queries=6, n_templates=3, L=32)
    b = synth.many_to_many(n_queries=6, n_templates=3, L=32)
    for k in ("queries", "templates", "source", "beta", "shift"):
        np.testing.assert_array_equal(a[k], b[k])
