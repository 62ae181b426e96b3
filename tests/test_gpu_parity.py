"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every comparison feeds both sides the same FP32 image values (the oracle gets
them converted exactly to float64), so that only the arithmetic differs.
Tolerances are explained in tests/parity.py.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign, synth
from tests.parity import REL_FP32, check_argmin, d2_tol, norm_scale, q_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def al():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = swalign.Aligner(0)
    yield a
    a.close()


def f32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def blobs(rng, count, L, ncomp=(2, 4)):
    p = synth.draw_mixtures(rng, count, L, ncomp=ncomp)
    return synth.render(p, L)


# ------------------------------------------------------------- projection

@pytest.mark.parametrize("L,n", [(16, 8), (33, 36), (64, 60), (128, 256), (200, 24),  # 4 angles/weight
                                 (231, 40), (256, 16), (300, 12),                   # two row bands
                                 (48, 30), (130, 18), (400, 8)])                    # generic, tiled
def test_project_matches_oracle(al, L, n):
    rng = np.random.default_rng(L * 1000 + n)
    imgs = blobs(rng, 3, L)
    imgs[1] -= 0.3 * imgs[1].max()  # negative pixels are clipped to 0
    imgs = f32(imgs)
    p = swalign.make_params(L, n, 8)
    got = al.project(imgs, p).cpu().numpy().astype(np.float64)
    for i in range(3):
        ref = oracle.project(np.maximum(imgs[i].astype(np.float64), 0.0), n)
        assert got[i].shape == ref.shape
        peak = ref.max()
        err = np.abs(got[i] - ref).max()
        assert err <= 5e-5 * peak, (i, err, peak)
        np.testing.assert_allclose(got[i].sum(axis=1), ref.sum(axis=1), rtol=2e-6)


@pytest.mark.parametrize("projector", ["splat", "slice"])
def test_project_scale_is_the_inverse_clipped_mass(al, projector):
    # ingest (a1): d_scale = 1 / sum max(pixel, 0) in FP64, NaN for an image
    # with no positive mass or a non-finite pixel
    rng = np.random.default_rng(77)
    L, n = 48, 12
    imgs = blobs(rng, 4, L)
    imgs[1] -= 0.3 * imgs[1].max()
    imgs[2] = -1.0
    imgs[3, 5, 7] = np.inf
    imgs = f32(imgs)
    p = swalign.make_params(L, n, 8, projector=projector)
    rows, scale = al.project(imgs, p, scale=True)
    scale = scale.cpu().numpy()
    for i in range(2):
        _, mass = oracle.prepare(imgs[i].astype(np.float64))
        assert scale[i] == pytest.approx(1.0 / mass, rel=1e-13)
        if projector == "splat":  # the splat keeps the mass exactly (the slice's
            # band-limited rows are clipped at zero, which adds the ringing's mass)
            np.testing.assert_allclose(rows[i].cpu().numpy().astype(np.float64).sum(axis=1)
                                       * scale[i], 1.0, rtol=2e-6)
    assert np.isnan(scale[2]) and np.isnan(scale[3])


# -------------------------------------------------------------- quantiles

@pytest.mark.parametrize("level_rule", [0, 1])
@pytest.mark.parametrize("L,n,M", [(16, 8, 5), (64, 36, 128), (128, 256, 128), (96, 60, 96)])
def test_quantiles_match_oracle(al, L, n, M, level_rule):
    rng = np.random.default_rng(7 + L + n + M)
    imgs = blobs(rng, 2, L)
    U = np.stack([oracle.project(im.astype(np.float64), n) for im in imgs])
    U32 = f32(U)
    p = swalign.make_params(L, n, M, level_rule=level_rule)
    q, center, norm = al.quantiles(U32, p)
    q, center, norm = q.cpu().numpy(), center.cpu().numpy(), norm.cpu().numpy()
    h = 2.0 / L
    for i in range(2):
        ref = oracle.quantiles(U32[i].astype(np.float64), h, M, level_rule)
        err = np.abs(q[i] - ref)
        assert np.all(err <= q_tol(ref)), (err / q_tol(ref)).max()
        a, Qc = oracle.center(q[i].astype(np.float64))
        np.testing.assert_allclose(center[i], a, rtol=0, atol=1e-12)
        np.testing.assert_allclose(norm[i], (Qc ** 2).sum(), rtol=1e-10)


# ---------------------------------------------------- single pair, full curve

@pytest.mark.parametrize("translation", [1, 0])
def test_single_pair_curve_matches_oracle(al, translation):
    d = synth.single_pair()  # 64 x 64, n = 360, M = 128
    f, g = f32(d["f"]), f32(d["g"])
    n, M = 360, 128
    p = swalign.make_params(64, n, M, translation=translation)
    D, S, best = al.align_all_rotations(f, g, p)
    D, S = D.cpu().numpy(), S.cpu().numpy()
    r = swalign.results_to_numpy(best)[0]
    ref, Dref, Sref = oracle.align_pair(f.astype(np.float64), g.astype(np.float64), n, M,
                                        translation=translation)
    Sc = norm_scale(f.astype(np.float64), g.astype(np.float64), n, M)
    tol = d2_tol(Dref, Sc)
    assert np.all(np.abs(D - Dref) <= tol), np.max(np.abs(D - Dref) / tol)
    np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-6)
    assert r["status"] == 0
    assert check_argmin(int(r["best_l"]), ref["best_l"], Dref, d2_tol(ref["d2"], Sc))
    assert abs(r["d2"] - Dref[r["best_l"]]) <= d2_tol(Dref[r["best_l"]], Sc)
    assert r["angle_rad"] == pytest.approx(2 * np.pi * r["best_l"] / n, rel=1e-6)


# ------------------------------------------------------------- many pairs

def compare_batch(al, q, t, n, M, translation=1, level_rule=0, n_bins=0, rel=REL_FP32,
                  precision="fp32"):
    L = q.shape[-1]
    p = swalign.make_params(L, n, M, n_bins=n_bins, translation=translation,
                            level_rule=level_rule, precision=precision)
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    B = n_bins or None
    ref = oracle.align_all_pairs(q.astype(np.float64), t.astype(np.float64), n, M, B=B,
                                 level_rule=level_rule, translation=translation)
    worst = 0.0
    for i in range(len(q)):
        for j in range(len(t)):
            gr, rr = got[i, j], ref[i, j]
            assert gr["status"] == rr["status"] == 0
            _, Dref, Sref = oracle.align_pair(q[i].astype(np.float64), t[j].astype(np.float64),
                                              n, M, B=B, level_rule=level_rule,
                                              translation=translation)
            Sc = norm_scale(q[i].astype(np.float64), t[j].astype(np.float64), n, M, level_rule)
            l = int(gr["best_l"])
            tol = d2_tol(rr["d2"], Sc, rel)
            assert check_argmin(l, int(rr["best_l"]), Dref, tol), (i, j, l, rr["best_l"])
            err = abs(gr["d2"] - Dref[l])
            assert err <= d2_tol(Dref[l], Sc, rel), (i, j, err, Dref[l], Sc)
            worst = max(worst, err / d2_tol(Dref[l], Sc, rel))
            np.testing.assert_allclose(gr["shift"], Sref[l], rtol=0, atol=1e-6)
    return worst


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_batch_ragged_tiles_match_oracle(al, precision):
    # FP32-accurate correlation on tcgen05 (FP16 split) and on the CUDA cores
    rng = np.random.default_rng(31)
    q = f32(blobs(rng, 5, 48))
    t = f32(blobs(rng, 70, 48))  # ragged against the 64-wide and 128-row tiles
    compare_batch(al, q, t, n=60, M=36, precision=precision)


@pytest.mark.parametrize("case", [
    dict(L=33, n=12, M=7, translation=1, level_rule=0, n_bins=0),
    dict(L=20, n=4, M=1, translation=1, level_rule=0, n_bins=0),
    dict(L=24, n=40, M=9, translation=0, level_rule=1, n_bins=0),
    dict(L=32, n=30, M=16, translation=1, level_rule=0, n_bins=60),
])
@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_batch_edge_parameters(al, case, precision):
    rng = np.random.default_rng(case["n"] * 7 + case["M"])
    case = dict(case)
    L = case.pop("L")
    q = f32(blobs(rng, 3, L))
    t = f32(blobs(rng, 4, L))
    compare_batch(al, q, t, precision=precision, **case)


def test_quarter_turn_is_exact(al):
    rng = np.random.default_rng(5)
    L, n, M = 64, 64, 32
    f = f32(blobs(rng, 1, L, ncomp=(3, 3))[0])
    g = np.ascontiguousarray(np.rot90(f, k=-1))  # g[r][c] = f[L-1-c][r]: g = R_{+90} f
    for r_ in range(L):
        for c_ in range(0, L, 17):
            assert g[r_, c_] == f[L - 1 - c_, r_]
    p = swalign.make_params(L, n, M)
    D, S, best = al.align_all_rotations(f, g, p)
    r = swalign.results_to_numpy(best)[0]
    assert r["best_l"] == 3 * n // 4
    Sc = norm_scale(f.astype(np.float64), g.astype(np.float64), n, M)
    assert abs(r["d2"]) <= d2_tol(0.0, Sc)  # exact in exact arithmetic
    np.testing.assert_allclose(r["shift"], 0.0, atol=1e-6)


@pytest.mark.parametrize("L", [16, 256])  # whole image in shared memory; two row bands
def test_status_flags(al, L):
    n, M = 8, 4
    rng = np.random.default_rng(1)
    good = f32(blobs(rng, 2, L))
    zero = np.zeros((L, L), np.float32)
    nan = good[0].copy()
    nan[L - 3, 4] = np.nan  # in the second band at L = 256
    neg = -good[1]
    q = f32(np.stack([good[0], zero, nan]))
    t = f32(np.stack([good[1], neg]))
    p = swalign.make_params(L, n, M)
    r = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(3, 2)
    assert r[0, 0]["status"] == 0 and np.isfinite(r[0, 0]["d2"])
    assert r[0, 1]["status"] == 2 and np.isnan(r[0, 1]["d2"])
    assert r[1, 0]["status"] == 1 and r[2, 0]["status"] == 1
    assert r[1, 1]["status"] == 1  # the query is reported first


def test_best_template_mode(al):
    rng = np.random.default_rng(77)
    L, n, M = 32, 24, 16
    q = f32(blobs(rng, 6, L))
    t = f32(blobs(rng, 40, L))
    p = swalign.make_params(L, n, M)
    allr = swalign.results_to_numpy(al.align_batch(q, t, p, mode=0)).reshape(6, 40)
    best = swalign.results_to_numpy(al.align_batch(q, t, p, mode=1))
    for i in range(6):
        j = int(np.argmin(allr[i]["d2"]))
        assert int(best[i]["template_index"]) == j
        assert best[i]["d2"] == allr[i, j]["d2"]
        assert best[i]["best_l"] == allr[i, j]["best_l"]


def test_pair_alone_equals_pair_in_batch(al):
    # Run to run the same batch is bitwise identical (no atomics, fixed
    # reduction orders).  A pair alone and in a batch agree within the parity
    # tolerance: the decision FFT packs two pairs per complex signal, so the
    # rounding of one depends on its partner.
    rng = np.random.default_rng(8)
    L, n, M = 64, 72, 32
    q = f32(blobs(rng, 9, L))
    t = f32(blobs(rng, 11, L))
    p = swalign.make_params(L, n, M)
    big = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(9, 11)
    again = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(9, 11)
    assert big.tobytes() == again.tobytes()
    for (i, j) in [(0, 0), (4, 7), (8, 10)]:
        one = swalign.results_to_numpy(al.align_batch(q[i:i + 1], t[j:j + 1], p))[0]
        _, Dref, _ = oracle.align_pair(q[i].astype(np.float64), t[j].astype(np.float64), n, M)
        Sc = norm_scale(q[i].astype(np.float64), t[j].astype(np.float64), n, M)
        tol = d2_tol(Dref[int(big[i, j]["best_l"])], Sc)
        assert check_argmin(int(one["best_l"]), int(big[i, j]["best_l"]), Dref, tol)
        assert abs(one["d2"] - big[i, j]["d2"]) <= 2 * tol


def test_invalid_arguments_are_rejected(al):
    x = torch.zeros((2, 16, 16), device="cuda")
    for bad in (swalign.make_params(16, 9, 4), swalign.make_params(16, 14, 4),
                swalign.make_params(600, 8, 4), swalign.make_params(16, 8, 0),
                swalign.make_params(16, 8, 4, n_bins=3), swalign.make_params(16, 8, 4, translation=2)):
        with pytest.raises(swalign.SwError) as e:
            al.project(x, bad)
        assert e.value.status == swalign.SW_ERR_INVALID_ARG
    p = swalign.make_params(16, 8, 4)
    buf = torch.zeros(2 * 16 * 16 + 1, device="cuda")
    out = torch.zeros((2, 8, p.n_bins or al.default_bins(16)), device="cuda")
    with pytest.raises(swalign.SwError) as e:  # misaligned image pointer
        al.call("sw_project", ctypes.byref(p), ctypes.c_void_p(buf.data_ptr() + 4), 2,
                ctypes.c_void_p(out.data_ptr()), None, ctypes.c_void_p(0))
    assert e.value.status == swalign.SW_ERR_INVALID_ARG


def test_workspace_limit_gives_oom_without_launch(al):
    rng = np.random.default_rng(2)
    q = f32(blobs(rng, 4, 32))
    p = swalign.make_params(32, 16, 8)
    al2 = swalign.Aligner(0)
    try:
        al2.set_workspace_limit(1024)
        out = torch.full((16, 40), 7, dtype=torch.uint8, device="cuda")
        with pytest.raises(swalign.SwError) as e:
            al2.align_batch(q, q, p, out=out)
        assert e.value.status == swalign.SW_ERR_OOM
        torch.cuda.synchronize()
        assert bool((out == 7).all())  # nothing ran
        al2.set_workspace_limit(0)
        r = swalign.results_to_numpy(al2.align_batch(q, q, p)).reshape(4, 4)
        assert np.all(r["status"] == 0)
    finally:
        al2.close()


# ----------------------------------------- full many-to-many size, sampled

def test_many_to_many_full_size_sampled(al):
    """4096 queries x 256 templates, 128 x 128, n = 256, M = 128, in the
    launch configuration of the benchmark; 40 sampled pairs against the
    oracle, and every query's own template found at its rotation."""
    d = synth.many_to_many()
    q, t = d["queries"], d["templates"]
    n, M = 256, 128
    p = swalign.make_params(128, n, M)
    res = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    assert np.all(res["status"] == 0)
    rng = np.random.default_rng(99)
    picks = [(int(i), int(d["source"][i])) for i in rng.integers(0, len(q), 20)]
    picks += [(int(i), int(j)) for i, j in zip(rng.integers(0, len(q), 20),
                                                rng.integers(0, len(t), 20))]
    for i, j in picks:
        fq, ft = q[i].astype(np.float64), t[j].astype(np.float64)
        rr, Dref, Sref = oracle.align_pair(fq, ft, n, M)
        Sc = norm_scale(fq, ft, n, M)
        gr = res[i, j]
        l = int(gr["best_l"])
        assert check_argmin(l, rr["best_l"], Dref, d2_tol(rr["d2"], Sc))
        assert abs(gr["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc)
    # property at full size: the query's own template is the best match for
    # nearly all queries, and its rotation matches the generated angle
    best_j = np.argmin(res["d2"], axis=1)
    assert np.mean(best_j == d["source"]) > 0.95
    own = res[np.arange(len(q)), d["source"]]
    l_true = np.round(d["beta"] * n / (2 * np.pi)) % n
    dl = np.abs(((own["best_l"] - l_true) + n / 2) % n - n / 2)
    assert np.mean(dl <= 3) > 0.95


def test_one_reference_full_size_sampled(al):
    """10,000 queries x 1 reference, 128 x 128, n = 512, M = 256, FP32:
    20 sampled queries against the oracle, and the generated rotation found
    for nearly all queries."""
    d = synth.one_reference_batch()
    q, ref = d["queries"], d["reference"]
    n, M = 512, 256
    p = swalign.make_params(128, n, M)
    res = swalign.results_to_numpy(al.align_batch(q, ref, p)).reshape(len(q))
    assert np.all(res["status"] == 0)
    fr = ref[0].astype(np.float64)
    for i in np.random.default_rng(11).integers(0, len(q), 20):
        fq = q[i].astype(np.float64)
        rr, Dref, Sref = oracle.align_pair(fq, fr, n, M)
        Sc = norm_scale(fq, fr, n, M)
        gr = res[i]
        l = int(gr["best_l"])
        assert check_argmin(l, rr["best_l"], Dref, d2_tol(rr["d2"], Sc)), (i, l, rr["best_l"])
        assert abs(gr["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc)
        np.testing.assert_allclose(gr["shift"], Sref[l], rtol=0, atol=1e-6)
    l_true = np.round(d["beta"] * n / (2 * np.pi)) % n
    dl = np.abs(((res["best_l"] - l_true) + n / 2) % n - n / 2)
    assert np.mean(dl <= 3) > 0.95


# ------------------------------------------------ empty batches, maximum sizes

def test_empty_batches_launch_nothing(al):
    p = swalign.make_params(16, 8, 4)
    x = torch.zeros((3, 16, 16), device="cuda")
    empty = torch.zeros((0, 16, 16), device="cuda")
    out = torch.zeros((1, 40), dtype=torch.uint8, device="cuda")
    n0 = al.launch_count()
    al.align_batch(empty, x, p, out=out)       # no queries
    al.align_batch(x, empty, p, out=out)       # no templates, all-pairs mode
    al.project(empty, p)
    assert al.launch_count() == n0
    with pytest.raises(swalign.SwError) as e:  # best template of nothing
        al.align_batch(x, empty, p, mode=1, out=out)
    assert e.value.status == swalign.SW_ERR_INVALID_ARG


def test_maximum_sizes_match_oracle(al):
    """L = 512, n = 1024, M = 1024 (the limits of sw_params): one pair on the
    CUDA-core path (sw_align_all_rotations, full curve) and on the tensor-core
    FP32 split path (sw_align_batch)."""
    rng = np.random.default_rng(512)
    L, n, M = 512, 1024, 1024
    f, g = f32(blobs(rng, 2, L))
    p = swalign.make_params(L, n, M)
    D, S, best = al.align_all_rotations(f, g, p)
    D = D.cpu().numpy()
    ref, Dref, Sref = oracle.align_pair(f.astype(np.float64), g.astype(np.float64), n, M)
    Sc = norm_scale(f.astype(np.float64), g.astype(np.float64), n, M)
    assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc))
    np.testing.assert_allclose(S.cpu().numpy(), Sref, rtol=0, atol=1e-6)
    r = swalign.results_to_numpy(al.align_batch(f[None], g[None], p))[0]
    assert check_argmin(int(r["best_l"]), ref["best_l"], Dref, d2_tol(ref["d2"], Sc))
    assert abs(r["d2"] - Dref[int(r["best_l"])]) <= d2_tol(Dref[int(r["best_l"])], Sc)


def test_largest_banded_ramp_filtered_size(al):
    """L = 312, the largest image the four-view projection takes in two row
    bands, with the ramp filter on its 450-bin grid (radices 2, 3, 3, 5, 5)."""
    rng = np.random.default_rng(312)
    L, n, M = 312, 60, 32
    f, g = f32(blobs(rng, 2, L))
    p = swalign.make_params(L, n, M, metric="rfsw2")
    B = swalign.bins_of(p)
    assert B == oracle.rfsw_bins(L) == 450
    D, S, best = al.align_all_rotations(f, g, p)
    D = D.cpu().numpy()
    ref, Dref, _ = oracle.align_pair_rfsw(f.astype(np.float64), g.astype(np.float64), n, M, B=B)
    from tests.parity import norm_scale_rfsw
    Sc = norm_scale_rfsw(f.astype(np.float64), g.astype(np.float64), n, M, B)
    assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc))
