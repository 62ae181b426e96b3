"""The Fourier-slice projector (sw_params.projector = SW_PROJ_SLICE) on the
CUDA path against the FP64 oracle (Sec. 2.3, Theorem proj_nufft).

Three levels:
- rows: sw_project against oracle.project_slice, whose slice samples are
  exact sums.  Bar per row, relative l2: ROW_TOL = 2 eps_nufft + (3 ceil(log2
  B) + W^2) u, where eps_nufft = 3.5e-7 is this kernel's measured NUFFT error
  in FP64 (W = 9 taps, grid N = B >= 1.5 L; the oracle-side measurement that
  chose W), u = 2^-24, and the FP32 terms bound the three FFT passes and the
  W^2-term tap sums.  Clipping at zero is 1-Lipschitz, so the bar holds
  for clipped rows too.
- quantiles end to end, in CDF space: a GPU quantile q at level z must sit at
  F_ref(q) = z up to 2 sqrt(B) ROW_TOL |U_ref|_2 / sum U_ref (the row error
  moves the normalised CDF by at most twice its l1 norm) plus the quantile's
  own FP32 error.
- everything after the projection (quantiles, spectra, GEMM, decision) is
  the code the splat path uses; it is checked at the usual FP32 bar against
  the oracle run on the GPU's own rows (bitwise the rows the pipeline uses:
  the kernel is deterministic and per image).
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign, synth
from tests.parity import REL_FP32, REL_LP, check_argmin, d2_tol, level_of

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_NUFFT = 3.5e-7
KW = 9
U32 = 2.0 ** -24


def row_tol(L, B):
    # the oversampled grid has N = B points
    return 2 * EPS_NUFFT + (3 * math.ceil(math.log2(B)) + KW * KW) * U32


@pytest.fixture(scope="module")
def al():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = swalign.Aligner(0)
    yield a
    a.close()


def blobs(rng, count, L, ncomp=(2, 5)):
    p = synth.draw_mixtures(rng, count, L, ncomp=ncomp)
    return np.ascontiguousarray(synth.render(p, L), dtype=np.float32)


def params(L, n, M, **kw):
    return swalign.make_params(L, n, M, projector="slice", **kw)


def ref_rows(img, n, B, clip):
    F, _ = oracle.prepare(img.astype(np.float64))
    U = oracle.project_slice(F, n, B)
    return np.maximum(U, 0.0) if clip else U


# ------------------------------------------------------------------- rows

@pytest.mark.parametrize("L,n,metric", [(3, 4, "sw2"), (16, 8, "sw2"), (33, 20, "sw2"),
                                        (48, 60, "sw2"), (64, 36, "rfsw2"), (100, 24, "rfsw2"),
                                        (128, 256, "sw2"),
                                        # grids in global memory (B = 256, 320, 384)
                                        (129, 12, "sw2"), (160, 8, "rfsw2"), (192, 12, "sw2"),
                                        (256, 8, "sw2")])
def test_slice_rows_match_oracle(al, L, n, metric):
    rng = np.random.default_rng(L * 7 + n)
    imgs = blobs(rng, 2, L)
    imgs[1] -= 0.2 * imgs[1].max()  # negative pixels are clipped to 0 on load
    p = params(L, n, 8, metric=metric)
    B = swalign.bins_of(p)
    assert B == oracle.bins_for(L, projector=1)
    got = al.project(imgs, p).cpu().numpy().astype(np.float64)
    tol = row_tol(L, B)
    for i in range(len(imgs)):
        mass = np.maximum(imgs[i].astype(np.float64), 0).sum()
        ref = ref_rows(imgs[i], n, B, clip=metric != "rfsw2") * mass
        err = np.linalg.norm(got[i] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= tol, (i, err.max(), tol)
        # theta + pi rows are the exact mirrors
        np.testing.assert_array_equal(got[i, n // 2:], got[i, :n // 2, ::-1])
        if metric != "rfsw2":
            assert got[i].min() >= 0.0


@pytest.mark.parametrize("L,n,M,level_rule", [(48, 60, 36, 0), (64, 128, 64, 0),
                                              (33, 12, 7, 1), (128, 32, 128, 0)])
def test_slice_quantiles_in_cdf_space(al, L, n, M, level_rule):
    rng = np.random.default_rng(L + n + M)
    imgs = blobs(rng, 3, L)
    p = params(L, n, M, level_rule=level_rule)
    B = swalign.bins_of(p)
    Q, _, _ = al.quantiles(al.project(imgs, p), p)
    Q = Q.cpu().numpy().astype(np.float64)
    h = 2.0 / L
    z = (np.arange(M) + 0.5) / M if level_rule == 0 else np.arange(M) / M
    tol_row = row_tol(L, B)
    for i in range(len(imgs)):
        U = ref_rows(imgs[i], n, B, clip=True)
        for k in range(n):
            tol = 2 * math.sqrt(B) * tol_row * np.linalg.norm(U[k]) / U[k].sum() + 1e-6
            lev = level_of(Q[i, k], U[k], h)
            if level_rule == 1:
                lev[0] = 0.0  # level 0 is the domain's left end on both sides
            assert np.abs(lev - z).max() <= tol, (i, k, np.abs(lev - z).max(), tol)


# ----------------------------------------- the pipeline on the GPU's own rows

def curve_from_rows(Rf, Rg, h, M, translation, level_rule=0):
    Qf = oracle.quantiles(Rf, h, M, level_rule)
    Qg = oracle.quantiles(Rg, h, M, level_rule)
    af, Qcf = oracle.center(Qf)
    ag, Qcg = oracle.center(Qg)
    n = Qf.shape[0]
    Sc = ((Qcf ** 2).sum() + (Qcg ** 2).sum()) / (n * M)
    if translation:
        D = oracle.rotation_curve(Qcf, Qcg)
        ang = 2 * np.pi * np.arange(n) / n
        c, s = np.cos(ang), np.sin(ang)
        S = np.stack([af[0] - (c * ag[0] - s * ag[1]), af[1] - (s * ag[0] + c * ag[1])], axis=1)
    else:
        D = oracle.rotation_curve(Qf, Qg)
        S = np.zeros((n, 2))
    return D, S, Sc


@pytest.mark.parametrize("translation", [1, 0])
def test_slice_curve_on_gpu_rows(al, translation):
    rng = np.random.default_rng(41 + translation)
    L, n, M = 64, 120, 64
    f, g = blobs(rng, 2, L)
    p = params(L, n, M, translation=translation)
    rows = al.project(np.stack([f, g]), p).cpu().numpy().astype(np.float64)
    D, S, best = al.align_all_rotations(f, g, p)
    D, S = D.cpu().numpy(), S.cpu().numpy()
    Dref, Sref, Sc = curve_from_rows(rows[0], rows[1], 2.0 / L, M, translation)
    tol = d2_tol(Dref, Sc)
    assert np.all(np.abs(D - Dref) <= tol), np.max(np.abs(D - Dref) / tol)
    np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-6)
    r = swalign.results_to_numpy(best)[0]
    assert r["status"] == 0
    lref = int(np.argmin(Dref))
    assert check_argmin(int(r["best_l"]), lref, Dref, d2_tol(Dref[lref], Sc))


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt", "bf16"])
def test_slice_batch_on_gpu_rows(al, precision):
    rng = np.random.default_rng(53)
    L, n, M = 48, 60, 36
    q = blobs(rng, 5, L)
    t = blobs(rng, 9, L)
    p = params(L, n, M, precision=precision)
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    rq = al.project(q, p).cpu().numpy().astype(np.float64)
    rt = al.project(t, p).cpu().numpy().astype(np.float64)
    rel = REL_LP if precision == "bf16" else REL_FP32
    near = 0
    for i in range(len(q)):
        for j in range(len(t)):
            Dref, Sref, Sc = curve_from_rows(rq[i], rt[j], 2.0 / L, M, 1)
            gr = got[i, j]
            assert gr["status"] == 0
            l = int(gr["best_l"])
            assert abs(gr["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc, rel), (i, j)
            np.testing.assert_allclose(gr["shift"], Sref[l], rtol=0, atol=1e-6)
            lref = int(np.argmin(Dref))
            if rel == REL_FP32:
                assert check_argmin(l, lref, Dref, d2_tol(Dref[lref], Sc, rel))
            else:
                near += abs((l - lref + n // 2) % n - n // 2) <= 1
    if rel != REL_FP32:
        assert near >= len(q) * len(t) - 1


def test_slice_ramp_filtered_curve_on_gpu_rows(al):
    rng = np.random.default_rng(67)
    L, n, M = 48, 60, 32
    f, g = blobs(rng, 2, L)
    p = params(L, n, M, metric="rfsw2")
    B = swalign.bins_of(p)
    rows = al.project(np.stack([f, g]), p).cpu().numpy().astype(np.float64)  # signed rows
    assert rows.min() < 0.0
    D, S, _ = al.align_all_rotations(f, g, p)
    D, S = D.cpu().numpy(), S.cpu().numpy()
    h = 2.0 / L
    Qs = []
    for R in rows:
        parts = oracle.rfsw_parts(R)
        Qs.append(np.stack([oracle.quantiles(parts[k], h, M) for k in range(2)]))
    Dref, Sref = oracle.rfsw_curve(Qs[0], Qs[1], translation=1)
    Sc = sum(((oracle.center(Q[k])[1]) ** 2).sum() for Q in Qs for k in range(2)) / (n * M)
    assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc)), B
    np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-6)


def test_slice_quarter_turn(al):
    rng = np.random.default_rng(71)
    L, n, M = 64, 64, 32
    f = blobs(rng, 1, L)[0]
    g = np.ascontiguousarray(np.rot90(f, k=-1))  # g[r, c] = f[L-1-c, r]
    p = params(L, n, M)
    _, _, best = al.align_all_rotations(f, g, p)
    r = swalign.results_to_numpy(best)[0]
    assert r["status"] == 0 and r["best_l"] == 3 * n // 4


def test_slice_bank_with_half_size_queries_equals_batch(al):
    rng = np.random.default_rng(73)
    L, n, M = 64, 60, 32
    t = blobs(rng, 7, L)
    qh = blobs(rng, 4, L // 2)
    qu = np.ascontiguousarray(np.repeat(np.repeat(qh, 2, axis=1), 2, axis=2) * 0.25)
    p = params(L, n, M)
    bank = swalign.Bank(al, t, p)
    try:
        a = swalign.results_to_numpy(bank.align(qh, q_L=L // 2))
    finally:
        bank.close()
    b = swalign.results_to_numpy(al.align_batch(qu, t, p))
    np.testing.assert_array_equal(a["best_l"], b["best_l"])
    np.testing.assert_allclose(a["d2"], b["d2"], rtol=1e-9, atol=1e-12)


def test_slice_global_grid_batch_on_gpu_rows(al):
    # 128 < L: the grids of chunks of images in global scratch; more images
    # than one chunk (1024) so that the chunk loop runs twice
    rng = np.random.default_rng(89)
    L, n, M = 192, 24, 32
    q = blobs(rng, 1030, L)
    t = blobs(rng, 3, L)
    p = params(L, n, M)
    assert swalign.bins_of(p) == 320
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    for i in (0, 7, 1023, 1024, 1029):
        rows = al.project(np.stack([q[i], t[1]]), p).cpu().numpy().astype(np.float64)
        Dref, Sref, Sc = curve_from_rows(rows[0], rows[1], 2.0 / L, M, 1)
        gr = got[i, 1]
        l = int(gr["best_l"])
        assert gr["status"] == 0
        assert abs(gr["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc), i
        np.testing.assert_allclose(gr["shift"], Sref[l], rtol=0, atol=1e-6)
        lref = int(np.argmin(Dref))
        assert check_argmin(l, lref, Dref, d2_tol(Dref[lref], Sc))


def upsample2(x):
    return np.ascontiguousarray(np.repeat(np.repeat(x, 2, axis=-2), 2, axis=-1) * 0.25)


@pytest.mark.parametrize("L,n", [(160, 10), (192, 8), (256, 12), (256, 20)])
def test_slice_upsampled_rows_match_oracle(al, L, n):
    # images of side L/2 through their own grid of B/2 points (128 < L): the
    # rows of the 2 x 2 upsampled image within the row bar, every target
    # wrapped into the half grid's period and folded by T(-s) = conj T(s)
    rng = np.random.default_rng(L * 3 + n)
    qh = blobs(rng, 2, L // 2)
    qh[1] -= 0.2 * qh[1].max()  # negative pixels are clipped to 0 on load
    p = params(L, n, 8)
    B = swalign.bins_of(p)
    n0 = al.launch_count()
    got = al.project_upsampled(qh, p).cpu().numpy().astype(np.float64)
    assert al.launch_count() - n0 == 1  # one CTA per image on the L/2 grid
    qu = upsample2(qh)
    tol = row_tol(L, B)
    plain = al.project(qu, p).cpu().numpy().astype(np.float64)
    for i in range(len(qh)):
        mass = np.maximum(qu[i].astype(np.float64), 0).sum()
        ref = ref_rows(qu[i], n, B, clip=True) * mass
        err = np.linalg.norm(got[i] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= tol, (i, err.max(), tol)
        np.testing.assert_array_equal(got[i, n // 2:], got[i, :n // 2, ::-1])
        assert got[i].min() >= 0.0
        # the L x L grid's rows of the upsampled image: both within the bar
        dif = np.linalg.norm(got[i] - plain[i], axis=1) / np.linalg.norm(ref, axis=1)
        assert dif.max() <= 2 * tol


def test_slice_upsampled_query_status(al):
    # a query of side L/2 with no mass or with a non-finite pixel is unusable
    rng = np.random.default_rng(98)
    L, n, M = 256, 8, 8
    t = blobs(rng, 2, L)
    qh = blobs(rng, 3, L // 2)
    qh[1] = 0.0
    qh[2, 3, 3] = np.inf
    bank = swalign.Bank(al, t, params(L, n, M))
    try:
        a = swalign.results_to_numpy(bank.align(qh, q_L=L // 2)).reshape(3, 2)
    finally:
        bank.close()
    assert np.all(a[0]["status"] == 0) and np.all(np.isfinite(a[0]["d2"]))
    assert np.all(a[1]["status"] == 1) and np.all(a[2]["status"] == 1)


def test_slice_bank_256_with_half_size_queries(al):
    # the serving setting: a bank at 256^2 and queries at 128^2 upsampled
    # 2 x 2; the pipeline after the rows at the FP32 bar on the GPU's own rows
    rng = np.random.default_rng(97)
    L, n, M = 256, 36, 32
    t = blobs(rng, 5, L)
    qh = blobs(rng, 3, L // 2)
    p = params(L, n, M)
    bank = swalign.Bank(al, t, p)
    try:
        a = swalign.results_to_numpy(bank.align(qh, q_L=L // 2)).reshape(3, 5)
        best = swalign.results_to_numpy(bank.align(qh, q_L=L // 2, mode=1))
    finally:
        bank.close()
    rq = al.project_upsampled(qh, p).cpu().numpy().astype(np.float64)
    rt = al.project(t, p).cpu().numpy().astype(np.float64)
    for i in range(3):
        dmin = []
        for j in range(5):
            Dref, Sref, Sc = curve_from_rows(rq[i], rt[j], 2.0 / L, M, 1)
            gr = a[i, j]
            l = int(gr["best_l"])
            assert gr["status"] == 0 and gr["template_index"] == j
            assert abs(gr["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc), (i, j)
            np.testing.assert_allclose(gr["shift"], Sref[l], rtol=0, atol=1e-6)
            lref = int(np.argmin(Dref))
            assert check_argmin(l, lref, Dref, d2_tol(Dref[lref], Sc))
            dmin.append(gr["d2"])
        assert best[i]["template_index"] == int(np.argmin(dmin))
        assert best[i]["d2"] == min(dmin)


def test_slice_status_flags(al):
    rng = np.random.default_rng(79)
    L, n, M = 32, 24, 16
    q = blobs(rng, 2, L)
    t = blobs(rng, 2, L)
    q[1, 3, 4] = np.nan
    t[1] = 0.0
    got = swalign.results_to_numpy(al.align_batch(q, t, params(L, n, M))).reshape(2, 2)
    assert got[0, 0]["status"] == 0
    assert got[1, 0]["status"] == 1 and got[1, 1]["status"] == 1
    assert got[0, 1]["status"] == 2


def test_slice_rejections(al):
    big = params(300, 16, 8)
    with pytest.raises(swalign.SwError) as e:
        al.project(np.zeros((1, 300, 300), np.float32), big)
    assert e.value.status == 2  # SW_ERR_UNSUPPORTED: built for L <= 256
    with pytest.raises(swalign.SwError) as e:  # above L = 128 only 256, 320 or 384 bins
        al.project(np.zeros((1, 160, 160), np.float32), params(160, 16, 8, n_bins=288))
    assert e.value.status == 1
    odd_bins = params(64, 16, 8, n_bins=94)  # not a multiple of 32 (the warp FFT's length)
    with pytest.raises(swalign.SwError) as e:
        al.project(np.zeros((1, 64, 64), np.float32), odd_bins)
    assert e.value.status == 1
    lib = swalign.load()
    p = params(32, 16, 8)
    f = torch.zeros((32, 32), dtype=torch.float32, device="cuda")
    out = torch.zeros((40,), dtype=torch.uint8, device="cuda")
    st = lib.sw_align_all_rotations_noalloc(ctypes.byref(p), ctypes.c_void_p(f.data_ptr()),
                                            ctypes.c_void_p(f.data_ptr()), None, None,
                                            ctypes.c_void_p(out.data_ptr()), None)
    assert st == 2


def test_slice_many_to_many_full_size_sampled(al):
    # The bench's workload (4096 x 256 pairs, L = 128, n = 256, M = 128, FP32)
    # in the bench's launch configuration, sampled pairs against the oracle on
    # the GPU's rows, and the rows of sampled images against the exact slice.
    data = synth.many_to_many()
    q, t = data["queries"], data["templates"]
    L, n, M = 128, 256, 128
    p = params(L, n, M)
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    rng = np.random.default_rng(83)
    pairs = [(int(rng.integers(len(q))), int(rng.integers(len(t)))) for _ in range(4)]
    for i, j in pairs:
        rows = al.project(np.stack([q[i], t[j]]), p).cpu().numpy().astype(np.float64)
        Dref, Sref, Sc = curve_from_rows(rows[0], rows[1], 2.0 / L, M, 1)
        gr = got[i, j]
        l = int(gr["best_l"])
        assert gr["status"] == 0
        assert abs(gr["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc), (i, j)
        lref = int(np.argmin(Dref))
        assert check_argmin(l, lref, Dref, d2_tol(Dref[lref], Sc))
    i = pairs[0][0]
    B = swalign.bins_of(p)
    rows = al.project(q[i:i + 1], p).cpu().numpy().astype(np.float64)[0]
    ref = ref_rows(q[i], n, B, clip=True) * np.maximum(q[i].astype(np.float64), 0).sum()
    err = np.linalg.norm(rows - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= row_tol(L, B)


def test_project_upsampled_rejects_odd_L(al):
    import ctypes
    p = params(65, 8, 8)
    x = torch.zeros((2, 32, 32), dtype=torch.float32, device="cuda")
    out = torch.empty((2, 8, swalign.bins_of(p)), dtype=torch.float32, device="cuda")
    with pytest.raises(swalign.SwError) as e:
        al.call("sw_project_upsampled", ctypes.byref(p), ctypes.c_void_p(x.data_ptr()), 2,
                ctypes.c_void_p(out.data_ptr()), None)
    assert e.value.status == 1 and "odd" in str(e.value)
    with pytest.raises(ValueError):
        al.project_upsampled(torch.zeros((2, 30, 30), device="cuda"), params(64, 8, 8))
