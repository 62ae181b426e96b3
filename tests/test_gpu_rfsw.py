"""Ramp-filtered sliced W2 (metric rfsw2) on the CUDA path against the FP64
oracle: quantiles of both parts, full curves, batches on every correlation
path (FP32 bar for fp32 / fp32_simt, reduced-precision bar for bf16), exact
quarter turns, bank == batch, and the many-to-many size sampled."""
import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign, synth
from tests.parity import (REL_FP32, REL_LP, check_argmin, d2_tol, level_of, norm_scale_rfsw,
                          rfsw_level_tol)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("L,n,M,level_rule", [(48, 60, 36, 0), (64, 256, 128, 0),
                                              (33, 12, 7, 1), (40, 20, 16, 1)])
def test_rfsw_quantiles_match_oracle(al, L, n, M, level_rule):
    rng = np.random.default_rng(L + n)
    imgs = blobs(rng, 4, L)
    p = swalign.make_params(L, n, M, level_rule=level_rule, metric="rfsw2")
    B = swalign.bins_of(p)
    assert B == oracle.rfsw_bins(L)
    proj = al.project(imgs, p)
    Q, C, N = al.quantiles(proj, p)
    Q, C, N = Q.cpu().numpy(), C.cpu().numpy(), N.cpu().numpy()
    h = 2.0 / L
    z = (np.arange(M) + 0.5) / M if level_rule == 0 else np.arange(M) / M
    for i in range(len(imgs)):
        F, _ = oracle.prepare(imgs[i].astype(np.float64))
        U = oracle.project(F, n, B)
        Ut = oracle.ramp_filter(U)
        parts = oracle.rfsw_parts(U)
        for part in range(2):
            Qr = oracle.quantiles(parts[part], h, M, level_rule)
            for k in range(n):
                tol = rfsw_level_tol(Ut[k], parts[part][k])
                lev = level_of(Q[i, part, k].astype(np.float64), parts[part][k], h)
                if level_rule == 1:
                    lev[0] = 0.0  # level 0 is the domain's left end on both sides
                assert np.abs(lev - z).max() <= tol, (i, part, k, np.abs(lev - z).max(), tol)
            a, Qc = oracle.center(Qr)
            np.testing.assert_allclose(C[i, part], a, atol=1e-4 * h)
            assert N[i, part] == pytest.approx((Qc ** 2).sum(), rel=1e-4)


def compare_rfsw(al, q, t, n, M, precision, translation=1, level_rule=0):
    L = q.shape[-1]
    p = swalign.make_params(L, n, M, translation=translation, level_rule=level_rule,
                            precision=precision, metric="rfsw2")
    B = swalign.bins_of(p)
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    rel = REL_LP if precision in ("bf16", "fp16") else REL_FP32
    ref = oracle.align_all_pairs_rfsw(q.astype(np.float64), t.astype(np.float64), n, M, B=B,
                                      level_rule=level_rule, translation=translation)
    near = 0
    for i in range(len(q)):
        for j in range(len(t)):
            gr, rr = got[i, j], ref[i, j]
            assert gr["status"] == rr["status"] == 0
            fq, ft = q[i].astype(np.float64), t[j].astype(np.float64)
            _, Dref, Sref = oracle.align_pair_rfsw(fq, ft, n, M, B=B, level_rule=level_rule,
                                                   translation=translation)
            Sc = norm_scale_rfsw(fq, ft, n, M, B, level_rule)
            l = int(gr["best_l"])
            assert abs(gr["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc, rel), (i, j, gr["d2"], Dref[l])
            np.testing.assert_allclose(gr["shift"], Sref[l], rtol=0, atol=1e-6)
            if rel == REL_FP32:
                assert check_argmin(l, int(rr["best_l"]), Dref, d2_tol(rr["d2"], Sc, rel))
            else:
                near += abs((l - int(rr["best_l"]) + n // 2) % n - n // 2) <= 1
    if rel != REL_FP32:
        assert near >= 0.99 * len(q) * len(t)


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt", "bf16"])
@pytest.mark.parametrize("translation", [1, 0])
def test_rfsw_batch_matches_oracle(al, precision, translation):
    rng = np.random.default_rng(17 + translation)
    q = blobs(rng, 5, 48)
    t = blobs(rng, 70, 48)  # ragged against the 64-wide and 128-row tiles
    compare_rfsw(al, q, t, n=60, M=36, precision=precision, translation=translation)


def test_rfsw_left_levels_odd_sizes(al):
    rng = np.random.default_rng(23)
    compare_rfsw(al, blobs(rng, 3, 33), blobs(rng, 4, 33), n=12, M=7, precision="fp32",
                 translation=1, level_rule=1)


def test_rfsw_curve_matches_oracle(al):
    rng = np.random.default_rng(29)
    f, g = blobs(rng, 2, 64)
    n, M = 128, 64
    for translation in (1, 0):
        p = swalign.make_params(64, n, M, translation=translation, metric="rfsw2")
        B = swalign.bins_of(p)
        D, S, best = al.align_all_rotations(f, g, p)
        D, S = D.cpu().numpy(), S.cpu().numpy()
        rr, Dref, Sref = oracle.align_pair_rfsw(f.astype(np.float64), g.astype(np.float64), n, M,
                                                B=B, translation=translation)
        Sc = norm_scale_rfsw(f.astype(np.float64), g.astype(np.float64), n, M, B)
        assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc))
        np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-6)
        r = swalign.results_to_numpy(best)[0]
        assert check_argmin(int(r["best_l"]), rr["best_l"], Dref, d2_tol(rr["d2"], Sc))


def test_rfsw_quarter_turn_is_exact(al):
    rng = np.random.default_rng(5)
    L, n, M = 64, 64, 32
    f = blobs(rng, 1, L)[0]
    g = np.ascontiguousarray(np.rot90(f, k=-1))  # g[r, c] = f[L-1-c, r]
    for translation in (1, 0):
        p = swalign.make_params(L, n, M, translation=translation, metric="rfsw2")
        r = swalign.results_to_numpy(al.align_batch(f[None], g[None], p))[0]
        assert r["best_l"] == 3 * n // 4
        Sc = norm_scale_rfsw(f.astype(np.float64), g.astype(np.float64), n, M,
                             swalign.bins_of(p))
        assert abs(r["d2"]) <= d2_tol(0.0, Sc)  # exact in exact arithmetic
        np.testing.assert_allclose(r["shift"], 0.0, atol=1e-6)


def test_rfsw_bank_equals_batch(al):
    rng = np.random.default_rng(31)
    L, n, M = 48, 60, 32
    t = blobs(rng, 9, L)
    q = blobs(rng, 4, L)
    for prec in ("fp32", "bf16"):
        p = swalign.make_params(L, n, M, precision=prec, metric="rfsw2")
        bank = swalign.Bank(al, t, p)
        try:
            a = swalign.results_to_numpy(al.align_batch(q, t, p))
            b = swalign.results_to_numpy(bank.align(q, q_L=L, mode=0))
            np.testing.assert_array_equal(a["best_l"], b["best_l"])
            np.testing.assert_array_equal(a["d2"], b["d2"])
        finally:
            bank.close()


def gpu_quantiles(al, img, p):
    """The quantiles the alignment path uses for one image: rows k < n/2 from
    sw_quantiles (the same packed rows and kernels), rows k + n/2 their
    mirror images Q_{k+n/2}(z_p) = -Q_k(z_{M-1-p}) (midpoint levels)."""
    Q = al.quantiles(al.project(img[None], p), p)[0].cpu().numpy()[0]
    nh = Q.shape[1] // 2
    Q[:, nh:, :] = -Q[:, :nh, ::-1]
    return Q


def check_levels(img, Q, n, M, B):
    F, _ = oracle.prepare(img)
    U = oracle.project(F, n, B)
    Ut = oracle.ramp_filter(U)
    parts = oracle.rfsw_parts(U)
    z = (np.arange(M) + 0.5) / M
    h = 2.0 / F.shape[0]
    for part in range(2):
        for k in range(n):
            lev = level_of(Q[part, k].astype(np.float64), parts[part][k], h)
            assert np.abs(lev - z).max() <= rfsw_level_tol(Ut[k], parts[part][k]), (part, k)


def test_rfsw_many_to_many_full_size_sampled(al):
    """4096 queries x 256 templates, 128 x 128, n = 256, M = 128 (per part),
    ramp-filtered: 16 sampled pairs against the oracle (where a part's
    quantile sits next to a flat CDF stretch, the GPU's quantiles are checked
    in CDF space and the distance against the oracle's curve on them); the
    query's own template is the best match for nearly all queries."""
    d = synth.many_to_many()
    q, t = d["queries"], d["templates"]
    n, M = 256, 128
    p = swalign.make_params(128, n, M, metric="rfsw2")
    B = swalign.bins_of(p)
    res = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    assert np.all(res["status"] == 0)
    rng = np.random.default_rng(99)
    picks = [(int(i), int(d["source"][i])) for i in rng.integers(0, len(q), 8)]
    picks += [(int(i), int(j)) for i, j in zip(rng.integers(0, len(q), 8),
                                                rng.integers(0, len(t), 8))]
    flat_pairs = 0
    for i, j in picks:
        fq, ft = q[i].astype(np.float64), t[j].astype(np.float64)
        rr, Dref, _ = oracle.align_pair_rfsw(fq, ft, n, M, B=B)
        Sc = norm_scale_rfsw(fq, ft, n, M, B)
        l = int(res[i, j]["best_l"])
        g = res[i, j]["d2"]
        if abs(g - Dref[l]) <= d2_tol(Dref[l], Sc):
            assert check_argmin(l, rr["best_l"], Dref, d2_tol(rr["d2"], Sc))
            continue
        # A part's CDF is flat across the other part's lobe, so its quantile
        # function jumps there; a level within rounding of the jump has two
        # correct quantiles.  Check the GPU's own quantiles in CDF space, then
        # the oracle's curve on exactly those quantiles.
        Qf, Qg = gpu_quantiles(al, q[i], p), gpu_quantiles(al, t[j], p)
        for img, Qi in ((fq, Qf), (ft, Qg)):
            check_levels(img, Qi, n, M, B)
        D, _ = oracle.rfsw_curve(Qf.astype(np.float64), Qg.astype(np.float64), 1)
        assert abs(g - D[l]) <= d2_tol(D[l], Sc), (i, j, g, D[l])
        assert check_argmin(l, int(np.argmin(D)), D, d2_tol(D.min(), Sc))
        flat_pairs += 1
    assert flat_pairs <= len(picks) // 4
    assert np.mean(np.argmin(res["d2"], axis=1) == d["source"]) > 0.9
