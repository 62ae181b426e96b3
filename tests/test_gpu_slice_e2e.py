"""The Fourier-slice path end to end against the FP64 oracle run from the
same FP32 images (Sec. 2.3 "Computation", Theorem proj_nufft; Eq.
discrete_sw2, Eq. discrete_rot_sw2).

Every comparison starts from the images on both sides: the CUDA path's
NUFFT rows, quantiles, angle spectra, correlation and decision against the
oracle's exact slice sums (orc_project_slice), sorted-mass quantiles and
direct O(n^2 M) rotation curve.  The bars are those of tests/parity.py:
  - FP32 (tcgen05 FP16 split, CUDA-core FP32): |d2 - D_ref(l)| <=
    1e-5 max(D_ref(l), 0.1 S); l identical or tied within that bar on the
    oracle's curve; s*(l) within 1e-6.
  - BF16 / FP16: the same with 1e-2; l within one bin (circularly) on
    >= 99% of the pairs.
The NUFFT's own error (relative l2 ~3.5e-7 per row) moves d2 by a few 1e-6
relative at most (measured on the full-size workload), inside the bar.
"""
import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign, synth, uneven
from tests.parity import REL_FP32, REL_LP, check_argmin, d2_tol

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


_SIDES = {}


class OracleSide:
    """The oracle's per-image transforms of a set of FP32 images (slice
    projector): uncentred and centred quantiles, centring vectors, norms."""

    def __init__(self, imgs, n, M, B, level_rule=0, projector=1):
        self.n, self.M = n, M
        key = (imgs.tobytes(), n, M, B, level_rule, projector)
        if key not in _SIDES:
            Q, A, ok = oracle.transform_images(imgs.astype(np.float64), n, M, B=B,
                                               level_rule=level_rule, projector=projector)
            assert ok.all()
            Qc = np.stack([oracle.center(x)[1] for x in Q])
            _SIDES[key] = (Q, A, Qc, (Qc ** 2).sum(axis=(1, 2)))
        self.Q, self.A, self.Qc, self.N = _SIDES[key]

    def take(self, idx):
        """The side of the images idx (a list of indices) only."""
        o = OracleSide.__new__(OracleSide)
        o.n, o.M = self.n, self.M
        o.Q, o.A, o.Qc, o.N = self.Q[idx], self.A[idx], self.Qc[idx], self.N[idx]
        return o


def check_pairs(got, fq, ft, pairs, translation, rel, stats=None):
    """got[i, j] (sw_result) against the oracle's curve of (query i,
    template j) for every pair; returns the number of pairs whose rotation
    is within one bin of the oracle's (the reduced-precision criterion)."""
    n, M = fq.n, fq.M
    near = 0
    for i, j in pairs:
        Qi = fq.Qc[i] if translation else fq.Q[i]
        Qj = ft.Qc[j] if translation else ft.Q[j]
        D = oracle.rotation_curve(Qi, Qj)
        S = (fq.N[i] + ft.N[j]) / (n * M)
        g = got[i, j]
        assert g["status"] == 0, (i, j)
        l = int(g["best_l"])
        lref = int(np.argmin(D))
        err = abs(g["d2"] - D[l])
        assert err <= d2_tol(D[l], S, rel), (i, j, l, g["d2"], D[l], S)
        dl = abs((l - lref + n // 2) % n - n // 2)
        near += dl <= 1
        if rel == REL_FP32:
            assert check_argmin(l, lref, D, d2_tol(D[lref], S, rel)), (i, j, l, lref)
        sref = oracle.shifts_of(fq.A[i], ft.A[j], n)[l] if translation else np.zeros(2)
        np.testing.assert_allclose(g["shift"], sref, rtol=0, atol=1e-6)
        assert g["template_index"] == j
        if stats is not None:
            stats.append((err / D[l], err / S, dl))
    return near


def run_batch(al, q, t, n, M, precision="fp32", translation=1, level_rule=0):
    L = q.shape[-1]
    p = swalign.make_params(L, n, M, precision=precision, translation=translation,
                            level_rule=level_rule, projector="slice")
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    return p, got


# ------------------------------------------------ small cases, every pair

@pytest.mark.parametrize("L,n,M,translation,level_rule", [
    (48, 60, 36, 1, 0), (48, 60, 36, 0, 1), (33, 12, 7, 1, 1),   # odd L
    (64, 120, 64, 1, 0), (96, 128, 96, 0, 0),
    (128, 64, 128, 1, 0), (128, 64, 128, 1, 1),                 # one CTA per image, L = 128
    (160, 32, 64, 1, 0), (192, 24, 32, 0, 0), (256, 16, 32, 1, 1),  # grids in global scratch
])
@pytest.mark.parametrize("precision", ["fp32", "fp32_simt", "bf16", "fp16"])
def test_slice_batch_matches_oracle_from_images(al, L, n, M, translation, level_rule, precision):
    rng = np.random.default_rng(L * 31 + n + M + translation)
    q = blobs(rng, 4, L)
    t = blobs(rng, 3, L)
    p, got = run_batch(al, q, t, n, M, precision, translation, level_rule)
    B = swalign.bins_of(p)
    assert B == oracle.bins_for(L, projector=1)
    fq = OracleSide(q, n, M, B, level_rule)
    ft = OracleSide(t, n, M, B, level_rule)
    rel = REL_LP if precision in ("bf16", "fp16") else REL_FP32
    pairs = [(i, j) for i in range(len(q)) for j in range(len(t))]
    near = check_pairs(got, fq, ft, pairs, translation, rel)
    assert near == len(pairs)


@pytest.mark.parametrize("precision", ["fp32", "fp32_simt"])
def test_slice_ragged_tiles_match_oracle_from_images(al, precision):
    # 70 templates: ragged against the correlation's 128-row and 256-column
    # tiles and the decision's 16-template blocks
    rng = np.random.default_rng(131)
    L, n, M = 40, 36, 24
    q = blobs(rng, 3, L)
    t = blobs(rng, 70, L)
    p, got = run_batch(al, q, t, n, M, precision)
    B = swalign.bins_of(p)
    fq, ft = OracleSide(q, n, M, B), OracleSide(t, n, M, B)
    check_pairs(got, fq, ft, [(i, j) for i in range(3) for j in range(70)], 1, REL_FP32)


@pytest.mark.parametrize("translation", [1, 0])
def test_slice_all_rotations_curve_matches_oracle_from_images(al, translation):
    rng = np.random.default_rng(141 + translation)
    L, n, M = 64, 120, 64
    f, g = blobs(rng, 2, L)
    p = swalign.make_params(L, n, M, translation=translation, projector="slice")
    D, S, best = al.align_all_rotations(f, g, p)
    D, S = D.cpu().numpy(), S.cpu().numpy()
    ref, Dref, Sref = oracle.align_pair(f.astype(np.float64), g.astype(np.float64), n, M,
                                        B=swalign.bins_of(p), translation=translation,
                                        projector=1)
    side = OracleSide(np.stack([f, g]), n, M, swalign.bins_of(p))
    Sc = side.N.sum() / (n * M)
    assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc)), np.max(np.abs(D - Dref) / d2_tol(Dref, Sc))
    np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-6)
    r = swalign.results_to_numpy(best)[0]
    assert r["status"] == 0
    assert check_argmin(int(r["best_l"]), ref["best_l"], Dref, d2_tol(ref["d2"], Sc))


def test_slice_ramp_filtered_matches_oracle_from_images(al):
    # RFSW2 on the Fourier-slice rows: signed rows, ramp filter, two parts
    rng = np.random.default_rng(151)
    L, n, M = 48, 60, 32
    q = blobs(rng, 2, L)
    t = blobs(rng, 3, L)
    p = swalign.make_params(L, n, M, metric="rfsw2", projector="slice")
    B = swalign.bins_of(p)
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    for i in range(len(q)):
        for j in range(len(t)):
            fq, ft = q[i].astype(np.float64), t[j].astype(np.float64)
            ref, Dref, Sref = oracle.align_pair_rfsw(fq, ft, n, M, B=B, projector=1)
            Sc = 0.0
            for img in (fq, ft):
                F, _ = oracle.prepare(img)
                for part in oracle.rfsw_parts(oracle.project_slice(F, n, B)):
                    Sc += float((oracle.center(oracle.quantiles(part, 2.0 / L, M))[1] ** 2).sum())
            Sc /= n * M
            g = got[i, j]
            l = int(g["best_l"])
            assert g["status"] == 0
            assert abs(g["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc), (i, j)
            assert check_argmin(l, ref["best_l"], Dref, d2_tol(ref["d2"], Sc))
            np.testing.assert_allclose(g["shift"], Sref[l], rtol=0, atol=1e-6)
    # the single-pair call gives the same curve
    D, S, _ = al.align_all_rotations(q[0], t[0], p)
    _, Dref, Sref = oracle.align_pair_rfsw(q[0].astype(np.float64), t[0].astype(np.float64),
                                           n, M, B=B, projector=1)
    assert np.all(np.abs(D.cpu().numpy() - Dref) <= d2_tol(Dref, Sc))


# --------------------------------------------- the headline workload, sampled

@pytest.fixture(scope="module")
def headline():
    return synth.many_to_many()


def test_slice_headline_workload_sampled_from_images(al, headline):
    """4096 x 256 pairs at 128^2, n = 256, M = 128, FP32 (tcgen05 split) in
    the benchmark's launch configuration: 8 pairs of queries with their own
    template (well aligned, d2 / S ~ 1e-4) and 8 random pairs, each against
    the oracle from the images."""
    q, t, src = headline["queries"], headline["templates"], headline["source"]
    n, M = 256, 128
    p, got = run_batch(al, q, t, n, M)
    assert np.all(got["status"] == 0)
    rng = np.random.default_rng(1729)
    I = rng.choice(len(q), 16, replace=False)
    J = np.unique(np.concatenate([src[I[:8]], rng.choice(len(t), 8, replace=False)]))
    B = swalign.bins_of(p)
    fq, ft = OracleSide(q[I], n, M, B), OracleSide(t[J], n, M, B)
    sub = got[np.ix_(I, J)]
    for a in range(len(I)):  # the stored template index is the column index
        sub[a]["template_index"] = np.arange(len(J))
    col = {int(j): c for c, j in enumerate(J)}
    pairs = [(a, col[int(src[I[a]])]) for a in range(8)]
    pairs += [(8 + a, int(c)) for a, c in enumerate(rng.integers(0, len(J), 8))]
    stats = []
    check_pairs(sub, fq, ft, pairs, 1, REL_FP32, stats)
    assert all(s[2] == 0 for s in stats)  # the same rotation index everywhere


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_headline_subset_64x16_low_precision(al, headline, precision):
    """The reduced-precision correlation on the headline workload (the
    first 64 queries x 16 templates of the 4096 x 256 batch, computed in the
    full batch): every pair within the 1e-2 bar of the oracle and within one
    bin of its rotation on >= 99%, and against the FP32 path on the same
    pairs."""
    q, t = headline["queries"], headline["templates"]
    n, M = 256, 128
    p, got = run_batch(al, q, t, n, M, precision)
    _, g32 = run_batch(al, q, t, n, M, "fp32")
    B = swalign.bins_of(p)
    fq, ft = OracleSide(q[:64], n, M, B), OracleSide(t[:16], n, M, B)
    pairs = [(i, j) for i in range(64) for j in range(16)]
    near = check_pairs(got, fq, ft, pairs, 1, REL_LP)
    assert near >= 0.99 * len(pairs)
    a, b = got[:64, :16], g32[:64, :16]
    S = (fq.N[:, None] + ft.N[None, :]) / (n * M)
    assert np.all(np.abs(a["d2"] - b["d2"]) <= 2 * d2_tol(b["d2"], S, REL_LP))
    dl = np.abs((a["best_l"] - b["best_l"] + n // 2) % n - n // 2)
    assert np.mean(dl <= 1) >= 0.99


# ------------------------------------------------ uneven batch, one graph

def test_slice_uneven_graph_sampled_from_images():
    """One CUDA graph over sizes L = 64 .. 256 (M = L, BF16 correlation) with
    the Fourier-slice projector: one sampled pair per size (a query and its
    own template) against the oracle from the images."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 256
    batch = synth.uneven_batch(n_queries=60, n_templates_per_L=3, seed=17)
    g = uneven.UnevenGraph(uneven.buckets_from(batch, n, "bf16", projector="slice"), mode=0)
    try:
        g.replay()
        res = g.results()
        for L, d in batch.items():
            q, t = d["queries"], d["templates"]
            r = res[L].reshape(len(q), len(t))
            i = 0
            j = int(d["source"][i])
            B = oracle.bins_for(L, projector=1)
            side = OracleSide(np.stack([q[i], t[j]]), n, L, B)
            got = r[i:i + 1, j:j + 1].copy()
            got[0, 0]["template_index"] = 0
            assert check_pairs(got, side.take([0]), side.take([1]), [(0, 0)], 1, REL_LP) == 1, L
    finally:
        g.close()
