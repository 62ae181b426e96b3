"""Max-sliced W2 over rotations (metric msw2) on the CUDA path against the
FP64 oracle's direct O(n^2 M) curve: batches (ragged row blocks and
template counts, every kernel shape n <= 256, <= 512, <= 1024), full
curves, exact quarter turns, the best-template mode and the unsupported
combinations."""
import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign, synth
from tests.parity import check_argmin, d2_tol, norm_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def al():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = swalign.Aligner(0)
    yield a
    a.close()


def blobs(rng, count, L):
    p = synth.draw_mixtures(rng, count, L, ncomp=(2, 4))
    return np.ascontiguousarray(synth.render(p, L, shift=rng.integers(-3, 4, (count, 2))),
                                dtype=np.float32)


def compare(al, q, t, n, M, translation=1, level_rule=0):
    L = q.shape[-1]
    p = swalign.make_params(L, n, M, translation=translation, level_rule=level_rule,
                            metric="msw2")
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    for i in range(len(q)):
        for j in range(len(t)):
            fq, ft = q[i].astype(np.float64), t[j].astype(np.float64)
            rr, D, S = oracle.align_pair_msw(fq, ft, n, M, level_rule=level_rule,
                                             translation=translation)
            Sc = norm_scale(fq, ft, n, M, level_rule)
            g = got[i, j]
            l = int(g["best_l"])
            assert g["status"] == 0
            assert check_argmin(l, rr["best_l"], D, d2_tol(rr["d2"], Sc)), (i, j, l, rr["best_l"])
            assert abs(g["d2"] - D[l]) <= d2_tol(D[l], Sc), (i, j, g["d2"], D[l])
            np.testing.assert_allclose(g["shift"], S[l], rtol=0, atol=1e-6)


@pytest.mark.parametrize("translation", [1, 0])
def test_msw_batch_matches_oracle(al, translation):
    rng = np.random.default_rng(40 + translation)
    compare(al, blobs(rng, 3, 40), blobs(rng, 70, 40), n=60, M=36, translation=translation)


@pytest.mark.parametrize("L,n,M", [(32, 360, 20), (24, 512, 12), (24, 1024, 8), (20, 12, 5)])
def test_msw_kernel_shapes(al, L, n, M):
    rng = np.random.default_rng(n + M)
    compare(al, blobs(rng, 2, L), blobs(rng, 3, L), n=n, M=M)


def test_msw_left_levels(al):
    rng = np.random.default_rng(8)
    compare(al, blobs(rng, 2, 32), blobs(rng, 3, 32), n=24, M=9, level_rule=1)


def test_msw_curve_matches_oracle(al):
    rng = np.random.default_rng(9)
    f, g = blobs(rng, 2, 48)
    n, M = 96, 48
    for translation in (1, 0):
        p = swalign.make_params(48, n, M, translation=translation, metric="msw2")
        D, S, best = al.align_all_rotations(f, g, p)
        D, S = D.cpu().numpy(), S.cpu().numpy()
        rr, Dref, Sref = oracle.align_pair_msw(f.astype(np.float64), g.astype(np.float64), n, M,
                                               translation=translation)
        Sc = norm_scale(f.astype(np.float64), g.astype(np.float64), n, M)
        assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc))
        np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-6)


def test_msw_quarter_turn_is_exact(al):
    rng = np.random.default_rng(5)
    L, n, M = 48, 48, 24
    f = blobs(rng, 1, L)[0]
    g = np.ascontiguousarray(np.rot90(f, k=-1))
    p = swalign.make_params(L, n, M, metric="msw2")
    r = swalign.results_to_numpy(al.align_batch(f[None], g[None], p))[0]
    assert r["best_l"] == 3 * n // 4
    assert r["d2"] <= 1e-12


def test_msw_best_template(al):
    rng = np.random.default_rng(6)
    q, t = blobs(rng, 5, 32), blobs(rng, 7, 32)
    p = swalign.make_params(32, 24, 16, metric="msw2")
    allp = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(5, 7)
    best = swalign.results_to_numpy(al.align_batch(q, t, p, mode=1))
    j = np.argmin(allp["d2"], axis=1)
    np.testing.assert_array_equal(best["d2"], allp["d2"][np.arange(5), j])


def test_msw_unsupported_combinations(al):
    q = blobs(np.random.default_rng(1), 2, 16)
    with pytest.raises(swalign.SwError):
        swalign.Bank(al, q, swalign.make_params(16, 8, 4, metric="msw2"))
    with pytest.raises(swalign.SwError):
        al.align_batch(q, q, swalign.make_params(16, 8, 4, metric="msw2", shift_grid=2,
                                                 shift_step_q=16))
