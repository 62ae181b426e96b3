"""Explicit translation sampling on the CUDA path (translation restricted to
a grid of whole or fractional pixels) against the oracle's brute force over
every grid point, for sliced W2 and the ramp-filtered distance."""
import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign, synth
from tests.parity import check_argmin, d2_tol, norm_scale, norm_scale_rfsw

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
    return np.ascontiguousarray(synth.render(p, L, shift=rng.integers(-4, 5, (count, 2))),
                                dtype=np.float32)


@pytest.mark.parametrize("metric", ["sw2", "rfsw2"])
# n = 64: the decision's register form (one warp per pair of curves)
@pytest.mark.parametrize("K,step_q,n", [(2, 16, 24), (6, 4, 24), (1, 48, 24), (2, 16, 64)])
def test_grid_batch_matches_oracle_brute_force(al, metric, K, step_q, n):
    rng = np.random.default_rng(K * 100 + step_q)
    L, M = 40, 16
    q, t = blobs(rng, 3, L), blobs(rng, 4, L)
    p = swalign.make_params(L, n, M, metric=metric, shift_grid=K, shift_step_q=step_q)
    B = swalign.bins_of(p)
    step = step_q * (2.0 / L) / 16
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(len(q), len(t))
    met = 1 if metric == "rfsw2" else 0
    for i in range(len(q)):
        for j in range(len(t)):
            fq, ft = q[i].astype(np.float64), t[j].astype(np.float64)
            rr, D, S = oracle.align_pair_grid(fq, ft, n, M, K, step, B=B, metric=met)
            Sc = (norm_scale_rfsw(fq, ft, n, M, B) if met else norm_scale(fq, ft, n, M))
            g = got[i, j]
            l = int(g["best_l"])
            assert g["status"] == 0
            assert check_argmin(l, rr["best_l"], D, d2_tol(rr["d2"], Sc)), (i, j)
            assert abs(g["d2"] - D[l]) <= d2_tol(D[l], Sc), (i, j, g["d2"], D[l])
            # the shift is a grid point, the oracle's unless two points tie
            ij = g["shift"] / step
            np.testing.assert_allclose(ij, np.rint(ij), atol=1e-9)
            assert np.all(np.abs(np.rint(ij)) <= K)
            # where the GPU picked another grid point than the brute force, the
            # two tie: its distance is already within the bar above


@pytest.mark.parametrize("n", [36, 64])
def test_grid_curve_matches_oracle(al, n):
    rng = np.random.default_rng(3)
    L, M = 48, 24
    f, g = blobs(rng, 2, L)
    K, step_q = 3, 8
    step = step_q * (2.0 / L) / 16
    p = swalign.make_params(L, n, M, shift_grid=K, shift_step_q=step_q)
    D, S, best = al.align_all_rotations(f, g, p)
    D, S = D.cpu().numpy(), S.cpu().numpy()
    _, Dref, Sref = oracle.align_pair_grid(f.astype(np.float64), g.astype(np.float64), n, M, K,
                                           step)
    Sc = norm_scale(f.astype(np.float64), g.astype(np.float64), n, M)
    assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc))
    same = np.all(np.isclose(S, Sref, atol=1e-9), axis=1)
    assert same.mean() >= 0.9  # elsewhere two grid points tie within rounding


def test_wide_grid_equals_closed_form(al):
    """A grid that contains every optimum: within rho step^2 / 2 of the
    unbounded closed form, and never below it."""
    rng = np.random.default_rng(4)
    L, n, M = 40, 24, 16
    q, t = blobs(rng, 2, L), blobs(rng, 3, L)
    free = swalign.results_to_numpy(al.align_batch(q, t, swalign.make_params(L, n, M)))
    p = swalign.make_params(L, n, M, shift_grid=200, shift_step_q=2)  # +-25 px
    grid = swalign.results_to_numpy(al.align_batch(q, t, p))
    step = 2 * (2.0 / L) / 16
    assert np.all(grid["d2"] >= free["d2"] - 1e-7)
    assert np.all(grid["d2"] - free["d2"] <= 0.5 * step ** 2 / 2 + 1e-7)


def test_grid_parameters_are_checked(al):
    q = np.ones((1, 16, 16), np.float32)
    with pytest.raises(swalign.SwError):
        al.align_batch(q, q, swalign.make_params(16, 8, 4, shift_grid=2, shift_step_q=0))
