"""Register form of the decision (Sec. 2.3, "Fast computation over
rotations": the inverse FFT over angle and the argmin of Eq. optimal_rotation).

For n_theta = 64, 128, 256 and 512 the decision's inverse FFT runs in the
registers of one warp per two templates (32 lanes); for n_theta = 60, 120,
180, 240, 360 and 480 on 30 lanes (a mixed-radix 2 x 3 x 5 transform across
the lanes).  Checked against the oracle at those
n: odd and even ragged template counts (8- and 16-byte staging of the spectra,
a zero-filled tail), both translation modes and both level rules, the full
single-pair curve, and unusable templates next to usable ones.  The
shared-memory form, forced through the autotune cache, is checked at the same
n against the same bar.
"""
import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign
from tests.parity import check_argmin, d2_tol, norm_scale
from tests.test_gpu_parity import blobs, compare_batch, f32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def al():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = swalign.Aligner(0)
    yield a
    a.close()


@pytest.mark.parametrize("n,M,nt,translation,level_rule", [
    (64, 24, 19, 1, 0),    # odd template count: 8-byte staging, two CTAs, ragged tail
    (128, 32, 22, 0, 0),   # even ragged count, rotation-only key
    (256, 16, 17, 1, 1),   # left-endpoint levels
    (256, 48, 33, 0, 1),
    (512, 40, 6, 1, 0),    # 16 values per lane
    # 30 lanes: n = 30 MW
    (60, 16, 9, 1, 0),
    (120, 24, 22, 0, 0),
    (180, 32, 17, 1, 1),
    (240, 24, 33, 0, 1),
    (360, 40, 19, 1, 0),   # the serving and single-pair angle count
    (360, 24, 16, 0, 0),
    (480, 32, 6, 1, 0),
])
def test_register_form_matches_oracle(al, n, M, nt, translation, level_rule):
    rng = np.random.default_rng(n + nt)
    L = 36
    q = f32(blobs(rng, 2, L))
    t = f32(blobs(rng, nt, L))
    compare_batch(al, q, t, n=n, M=M, translation=translation, level_rule=level_rule)


@pytest.mark.parametrize("translation", [1, 0])
@pytest.mark.parametrize("n", [128, 256, 360, 120])
def test_register_form_single_pair_curve(al, n, translation):
    rng = np.random.default_rng(n + translation)
    L, M = 48, 40
    f, g = f32(blobs(rng, 2, L))
    p = swalign.make_params(L, n, M, translation=translation)
    D, S, best = al.align_all_rotations(f, g, p)
    D, S = D.cpu().numpy(), S.cpu().numpy()
    r = swalign.results_to_numpy(best)[0]
    f64, g64 = f.astype(np.float64), g.astype(np.float64)
    ref, Dref, Sref = oracle.align_pair(f64, g64, n, M, translation=translation)
    Sc = norm_scale(f64, g64, n, M)
    assert np.all(np.abs(D - Dref) <= d2_tol(Dref, Sc)), np.max(np.abs(D - Dref))
    np.testing.assert_allclose(S, Sref, rtol=0, atol=1e-6)
    assert r["status"] == 0
    assert check_argmin(int(r["best_l"]), ref["best_l"], Dref, d2_tol(ref["d2"], Sc))
    assert r["d2"] == D[r["best_l"]]


def test_unusable_partner_template_leaves_its_pair_unchanged(al):
    """Templates 2s and 2s + 1 share one complex transform: an unusable one
    (negative mass) is zeroed, so the other's result is that of a batch
    without it, bit for bit."""
    rng = np.random.default_rng(12)
    L, n, M = 32, 64, 16
    q = f32(blobs(rng, 2, L))
    good = f32(blobs(rng, 3, L))
    t = f32(np.stack([good[0], -good[1], good[2]]))  # template 1 is the partner of 0
    p = swalign.make_params(L, n, M)
    r = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(2, 3)
    alone = swalign.results_to_numpy(al.align_batch(q, t[:1], p)).reshape(2, 1)
    for i in range(2):
        assert r[i, 0]["status"] == 0 and r[i, 2]["status"] == 0
        assert r[i, 1]["status"] == 2 and np.isnan(r[i, 1]["d2"])
        assert r[i, 0]["best_l"] == alone[i, 0]["best_l"]
        assert r[i, 0]["d2"] == alone[i, 0]["d2"]


@pytest.mark.parametrize("n,dec", [(64, 8), (256, 4), (512, 16), (360, 8), (60, 16)])
def test_shared_memory_form_at_register_sizes(al, tmp_path, n, dec):
    """The shared-memory form, taken through the autotune cache, at n where
    the register form is the default: both meet the oracle's bar."""
    rng = np.random.default_rng(n * 3 + dec)
    L, M = 32, 24
    q = f32(blobs(rng, 2, L))
    t = f32(blobs(rng, 7, L))
    p = swalign.make_params(L, n, M)
    dev = torch.cuda.get_device_name(0).replace(" ", "_").replace("\t", "_")
    B = p.n_bins or al.default_bins(p.L)
    cache = tmp_path / "tune.txt"
    for form in (dec, 1):
        cache.write_text(f"swtune2 {dev} L={p.L} n={p.n_theta} M={p.n_levels} B={B} "
                         f"prec={p.gemm_precision} 304 8 {form} 0 0 0\n")
        assert al.autotune(p, cache)[2] == form
        compare_batch(al, q, t, n=n, M=M)
