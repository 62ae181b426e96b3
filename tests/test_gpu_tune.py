"""Autotuned launch shapes (sw_autotune).

The choice is kept per parameter set and read back from the cache file
without timing; every candidate launch shape and every FFT plan (radix order,
radix-4 or radix-8 stages) gives results within the FP32 parity bar of the
oracle (the plan changes the rounding only); a bank keeps the shapes it was
created with.
"""
import numpy as np
import pytest

from paper_2503_13756_gb300 import swalign
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


def cache_key(al, p):
    dev = torch.cuda.get_device_name(0).replace(" ", "_").replace("\t", "_")
    B = p.n_bins or al.default_bins(p.L)
    return f"swtune2 {dev} L={p.L} n={p.n_theta} M={p.n_levels} B={B} prec={p.gemm_precision}"


def test_autotune_keeps_and_caches_its_choice(al, tmp_path):
    p = swalign.make_params(48, 60, 32)  # n = 60 = 4 * 3 * 5: the radix orders differ
    cache = tmp_path / "tune.txt"
    assert al.tune_choice(p) == (0, 0, 0, 0, 0, 0)
    want, spec, dec, plan, tile_s, tile_l = al.autotune(p, cache)
    # n = 60 = 30 x 2: the register form (1) is a candidate beside the shared widths
    assert want in (304, 456, 912) and spec in (4, 8, 16) and dec in (1, 8, 16)
    assert plan in range(8)
    assert tile_s in (128, 256) and tile_l in (128, 256)  # FP32 split on the tensor cores
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith(cache_key(al, p) + " ")
    # a second context reads the cache and launches nothing
    b = swalign.Aligner(0)
    try:
        n0 = b.launch_count()
        assert b.autotune(p, cache) == (want, spec, dec, plan, tile_s, tile_l)
        assert b.launch_count() == n0
        # other parameters are untouched
        assert b.tune_choice(swalign.make_params(48, 60, 16)) == (0, 0, 0, 0, 0, 0)
    finally:
        b.close()
    assert len(cache.read_text().splitlines()) == 1


@pytest.mark.parametrize("n,plan,spec,dec", [
    (60, 0, 16, 8), (60, 1, 8, 16), (60, 2, 4, 4), (60, 3, 16, 16),
    (36, 1, 4, 16), (36, 3, 8, 4), (256, 0, 4, 16), (40, 2, 8, 8),
    # radix-8 plans: 256 = 8 8 4, 512 = 8 8 8, 120 = 8 3 5 / 5 3 8, 1024 = 8 8 8 2
    (256, 4, 8, 8), (512, 6, 16, 4), (120, 5, 4, 8), (120, 7, 16, 16), (1024, 4, 8, 16),
])
def test_every_launch_shape_matches_oracle(al, tmp_path, n, plan, spec, dec):
    rng = np.random.default_rng(n * 10 + plan)
    L, M = 40, 24
    q = f32(blobs(rng, 3, L))
    t = f32(blobs(rng, 5, L))
    p = swalign.make_params(L, n, M)
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{cache_key(al, p)} 304 {spec} {dec} {plan} 0 0\n")
    assert al.autotune(p, cache) == (304, spec, dec, plan, 0, 0)
    compare_batch(al, q, t, n=n, M=M)


def test_bank_keeps_its_launch_shapes(al, tmp_path):
    rng = np.random.default_rng(8)
    L, n, M = 48, 60, 32
    t = f32(blobs(rng, 9, L))
    q = f32(blobs(rng, 4, L))
    p = swalign.make_params(L, n, M)
    cache = tmp_path / "tune.txt"
    cache.write_text(f"{cache_key(al, p)} 456 8 16 3 128 128\n")
    al.autotune(p, cache)
    bank = swalign.Bank(al, t, p)
    try:
        batch = swalign.results_to_numpy(al.align_batch(q, t, p))
        # retune the context: the bank keeps the shapes it was built with
        cache.write_text(f"{cache_key(al, p)} 456 16 8 0 256 256\n")
        al.autotune(p, cache)
        viab = swalign.results_to_numpy(bank.align(q, q_L=L, mode=0))
        np.testing.assert_array_equal(viab["best_l"], batch["best_l"])
        np.testing.assert_array_equal(viab["d2"], batch["d2"])
    finally:
        bank.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("Nt", [9, 64, 70, 130])
def test_both_correlation_tiles_match_oracle(al, tmp_path, precision, Nt):
    # the tensor-core correlation's 128- and 256-column tiles give the same
    # pairs within the bar, for template counts in either class and ragged
    # against either tile
    from tests.parity import REL_FP32, REL_LP
    rng = np.random.default_rng(Nt + len(precision))
    L, n, M = 32, 24, 16
    q = f32(blobs(rng, 3, L))
    t = f32(blobs(rng, Nt, L))
    p = swalign.make_params(L, n, M, precision=precision)
    cache = tmp_path / "tune.txt"
    rel = REL_FP32 if precision == "fp32" else REL_LP
    outs = []
    for tile in (128, 256):
        cache.write_text(f"{cache_key(al, p)} 304 8 8 0 {tile} {tile}\n")
        assert al.autotune(p, cache)[4:] == (tile, tile)
        outs.append(swalign.results_to_numpy(al.align_batch(q, t, p)))
        compare_batch(al, q, t, n=n, M=M, rel=rel, precision=precision)
    a, b = outs
    np.testing.assert_array_equal(a["status"], b["status"])
    # the tile changes neither the products nor their order along K
    np.testing.assert_array_equal(a["best_l"], b["best_l"])
    np.testing.assert_allclose(a["d2"], b["d2"], rtol=1e-6, atol=1e-12)


def test_autotune_times_the_correlation_tile(al):
    # BF16 correlation: the autotuner picks a tile for each template class
    p = swalign.make_params(32, 24, 16, precision="bf16")
    choice = al.autotune(p)
    assert choice[4] in (128, 256) and choice[5] in (128, 256)
