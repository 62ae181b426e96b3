"""Template bank and serving loop (continuous batching) on the GPU."""
import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import serving, swalign, synth
from tests.parity import REL_FP32, REL_LP, check_argmin, d2_tol, norm_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def al():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = swalign.Aligner(0)
    yield a
    a.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp32_simt"])
def test_bank_equals_batch(al, precision):
    rng = np.random.default_rng(4)
    L, n, M = 64, 60, 32
    tp = synth.draw_mixtures(rng, 37, L, ncomp=(2, 4))
    t = synth.render(tp, L)
    q = synth.render(tp, L, idx=rng.integers(0, 37, 21), beta=rng.uniform(0, 6.28, 21))
    p = swalign.make_params(L, n, M, precision=precision)
    bank = swalign.Bank(al, t, p)
    try:
        got = swalign.results_to_numpy(bank.align(q))
        ref = swalign.results_to_numpy(al.align_batch(q, t, p))
        assert got.tobytes() == ref.tobytes()  # same kernels, same spectra
        best = swalign.results_to_numpy(bank.align(q, mode=1))
        refb = swalign.results_to_numpy(al.align_batch(q, t, p, mode=1))
        assert best.tobytes() == refb.tobytes()
    finally:
        bank.close()


def test_bank_upsamples_half_size_queries(al):
    # A query at L/2 is upsampled 2x2 on load (each cell split into four of a
    # quarter of its value): the same as aligning the upsampled image.
    rng = np.random.default_rng(5)
    L, n, M = 64, 36, 16
    tp = synth.draw_mixtures(rng, 9, L)
    t = synth.render(tp, L)
    qh = synth.render(synth.draw_mixtures(rng, 5, L // 2), L // 2)
    p = swalign.make_params(L, n, M)
    bank = swalign.Bank(al, t, p)
    try:
        got = swalign.results_to_numpy(bank.align(qh, q_L=L // 2))
        ref = swalign.results_to_numpy(al.align_batch(synth.upsample2(qh), t, p))
        assert got.tobytes() == ref.tobytes()
        # and against the oracle on the upsampled image
        r0 = oracle.align_pair(synth.upsample2(qh[0]).astype(np.float64),
                               t[0].astype(np.float64), n, M)
        assert got[0]["best_l"] == r0[0]["best_l"]
    finally:
        bank.close()


@pytest.mark.parametrize("projector,precision", [("splat", "fp32"), ("slice", "fp32"),
                                                ("slice", "bf16")])
def test_serving_results_are_the_same_alone_and_in_the_mix(projector, precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(6)
    L, n, M = 64, 60, 32
    proj = int(projector == "slice")
    rel = REL_FP32 if precision == "fp32" else REL_LP
    bank = synth.serving_bank(n_templates=48, L=L, seed=rng)
    pool = synth.serving_pool(bank, pool_size=64, seed=rng, max_shift_px=3, warp_amp_px=1.0)
    sched = synth.serving_schedule(24, rate_hz=2000.0, max_images=40, Lb=L, seed=rng)
    reqs = serving.make_requests(pool, sched)
    p = swalign.make_params(L, n, M, precision=precision, projector=projector)
    eng = serving.ServingEngine(bank["templates"], p, n_slots=3, max_batch_images=64)
    try:
        stats = eng.run(reqs, realtime=True)
        assert stats["requests"] == 24 and stats["batches"] >= 2
        assert all(r.t_done >= r.t_arrive for r in reqs)
        for r in reqs[::5]:  # alone: the request as its own batch
            alone = swalign.results_to_numpy(
                eng.bank.align(r.images, q_L=r.images.shape[-1], mode=1))
            for k in range(len(r.images)):
                a, b = alone[k], r.results[k]
                assert a["status"] == b["status"] == 0
                assert int(a["template_index"]) == int(b["template_index"])  # same best template
                j = int(a["template_index"])
                img = r.images[k] if r.images.shape[-1] == L else synth.upsample2(r.images[k])
                _, Dref, _ = oracle.align_pair(img.astype(np.float64),
                                               bank["templates"][j].astype(np.float64), n, M,
                                               projector=proj)
                Sc = norm_scale(img.astype(np.float64),
                                bank["templates"][j].astype(np.float64), n, M, projector=proj)
                # alone and in the mix agree within the bar, and both match the
                # oracle from the images at their rotation
                tol = d2_tol(Dref[int(a["best_l"])], Sc, rel)
                if precision == "fp32":
                    assert check_argmin(int(b["best_l"]), int(a["best_l"]), Dref, tol)
                else:
                    dl = (int(b["best_l"]) - int(a["best_l"]) + n // 2) % n - n // 2
                    assert abs(dl) <= 1
                assert abs(a["d2"] - b["d2"]) <= 2 * tol
                for x in (a, b):
                    assert abs(x["d2"] - Dref[int(x["best_l"])]) <= d2_tol(
                        Dref[int(x["best_l"])], Sc, rel)
        # most queries find their own source template
        hits = np.mean([np.mean(r.results["template_index"].astype(int) == r.source) for r in reqs])
        assert hits > 0.9
    finally:
        eng.close()


def test_serving_memory_admission_limits_batches():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(7)
    L, n, M = 32, 24, 16
    bank = synth.serving_bank(n_templates=16, L=L, seed=rng)
    pool = synth.serving_pool(bank, pool_size=16, seed=rng)
    reqs = serving.make_requests(pool, synth.serving_schedule(10, 1000.0, 30, Lb=L, seed=rng))
    p = swalign.make_params(L, n, M)
    eng = serving.ServingEngine(bank["templates"], p, n_slots=2, max_batch_images=64,
                                mem_fraction=1e-9)  # budget below one batch of 64
    try:
        assert eng.max_batch < 64
        stats = eng.run(reqs, realtime=False)
        assert all(r.t_done >= 0 for r in reqs)
        assert stats["mean_batch_images"] <= eng.max_batch
    finally:
        eng.close()


def test_serving_256_bank_half_size_queries_alone_equal_the_mix():
    # the serving setting's shapes: a bank at 256^2 with queries at 128^2
    # (projected on their own grid) and at 256^2, batched by the engine across
    # slots; every image is computed on its own, so a request's results in
    # the mix are bitwise those of the request alone
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(16)
    L, n, M = 256, 36, 32
    bank = synth.serving_bank(n_templates=20, L=L, seed=rng)
    pool = synth.serving_pool(bank, pool_size=24, seed=rng, max_shift_px=4, warp_amp_px=1.0)
    sched = synth.serving_schedule(16, rate_hz=4000.0, max_images=24, Lb=L, seed=rng)
    reqs = serving.make_requests(pool, sched)
    assert {r.images.shape[-1] for r in reqs} == {L, L // 2}
    p = swalign.make_params(L, n, M, precision="bf16", projector="slice")
    eng = serving.ServingEngine(bank["templates"], p, n_slots=3, max_batch_images=32)
    try:
        eng.run(reqs, realtime=False)
        for r in reqs:
            alone = swalign.results_to_numpy(
                eng.bank.align(r.images, q_L=r.images.shape[-1], mode=1))
            assert np.all(alone["status"] == 0)
            assert alone.tobytes() == r.results.tobytes()
        hits = np.mean(np.concatenate(
            [r.results["template_index"].astype(int) == r.source for r in reqs]))
        assert hits > 0.9
    finally:
        eng.close()
