"""Uneven batches (queries of several sizes, each size against its own
templates, M = L levels, BF16 GEMM) captured as one CUDA graph.

The graph replay gives bitwise the results of the same calls made eagerly,
and sampled pairs of every size agree with the FP64 oracle within the
reduced-precision bar (tests/parity.py); at the full size (20,000 queries x
64 templates per size) the query's own template is found for nearly all
queries.
"""
import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign, synth, uneven
from tests.parity import REL_LP, d2_tol, norm_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_THETA = 256


@pytest.fixture(autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def check_sampled(batch, res, picks_per_L, rng):
    """|d2 - D_ref(l_gpu)| within the reduced-precision bar, l_gpu within one
    bin of the oracle's argmin (circularly), on sampled pairs."""
    near = 0
    total = 0
    for L, d in batch.items():
        q, t = d["queries"], d["templates"]
        r = res[L].reshape(len(q), len(t))
        for _ in range(picks_per_L):
            i, j = int(rng.integers(len(q))), int(rng.integers(len(t)))
            if rng.random() < 0.5:
                j = int(d["source"][i])
            fq, ft = q[i].astype(np.float64), t[j].astype(np.float64)
            rr, Dref, _ = oracle.align_pair(fq, ft, N_THETA, L)
            Sc = norm_scale(fq, ft, N_THETA, L)
            g = r[i, j]
            assert g["status"] == 0
            l = int(g["best_l"])
            assert abs(g["d2"] - Dref[l]) <= d2_tol(Dref[l], Sc, REL_LP), (L, i, j)
            dl = abs((l - int(rr["best_l"]) + N_THETA // 2) % N_THETA - N_THETA // 2)
            near += dl <= 1
            total += 1
    assert near >= 0.95 * total, (near, total)


@pytest.mark.parametrize("concurrent", [True, False])
def test_graph_replay_equals_eager_calls_and_oracle(concurrent):
    # concurrent: one branch (context and stream) per size inside the graph
    batch = synth.uneven_batch(n_queries=150, n_templates_per_L=6)
    g = uneven.UnevenGraph(uneven.buckets_from(batch, N_THETA, "bf16"), mode=0,
                           concurrent=concurrent)
    try:
        assert g.launches_per_replay == 5 * 5  # five kernels per size, all in the graph
        for b in g.buckets:
            b.out.zero_()
        g.replay()
        replay = g.results()
        g.run_eager()
        eager = g.results()
        for L in batch:
            np.testing.assert_array_equal(replay[L]["best_l"], eager[L]["best_l"])
            np.testing.assert_array_equal(replay[L]["d2"], eager[L]["d2"])
            np.testing.assert_array_equal(replay[L]["shift"], eager[L]["shift"])
        check_sampled(batch, replay, 4, np.random.default_rng(1))
        # refill the inputs in place and replay: new results, same graph
        b = g.buckets[0]
        b.queries.copy_(torch.flip(b.queries, dims=(-1,)))
        g.replay()
        flipped = g.results()[b.L]
        ref = swalign.results_to_numpy(
            g.al.align_batch(b.queries, b.templates, b.params)).reshape(-1)
        np.testing.assert_array_equal(flipped["d2"], ref["d2"])
    finally:
        g.close()


def test_graph_with_the_slice_projector_equals_eager_calls():
    # the Fourier-slice projector: L <= 128 in one launch, 192 and 256 with
    # the grids in the context's scratch (two launches per chunk of images),
    # reserved before the capture
    batch = synth.uneven_batch(n_queries=120, n_templates_per_L=4, seed=11)
    g = uneven.UnevenGraph(uneven.buckets_from(batch, N_THETA, "bf16", projector="slice"),
                           mode=0)
    try:
        assert g.launches_per_replay == 5 * 5 + 2 * 2  # L = 192 and 256: grid, tile and row kernels
        for b in g.buckets:
            b.out.zero_()
        g.replay()
        replay = g.results()
        g.run_eager()
        eager = g.results()
        for L in batch:
            assert np.all(replay[L]["status"] == 0)
            np.testing.assert_array_equal(replay[L]["best_l"], eager[L]["best_l"])
            np.testing.assert_array_equal(replay[L]["d2"], eager[L]["d2"])
    finally:
        g.close()


def test_graph_best_template_mode():
    batch = synth.uneven_batch(n_queries=100, n_templates_per_L=5, seed=7)
    g = uneven.UnevenGraph(uneven.buckets_from(batch, N_THETA, "bf16"), mode=1)
    try:
        g.replay()
        best = g.results()
        al = g.al
        for b in g.buckets:
            allp = swalign.results_to_numpy(al.align_batch(b.queries, b.templates, b.params))
            allp = allp.reshape(b.queries.shape[0], b.templates.shape[0])
            j = np.argmin(allp["d2"], axis=1)
            np.testing.assert_array_equal(best[b.L]["d2"], allp["d2"][np.arange(len(j)), j])
    finally:
        g.close()


def test_uneven_full_size_sampled():
    """20,000 queries with L in {64, 96, 128, 192, 256} (0.3/0.25/0.2/0.15/
    0.1), 64 templates per size, n = 256, M = L, BF16 GEMM: one graph."""
    batch = synth.uneven_batch()
    assert sum(len(d["queries"]) for d in batch.values()) == 20000
    g = uneven.UnevenGraph(uneven.buckets_from(batch, N_THETA, "bf16"), mode=0)
    try:
        g.replay()
        res = g.results()
        check_sampled(batch, res, 6, np.random.default_rng(2))
        for L, d in batch.items():
            r = res[L].reshape(len(d["queries"]), len(d["templates"]))
            assert np.all(r["status"] == 0)
            assert np.mean(np.argmin(r["d2"], axis=1) == d["source"]) > 0.9, L
    finally:
        g.close()
