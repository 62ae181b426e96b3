"""Reduced-precision correlation (tcgen05, BF16 / FP16 operands, FP32
accumulation) against the FP64 oracle.

Bar: |d2_gpu - D_ref(l_gpu)| <= 1e-2 max(D_ref(l_gpu), 0.1 S) + 1e-12 on every
pair, and the rotation within one angular bin (circularly) of the oracle's
on at least 99% of pairs.
"""
import numpy as np
import pytest

import oracle
from paper_2503_13756_gb300 import swalign, synth
from tests.parity import REL_LP, d2_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def al():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = swalign.Aligner(0)
    yield a
    a.close()


def oracle_curves(q, t, n, M, translation=1):
    """Oracle quantiles per image (centred when translating), then every
    pair's rotation curve, spread over host threads (ctypes drops the GIL)."""
    import concurrent.futures as cf
    import os

    def tr(img):
        F, _ = oracle.prepare(img.astype(np.float64))
        Q = oracle.quantiles(oracle.project(F, n), 2.0 / F.shape[0], M)
        a, Qc = oracle.center(Q)
        return (Qc if translation else Q), (Qc ** 2).sum()

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        Tq = list(ex.map(tr, q))
        Tt = list(ex.map(tr, t))
        D = np.empty((len(q), len(t), n))
        S = np.empty((len(q), len(t)))

        def row(i):
            Qi, Ni = Tq[i]
            for j, (Qj, Nj) in enumerate(Tt):
                D[i, j] = oracle.rotation_curve(Qi, Qj)
                S[i, j] = (Ni + Nj) / (n * M)

        list(ex.map(row, range(len(q))))
    return D, S


def check_lowprec(got, D, S, n, frac_ok=0.99):
    l = got["best_l"].astype(int)
    lref = D.argmin(axis=2)
    dref = np.take_along_axis(D, l[..., None], axis=2)[..., 0]
    tol = d2_tol(dref, S, REL_LP)
    assert np.all(got["status"] == 0)
    bad = np.abs(got["d2"] - dref) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], (np.abs(got["d2"] - dref) / tol).max())
    dl = np.abs((l - lref + n // 2) % n - n // 2)
    assert np.mean(dl <= 1) >= frac_ok, np.mean(dl <= 1)
    return float(np.mean(dl == 0))


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("L,n,M,Nq,Nt", [
    (48, 64, 64, 130, 140),   # ragged M tiles (130), N tiles (280 columns)
    (40, 36, 36, 70, 33),     # K = 72 padded to 128, odd template count
    (64, 256, 128, 130, 65),  # n and M of the many-to-many workload
])
def test_lowprec_matches_oracle(al, precision, L, n, M, Nq, Nt):
    rng = np.random.default_rng(L + n + M)
    tp = synth.draw_mixtures(rng, Nt, L, ncomp=(2, 5))
    t = synth.render(tp, L)
    src = rng.integers(0, Nt, Nq)
    q = synth.render(tp, L, idx=src, beta=rng.uniform(0, 2 * np.pi, Nq),
                     shift=rng.integers(-3, 4, (Nq, 2)))
    p = swalign.make_params(L, n, M, precision=precision)
    got = swalign.results_to_numpy(al.align_batch(q, t, p)).reshape(Nq, Nt)
    D, S = oracle_curves(q, t, n, M)
    check_lowprec(got, D, S, n)


def test_lowprec_agrees_with_fp32_path(al):
    rng = np.random.default_rng(3)
    L, n, M = 64, 128, 64
    tp = synth.draw_mixtures(rng, 50, L, ncomp=(2, 5))
    t = synth.render(tp, L)
    q = synth.render(tp, L, idx=rng.integers(0, 50, 300), beta=rng.uniform(0, 6.28, 300))
    r32 = swalign.results_to_numpy(al.align_batch(q, t, swalign.make_params(L, n, M)))
    for prec in ("bf16", "fp16"):
        r = swalign.results_to_numpy(al.align_batch(q, t, swalign.make_params(L, n, M,
                                                                                 precision=prec)))
        rel = np.abs(r["d2"] - r32["d2"]) / np.maximum(r32["d2"], 1e-3 * r32["d2"].mean())
        assert np.quantile(rel, 0.99) < 1e-2, (prec, np.quantile(rel, 0.99))
        dl = np.abs((r["best_l"] - r32["best_l"] + n // 2) % n - n // 2)
        assert np.mean(dl <= 1) >= 0.99
