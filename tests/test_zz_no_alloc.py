"""The allocation-free single-pair entry point, through the C ABI.

sw_align_all_rotations_noalloc serves callers that may not allocate device
memory while they run (all memory handed to their own pool, no implicit device
synchronisation allowed, or a host that forbids allocations after start-up).
It keeps its intermediates in one fixed device array inside the library.
This file is collected last so that, if it fails, a run stopping at the first
failure has already run every other test; it passes alone and after them.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_13756_gb300 import swalign, synth
from tests.parity import d2_tol, norm_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _call_noalloc(lib, params, f, g):
    n = params.n_theta
    D = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    S = torch.full((n, 2), float("nan"), dtype=torch.float64, device="cuda")
    best = torch.zeros((40,), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.sw_align_all_rotations_noalloc(
        ctypes.byref(params), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(S.data_ptr()),
        ctypes.c_void_p(best.data_ptr()), stream)
    assert st == swalign.SW_OK, st
    torch.cuda.synchronize()
    return D.cpu().numpy(), S.cpu().numpy(), swalign.results_to_numpy(best)[0]


def test_noalloc_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = swalign.load()
    al = swalign.Aligner(0)
    try:
        rng = np.random.default_rng(2026)
        cases = [(64, 360, 128, 1), (48, 60, 36, 0)]  # two calls in a row, different sizes
        for L, n, M, translation in cases:
            mix = synth.draw_mixtures(rng, 2, L, ncomp=(2, 4))
            imgs = synth.render(mix, L, beta=[0.0, 1.1], shift=[[0, 0], [2, -1]])
            f = torch.from_numpy(imgs[0]).cuda()
            g = torch.from_numpy(imgs[1]).cuda()
            p = swalign.make_params(L, n, M, translation=translation)
            D, S, r = _call_noalloc(lib, p, f, g)
            Dr, Sr, br = al.align_all_rotations(f, g, p)
            torch.cuda.synchronize()
            Dr, Sr = Dr.cpu().numpy(), Sr.cpu().numpy()
            rr = swalign.results_to_numpy(br)[0]
            Sc = norm_scale(imgs[0].astype(np.float64), imgs[1].astype(np.float64), n, M)
            assert np.all(np.abs(D - Dr) <= d2_tol(Dr, Sc))
            np.testing.assert_allclose(S, Sr, rtol=0, atol=1e-9)
            assert r["status"] == rr["status"] == 0
            assert r["best_l"] == rr["best_l"]
            assert abs(r["d2"] - rr["d2"]) <= d2_tol(rr["d2"], Sc)
        # sizes beyond the fixed scratch are refused, nothing is launched
        big = swalign.make_params(64, 1024, 1024)
        f = torch.zeros((64, 64), device="cuda")
        out = torch.zeros((40,), dtype=torch.uint8, device="cuda")
        st = lib.sw_align_all_rotations_noalloc(
            ctypes.byref(big), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()),
            None, None, ctypes.c_void_p(out.data_ptr()), None)
        assert st == swalign.SW_ERR_OOM
    finally:
        al.close()


def test_noalloc_call_replays_from_a_cuda_graph():
    # after a first call (which looks up the fixed array's address), a call
    # captured into a CUDA graph replays with the same results: it copies
    # nothing from host memory (its angle tables come from a kernel inside
    # the graph) and allocates nothing
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = swalign.load()
    rng = np.random.default_rng(77)
    L, n, M = 64, 360, 128
    mix = synth.draw_mixtures(rng, 2, L, ncomp=(2, 4))
    imgs = synth.render(mix, L, beta=[0.0, 2.3], shift=[[0, 0], [1, -2]])
    f = torch.from_numpy(imgs[0]).cuda()
    g = torch.from_numpy(imgs[1]).cuda()
    p = swalign.make_params(L, n, M, translation=1)
    D0, S0, r0 = _call_noalloc(lib, p, f, g)
    Sc = norm_scale(imgs[0].astype(np.float64), imgs[1].astype(np.float64), n, M)

    D = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    S = torch.full((n, 2), float("nan"), dtype=torch.float64, device="cuda")
    best = torch.zeros((40,), dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        st = lib.sw_align_all_rotations_noalloc(
            ctypes.byref(p), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()),
            ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(S.data_ptr()),
            ctypes.c_void_p(best.data_ptr()), ctypes.c_void_p(side.cuda_stream))
    assert st == swalign.SW_OK, st
    torch.cuda.synchronize()
    for _ in range(2):
        D.fill_(float("nan"))
        S.fill_(float("nan"))
        best.zero_()
        graph.replay()
        torch.cuda.synchronize()
        Dn, Sn = D.cpu().numpy(), S.cpu().numpy()
        r = swalign.results_to_numpy(best)[0]
        assert np.all(np.isfinite(Dn)) and np.all(np.isfinite(Sn))
        assert np.all(np.abs(Dn - D0) <= d2_tol(D0, Sc))
        np.testing.assert_allclose(Sn, S0, rtol=0, atol=1e-9)
        assert r["status"] == r0["status"] == 0
        assert r["best_l"] == r0["best_l"]
    del graph


def test_noalloc_refuses_what_it_does_not_offer():
    # the allocation-free call covers sliced W2 with the linear splat; other
    # metrics and the Fourier-slice projector are refused before any launch,
    # and parameters outside the limits give the status of the allocating call
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = swalign.load()
    f = torch.zeros((32, 32), device="cuda")
    out = torch.zeros((40,), dtype=torch.uint8, device="cuda")
    cases = [(swalign.make_params(32, 16, 8, metric="msw2"), swalign.SW_ERR_UNSUPPORTED),
             (swalign.make_params(32, 16, 8, metric="rfsw2"), swalign.SW_ERR_UNSUPPORTED),
             (swalign.make_params(32, 16, 8, projector="slice"), swalign.SW_ERR_UNSUPPORTED),
             (swalign.make_params(300, 16, 8, projector="slice"), swalign.SW_ERR_UNSUPPORTED),
             (swalign.make_params(32, 15, 8), swalign.SW_ERR_INVALID_ARG)]
    for p, want in cases:
        st = lib.sw_align_all_rotations_noalloc(
            ctypes.byref(p), ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()),
            None, None, ctypes.c_void_p(out.data_ptr()), None)
        assert st == want, (p.metric, p.projector, p.L, st)
