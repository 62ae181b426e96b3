"""FP64 CPU oracle for sliced-2-Wasserstein rigid alignment (arXiv 2503.13756).

TEST INFRASTRUCTURE ONLY.  The product path never imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may.  The oracle shares no code with the CUDA library;
``sw_oracle.c`` is plain C compiled with gcc into ``oracle/_build``.

Every routine follows a passage of the paper (cited in the C source):
projection (Eq. radon_transform, Sec. 2.1; the linear splat, or the
band-limited Fourier-slice projection of Sec. 2.3 and Theorem proj_nufft), CDF / ICDF by cumulative sum and
linear interpolation (Sec. 2.3), the discrete SW2 and its rotation search
(Eq. discrete_sw2, Eq. discrete_rot_sw2), and the translation centring derived
from the shift lemma of App. B.  All routines are pinned by ``tests/
test_oracle_pins.py`` against closed forms, invariants and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrcResult(ctypes.Structure):
    _fields_ = [
        ("best_l", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("angle", ctypes.c_double),
        ("shift", ctypes.c_double * 2),
        ("d2", ctypes.c_double),
    ]


RESULT_DTYPE = np.dtype(
    [("best_l", "<i4"), ("status", "<i4"), ("angle", "<f8"),
     ("shift", "<f8", (2,)), ("d2", "<f8")],
    align=True,
)
assert RESULT_DTYPE.itemsize == ctypes.sizeof(OrcResult)


def build(force: bool = False) -> str:
    """Compile ``sw_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, IEEE)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ci = ctypes.c_int
            lib.orc_default_bins.argtypes = [ci]
            lib.orc_default_bins.restype = ci
            lib.orc_prepare.argtypes = [dp, ci, dp]
            lib.orc_prepare.restype = ctypes.c_double
            lib.orc_project.argtypes = [dp, ci, ci, ci, dp]
            lib.orc_project.restype = None
            lib.orc_quantiles.argtypes = [dp, ci, ci, ctypes.c_double, ci, ci, dp]
            lib.orc_quantiles.restype = ci
            lib.orc_w2_hist_exact.argtypes = [dp, dp, ci, ctypes.c_double]
            lib.orc_w2_hist_exact.restype = ctypes.c_double
            lib.orc_center.argtypes = [dp, ci, ci, dp, dp]
            lib.orc_center.restype = None
            lib.orc_rotation_curve.argtypes = [dp, dp, ci, ci, dp]
            lib.orc_rotation_curve.restype = None
            lib.orc_project_slice.argtypes = [dp, ci, ci, ci, dp]
            lib.orc_project_slice.restype = None
            lib.orc_align_pair.argtypes = [dp, dp, ci, ci, ci, ci, ci, ci, ci, dp, dp,
                                           ctypes.POINTER(OrcResult)]
            lib.orc_align_pair.restype = None
            lib.orc_align_all_pairs.argtypes = [dp, ci, dp, ci, ci, ci, ci, ci, ci,
                                                ci, ci, ci, ctypes.c_void_p]
            lib.orc_align_all_pairs.restype = ci
            lib.orc_transform_images.argtypes = [dp, ci, ci, ci, ci, ci, ci, ci, ci, dp, dp,
                                                 ctypes.POINTER(ctypes.c_int)]
            lib.orc_transform_images.restype = ci
            lib.orc_ramp_filter.argtypes = [dp, ci, ci, dp]
            lib.orc_ramp_filter.restype = None
            lib.orc_rfsw_parts.argtypes = [dp, ci, ci, dp, dp]
            lib.orc_rfsw_parts.restype = None
            lib.orc_rfsw_curve.argtypes = [dp, dp, ci, ci, ci, dp, dp]
            lib.orc_rfsw_curve.restype = None
            lib.orc_align_pair_rfsw.argtypes = lib.orc_align_pair.argtypes
            lib.orc_align_pair_rfsw.restype = None
            lib.orc_align_all_pairs_rfsw.argtypes = lib.orc_align_all_pairs.argtypes
            lib.orc_align_all_pairs_rfsw.restype = ci
            lib.orc_grid_curve.argtypes = [dp, dp, ci, ci, ci, ci, ctypes.c_double, dp, dp]
            lib.orc_grid_curve.restype = None
            lib.orc_align_pair_grid.argtypes = [dp, dp, ci, ci, ci, ci, ci, ci, ci,
                                                ctypes.c_double, ci, dp, dp,
                                                ctypes.POINTER(OrcResult)]
            lib.orc_align_pair_grid.restype = None
            lib.orc_msw_curve.argtypes = [dp, dp, ci, ci, dp]
            lib.orc_msw_curve.restype = None
            lib.orc_align_pair_msw.argtypes = lib.orc_align_pair.argtypes
            lib.orc_align_pair_msw.restype = None
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def default_bins(L: int) -> int:
    return int(_load().orc_default_bins(int(L)))


def prepare(img) -> tuple[np.ndarray, float]:
    """Clamp at 0 and normalise to unit mass; returns (image, mass)."""
    img = _f64(img)
    L = img.shape[-1]
    out = np.empty_like(img)
    mass = _load().orc_prepare(_dp(img), L, _dp(out))
    return out, float(mass)


def project(F, n: int, B: int | None = None) -> np.ndarray:
    """Pixel-driven linear-splat Radon projection, [n][B] float64."""
    F = _f64(F)
    L = F.shape[-1]
    B = default_bins(L) if B is None else int(B)
    U = np.empty((n, B), dtype=np.float64)
    _load().orc_project(_dp(F), L, int(n), B, _dp(U))
    return U


def project_slice(F, n: int, B: int | None = None) -> np.ndarray:
    """Band-limited Fourier-slice projection (signed rows), [n][B] float64:
    U[k][b] = h g~(s_b), g~ the trigonometric polynomial on the period B h
    whose coefficients are the exact slice samples of the cell image."""
    F = _f64(F)
    L = F.shape[-1]
    B = bins_for(L, projector=1) if B is None else int(B)
    U = np.empty((n, B), dtype=np.float64)
    _load().orc_project_slice(_dp(F), L, int(n), B, _dp(U))
    return U


def bins_for(L: int, metric: int = 0, projector: int = 0) -> int:
    """Default bin count.  Fourier-slice projector: the smallest multiple of
    32 that is at least the default B and 1.5 L (the CUDA path's grid length;
    the oracle's direct sums take any B).  Ramp-filtered rows (metric 1):
    the smallest even 2/3/5-smooth count >= the default B.  Otherwise the
    default B."""
    if projector:
        need = max(default_bins(L), (3 * L + 1) // 2)
        m = (need + 31) // 32
        if m > 6:  # the CUDA path's grids above L = 128: 256, 320 or 384
            m = 8 if m <= 8 else (10 if m <= 10 else 12)
        return 32 * m
    return rfsw_bins(L) if metric == 1 else default_bins(L)


def quantiles(U, h: float, M: int, level_rule: int = 0) -> np.ndarray:
    """Quantile functions of the rows of ``U`` ([n][B]) at M levels -> [n][M]."""
    U = _f64(U)
    n, B = U.shape
    Q = np.empty((n, M), dtype=np.float64)
    ok = _load().orc_quantiles(_dp(U), n, B, float(h), int(M), int(level_rule), _dp(Q))
    if not ok:
        raise ValueError("a projection has no positive mass")
    return Q


def w2_hist_exact(Ua, Ub, h: float) -> float:
    Ua, Ub = _f64(Ua), _f64(Ub)
    return float(_load().orc_w2_hist_exact(_dp(Ua), _dp(Ub), Ua.shape[-1], float(h)))


def center(Q) -> tuple[np.ndarray, np.ndarray]:
    """Translation centring: returns (a, Q - <a, e_k>)."""
    Q = _f64(Q)
    n, M = Q.shape
    a = np.empty(2, dtype=np.float64)
    Qc = np.empty_like(Q)
    _load().orc_center(_dp(Q), n, M, _dp(a), _dp(Qc))
    return a, Qc


def rotation_curve(Qf, Qg) -> np.ndarray:
    """D[l] = 1/(nM) sum_k sum_p (Qf[k,p] - Qg[(k-l) mod n, p])^2 (direct)."""
    Qf, Qg = _f64(Qf), _f64(Qg)
    n, M = Qf.shape
    D = np.empty(n, dtype=np.float64)
    _load().orc_rotation_curve(_dp(Qf), _dp(Qg), n, M, _dp(D))
    return D


def align_pair(f, g, n: int, M: int, B: int | None = None, level_rule: int = 0,
               translation: int = 1, projector: int = 0):
    """Full curve for one pair.  Returns (result dict, D[n], shifts[n][2]).
    projector 0: linear splat; 1: Fourier slice, clipped at zero."""
    f, g = _f64(f), _f64(g)
    L = f.shape[-1]
    B = bins_for(L, 0, projector) if B is None else int(B)
    D = np.empty(n, dtype=np.float64)
    S = np.empty((n, 2), dtype=np.float64)
    res = OrcResult()
    _load().orc_align_pair(_dp(f), _dp(g), L, int(n), int(M), B, int(level_rule),
                           int(translation), int(projector), _dp(D), _dp(S),
                           ctypes.byref(res))
    out = {"best_l": res.best_l, "status": res.status, "angle": res.angle,
           "shift": np.array([res.shift[0], res.shift[1]]), "d2": res.d2}
    return out, D, S


def align_all_pairs(queries, templates, n: int, M: int, B: int | None = None,
                    level_rule: int = 0, translation: int = 1,
                    nthreads: int | None = None, projector: int = 0) -> np.ndarray:
    """All pairs: result[i, j] aligns template j onto query i (structured array)."""
    q, t = _f64(queries), _f64(templates)
    Nq, Nt, L = q.shape[0], t.shape[0], q.shape[-1]
    B = bins_for(L, 0, projector) if B is None else int(B)
    nthreads = os.cpu_count() or 1 if nthreads is None else int(nthreads)
    out = np.zeros((Nq, Nt), dtype=RESULT_DTYPE)
    ok = _load().orc_align_all_pairs(_dp(q), Nq, _dp(t), Nt, L, int(n), int(M), B,
                                     int(level_rule), int(translation), int(projector),
                                     nthreads, out.ctypes.data)
    if not ok:
        raise MemoryError("oracle allocation failed")
    return out


def transform_images(imgs, n: int, M: int, B: int | None = None, level_rule: int = 0,
                     projector: int = 0, nthreads: int | None = None):
    """The per-image steps of ``align_pair`` (prepare, project, quantiles,
    centring vector) for every image, in parallel.  Returns (Q [N][n][M]
    uncentred quantiles, A [N][2] centring vectors, ok [N] bool)."""
    x = _f64(imgs)
    N, L = x.shape[0], x.shape[-1]
    B = bins_for(L, 0, projector) if B is None else int(B)
    nthreads = os.cpu_count() or 1 if nthreads is None else int(nthreads)
    Q = np.zeros((N, n, M), dtype=np.float64)
    A = np.zeros((N, 2), dtype=np.float64)
    ok = np.zeros(N, dtype=np.intc)
    _load().orc_transform_images(_dp(x), N, L, int(n), int(M), B, int(level_rule),
                                 int(projector), nthreads, _dp(Q), _dp(A),
                                 ok.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return Q, A, ok.astype(bool)


def shifts_of(af, ag, n: int) -> np.ndarray:
    """s*(l) = a_f - R_{alpha_l} a_g for every l (the closed-form optimal
    translation, derived from the shift lemma of App. B), [n][2]."""
    ang = 2.0 * np.pi * np.arange(n) / n
    c, s = np.cos(ang), np.sin(ang)
    q = n // 4 if n % 4 == 0 else None
    if q is not None:  # exact axis directions at quarter turns, as the oracle's table
        for k, (cc, ss) in zip(range(0, n, q), ((1, 0), (0, 1), (-1, 0), (0, -1))):
            c[k], s[k] = cc, ss
    return np.stack([af[0] - (c * ag[0] - s * ag[1]), af[1] - (s * ag[0] + c * ag[1])], axis=1)


# ---------------------------------------------------------------------------
# Ramp-filtered sliced W2 (Sec. 2.1 "High-pass filter", Eq.
# signed_sliced_wasserstein, Eq. discrete_rot_signed_sw2).

def rfsw_bins(L: int) -> int:
    """Bins of the ramp-filtered path: the smallest even 2/3/5-smooth count at
    least the default B (the filter is circular on the bin grid, so B is part
    of the definition; a smooth B lets the CUDA path use its FFT)."""
    B = default_bins(L)
    while True:
        m = B
        for q in (2, 3, 5):
            while m % q == 0:
                m //= q
        if m == 1 and B % 2 == 0:
            return B
        B += 1


def ramp_filter(U) -> np.ndarray:
    """Rows of U filtered by |xi| circularly on the bin grid (plain DFT sums)."""
    U = _f64(U)
    rows = U.reshape(-1, U.shape[-1])
    out = np.empty_like(rows)
    _load().orc_ramp_filter(_dp(rows), rows.shape[0], rows.shape[1], _dp(out))
    return out.reshape(U.shape)


def rfsw_parts(U) -> tuple[np.ndarray, np.ndarray]:
    """Positive part and absolute negative part of the filtered rows."""
    U = _f64(U)
    rows = U.reshape(-1, U.shape[-1])
    up, um = np.empty_like(rows), np.empty_like(rows)
    _load().orc_rfsw_parts(_dp(rows), rows.shape[0], rows.shape[1], _dp(up), _dp(um))
    return up.reshape(U.shape), um.reshape(U.shape)


def rfsw_curve(Qf, Qg, translation: int = 1):
    """Qf, Qg: [2][n][M] quantiles of the two parts (uncentred).  Returns
    (D[n], shifts[n][2]) from the definition (s* per rotation)."""
    Qf, Qg = _f64(Qf), _f64(Qg)
    _, n, M = Qf.shape
    D = np.empty(n, dtype=np.float64)
    S = np.empty((n, 2), dtype=np.float64)
    _load().orc_rfsw_curve(_dp(Qf), _dp(Qg), n, M, int(translation), _dp(D), _dp(S))
    return D, S


def align_pair_rfsw(f, g, n: int, M: int, B: int | None = None, level_rule: int = 0,
                    translation: int = 1, projector: int = 0):
    """RFSW curve for one pair.  Returns (result dict, D[n], shifts[n][2])."""
    f, g = _f64(f), _f64(g)
    L = f.shape[-1]
    B = rfsw_bins(L) if B is None else int(B)
    D = np.empty(n, dtype=np.float64)
    S = np.empty((n, 2), dtype=np.float64)
    res = OrcResult()
    _load().orc_align_pair_rfsw(_dp(f), _dp(g), L, int(n), int(M), B, int(level_rule),
                                int(translation), int(projector), _dp(D), _dp(S),
                                ctypes.byref(res))
    out = {"best_l": res.best_l, "status": res.status, "angle": res.angle,
           "shift": np.array([res.shift[0], res.shift[1]]), "d2": res.d2}
    return out, D, S


def align_all_pairs_rfsw(queries, templates, n: int, M: int, B: int | None = None,
                         level_rule: int = 0, translation: int = 1,
                         nthreads: int | None = None, projector: int = 0) -> np.ndarray:
    q, t = _f64(queries), _f64(templates)
    Nq, Nt, L = q.shape[0], t.shape[0], q.shape[-1]
    B = rfsw_bins(L) if B is None else int(B)
    nthreads = os.cpu_count() or 1 if nthreads is None else int(nthreads)
    out = np.zeros((Nq, Nt), dtype=RESULT_DTYPE)
    ok = _load().orc_align_all_pairs_rfsw(_dp(q), Nq, _dp(t), Nt, L, int(n), int(M), B,
                                          int(level_rule), int(translation), int(projector),
                                          nthreads, out.ctypes.data)
    if not ok:
        raise MemoryError("oracle allocation failed")
    return out


# ---------------------------------------------------------------------------
# Explicit translation sampling: the translation restricted to the grid
# (i, j) * step, |i|, |j| <= K, by brute force over the grid.

def grid_curve(Qf, Qg, K: int, step: float):
    """Qf, Qg: [parts][n][M] uncentred quantiles.  Returns (D[n], shifts[n][2])."""
    Qf, Qg = _f64(Qf), _f64(Qg)
    parts, n, M = Qf.shape
    D = np.empty(n, dtype=np.float64)
    S = np.empty((n, 2), dtype=np.float64)
    _load().orc_grid_curve(_dp(Qf), _dp(Qg), parts, n, M, int(K), float(step), _dp(D), _dp(S))
    return D, S


def align_pair_grid(f, g, n: int, M: int, K: int, step: float, B: int | None = None,
                    level_rule: int = 0, metric: int = 0, projector: int = 0):
    """One pair with the translation on the grid.  step in domain units
    (the image spans [-1, 1]); metric 0 sliced W2, 1 ramp-filtered."""
    f, g = _f64(f), _f64(g)
    L = f.shape[-1]
    if B is None:
        B = bins_for(L, metric, projector)
    D = np.empty(n, dtype=np.float64)
    S = np.empty((n, 2), dtype=np.float64)
    res = OrcResult()
    _load().orc_align_pair_grid(_dp(f), _dp(g), L, int(n), int(M), int(B), int(level_rule),
                                int(metric), int(K), float(step), int(projector), _dp(D),
                                _dp(S), ctypes.byref(res))
    out = {"best_l": res.best_l, "status": res.status, "angle": res.angle,
           "shift": np.array([res.shift[0], res.shift[1]]), "d2": res.d2}
    return out, D, S


# ---------------------------------------------------------------------------
# Max-sliced W2 over rotations (Eq. max_sliced_wasserstein).

def msw_curve(Qf, Qg) -> np.ndarray:
    """D[l] = max_k (1/M) sum_p (Qf[k,p] - Qg[(k-l) mod n, p])^2 (direct)."""
    Qf, Qg = _f64(Qf), _f64(Qg)
    n, M = Qf.shape
    D = np.empty(n, dtype=np.float64)
    _load().orc_msw_curve(_dp(Qf), _dp(Qg), n, M, _dp(D))
    return D


def align_pair_msw(f, g, n: int, M: int, B: int | None = None, level_rule: int = 0,
                   translation: int = 1, projector: int = 0):
    """Max-sliced curve for one pair.  Returns (result dict, D[n], shifts[n][2])."""
    f, g = _f64(f), _f64(g)
    L = f.shape[-1]
    B = bins_for(L, 0, projector) if B is None else int(B)
    D = np.empty(n, dtype=np.float64)
    S = np.empty((n, 2), dtype=np.float64)
    res = OrcResult()
    _load().orc_align_pair_msw(_dp(f), _dp(g), L, int(n), int(M), B, int(level_rule),
                               int(translation), int(projector), _dp(D), _dp(S),
                               ctypes.byref(res))
    out = {"best_l": res.best_l, "status": res.status, "angle": res.angle,
           "shift": np.array([res.shift[0], res.shift[1]]), "d2": res.d2}
    return out, D, S
