"""Thin ctypes binding of the C ABI in ``include/swalign.h``.

Argument marshalling only: tensors are passed as device pointers with the
current torch CUDA stream; every step of the alignment runs in the CUDA
library.  There is no fallback: if the library cannot be built or loaded,
or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

from . import build as _build

SW_OK, SW_ERR_INVALID_ARG, SW_ERR_UNSUPPORTED, SW_ERR_OOM, SW_ERR_CUDA, SW_ERR_TIMEOUT = range(6)
PREC = {"fp32": 0, "bf16": 1, "fp16": 2, "fp32_simt": 3}

RESULT_DTYPE = np.dtype(
    [("best_l", "<i4"), ("status", "<i4"), ("angle_rad", "<f4"), ("template_index", "<i4"),
     ("shift", "<f8", (2,)), ("d2", "<f8")],
    align=True,
)
assert RESULT_DTYPE.itemsize == 40


class Params(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in
                ("L", "n_theta", "n_levels", "n_bins", "translation", "level_rule",
                 "gemm_precision", "metric", "shift_grid", "shift_step_q", "projector")]


METRIC = {"sw2": 0, "rfsw2": 1, "msw2": 2}
PROJECTOR = {"splat": 0, "slice": 1}


def make_params(L, n_theta, n_levels, n_bins=0, translation=1, level_rule=0,
                precision="fp32", metric="sw2", shift_grid=0, shift_step_q=0,
                projector="splat") -> Params:
    """shift_grid = K > 0 restricts the translation to the grid (i, j) * step,
    |i|, |j| <= K, step = shift_step_q / 16 pixel.  projector "splat" (linear
    splat) or "slice" (band-limited Fourier-slice projection, L <= 256)."""
    prec = PREC[precision] if isinstance(precision, str) else int(precision)
    met = METRIC[metric] if isinstance(metric, str) else int(metric)
    proj = PROJECTOR[projector] if isinstance(projector, str) else int(projector)
    return Params(int(L), int(n_theta), int(n_levels), int(n_bins), int(translation),
                  int(level_rule), prec, met, int(shift_grid), int(shift_step_q), proj)


def bins_of(params: Params) -> int:
    """Bin count B the library uses for params (sw_params.n_bins, else the
    default; the ramp-filtered metric rounds the default up to an even
    2/3/5-smooth count, the Fourier-slice projector to a multiple of 32 that
    is at least 1.5 L)."""
    if params.n_bins:
        return int(params.n_bins)
    L = int(params.L)
    B = 2 * math.ceil((L - 1) / math.sqrt(2.0)) + 2 if L >= 1 else 0
    if params.projector == PROJECTOR["slice"]:
        # the slice projector's bins are its oversampled grid: a multiple of
        # 32 that is at least 1.5 L
        need = max(B, (3 * L + 1) // 2)
        m = (need + 31) // 32
        if m > 6:  # grids in global memory: 256, 320 or 384 bins
            m = 8 if m <= 8 else (10 if m <= 10 else 12)
        return 32 * m
    if params.metric == METRIC["rfsw2"]:
        def smooth(m):
            for q in (2, 3, 5):
                while m % q == 0:
                    m //= q
            return m == 1
        while B % 2 or not smooth(B):
            B += 1
    return B


class SwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"swalign status {status}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

EXPORTS = (
    "sw_create", "sw_destroy", "sw_last_error", "sw_default_bins", "sw_set_workspace_limit",
    "sw_batch_workspace_bytes", "sw_reserve", "sw_project", "sw_quantiles",
    "sw_align_all_rotations", "sw_align_batch", "sw_bank_create", "sw_bank_align",
    "sw_bank_size", "sw_bank_destroy", "sw_profile", "sw_profile_read", "sw_launch_count",
    "sw_align_all_rotations_noalloc", "sw_bank_workspace_bytes", "sw_autotune",
    "sw_autotune_get", "sw_set_wait_limit", "sw_set_correlation_stall", "sw_measure_fp32_fma",
    "sw_project_upsampled",
)
STAGES = ("project", "quantile", "spectrum", "corr", "decide", "best", "ramp")


def load(path: str | None = None):
    """Builds (if stale) and loads the library; returns the ctypes handle."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(path or _build.build())
            vp, ci, P = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Params)
            sig = {
                "sw_create": ([ci, ctypes.POINTER(vp)], ci),
                "sw_destroy": ([vp], None),
                "sw_last_error": ([vp], ctypes.c_char_p),
                "sw_default_bins": ([ci], ci),
                "sw_set_workspace_limit": ([vp, ctypes.c_size_t], ci),
                "sw_batch_workspace_bytes": ([P, ci, ci], ctypes.c_size_t),
                "sw_reserve": ([vp, P, ci, ci], ci),
                "sw_project": ([vp, P, vp, ci, vp, vp, vp], ci),
                "sw_project_upsampled": ([vp, P, vp, ci, vp, vp], ci),
                "sw_quantiles": ([vp, P, vp, ci, vp, vp, vp, vp], ci),
                "sw_align_all_rotations": ([vp, P, vp, vp, vp, vp, vp, vp], ci),
                "sw_align_batch": ([vp, P, vp, ci, vp, ci, ci, vp, vp], ci),
                "sw_bank_create": ([vp, P, vp, ci, ctypes.POINTER(vp), vp], ci),
                "sw_bank_align": ([vp, vp, vp, ci, ci, ci, vp, vp], ci),
                "sw_bank_size": ([vp], ci),
                "sw_bank_destroy": ([vp], None),
                "sw_profile": ([vp, ci], ci),
                "sw_profile_read": ([vp, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int64)], ci),
                "sw_launch_count": ([vp], ctypes.c_int64),
                "sw_align_all_rotations_noalloc": ([P, vp, vp, vp, vp, vp, vp], ci),
                "sw_bank_workspace_bytes": ([vp, ci, ci], ctypes.c_size_t),
                "sw_autotune": ([vp, P, ctypes.c_char_p], ci),
                "sw_autotune_get": ([vp, P, ctypes.POINTER(ci)], ci),
                "sw_set_wait_limit": ([vp, ctypes.c_int64], ci),
                "sw_set_correlation_stall": ([vp, ci], ci),
                "sw_measure_fp32_fma": ([ci, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)], ci),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f32(x, device):
    import torch
    t = torch.as_tensor(x, dtype=torch.float32, device=device)
    return t.contiguous()


class Aligner:
    """One library context (one device, one workspace).  Use one per stream."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("swalign needs a CUDA device; none is visible")
        self.lib = load()
        self.device = device
        self.torch_device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        self._check(self.lib.sw_create(device, ctypes.byref(h)), None)
        self.ctx = h

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.sw_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, status, ctx):
        if status != SW_OK:
            msg = self.lib.sw_last_error(ctx).decode() if ctx else ""
            raise SwError(status, msg)

    def call(self, name, *args):
        self._check(getattr(self.lib, name)(self.ctx, *args), self.ctx)

    # ---------------------------------------------------------------- API
    def autotune(self, params: Params, cache_path: str | None = None):
        """Times candidate launch shapes for params and keeps the fastest
        (sw_autotune); returns the choice (projection CTA target, spectrum
        width, decision width, FFT plan: radix order, radix-4 or radix-8
        stages, correlation tile width for <= 64 and for more templates)."""
        path = None if cache_path is None else str(cache_path).encode()
        self.call("sw_autotune", ctypes.byref(params), path)
        return self.tune_choice(params)

    def tune_choice(self, params: Params):
        out = (ctypes.c_int * 6)()
        self.call("sw_autotune_get", ctypes.byref(params), out)
        return tuple(int(v) for v in out)

    def profile(self, enable: bool):
        self.call("sw_profile", int(bool(enable)))

    def profile_read(self):
        """{stage: (total ms, launches)} since the last read (waits for them)."""
        ms = (ctypes.c_double * 8)()
        cnt = (ctypes.c_int64 * 8)()
        self.call("sw_profile_read", ms, cnt)
        return {name: (ms[i], cnt[i]) for i, name in enumerate(STAGES) if cnt[i]}

    def launch_count(self) -> int:
        return int(self.lib.sw_launch_count(self.ctx))

    def default_bins(self, L: int) -> int:
        return int(self.lib.sw_default_bins(int(L)))

    def set_wait_limit(self, cycles: int):
        """Limit (SM cycles) of the tensor-core pipeline's bounded waits;
        0 restores the default (sw_set_wait_limit)."""
        self.call("sw_set_wait_limit", ctypes.c_int64(int(cycles)))

    def set_correlation_stall(self, enable: bool):
        """Test hook: tensor-core correlations issue no copies while enabled,
        so their bounded waits run out (sw_set_correlation_stall)."""
        self.call("sw_set_correlation_stall", int(bool(enable)))

    def set_workspace_limit(self, nbytes: int):
        self.call("sw_set_workspace_limit", ctypes.c_size_t(int(nbytes)))

    def reserve(self, params: Params, Nq: int, Nt: int):
        self.call("sw_reserve", ctypes.byref(params), int(Nq), int(Nt))

    def project(self, imgs, params: Params, out=None, stream=None, scale=False):
        """Projection rows [nb][n][B]; with scale=True also the FP64 scales
        1 / mass [nb] (NaN for an unusable image)."""
        import torch
        x = _f32(imgs, self.torch_device)
        nb = x.shape[0]
        B = bins_of(params)
        if out is None:
            out = torch.empty((nb, params.n_theta, B), dtype=torch.float32, device=x.device)
        sc = torch.empty((nb,), dtype=torch.float64, device=x.device) if scale else None
        self.call("sw_project", ctypes.byref(params), _ptr(x), nb, _ptr(out), _ptr(sc),
                  _stream(stream))
        return (out, sc) if scale else out

    def project_upsampled(self, imgs, params: Params, out=None, stream=None):
        """Projection rows [nb][n][B] of images of side L/2 upsampled 2 x 2
        (each pixel split into four cells of a quarter of its value)."""
        import torch
        x = _f32(imgs, self.torch_device)
        nb = x.shape[0]
        if x.shape[-1] * 2 != params.L:
            raise ValueError(f"images of side {x.shape[-1]}: want L/2 = {params.L // 2}")
        B = bins_of(params)
        if out is None:
            out = torch.empty((nb, params.n_theta, B), dtype=torch.float32, device=x.device)
        self.call("sw_project_upsampled", ctypes.byref(params), _ptr(x), nb, _ptr(out),
                  _stream(stream))
        return out

    def quantiles(self, proj, params: Params, stream=None):
        import torch
        x = _f32(proj, self.torch_device)
        nb = x.shape[0]
        parts = (2,) if params.metric == METRIC["rfsw2"] else ()
        q = torch.empty((nb, *parts, params.n_theta, params.n_levels), dtype=torch.float32,
                        device=x.device)
        center = torch.empty((nb, *parts, 2), dtype=torch.float64, device=x.device)
        norm = torch.empty((nb, *parts), dtype=torch.float64, device=x.device)
        self.call("sw_quantiles", ctypes.byref(params), _ptr(x), nb, _ptr(q), _ptr(center),
                  _ptr(norm), _stream(stream))
        return q, center, norm

    def align_all_rotations(self, f, g, params: Params, stream=None):
        import torch
        F, G = _f32(f, self.torch_device), _f32(g, self.torch_device)
        n = params.n_theta
        D = torch.empty((n,), dtype=torch.float64, device=F.device)
        S = torch.empty((n, 2), dtype=torch.float64, device=F.device)
        best = torch.empty((40,), dtype=torch.uint8, device=F.device)
        self.call("sw_align_all_rotations", ctypes.byref(params), _ptr(F), _ptr(G), _ptr(D),
                  _ptr(S), _ptr(best), _stream(stream))
        return D, S, best

    def align_batch(self, queries, templates, params: Params, mode=0, out=None, stream=None):
        import torch
        q = _f32(queries, self.torch_device)
        t = _f32(templates, self.torch_device)
        Nq, Nt = q.shape[0], t.shape[0]
        rows = Nq * Nt if mode == 0 else Nq
        if out is None:
            out = torch.empty((rows, 40), dtype=torch.uint8, device=q.device)
        self.call("sw_align_batch", ctypes.byref(params), _ptr(q), Nq, _ptr(t), Nt, int(mode),
                  _ptr(out), _stream(stream))
        return out


class Bank:
    """Device-resident angle spectra of a template set (sw_bank_create)."""

    def __init__(self, aligner: "Aligner", templates, params: Params, stream=None):
        self.al = aligner
        self.params = params
        t = _f32(templates, aligner.torch_device)
        self.Nt = t.shape[0]
        h = ctypes.c_void_p()
        aligner.call("sw_bank_create", ctypes.byref(params), _ptr(t), self.Nt, ctypes.byref(h),
                     _stream(stream))
        self.handle = h

    def workspace_bytes(self, Nq: int, mode: int = 0) -> int:
        return int(self.al.lib.sw_bank_workspace_bytes(self.handle, int(Nq), int(mode)))

    def align(self, queries, q_L=None, mode=0, out=None, stream=None, aligner=None):
        import torch
        al = aligner or self.al
        q = _f32(queries, al.torch_device)
        Nq = q.shape[0]
        q_L = q.shape[-1] if q_L is None else q_L
        rows = Nq * self.Nt if mode == 0 else Nq
        if out is None:
            out = torch.empty((rows, 40), dtype=torch.uint8, device=q.device)
        al.call("sw_bank_align", self.handle, _ptr(q), Nq, int(q_L), int(mode), _ptr(out),
                _stream(stream))
        return out

    def close(self):
        if getattr(self, "handle", None):
            self.al.lib.sw_bank_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_fp32_fma(device: int = 0):
    """(TFLOP/s, ms per probe launch) of FP32 FMAs on the device
    (sw_measure_fp32_fma)."""
    lib = load()
    tf, ms = ctypes.c_double(), ctypes.c_double()
    st = lib.sw_measure_fp32_fma(int(device), ctypes.byref(tf), ctypes.byref(ms))
    if st != SW_OK:
        raise SwError(st, "sw_measure_fp32_fma failed")
    return tf.value, ms.value


def results_to_numpy(buf) -> np.ndarray:
    """Device result buffer ([N][40] uint8) -> structured numpy array."""
    a = buf.detach().cpu().numpy().reshape(-1)
    return a.view(RESULT_DTYPE)
