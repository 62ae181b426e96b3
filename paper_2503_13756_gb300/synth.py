"""Seeded synthetic inputs shaped like the paper's workloads.

The paper aligns rotated, shifted, deformed MNIST digits and projection images
of a cryo-EM volume (Sec. 5.3, Sec. 5.4); neither dataset is available, so
these generators stand in for them with heterogeneous, nonnegative, unit-mass
images: mixtures of anisotropic Gaussian blobs, copies of them that are
rotated, shifted by whole pixels, warped by a smooth random displacement
field and perturbed by noise, then clipped at 0 and renormalised.  The
random-dense images of the paper's timing tables (Sec. 5.1, Tables 2-3) are
also provided.

This module holds none of the alignment method's arithmetic: it only draws
random numbers and evaluates Gaussians.  Both the CUDA path's tests and the
oracle's tests consume its arrays.

Length units are pixels unless stated.  The image grid is the cell grid of
the library: row r, column c, cell centre at (c + 1/2 - L/2, r + 1/2 - L/2)
pixels from the image centre, y growing with the row index.
"""
from __future__ import annotations

import numpy as np

try:  # scipy's pocketfft build is far faster than numpy's for batched 2-D FFTs
    from scipy import fft as _fft
    _FFT_KW = {"workers": -1}
except ImportError:  # pragma: no cover
    _fft = np.fft
    _FFT_KW = {}

SEED_BASE = 20250317


def _rng(seed):
    return seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)


def _grid(L):
    x = np.arange(L) + 0.5 - L / 2
    X, Y = np.meshgrid(x, x)  # X along columns, Y along rows
    return X, Y


def draw_mixtures(rng, count, L, ncomp=(3, 3), box_px=None, sigma_px=None):
    """Parameters of ``count`` blob mixtures.

    ncomp: inclusive range of the number of components.  box_px: side of the
    central square holding the centres (40 px at L = 64, scaled with L).
    sigma_px: range of the per-axis standard deviations (3-8 px at L = 64,
    scaled with L).  Weights ~ U(0.5, 1), orientations ~ U(0, pi).
    """
    s = L / 64.0
    box = 40.0 * s if box_px is None else float(box_px)
    sig = (3.0 * s, 8.0 * s) if sigma_px is None else sigma_px
    kmax = ncomp[1]
    k = rng.integers(ncomp[0], ncomp[1] + 1, size=count)
    active = np.arange(kmax)[None, :] < k[:, None]
    mu = rng.uniform(-box / 2, box / 2, size=(count, kmax, 2))
    sd = rng.uniform(sig[0], sig[1], size=(count, kmax, 2))
    phi = rng.uniform(0.0, np.pi, size=(count, kmax))
    w = rng.uniform(0.5, 1.0, size=(count, kmax)) * active
    return {"mu": mu, "sd": sd, "phi": phi, "w": w}


def _smooth_field(rng, count, L, sigma_px, amp_px):
    """Displacement fields [count][2][L][L]: white noise filtered by a
    Gaussian of std sigma_px (periodic), scaled so max |d| = amp_px.  Chunks
    of 256 fields draw from their own child generators (spawned in order from
    rng) and run on a thread pool, so the result does not depend on the
    number of threads."""
    out = np.zeros((count, 2, L, L), dtype=np.float32)
    if amp_px == 0.0:
        return out
    f = np.fft.fftfreq(L)
    g = np.exp(-2.0 * (np.pi * sigma_px) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    g = g[:, : L // 2 + 1].astype(np.float32)
    starts = list(range(0, count, 256))
    kids = rng.spawn(len(starts))

    def chunk(c0, kid):
        c1 = min(count, c0 + 256)
        noise = kid.standard_normal((c1 - c0, 2, L, L), dtype=np.float32)
        d = _fft.irfft2(_fft.rfft2(noise) * g, s=(L, L))
        mag = np.sqrt((d ** 2).sum(axis=1)).reshape(c1 - c0, -1).max(axis=1)
        out[c0:c1] = d * (amp_px / np.maximum(mag, 1e-30))[:, None, None, None]

    _parallel(chunk, zip(starts, kids))
    return out


def _parallel(fn, items):
    import concurrent.futures as cf
    import os
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        for fut in [ex.submit(fn, *it) for it in items]:
            fut.result()


def render(params, L, idx=None, beta=None, shift=None, warp=None, noise_std=0.0,
           rng=None, dtype=np.float32):
    """Evaluate mixtures on the L x L grid.

    For each image i (mixture ``idx[i]``), the value at cell centre p is
    A(R(-beta_i) (p + d_i(p) - shift_i)), i.e. the mixture rotated by beta_i,
    shifted by shift_i and warped by the displacement field d_i.  Then
    N(0, noise_std) is added (the blob peaks are the weights, <= 1), the image
    is clipped at 0 and renormalised to unit mass.
    """
    count = params["w"].shape[0] if idx is None else len(idx)
    idx = np.arange(count) if idx is None else np.asarray(idx)
    beta = np.zeros(count) if beta is None else np.asarray(beta, dtype=float)
    shift = np.zeros((count, 2)) if shift is None else np.asarray(shift, dtype=float)
    wt = np.float64 if np.dtype(dtype) == np.float64 else np.float32  # working type
    X, Y = (a.astype(wt) for a in _grid(L))
    out = np.empty((count, L, L), dtype=dtype)

    def col(a):
        return np.asarray(a, dtype=wt)[:, None, None]

    def chunk(sl, noise):
        n = sl.stop - sl.start
        px = X[None] - col(shift[sl, 0])
        py = Y[None] - col(shift[sl, 1])
        if warp is not None:
            px = px + warp[sl, 0].astype(wt)
            py = py + warp[sl, 1].astype(wt)
        cb, sb = col(np.cos(beta[sl])), col(np.sin(beta[sl]))
        qx = cb * px + sb * py       # R(-beta) p
        qy = -sb * px + cb * py
        img = np.zeros((n, L, L), dtype=wt)
        ii = idx[sl]
        for j in range(params["w"].shape[1]):
            w = params["w"][ii, j]
            if not np.any(w):
                continue
            # exponent -1/2 (dx, dy) P (dx, dy)^T with P = R diag(1/sx^2, 1/sy^2) R^T
            cp, sp = np.cos(params["phi"][ii, j]), np.sin(params["phi"][ii, j])
            ix, iy = 1.0 / params["sd"][ii, j, 0] ** 2, 1.0 / params["sd"][ii, j, 1] ** 2
            pxx = col(-0.5 * (cp * cp * ix + sp * sp * iy))
            pyy = col(-0.5 * (sp * sp * ix + cp * cp * iy))
            pxy = col(-(cp * sp * (ix - iy)))
            dx = qx - col(params["mu"][ii, j, 0])
            dy = qy - col(params["mu"][ii, j, 1])
            e = pxx * dx * dx + pyy * dy * dy + pxy * dx * dy
            img += col(w) * np.exp(e)
        if noise is not None:
            img += noise
        np.maximum(img, 0.0, out=img)
        mass = img.reshape(n, -1).sum(axis=1, dtype=np.float64)
        img /= col(np.where(mass > 0, mass, 1.0))
        out[sl] = img

    # chunks of 128 images run on a thread pool (numpy releases the GIL); each
    # draws its noise from its own child generator, spawned in order from rng
    starts = list(range(0, count, 128))
    kids = rng.spawn(len(starts)) if noise_std > 0.0 else [None] * len(starts)

    def run(c0, kid):
        sl = slice(c0, min(count, c0 + 128))
        noise = None
        if kid is not None:
            noise = kid.normal(0.0, noise_std, size=(sl.stop - sl.start, L, L)).astype(wt)
        chunk(sl, noise)

    _parallel(run, zip(starts, kids))
    return out


def _perturbed_copies(rng, params, L, idx, max_shift_px, warp_amp_px, warp_sigma_px,
                      noise_std, dtype):
    count = len(idx)
    beta = rng.uniform(0.0, 2 * np.pi, size=count)
    shift = rng.integers(-max_shift_px, max_shift_px + 1, size=(count, 2)).astype(float)
    warp = _smooth_field(rng, count, L, warp_sigma_px, warp_amp_px)
    imgs = render(params, L, idx=idx, beta=beta, shift=shift, warp=warp,
                  noise_std=noise_std, rng=rng, dtype=dtype)
    return imgs, beta, shift


def single_pair(L=64, seed=SEED_BASE + 0, dtype=np.float64):
    """One reference and one rotated/shifted/warped/noisy copy.

    Reference: 3 anisotropic blobs (centres in the central 40 x 40 px box at
    L = 64, sigmas 3-8 px).  Copy: random rotation, integer shift <= 4 px,
    displacement field of max amplitude 2 px (Gaussian-filtered noise, std
    6 px), noise N(0, 0.01), clipped and renormalised.
    """
    rng = _rng(seed)
    p = draw_mixtures(rng, 1, L, ncomp=(3, 3))
    ref = render(p, L, dtype=dtype)
    q, beta, shift = _perturbed_copies(rng, p, L, [0], 4 * L // 64, 2.0 * L / 64,
                                       6.0 * L / 64, 0.01, dtype)
    return {"f": ref[0], "g": q[0], "beta": beta[0], "shift": shift[0]}


def one_reference_batch(n_queries=10000, L=128, seed=SEED_BASE + 1, dtype=np.float32):
    """One reference and ``n_queries`` perturbed copies of it (shift <= 8 px,
    warp 3 px, noise N(0, 0.02))."""
    rng = _rng(seed)
    p = draw_mixtures(rng, 1, L, ncomp=(3, 3))
    ref = render(p, L, dtype=dtype)
    q, beta, shift = _perturbed_copies(rng, p, L, np.zeros(n_queries, dtype=int), 8,
                                       3.0, 6.0 * L / 64, 0.02, dtype)
    return {"reference": ref, "queries": q, "beta": beta, "shift": shift}


def many_to_many(n_queries=4096, n_templates=256, L=128, seed=SEED_BASE + 2,
                 dtype=np.float32):
    """Templates: 2-6 blob mixtures.  Queries: rotated, shifted (<= 8 px) and
    warped (3 px) copies of randomly chosen templates."""
    rng = _rng(seed)
    p = draw_mixtures(rng, n_templates, L, ncomp=(2, 6))
    templates = render(p, L, dtype=dtype)
    src = rng.integers(0, n_templates, size=n_queries)
    q, beta, shift = _perturbed_copies(rng, p, L, src, 8, 3.0, 6.0 * L / 64, 0.0, dtype)
    return {"templates": templates, "queries": q, "source": src, "beta": beta,
            "shift": shift}


UNEVEN_SIZES = (64, 96, 128, 192, 256)
UNEVEN_WEIGHTS = (0.30, 0.25, 0.20, 0.15, 0.10)


def uneven_batch(n_queries=20000, n_templates_per_L=64, seed=SEED_BASE + 3,
                 dtype=np.float32):
    """Queries with L drawn from {64, 96, 128, 192, 256} (0.3/0.25/0.2/0.15/
    0.1), each bucket with its own templates.  Returns a dict keyed by L."""
    rng = _rng(seed)
    Ls = rng.choice(UNEVEN_SIZES, size=n_queries, p=UNEVEN_WEIGHTS)
    out = {}
    for L in UNEVEN_SIZES:
        nq = int((Ls == L).sum())
        p = draw_mixtures(rng, n_templates_per_L, L, ncomp=(2, 6))
        t = render(p, L, dtype=dtype)
        src = rng.integers(0, n_templates_per_L, size=nq)
        q, beta, shift = _perturbed_copies(rng, p, L, src, 8 * L // 128, 3.0 * L / 128,
                                           6.0 * L / 64, 0.0, dtype)
        out[L] = {"templates": t, "queries": q, "source": src, "beta": beta,
                  "shift": shift}
    return out


def upsample2(img):
    """2 x 2 replication with value / 4: the same cell-average image on a
    grid twice as fine (exact under the cell-average model)."""
    return np.repeat(np.repeat(img, 2, axis=-1), 2, axis=-2) / 4.0


def serving_bank(n_templates=1000, L=256, seed=SEED_BASE + 4, dtype=np.float32):
    rng = _rng(seed)
    p = draw_mixtures(rng, n_templates, L, ncomp=(2, 6))
    return {"templates": render(p, L, dtype=dtype), "params": p, "rng": rng}


def serving_pool(bank, pool_size=256, seed=SEED_BASE + 5, max_shift_px=8, warp_amp_px=3.0):
    """Perturbed copies of bank templates (random rotation, shift, warp) at
    the bank's side L and at L/2 (rendered at L and block-averaged 2 x 2),
    from which serving requests draw their images."""
    rng = _rng(seed)
    p = bank["params"]
    Lb = bank["templates"].shape[-1]
    nt = bank["templates"].shape[0]
    out = {}
    for L in (Lb, Lb // 2):
        src = rng.integers(0, nt, size=pool_size)
        beta = rng.uniform(0, 2 * np.pi, size=pool_size)
        shift = rng.integers(-max_shift_px, max_shift_px + 1, size=(pool_size, 2)).astype(float)
        warp = _smooth_field(rng, pool_size, Lb, 6.0 * Lb / 64, warp_amp_px)
        fine = render(p, Lb, idx=src, beta=beta, shift=shift, warp=warp, dtype=np.float32)
        if L != Lb:
            k = Lb // L
            fine = fine.reshape(pool_size, L, k, L, k).sum(axis=(2, 4), dtype=np.float64)
            fine = fine.astype(np.float32)
        out[L] = {"images": fine, "source": src, "beta": beta}
    return out


def serving_schedule(n_requests, rate_hz=200.0, max_images=512, Lb=256, seed=SEED_BASE + 6):
    """Poisson arrivals at rate_hz; per request a count log-uniform on
    [1, max_images] and L = Lb or Lb/2 with equal odds."""
    rng = _rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    counts = np.clip(np.round(np.exp(rng.uniform(0, np.log(max_images), n_requests))), 1,
                     max_images).astype(int)
    Ls = np.where(rng.random(n_requests) < 0.5, Lb, Lb // 2)
    picks = [rng.integers(0, 1 << 30, size=c) for c in counts]
    return t, counts, Ls, picks


def random_dense(L, count=2, seed=SEED_BASE + 9, dtype=np.float32):
    """The timing workload of Tables 2-3: pixels ~ U[0, 1), unit mass."""
    rng = _rng(seed)
    x = rng.random((count, L, L))
    x /= x.reshape(count, -1).sum(axis=1)[:, None, None]
    return x.astype(dtype)
