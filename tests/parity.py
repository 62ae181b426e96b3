"""Tolerances for comparing the CUDA path with the FP64 oracle.

Distances (FP32 correlation path): |d2_gpu - d2_ref| <= 1e-5 * max(d2_ref, 0.1 S),
S = (N_f + N_g) / (n M) with N the centred quantile norm.  The relative bound
1e-5 is the stated FP32 target; the floor 0.1 S covers the cancellation in
N_f + N_g - 2 corr, whose FP32 rounding scales with S, not with d2 (so a
relative bound alone is undefined as d2 -> 0, e.g. for self-comparisons).
Reduced precision (BF16/FP16 correlation): the same with 1e-2.  Both carry an
absolute floor of 1e-12: the quantiles are FP32 values of magnitude <= 2
(half an ulp <= 1.2e-7), and when both the distance and the centred norms
vanish (e.g. M = 1, n = 4, where every centred quantile is 0) only the squared
rounding of the quantiles remains.

Quantiles: |Q_gpu - Q_ref| <= 2.5e-7 |Q_ref| + 1e-7 -- the FP32 bin width h
(relative error <= 6e-8), the node e_j = (j - B/2) h (one more rounding) and
the final rounding of Q (half an ulp), plus the interpolation fraction.

Argmin: identical, except at ties -- the GPU's choice l_gpu is accepted when
the oracle's own curve puts it within the distance tolerance of the optimum,
D_ref(l_gpu) - D_ref(l_ref) <= tol (several rotations are then correct).
"""
import numpy as np

import oracle

REL_FP32 = 1e-5
REL_LP = 1e-2


def norm_scale(f, g, n, M, level_rule=0, projector=0):
    """S = (N_f + N_g) / (n M) from the oracle's centred quantiles (projector
    0: linear splat; 1: Fourier slice, rows clipped at zero)."""
    tot = 0.0
    for img in (f, g):
        F, mass = oracle.prepare(img)
        if mass <= 0:
            return np.nan
        if projector:
            U = np.maximum(oracle.project_slice(F, n), 0.0)
        else:
            U = oracle.project(F, n)
        Q = oracle.quantiles(U, 2.0 / F.shape[0], M, level_rule)
        _, Qc = oracle.center(Q)
        tot += float((Qc ** 2).sum())
    return tot / (n * M)


def norm_scale_rfsw(f, g, n, M, B, level_rule=0):
    """S for the ramp-filtered distance: both parts' centred norms."""
    tot = 0.0
    for img in (f, g):
        F, mass = oracle.prepare(img)
        if mass <= 0:
            return np.nan
        for part in oracle.rfsw_parts(oracle.project(F, n, B)):
            Q = oracle.quantiles(part, 2.0 / F.shape[0], M, level_rule)
            _, Qc = oracle.center(Q)
            tot += float((Qc ** 2).sum())
    return tot / (n * M)


# Quantiles of the ramp-filtered parts are checked in CDF space: the FP32
# FFT filter leaves an absolute error of at most (2 ceil(log2 B) + 2) u
# max|Ut| in every filtered bin (u = 2^-24, forward and inverse transform),
# so the part's normalised CDF is off by at most B times that over its mass
# T; a GPU quantile q must then sit at a level F_ref(q) within that of its
# own level z_p.  (A bar on q itself would be unbounded where a part is thin:
# the negative part's tails hold ~1e-3 of the peak per bin.)  The distances,
# which average over levels and angles, stay within the FP32 bar above.
def rfsw_level_tol(Ut_row, part_row):
    B = Ut_row.size
    gamma = (2 * np.ceil(np.log2(B)) + 2) * 2.0 ** -24
    return B * gamma * np.abs(Ut_row).max() / part_row.sum()


def level_of(q, part_row, h):
    """The oracle's normalised CDF of a part row at positions q (nodes
    e_j = (j - B/2) h, linear in between)."""
    B = part_row.size
    F = np.concatenate([[0.0], np.cumsum(part_row)]) / part_row.sum()
    e = (np.arange(B + 1) - 0.5 * B) * h
    return np.interp(q, e, F)


ABS_FLOOR = 1e-12


def d2_tol(d2_ref, S, rel=REL_FP32):
    return rel * np.maximum(d2_ref, 0.1 * S) + ABS_FLOOR


def q_tol(q_ref):
    return 2.5e-7 * np.abs(q_ref) + 1e-7


def check_argmin(l_gpu, l_ref, D_ref, tol):
    """True when l_gpu is l_ref or ties with it within tol on the oracle curve."""
    if l_gpu == l_ref:
        return True
    return D_ref[l_gpu] - D_ref[l_ref] <= tol

