"""Closed-form projections of Gaussian mixtures, used to pin the oracle.

A 2-D Gaussian N(mu, S) projects onto the direction e = (cos t, sin t) as the
1-D Gaussian N(<mu, e>, e^T S e) (the Radon transform of Eq. radon_transform,
Sec. 2.1, applied to a Gaussian).  Its mass in a bin [e_j, e_{j+1}] is a
difference of normal CDFs.  Nothing here comes from the oracle.
"""
import numpy as np

try:
    from scipy.special import ndtr
except ImportError:  # pragma: no cover - scipy is present on both machines
    ndtr = None


def rot(beta):
    c, s = np.cos(beta), np.sin(beta)
    return np.array([[c, -s], [s, c]])


def mixture_hist(weights, means, covs, thetas, B, h):
    """Bin masses [len(thetas)][B] on nodes e_j = (j - B/2) h."""
    edges = (np.arange(B + 1) - B / 2) * h
    out = np.zeros((len(thetas), B))
    for k, t in enumerate(thetas):
        e = np.array([np.cos(t), np.sin(t)])
        for w, mu, S in zip(weights, means, covs):
            m = float(e @ mu)
            sd = float(np.sqrt(e @ S @ e))
            out[k] += w * np.diff(ndtr((edges - m) / sd))
    return out


def random_mixture(rng, ncomp, spread=0.25, smin=0.04, smax=0.10):
    weights = rng.uniform(0.5, 1.0, ncomp)
    means = [rng.uniform(-spread, spread, 2) for _ in range(ncomp)]
    covs = []
    for _ in range(ncomp):
        sx, sy = rng.uniform(smin, smax, 2)
        R = rot(rng.uniform(0, np.pi))
        covs.append(R @ np.diag([sx * sx, sy * sy]) @ R.T)
    return weights, means, covs


def transform_mixture(mix, beta=0.0, shift=(0.0, 0.0)):
    """Mixture of T_shift R_beta f: means R mu + shift, covariances R S R^T."""
    w, means, covs = mix
    R = rot(beta)
    s = np.asarray(shift, dtype=float)
    return w, [R @ m + s for m in means], [R @ S @ R.T for S in covs]


def pixel_image(mix, L):
    """Point samples of the mixture density at the L x L cell centres."""
    h = 2.0 / L
    x = -1.0 + (np.arange(L) + 0.5) * h
    X, Y = np.meshgrid(x, x)  # X varies along columns, Y along rows
    img = np.zeros((L, L))
    for w, mu, S in zip(*mix):
        P = np.linalg.inv(S)
        dx, dy = X - mu[0], Y - mu[1]
        q = P[0, 0] * dx * dx + 2 * P[0, 1] * dx * dy + P[1, 1] * dy * dy
        img += w * np.exp(-0.5 * q) / (2 * np.pi * np.sqrt(np.linalg.det(S)))
    return img
