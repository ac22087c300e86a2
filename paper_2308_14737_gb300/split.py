"""Splitting and removal of Gaussians between optimisation rounds (paper Sec. 8).

Host-side logic over the K Gaussians of an object (O(K), run between rounds); the
per-Gaussian loss it needs -- a sum over a batch of rays of the ray's loss times
the Gaussian's normalised weight on that ray -- comes from the library's
``fmb_loss_attribution`` kernel (``Renderer.attribution``).

* removal (Eq. 18): lambda_i <= mean(lambda) - z_lambda std(lambda), z_lambda = 2;
* splitting (Eq. 19): l_i >= mean(l) + z_l std(l), z_l = 1, with l_i the average
  loss attributed to Gaussian i over the batch of M rays;
* a split (Eq. 20-23) replaces a Gaussian by two: means shifted by
  +- sigma_1 sqrt(2/pi) along the dominant eigenvector v_1 of its covariance, the
  dominant standard deviation scaled by sqrt(1 - 2/pi) (the half-normal's moments),
  the other axes kept, log(lambda) plus N(0, 0.1) noise each.

sigma_1 is read as the dominant standard deviation (the square root of the
covariance's largest eigenvalue): the half-normal's mean offset sigma sqrt(2/pi)
and deviation sigma sqrt(1 - 2/pi) are in units of a standard deviation.  With it
the two halves, equally weighted, keep the original mean and covariance.
"""

from __future__ import annotations

import numpy as np

HALF_NORMAL_SHIFT = np.sqrt(2.0 / np.pi)  # ~0.8
HALF_NORMAL_SCALE = np.sqrt(1.0 - 2.0 / np.pi)  # ~0.6


def remove_mask(weights, z: float = 2.0) -> np.ndarray:
    """Eq. 18: Gaussians whose weight lies z standard deviations below the mean."""
    lam = np.asarray(weights, dtype=np.float64)
    return lam <= lam.mean() - z * lam.std()


def split_mask(attribution, n_rays: int, z: float = 1.0) -> np.ndarray:
    """Eq. 19: Gaussians whose average attributed loss (attribution / n_rays) lies
    z standard deviations above the mean."""
    l = np.asarray(attribution, dtype=np.float64) / max(int(n_rays), 1)
    return l >= l.mean() + z * l.std()


def _unpack(c):
    L = np.zeros(c.shape[:-1] + (3, 3))
    L[..., 0, 0], L[..., 1, 0], L[..., 1, 1] = c[..., 0], c[..., 1], c[..., 2]
    L[..., 2, 0], L[..., 2, 1], L[..., 2, 2] = c[..., 3], c[..., 4], c[..., 5]
    return L


def _pack(L):
    return np.stack([L[..., 0, 0], L[..., 1, 0], L[..., 1, 1], L[..., 2, 0], L[..., 2, 1], L[..., 2, 2]], -1)


def split_gaussians(means, chol, weights, idx, rng=None, noise: float = 0.1):
    """Eq. 20-23 for the Gaussians ``idx``: returns (means, chol, weights) of the
    2 len(idx) replacements, the pair of Gaussian idx[k] at rows 2k and 2k + 1.
    ``chol`` packs the lower-triangular factor of the precision (Sigma^-1 = L L^T)."""
    rng = rng if rng is not None else np.random.default_rng(0)
    idx = np.asarray(idx, dtype=np.int64)
    mu = np.asarray(means, dtype=np.float64)[idx]
    L = _unpack(np.asarray(chol, dtype=np.float64)[idx])
    prec = L @ np.swapaxes(L, -1, -2)
    cov = np.linalg.inv(prec)
    evals, evecs = np.linalg.eigh(cov)  # ascending: the last is dominant
    sig1 = np.sqrt(evals[:, -1])
    v1 = evecs[:, :, -1]
    shift = (sig1 * HALF_NORMAL_SHIFT)[:, None] * v1
    new_evals = evals.copy()
    new_evals[:, -1] = evals[:, -1] * HALF_NORMAL_SCALE ** 2
    new_cov = evecs @ (new_evals[:, :, None] * np.swapaxes(evecs, -1, -2))
    new_L = np.linalg.cholesky(np.linalg.inv(new_cov))
    out_mu = np.empty((2 * len(idx), 3))
    out_mu[0::2] = mu + shift
    out_mu[1::2] = mu - shift
    out_chol = np.repeat(_pack(new_L), 2, axis=0)
    lam = np.asarray(weights, dtype=np.float64)[idx]
    out_w = np.exp(np.log(np.repeat(lam, 2)) + rng.normal(0.0, noise, 2 * len(idx)))
    return out_mu, out_chol, out_w


def apply(means, chol, weights, attribution, n_rays, rng=None, z_remove: float = 2.0, z_split: float = 1.0):
    """One removal + splitting round: drops the Eq. 18 Gaussians, replaces the
    Eq. 19 ones (among the kept) by their Eq. 20-23 halves.  Returns float32
    (means, chol, weights) and the (removed, split) masks."""
    rm = remove_mask(weights, z_remove)
    sp = split_mask(attribution, n_rays, z_split) & ~rm
    keep = ~rm & ~sp
    m2, c2, w2 = split_gaussians(means, chol, weights, np.nonzero(sp)[0], rng)
    f = lambda a, b: np.concatenate([np.asarray(a, dtype=np.float64)[keep], b]).astype(np.float32)
    return f(means, m2), f(chol, c2), f(weights, w2), rm, sp
