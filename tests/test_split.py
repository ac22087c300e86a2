"""Host-side splitting and removal of Gaussians (Sec. 8): moment preservation of a
split (half-normal shift and scale, Eq. 20-21), the z-score criteria (Eq. 18-19)
and the bookkeeping of one round."""

import numpy as np

from paper_2308_14737_gb300 import split, synth


def _cov(c):
    L = split._unpack(np.asarray(c, dtype=np.float64))
    return np.linalg.inv(L @ np.swapaxes(L, -1, -2))


def test_split_keeps_mean_and_covariance():
    """Two halves of equal weight: their mixture has the original mean and
    covariance (sigma_1^2 (1 - 2/pi) + (sigma_1 sqrt(2/pi))^2 = sigma_1^2 along
    v_1, the other axes untouched), and the halves differ only along v_1."""
    rng = np.random.default_rng(0)
    mu, chol, lam = synth.random_gaussians(rng, 6, "cholesky")
    m2, c2, w2 = split.split_gaussians(mu, chol, lam, np.arange(6), np.random.default_rng(1))
    for i in range(6):
        a, b = m2[2 * i], m2[2 * i + 1]
        np.testing.assert_allclose((a + b) / 2, mu[i], atol=1e-6)
        ca = _cov(c2[2 * i])
        mix = ca + 0.25 * np.outer(a - b, a - b)  # equal-weight mixture of N(a, ca), N(b, ca)
        np.testing.assert_allclose(mix, _cov(chol[i]), rtol=1e-5, atol=1e-9)
        ev, V = np.linalg.eigh(_cov(chol[i]))
        d = (a - b) / np.linalg.norm(a - b)
        assert abs(abs(d @ V[:, -1]) - 1) < 1e-9  # along the dominant eigenvector
        np.testing.assert_allclose(np.linalg.norm(a - b) / 2, np.sqrt(ev[-1]) * np.sqrt(2 / np.pi), rtol=1e-9)
        np.testing.assert_allclose(np.linalg.eigvalsh(ca)[-1] <= ev[-1], True)
    # log-weights: the original plus N(0, 0.1) noise
    dl = np.log(w2) - np.log(np.repeat(lam, 2))
    assert np.all(np.abs(dl) < 0.6) and np.std(dl) > 0.01


def test_criteria_z_scores():
    lam = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 1.0, 0.01])
    rm = split.remove_mask(lam)
    assert rm.tolist() == [False] * 7 + [True]
    att = np.array([1.0, 1.0, 1.0, 9.0, 1.0])
    sp = split.split_mask(att * 10, 10)
    assert sp.tolist() == [False, False, False, True, False]


def test_apply_round():
    rng = np.random.default_rng(2)
    mu, chol, lam = synth.random_gaussians(rng, 10, "cholesky")
    lam[3] = 1e-4
    att = np.ones(10)
    att[7] = 50.0
    m, c, w, rm, sp = split.apply(mu, chol, lam, att, 1)
    assert rm[3] and sp[7] and rm.sum() == 1 and sp.sum() == 1
    assert m.shape == (10 - 1 - 1 + 2, 3) and c.shape == (10, 6) and w.shape == (10,)
    np.testing.assert_array_equal(m[:8], np.delete(mu, [3, 7], axis=0))
