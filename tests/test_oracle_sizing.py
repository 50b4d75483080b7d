"""Pins of the oracle's Eq. 7 sizing field (Sec. 3.3): closed forms and the
properties that define it (a K-Lipschitz function not above lfs on the
samples, attained by some sample)."""
import numpy as np

import oracle as O


def test_single_sample_is_a_cone():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-1, 1, 1000), rng.uniform(-1, 1, 1000)
    mu = O.sizing_field([[0.2, -0.3]], [0.05], 0.1, x, y)
    assert np.allclose(mu, 0.1 * np.hypot(x - 0.2, y + 0.3) + 0.05, rtol=0, atol=1e-16)


def test_zero_gradation_is_uniform():
    rng = np.random.default_rng(1)
    s = rng.uniform(-1, 1, (200, 2))
    lfs = rng.uniform(0.01, 0.2, 200)
    mu = O.sizing_field(s, lfs, 0.0, rng.uniform(-1, 1, 500), rng.uniform(-1, 1, 500))
    assert np.all(mu == lfs.min())


def test_lipschitz_bounded_by_lfs_and_attained():
    rng = np.random.default_rng(2)
    s = rng.uniform(-1, 1, (300, 2))
    lfs = rng.uniform(0.001, 0.3, 300)
    K = 0.2
    x, y = rng.uniform(-1.2, 1.2, 2000), rng.uniform(-1.2, 1.2, 2000)
    mu = O.sizing_field(s, lfs, K, x, y)
    # K-Lipschitz
    i, j = rng.integers(0, 2000, 5000), rng.integers(0, 2000, 5000)
    assert np.all(np.abs(mu[i] - mu[j]) <= K * np.hypot(x[i] - x[j], y[i] - y[j]) + 1e-14)
    # not above lfs on the samples
    assert np.all(O.sizing_field(s, lfs, K, s[:, 0], s[:, 1]) <= lfs)
    # attained: some sample gives the value (the smallest gap is rounding only)
    gap = np.min(K * np.hypot(x[:, None] - s[None, :, 0], y[:, None] - s[None, :, 1]) + lfs[None, :] - mu[:, None], 1)
    assert np.all(np.abs(gap) <= 1e-15)
