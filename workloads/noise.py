"""Complex white Gaussian measurement noise at a stated SNR."""

import numpy as np


def noise_sigma_for_snr(y_clean, snr_db):
    """Per-complex-sample noise standard deviation sigma.

    sigma^2 = mean(|y_clean|^2) / 10^(snr_db / 10); each real and imaginary
    part then has variance sigma^2 / 2.
    """
    p = float(np.mean(np.abs(y_clean) ** 2))
    return np.sqrt(p / 10.0 ** (snr_db / 10.0))


def complex_noise(shape, sigma, seed=0):
    rng = np.random.default_rng(seed)
    s = sigma / np.sqrt(2.0)
    return rng.normal(0.0, s, size=shape) + 1j * rng.normal(0.0, s, size=shape)
