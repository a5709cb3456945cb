"""Random complex coefficient vectors and images (seeded)."""

import numpy as np


def random_coefficients(C, q, seed=0, decay=True):
    """alpha of shape (C, q), complex128.

    With ``decay`` the variance of coefficient j falls as 1 / (1 + j), which
    mimics the spectral ordering of an SVD-built basis (low index = smooth).
    """
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(C, q)) + 1j * rng.normal(size=(C, q))
    if decay:
        a = a / np.sqrt(1.0 + np.arange(q))[None, :]
    return a / np.sqrt(2.0)


def random_image(shape, seed=0):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)) / np.sqrt(2.0)
