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


def random_excitations(n_dipoles, L, seed=0):
    """Complex Gaussian excitation amplitudes (n_dipoles x L, unit variance): the
    random amplitudes and phases of the boundary dipoles that sample the range
    of the field operator (complex128)."""
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n_dipoles, L)) + 1j * rng.normal(size=(n_dipoles, L))) / np.sqrt(2.0)
