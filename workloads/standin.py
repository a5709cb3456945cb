"""Smooth orthonormal stand-in bases for timing runs.

The Maxwell basis itself (dipole fields through the free-space Green's function
followed by an SVD, "Maxwell Regularization" section) is built by the FP64
oracle.  Benchmarks only need a basis of the same shape and kind: orthonormal
columns of smooth complex fields, ordered from slow to fast spatial variation.
These generators give exactly that with plain numpy QR, and nothing of the
paper's construction.
"""

import numpy as np


def _low_modes_1d(n, r):
    k = np.arange(n) - n // 2
    order = np.argsort(np.abs(k) + 0.25 * (k < 0), kind="stable")[:r]
    t = np.arange(n)
    return np.exp(2j * np.pi * np.outer(t, k[order]) / n)


def smooth_orthonormal_basis(ny, nx, q, seed=0):
    """U of shape (ny * nx, q), complex128, orthonormal columns.

    Columns span the q lowest 2D Fourier modes (ordered by |k|) times a smooth
    random complex envelope, orthonormalised by QR.
    """
    rng = np.random.default_rng(seed)
    ky = np.arange(ny) - ny // 2
    kx = np.arange(nx) - nx // 2
    KY, KX = np.meshgrid(ky, kx, indexing="ij")
    kr = KY.astype(float) ** 2 + KX.astype(float) ** 2
    order = np.lexsort((KX.ravel(), KY.ravel(), kr.ravel()))[:q]
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    env_phase = np.zeros((ny, nx))
    env_amp = np.ones((ny, nx))
    for _ in range(3):
        fy, fx = rng.integers(0, 3, size=2)
        a, b = rng.normal(size=2)
        env_phase += a * np.cos(2 * np.pi * (fy * y / ny + fx * x / nx) + b)
        env_amp += 0.1 * rng.normal() * np.sin(2 * np.pi * (fy * y / ny + fx * x / nx))
    env = (env_amp * np.exp(1j * env_phase)).ravel()
    modes = np.exp(
        2j * np.pi * (np.outer(y.ravel(), KY.ravel()[order])[:, None, :] / ny
                      + np.outer(x.ravel(), KX.ravel()[order])[None, :, :] / nx)
    ).reshape(ny * nx, q)
    Q, _ = np.linalg.qr(env[:, None] * modes)
    return Q


def smooth_tucker_basis(n, r, q, seed=0):
    """Tucker-factored orthonormal basis: core (r1, r2, r3, q) and factors U_k (n_k, r_k).

    The expanded basis column j is core[..., j] x1 U1 x2 U2 x3 U3; with
    orthonormal factors and a core whose unfolding (r1 r2 r3, q) has
    orthonormal columns, the expanded columns are orthonormal too.
    """
    rng = np.random.default_rng(seed)
    factors = []
    for nk, rk in zip(n, r):
        env = np.exp(1j * rng.normal() * np.cos(2 * np.pi * np.arange(nk) / nk))
        Qk, _ = np.linalg.qr(env[:, None] * _low_modes_1d(nk, rk))
        factors.append(Qk)
    R = r[0] * r[1] * r[2]
    g = rng.normal(size=(R, q)) + 1j * rng.normal(size=(R, q))
    Qc, _ = np.linalg.qr(g)
    core = Qc.reshape(r[0], r[1], r[2], q)
    return core, factors
