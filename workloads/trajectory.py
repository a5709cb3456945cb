"""Golden-angle radial trajectories (Results, "2D synthetic radial sequences").

Samples are in radians per pixel on [-pi, pi); spoke s has angle
s * pi * (sqrt(5) - 1) / 2 (the golden angle, about 111.246 degrees) and every
spoke passes through the k-space centre.
"""

import numpy as np


def golden_angle_radial(n_spokes, n_readout):
    """Return k of shape (n_spokes * n_readout, 2) as (kx, ky), float64.

    Readout sample j of a spoke sits at radius pi * (j - n_readout/2) / (n_readout/2).
    """
    ga = np.pi * (np.sqrt(5.0) - 1.0) / 2.0
    theta = np.arange(n_spokes) * ga
    kr = np.pi * (np.arange(n_readout) - n_readout // 2) / (n_readout / 2.0)
    kx = kr[None, :] * np.cos(theta)[:, None]
    ky = kr[None, :] * np.sin(theta)[:, None]
    return np.stack([kx.ravel(), ky.ravel()], axis=1)
