"""Dipole site geometry for the Maxwell-basis workloads (inputs: where the
boundary sources sit; none of the field arithmetic lives here)."""

import numpy as np


def circle_sites(n_sites, radius, z=0.0):
    """n_sites points evenly spaced on a circle in the plane z."""
    th = 2.0 * np.pi * np.arange(n_sites) / n_sites
    return np.stack([radius * np.cos(th), radius * np.sin(th), np.full(n_sites, z)], axis=1)


def sphere_sites(n_sites, radius):
    """n_sites points spread over a sphere (the Fibonacci lattice)."""
    i = np.arange(n_sites) + 0.5
    zc = 1.0 - 2.0 * i / n_sites
    rho = np.sqrt(1.0 - zc ** 2)
    th = np.pi * (3.0 - np.sqrt(5.0)) * i
    return radius * np.stack([rho * np.cos(th), rho * np.sin(th), zc], axis=1)
