"""Random-ellipse phantoms (seeded), standing in for the paper's density images.

The paper's radial experiment uses a Shepp-Logan model (Results, "2D synthetic
radial sequences"); the workloads here use seeded random ellipses of the same
kind: real-valued piecewise-constant densities on an n x n grid.
"""

import numpy as np


def random_ellipses(ny, nx, n_ellipses=8, seed=0, nz=None):
    """Return a real phantom of shape (ny, nx) (or (nz, ny, nx) when nz is set).

    Painter's order: a background ellipse of intensity 0.2 is drawn first, then
    ``n_ellipses`` ellipses with centres U[-0.5, 0.5], semi-axes U[0.1, 0.5],
    angle U[0, pi) and intensity U[0.1, 1] overwrite what lies under them.
    Coordinates are normalised to [-1, 1) across the field of view.
    """
    rng = np.random.default_rng(seed)
    if nz is None:
        yy, xx = np.meshgrid(
            (np.arange(ny) - ny / 2) / (ny / 2),
            (np.arange(nx) - nx / 2) / (nx / 2),
            indexing="ij",
        )
        img = np.zeros((ny, nx))
        img[(yy / 0.9) ** 2 + (xx / 0.8) ** 2 <= 1.0] = 0.2
        for _ in range(n_ellipses):
            cy, cx = rng.uniform(-0.5, 0.5, size=2)
            ay, ax = rng.uniform(0.1, 0.5, size=2)
            th = rng.uniform(0.0, np.pi)
            val = rng.uniform(0.1, 1.0)
            dy, dx = yy - cy, xx - cx
            u = dx * np.cos(th) + dy * np.sin(th)
            v = -dx * np.sin(th) + dy * np.cos(th)
            img[(u / ax) ** 2 + (v / ay) ** 2 <= 1.0] = val
        return img
    zz, yy, xx = np.meshgrid(
        (np.arange(nz) - nz / 2) / (nz / 2),
        (np.arange(ny) - ny / 2) / (ny / 2),
        (np.arange(nx) - nx / 2) / (nx / 2),
        indexing="ij",
    )
    img = np.zeros((nz, ny, nx))
    img[(zz / 0.9) ** 2 + (yy / 0.9) ** 2 + (xx / 0.8) ** 2 <= 1.0] = 0.2
    for _ in range(n_ellipses):
        c = rng.uniform(-0.5, 0.5, size=3)
        a = rng.uniform(0.1, 0.5, size=3)
        val = rng.uniform(0.1, 1.0)
        r2 = ((zz - c[0]) / a[0]) ** 2 + ((yy - c[1]) / a[1]) ** 2 + ((xx - c[2]) / a[2]) ** 2
        img[r2 <= 1.0] = val
    return img
