"""Seeded Cartesian sampling masks.

The paper names its sampling schemes (1D Cartesian with ACS lines, 2D
variable-density Poisson-disc, 3D Poisson-disc over the two phase-encode axes)
without giving generators; these are plain seeded generators of that kind.  A
mask is a boolean array over the k-space grid in centred order (index n/2 is
the DC sample); ``mask_to_indices`` turns it into the sorted raster index list
the operator consumes.  All counts are exact: ``round(N_pe / R)`` sampled
phase-encode positions, calibration region always included.
"""

import numpy as np


def mask_to_indices(mask):
    """Sorted raster-order flat indices of the True entries (int32)."""
    return np.flatnonzero(np.asarray(mask).ravel()).astype(np.int32)


def vd_lines_mask(ny, nx, R, n_acs, seed=0):
    """1D variable-density line mask (phase encode along y, readout along x).

    ``round(ny / R)`` lines in total: the ``n_acs`` central lines plus lines
    drawn without replacement with probability proportional to
    (1 - |k| / k_max)^2.
    """
    rng = np.random.default_rng(seed)
    n_lines = int(round(ny / R))
    if n_acs > n_lines:
        raise ValueError("more ACS lines than sampled lines")
    k = np.arange(ny) - ny // 2
    acs = np.abs(k + 0.5) < n_acs / 2.0
    acs_idx = np.flatnonzero(acs)
    if acs_idx.size != n_acs:  # odd n_acs: widen on the negative side
        acs = (k >= -(n_acs // 2) - (n_acs % 2)) & (k < n_acs // 2)
        acs_idx = np.flatnonzero(acs)
    rest = np.flatnonzero(~acs)
    w = (1.0 - np.abs(k[rest]) / (ny / 2.0 + 1.0)) ** 2
    chosen = rng.choice(rest, size=n_lines - acs_idx.size, replace=False, p=w / w.sum())
    lines = np.zeros(ny, dtype=bool)
    lines[acs_idx] = True
    lines[chosen] = True
    mask = np.zeros((ny, nx), dtype=bool)
    mask[lines, :] = True
    return mask


def _mis_poisson(rad, prio, rounds=64):
    """Greedy parallel maximal independent set on the disc-conflict graph.

    Two grid points conflict when their distance is below the mean of their
    radii.  In each round every still-free point whose priority beats all free
    conflicting neighbours is accepted and its neighbours are removed.
    """
    ny, nx = rad.shape
    rmax = int(np.ceil(rad.max()))
    offs = [
        (dy, dx)
        for dy in range(-rmax, rmax + 1)
        for dx in range(-rmax, rmax + 1)
        if (dy or dx) and dy * dy + dx * dx < (rmax + 0.0) ** 2
    ]
    pad = rmax
    free = np.ones((ny, nx), dtype=bool)
    acc = np.zeros((ny, nx), dtype=bool)
    P = np.full((ny + 2 * pad, nx + 2 * pad), -1.0)
    Rp = np.zeros((ny + 2 * pad, nx + 2 * pad))
    Rp[pad:pad + ny, pad:pad + nx] = rad
    for _ in range(rounds):
        if not free.any():
            break
        P[pad:pad + ny, pad:pad + nx] = np.where(free, prio, -1.0)
        win = free.copy()
        for dy, dx in offs:
            nb_p = P[pad + dy:pad + dy + ny, pad + dx:pad + dx + nx]
            nb_r = Rp[pad + dy:pad + dy + ny, pad + dx:pad + dx + nx]
            conflict = (dy * dy + dx * dx) < (0.5 * (rad + nb_r)) ** 2
            win &= ~(conflict & (nb_p > prio))
        acc |= win
        A = np.zeros((ny + 2 * pad, nx + 2 * pad), dtype=bool)
        A[pad:pad + ny, pad:pad + nx] = win
        block = win.copy()
        for dy, dx in offs:
            nb_a = A[pad + dy:pad + dy + ny, pad + dx:pad + dx + nx]
            nb_r = Rp[pad + dy:pad + dy + ny, pad + dx:pad + dx + nx]
            block |= nb_a & ((dy * dy + dx * dx) < (0.5 * (rad + nb_r)) ** 2)
        free &= ~block
    return acc


def _exact_count(mask, keep, target, rng):
    """Add or drop random non-calibration points until ``mask.sum() == target``."""
    mask = mask | keep
    cnt = int(mask.sum())
    if cnt > target:
        cand = np.flatnonzero((mask & ~keep).ravel())
        drop = rng.choice(cand, size=cnt - target, replace=False)
        mask.ravel()[drop] = False
    elif cnt < target:
        cand = np.flatnonzero((~mask).ravel())
        add = rng.choice(cand, size=target - cnt, replace=False)
        mask.ravel()[add] = True
    return mask


def _pd_plane(n0, n1, R, calib, seed):
    rng = np.random.default_rng(seed)
    target = int(round(n0 * n1 / R))
    k0 = (np.arange(n0) - n0 // 2) / (n0 / 2.0)
    k1 = (np.arange(n1) - n1 // 2) / (n1 / 2.0)
    kr = np.sqrt(k0[:, None] ** 2 + k1[None, :] ** 2)
    prio = rng.random((n0, n1))
    keep = np.zeros((n0, n1), dtype=bool)
    c0, c1 = min(calib[0], n0), min(calib[1], n1)
    keep[n0 // 2 - c0 // 2:n0 // 2 - c0 // 2 + c0, n1 // 2 - c1 // 2:n1 // 2 - c1 // 2 + c1] = True
    if target < keep.sum():
        raise ValueError("calibration region larger than the sample budget")
    # Variable density: the disc radius grows linearly with |k|.  Bisection on
    # the radius scale brings the count near the target; the last step makes it
    # exact.
    lo, hi = 0.3, 8.0
    best = None
    for _ in range(7):
        s = 0.5 * (lo + hi)
        m = _mis_poisson(s * (1.0 + 1.5 * kr), prio) | keep
        best = m
        if m.sum() > target:
            lo = s
        else:
            hi = s
    return _exact_count(best, keep, target, rng)


def poisson_disc_mask(ny, nx, R, calib=(24, 24), seed=0):
    """2D variable-density Poisson-disc mask over (ky, kx), exact count."""
    return _pd_plane(ny, nx, R, calib, seed)


def poisson_disc_mask_3d(nz, ny, nx, R, calib=(24, 24), seed=0):
    """3D mask: Poisson-disc over the (kz, ky) phase-encode plane, kx fully sampled.

    Sample count = nx * round(nz * ny / R).
    """
    plane = _pd_plane(nz, ny, R, calib, seed)
    return np.repeat(plane[:, :, None], nx, axis=2)
