"""Seeded truth of the reconstruction workloads (input generation only).

Used by tests/golden/make_recon_golden.py (which makes the data and the FP64
oracle's reconstruction of it) and by bench.py (which reads those fixtures).
"""

import numpy as np

from .coefs import random_coefficients
from .configs import workload
from .masks import mask_to_indices, poisson_disc_mask, vd_lines_mask
from .phantom import random_ellipses
from .standin import smooth_orthonormal_basis
from .trajectory import golden_angle_radial

RECON_SEED = 20200820 + 500


def recon_case(name):
    """(cfg, U [N][q] complex128 of complex64 values, sampling, alpha_true, p_true):
    the sampling is the sorted sample indices of a Cartesian workload or the
    (M, 2) float32 k-space trajectory (rad/pixel) of a radial one."""
    cfg = workload(name)
    ny, nx = cfg["dims"]
    C, q = cfg["C"], cfg["q"]
    base = RECON_SEED
    U = smooth_orthonormal_basis(ny, nx, q, seed=base).astype(np.complex64).astype(np.complex128)
    if cfg["kind"] == "radial":
        k = golden_angle_radial(cfg["spokes"], cfg["readout"]).astype(np.float32)
        a_true = random_coefficients(C, q, seed=base + 2)
        p_true = random_ellipses(ny, nx, seed=base + 3).ravel().astype(np.complex128)
        return cfg, U, k, a_true, p_true
    if cfg["mask"] == "poisson":
        mask = poisson_disc_mask(ny, nx, cfg["R"], calib=cfg["calib"], seed=base + 1)
    else:
        mask = vd_lines_mask(ny, nx, cfg["R"], cfg["acs"], seed=base + 1)
    idx = mask_to_indices(mask)
    a_true = random_coefficients(C, q, seed=base + 2)
    p_true = random_ellipses(ny, nx, seed=base + 3).ravel().astype(np.complex128)
    return cfg, U, idx, a_true, p_true
