"""Seeded synthetic inputs for the encoding-operator workloads.

This package is shared by the FP64 oracle, the tests and the benchmark.  It
holds only input generation: phantoms, sampling masks, radial trajectories,
measurement noise, random coefficients, dipole-site geometry and a smooth
orthonormal stand-in basis.
None of the method's arithmetic (basis construction from Green's functions,
the encoding operator, the solvers) lives here.

Every generator takes an explicit integer seed and uses
``numpy.random.default_rng(seed)``, so both sides of a parity test see the same
bytes.
"""

from .phantom import random_ellipses  # noqa: F401
from .masks import (  # noqa: F401
    vd_lines_mask,
    poisson_disc_mask,
    poisson_disc_mask_3d,
    mask_to_indices,
)
from .trajectory import golden_angle_radial  # noqa: F401
from .noise import complex_noise, noise_sigma_for_snr  # noqa: F401
from .coefs import random_coefficients, random_excitations, random_image  # noqa: F401
from .standin import smooth_orthonormal_basis, smooth_tucker_basis  # noqa: F401
from .sources import circle_sites, sphere_sites  # noqa: F401
from .configs import WORKLOADS, workload  # noqa: F401
from .recon import RECON_SEED, recon_case  # noqa: F401

BASE_SEED = 20200820
