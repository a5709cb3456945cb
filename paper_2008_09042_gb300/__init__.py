"""GB300-native (sm_103a) Maxwell Parallel Imaging encoding operator.

The operator G(p, alpha) = [F_s(U alpha_k (.) p)]_k, its adjoint, Jacobian and
Jacobian-adjoint, and the two solvers built on them, all run in the CUDA
kernels of ``libmpi_gb300.so`` behind the C ABI declared in
``include/mpi_gb300.h``.  This package only marshals arguments.
"""

from ._lib import MpiError, load  # noqa: F401
from .api import (  # noqa: F401
    Basis,
    Batch,
    Context,
    MPIOperator,
    Plan,
    TuckerBasis,
    adjoint,
    basis_expand,
    basis_project,
    maxwell_basis_2d,
    maxwell_basis_3d,
    tucker_compress,
    forward_maps,
    adjoint_maps,
    jacobian_maps,
    jacobian_adjoint_maps,
    sm_estimate_maps,
    expand_path,
    forward,
    forward_host,
    adjoint_host,
    jacobian,
    jacobian_adjoint,
    image_solve,
    image_solve_dynamic,
    mpi_operator,
    sm_estimate,
    tv_prox,
)
