// Solvers placeholder (filled in by the solver translation unit).
#include "mpi_internal.h"

extern "C" mpi_status mpi_sm_estimate(mpi_ctx* ctx, const mpi_plan*, const mpi_basis*, const mpi_c32*, int,
                                      const mpi_irgn_params*, mpi_c32*, mpi_c32*, double*, mpi_precision) {
  return set_err(ctx, MPI_ERR_UNSUPPORTED, "not built");
}
extern "C" mpi_status mpi_image_solve(mpi_ctx* ctx, const mpi_plan*, const mpi_basis*, const mpi_c32*, int,
                                      const mpi_c32*, const double*, const mpi_admm_params*, mpi_c32*, double*,
                                      mpi_precision) {
  return set_err(ctx, MPI_ERR_UNSUPPORTED, "not built");
}
extern "C" mpi_status mpi_tv_prox(mpi_ctx* ctx, const mpi_plan*, const mpi_c32*, double, int, mpi_c32*) {
  return set_err(ctx, MPI_ERR_UNSUPPORTED, "not built");
}
extern "C" mpi_status mpi_basis_project(mpi_ctx* ctx, const mpi_basis*, const mpi_c32*, int, mpi_c32*) {
  return set_err(ctx, MPI_ERR_UNSUPPORTED, "not built");
}
