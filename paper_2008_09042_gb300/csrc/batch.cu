// Batched operator application over many slices of uneven grid size and coil
// count, replayed as one CUDA graph.
//
// mpi_batch_create orders the slices by basis (slices of the same grid share
// one Maxwell basis, which then stays L2-resident across consecutive slices),
// sizes the context workspace for the largest slice, and records every kernel
// of every slice's operator calls into one graph by stream capture on a private
// stream.  mpi_batch_run launches that graph on the context's stream.  The
// captured pointers are the caller's buffers, which must stay valid for the
// life of the batch.
#include <algorithm>
#include <numeric>
#include <vector>

#include "mpi_internal.h"

struct mpi_batch {
  mpi_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int n = 0;
  int64_t kernels = 0;  // kernels per replay
};

namespace {

mpi_status record_slice(mpi_ctx* ctx, const mpi_batch_slice& s, int kind, mpi_precision prec) {
  mpi_status st = MPI_OK;
  if (kind & MPI_BATCH_FORWARD)
    st = mpi_forward(ctx, s.plan, s.basis, s.alpha, s.C, s.p, s.y, prec);
  if (st == MPI_OK && (kind & MPI_BATCH_ADJOINT))
    st = mpi_adjoint(ctx, s.plan, s.basis, s.alpha, s.C, s.y, s.x, prec);
  return st;
}

}  // namespace

extern "C" mpi_status mpi_batch_create(mpi_ctx* ctx, const mpi_batch_slice* slices, int n, int kind,
                                       mpi_precision prec, mpi_batch** out) {
  if (!ctx) return MPI_ERR_ARG;
  if (!slices || n < 1 || !out || kind < 1 || kind > 3) return set_err(ctx, MPI_ERR_ARG, "batch: bad argument");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  for (int i = 0; i < n; ++i) {
    const mpi_batch_slice& s = slices[i];
    if (!s.plan || !s.basis || !s.alpha || s.C < 1 || !s.p || !s.x || (s.plan->M > 0 && !s.y))
      return set_err(ctx, MPI_ERR_ARG, "batch: incomplete slice " + std::to_string(i));
    // reserve the workspace outside the capture (no allocation may happen inside it)
    mpi_status st = mpi_ctx_reserve(ctx, s.plan, s.basis, s.C);
    if (st) return st;
  }
  // tune the slices' FFT line passes now: no tuning happens inside the capture
  for (int i = 0; i < n; ++i) {
    mpi_status st = mpi_ctx_reserve(ctx, slices[i].plan, slices[i].basis, slices[i].C);
    if (st == MPI_OK) st = tune_line_passes(ctx, slices[i].plan, slices[i].C);
    if (st) return st;
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return slices[a].basis < slices[b].basis; });

  mpi_batch* bt = new mpi_batch();
  bt->ctx = ctx;
  bt->n = n;
  cudaStream_t cap = nullptr, user = ctx->stream;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete bt;
    return cuda_check(ctx, e, "batch stream");
  }
  // the capture must not wait on work still queued on the user's stream
  e = cudaStreamSynchronize(user);
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  ctx->stream = cap;
  const int64_t l0 = ctx->launches;
  mpi_status st = MPI_OK;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    for (int i = 0; i < n && st == MPI_OK; ++i) st = record_slice(ctx, slices[order[i]], kind, prec);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (st == MPI_OK && e2 == cudaSuccess) {
      bt->graph = g;
      e2 = cudaGraphInstantiate(&bt->exec, g, 0);
    } else if (g) {
      cudaGraphDestroy(g);
    }
    if (st == MPI_OK && e2 != cudaSuccess) st = cuda_check(ctx, e2, "batch graph capture");
  } else {
    st = cuda_check(ctx, e, "batch capture begin");
  }
  bt->kernels = ctx->launches - l0;
  ctx->launches = l0;
  ctx->stream = user;
  ctx->profiling = prof;
  cudaStreamDestroy(cap);
  if (st != MPI_OK) {
    mpi_batch_destroy(bt);
    return st;
  }
  ctx_adopt(ctx, &bt->ctx);
  *out = bt;
  return MPI_OK;
}

extern "C" mpi_status mpi_batch_run(mpi_ctx* ctx, mpi_batch* bt) {
  if (!ctx) return MPI_ERR_ARG;
  if (!bt || bt->ctx != ctx || !bt->exec) return set_err(ctx, MPI_ERR_ARG, "batch: bad handle");
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaGraphLaunch(bt->exec, ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "batch graph launch");
  ctx->launches += bt->kernels;
  return MPI_OK;
}

extern "C" int64_t mpi_batch_kernel_count(const mpi_batch* bt) { return bt ? bt->kernels : -1; }

extern "C" mpi_status mpi_batch_destroy(mpi_batch* bt) {
  if (!bt) return MPI_ERR_ARG;
  ctx_release(&bt->ctx);
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  delete bt;
  return MPI_OK;
}
