// mpi_forward_noalloc: the Cartesian forward operator with its scratch in a
// fixed, file-scope device array instead of the context's growable workspace.
//
// Some callers cannot call cudaMalloc once they are running: a reconstruction
// service whose device memory is divided up at start-up by its own pool
// allocator, or a real-time loop that must not block in the driver's allocator
// (cudaMalloc may synchronise the device and can fail at an unpredictable point
// under memory pressure).  mpi_forward grows the context workspace on demand;
// this entry point never allocates: the per-coil intermediate lives in
// g_noalloc_scratch below, which every GPU that loads the library holds until
// the process exits.
#include <mutex>

#include "mpi_internal.h"

namespace {

// 16 MiB of scratch: the [C][N] complex64 image-side intermediate between the
// expansion pass and the FFT passes, so C * N <= 2,097,152.
constexpr size_t kNoallocScratchElems = (size_t)2 << 20;
static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
float2* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch is only a host-side stand-in, so the real address is looked
// up once per device with that device current.
mpi_status noalloc_scratch(mpi_ctx* ctx, float2** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(ctx, e, "noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_err(ctx, MPI_ERR_UNSUPPORTED, "noalloc: device index too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_check(ctx, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                            "noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = (float2*)p;
  }
  *out = g_noalloc_ptr[dev];
  return MPI_OK;
}

}  // namespace

extern "C" mpi_status mpi_forward_noalloc(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                          const mpi_c32* alpha, int C, const mpi_c32* p, mpi_c32* y) {
  if (!ctx) return MPI_ERR_ARG;
  if (!plan || !basis || !alpha || !p || C < 1 || (plan->M > 0 && !y))
    return set_err(ctx, MPI_ERR_ARG, "forward_noalloc: bad argument");
  if (plan->ctx != ctx || basis->ctx != ctx) return set_err(ctx, MPI_ERR_ARG, "plan/basis from another context");
  if (basis->N != plan->N) return set_err(ctx, MPI_ERR_SHAPE, "basis N differs from plan N");
  if (plan->kind != MPI_TRAJ_CARTESIAN)
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "forward_noalloc: Cartesian plans only");
  if (basis->tucker) return set_err(ctx, MPI_ERR_UNSUPPORTED, "forward_noalloc: dense bases only");
  if ((size_t)C * (size_t)plan->N > kNoallocScratchElems)
    return set_err(ctx, MPI_ERR_SHAPE,
                   "forward_noalloc: C * N exceeds the 2,097,152-element (16 MiB) static scratch");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_check(ctx, e, "noalloc: cudaSetDevice");
  float2* v = nullptr;
  mpi_status st = noalloc_scratch(ctx, &v);
  if (st) return st;
  // The expansion pass writes all C * N scratch entries before the FFT passes
  // read them, so nothing left from an earlier call needs clearing.
  ExpandArgs a;
  a.U = basis->U;
  a.N = basis->N;
  a.q = basis->q;
  a.nx = plan->nx;
  a.ny = plan->ny;
  a.C = C;
  a.centre = 1;
  a.scale = 1.0f / sqrtf((float)plan->N);
  a.alpha = (const float2*)alpha;
  a.p = (const float2*)p;
  a.out = v;
  if ((st = launch_expand(ctx, EX_FWD, a))) return st;
  if (plan->ndim == 3 && (st = launch_fft_z(ctx, v, C, plan->nz, plan->ny, plan->nx, false))) return st;
  if ((st = launch_fft_cols(ctx, v, C, plan->nz, plan->ny, plan->nx, false))) return st;
  return launch_rows_fwd_gather(ctx, plan, v, C, (float2*)y);
}
