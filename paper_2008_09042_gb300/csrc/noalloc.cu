// mpi_forward_noalloc: the Cartesian forward operator with its scratch in a
// fixed, file-scope device array instead of the context's growable workspace.
//
// Some callers cannot call cudaMalloc once they are running: a reconstruction
// service whose device memory is divided up at start-up by its own pool
// allocator, or a real-time loop that must not block in the driver's allocator
// (cudaMalloc may synchronise the device and can fail at an unpredictable point
// under memory pressure).  mpi_forward grows the context workspace on demand;
// this entry point never allocates: the per-coil intermediate lives in
// g_noalloc_scratch below, which every GPU on which a context of this library
// is created holds from that moment until the process exits.
#include "mpi_internal.h"

namespace {

// 16 MiB of scratch: the [C][N] complex64 image-side intermediate between the
// expansion pass and the FFT passes, so C * N <= 2,097,152.
constexpr size_t kNoallocScratchElems = (size_t)2 << 20;
static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchElems];

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch is only a host-side stand-in, so the real address is asked
// for with the device current.  The driver loads the library's modules lazily:
// the first lookup on a device loads the module that holds the array, which
// reserves its 16 MiB.  mpi_ctx_create does that first lookup (noalloc_preload),
// so that an mpi_forward_noalloc call only reads the address of a module that is
// already resident.  The address is looked up on every call, not cached, so a
// module loaded anew after a device reset is found where it now is.
mpi_status noalloc_scratch(mpi_ctx* ctx, float2** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    return cuda_check(ctx, e == cudaSuccess ? cudaErrorInvalidSymbol : e, "noalloc: cudaGetSymbolAddress");
  *out = (float2*)p;
  return MPI_OK;
}

}  // namespace

cudaError_t noalloc_preload() {
  void* p = nullptr;
  return cudaGetSymbolAddress(&p, g_noalloc_scratch);
}

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
  // read them, so nothing left from an earlier call needs clearing.  The FP32
  // expansion is the same one mpi_forward runs (3xTF32 on the tensor cores where
  // the shape fits, else the CUDA-core kernel); its operand copy and tensor map
  // were made with the basis, so it allocates nothing here.
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
  // No launch-shape tuning here (it times candidates with events on scratch
  // memory): the passes take a shape tuned by an earlier call, or the default.
  void* scratch = ctx->tune_scratch;
  ctx->tune_scratch = nullptr;
  struct Restore {
    mpi_ctx* c;
    void* s;
    ~Restore() { c->tune_scratch = s; }
  } restore{ctx, scratch};
  if ((st = expand(ctx, basis, EX_FWD, a, MPI_PREC_FP32))) return st;
  if (plan->ndim == 3 && (st = launch_fft_z(ctx, v, C, plan->nz, plan->ny, plan->nx, false))) return st;
  if ((st = launch_fft_cols(ctx, v, C, plan->nz, plan->ny, plan->nx, false))) return st;
  return launch_rows_fwd_gather(ctx, plan, v, C, (float2*)y);
}
