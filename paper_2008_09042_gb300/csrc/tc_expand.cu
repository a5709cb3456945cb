// BF16 tensor-core basis expansion (tcgen05 + TMA + TMEM), the dense
// contraction of the operator: S = U A^T with U in C^{N x q}, A = [alpha_k]
// (Maxwell Regularization section, s_k = U alpha_k), fused with the point-wise
// products of the forward, adjoint and Jacobian passes (Eqs. 5 and 7 and the
// Jacobian-adjoint display after Eq. 7).
//
// Complex to real: a pixel row of the BF16 operand is [Re U[n][0..q) | Im U[n][0..q) | 0-pad]
// (K = 2q padded to a multiple of 64), and the coefficient operand has, per
// coil c, the two K-major rows [Re a_c, -Im a_c] and [Im a_c, Re a_c], so that
// accumulator columns 2c and 2c+1 hold Re and Im of s_c.  BF16 operands, FP32
// accumulation in tensor memory.
//
// CTA = 6 warps: warp 0 streams 128-pixel x 64-element tiles of U with TMA
// (128-byte swizzle) into a ring of shared-memory stages; warp 1 owns the TMEM
// accumulator and one thread issues tcgen05.mma (M = 128, N = padded 2C or 4C,
// K = 16 per instruction); warps 2-5 read the accumulator with tcgen05.ld
// (warp w owns TMEM lanes 32 (w % 4) ..) and apply the epilogue, one pixel per
// thread.  The epilogue warps first write the coefficient operand into shared
// memory (swizzled K-major layout) while the first tiles of U are in flight.
// Persistent CTAs walk the pixel tiles; the ring is as deep as shared memory
// allows.
// Every mbarrier wait is bounded (kWaitCycles); on a timeout the CTA records
// the error, drains what it issued (bounded) and frees its TMEM.
#include <cuda.h>

#include <algorithm>

#include "mpi_internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace {

using namespace mpi_tc;

constexpr int kKChunk = 64;  // BF16 elements per 128-byte swizzle row
constexpr int kMaxStages = 12;
constexpr int kThreads = 192;

template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) k_expand_tc(const __grid_constant__ CUtensorMap tmap, TcArgs a_in,
                                                            int stages) {
  TcArgs a = a_in;
  if (a.rows) {  // grouped launch: this row's slice
    const ExpandRow r = a.rows[blockIdx.y];
    a.alpha = r.alpha;
    a.p = r.p;
    a.w = r.w;
    a.out = r.out;
    a.C = r.C;
  }
  extern __shared__ unsigned char smem_raw[];
  // aligned by an offset from the shared array, so that accesses stay shared-memory ones
  unsigned char* smem = smem_raw + ((1024u - (mpi_ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  const int Kp = a.KC * kKChunk;
  const uint32_t b_bytes = (uint32_t)a.n_gemm * Kp * 2;
  unsigned char* sB = smem;
  unsigned char* sA = smem + ((b_bytes + 1023) & ~1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(sA + stages * kStageBytes);
  uint64_t* empty = full + stages;
  uint64_t* acc_full = empty + stages;  // [2]: double-buffered accumulator
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint64_t* drain = acc_empty + 2;
  uint64_t* bfull = drain + 1;  // coefficient operand landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bfull + 1);
  __shared__ int s_failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // Launched with programmatic stream serialization: set-up and the TMA stream of
  // the (constant) basis start at once; only the epilogue warps, which read
  // the coefficients and per-pixel data and write the outputs, wait for the
  // previous kernel.
  mpi_ptx::pdl_trigger();
  if (tid == 0) {
    s_failed = 0;
    for (int s = 0; s < stages; ++s) {
      mpi_ptx::mbar_init(&full[s], 1);
      mpi_ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mpi_ptx::mbar_init(&acc_full[b], 1);
      mpi_ptx::mbar_init(&acc_empty[b], 4);
    }
    mpi_ptx::mbar_init(drain, 1);
    mpi_ptx::mbar_init(bfull, 4);  // one arrival per epilogue warp once the coefficient operand is written
    mpi_ptx::fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     mpi_ptx::smem_addr(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  const int n_tiles = (a.N + kTileM - 1) / kTileM;
  if (warp == 0 && lane == 0) {
    // ---------------- producer: TMA tiles of U
    int it = 0;
    RingPos r;
    bool ok = true;
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      for (int kc = 0; kc < a.KC; ++kc, ++it) {
        if (!mpi_ptx::mbar_wait(&empty[r.s], r.ph ^ 1u, a.err, a.wait_cycles)) {
          ok = false;
          break;
        }
        mpi_ptx::mbar_arrive_expect_tx(&full[r.s], kStageBytes);
        tma_load_2d(sA + r.s * kStageBytes, &tmap, kc * kKChunk, t * kTileM, &full[r.s]);
        r.next(stages);
      }
    }
    if (!ok) {
      s_failed = 1;
      // bounded wait for the fills still in flight
      for (int g = (it > stages ? it - stages : 0); g < it; ++g)
        mpi_ptx::mbar_wait(&full[g % stages], (uint32_t)((g / stages) & 1), nullptr, a.wait_cycles);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    // A descriptor of base + off is desc(base) + (off >> 4): the 14-bit start
    // address field holds every shared-memory address, so the sum never carries.
    const uint32_t idesc = idesc_bf16(kTileM, a.n_gemm);
    const uint64_t a0 = sdesc_sw128(mpi_ptx::smem_addr(sA));
    const uint64_t b0 = sdesc_sw128(mpi_ptx::smem_addr(sB));
    const uint32_t b_chunk = (uint32_t)(a.n_gemm * 128) >> 4;  // descriptor step per K chunk
    RingPos r;
    int tc = 0;
    bool ok = mpi_ptx::mbar_wait(bfull, 0, a.err, a.wait_cycles);
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      const uint32_t tacc = tmem + (uint32_t)(buf * a.half_cols);
      if (!mpi_ptx::mbar_wait(&acc_empty[buf], (uint32_t)(((tc >> 1) & 1) ^ 1), a.err, a.wait_cycles)) {
        ok = false;
        break;
      }
      fence_after();
      for (int kc = 0; kc < a.KC; ++kc) {
        const int s = r.s;
        if (!mpi_ptx::mbar_wait(&full[s], r.ph, a.err, a.wait_cycles)) {
          ok = false;
          break;
        }
        r.next(stages);
        fence_after();
        // four K = 16 steps of this 64-element chunk (32 bytes apart in the swizzled rows)
        const uint64_t ad = a0 + (uint32_t)(s * (kStageBytes >> 4));
        const uint64_t bd = b0 + (uint32_t)kc * b_chunk;
        mma_bf16(tacc, ad, bd, idesc, kc != 0);
        mma_bf16_acc(tacc, ad + 2, bd + 2, idesc);
        mma_bf16_acc(tacc, ad + 4, bd + 4, idesc);
        mma_bf16_acc(tacc, ad + 6, bd + 6, idesc);
        mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
      }
      if (ok) mma_commit(&acc_full[buf]);
    }
    // all MMAs issued by this thread have completed once `drain` fires
    mma_commit(drain);
    mpi_ptx::mbar_wait(drain, 0, a.err, a.wait_cycles);
    if (!ok) s_failed = 1;
  } else if (warp >= 2) {
    mpi_ptx::pdl_wait();  // alpha, p and w may come from the previous kernel
    build_coef_smem<false>(a, sB, Kp, MODE == EX_JFWD, tid - 64, bfull);
    tc_epilogue<MODE>(a, tmem, warp, lane, acc_full, acc_empty, n_tiles, &s_failed);
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

__global__ void k_basis_to_bf16(const float2* __restrict__ U, int N, int q, int Kp, __nv_bfloat16* __restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)N * Kp) return;
  const int n = (int)(e / Kp), k = (int)(e % Kp);
  float v = 0.f;
  if (k < q) v = U[(size_t)k * N + n].x;
  else if (k < 2 * q) v = U[(size_t)(k - q) * N + n].y;
  out[e] = __float2bfloat16_rn(v);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// BF16 operand copy of the basis and its tensor map (called at basis load).
mpi_status tc_basis_prepare(mpi_ctx* ctx, mpi_basis* b) {
  const int Kp = round_up(2 * b->q, kKChunk);
  b->Ubf_bytes = (size_t)b->N * Kp * sizeof(__nv_bfloat16);
  cudaError_t e = cudaMalloc(&b->Ubf, b->Ubf_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->Ubf = nullptr;
    return set_err(ctx, MPI_ERR_OOM, "BF16 basis copy");
  }
  const size_t total = (size_t)b->N * Kp;
  MPI_PROF(ctx, KF_OTHER);
  k_basis_to_bf16<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(b->U, b->N, b->q, Kp, b->Ubf);
  MPI_LAUNCH_CHECK(ctx, "k_basis_to_bf16");
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
  }
  CUtensorMap* map = new CUtensorMap;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)b->N};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {(cuuint32_t)kKChunk, (cuuint32_t)kTileM};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = ((EncodeTiledFn)fn)(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, b->Ubf, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    delete map;
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "tensor map encoding failed");
  }
  b->tmap = map;
  b->Kp = Kp;
  return MPI_OK;
}

bool tc_encode_operand_map(void* map, void* ptr, long rows, int Kp) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {(cuuint32_t)kKChunk, (cuuint32_t)kTileM};
  const cuuint32_t estr[2] = {1, 1};
  return ((EncodeTiledFn)fn)((CUtensorMap*)map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_encode_operand_map_k(void* map, void* ptr, long rows, int K) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn || K % 8) {
    cudaGetLastError();
    return false;
  }
  // K columns stored; boxes past K (up to the kernel's Kp) read as zeros
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(__nv_bfloat16)};
  const cuuint32_t box[2] = {(cuuint32_t)kKChunk, (cuuint32_t)kTileM};
  const cuuint32_t estr[2] = {1, 1};
  return ((EncodeTiledFn)fn)((CUtensorMap*)map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void tc_basis_release(mpi_basis* b) {
  delete (CUtensorMap*)b->tmap;
  b->tmap = nullptr;
}

mpi_status launch_expand_tc(mpi_ctx* ctx, const mpi_basis* b, int mode, const ExpandArgs& x) {
  if (!b->Ubf || !b->tmap) return set_err(ctx, MPI_ERR_UNSUPPORTED, "basis has no BF16 operand copy");
  if (x.N <= 0 || x.C <= 0) return MPI_OK;
  TcArgs a{};  // every field not set below is zero (no K offset, no split)
  a.N = x.N;
  a.q = x.q;
  a.C = x.C;
  a.KC = b->Kp / kKChunk;
  const int cols = round_up(2 * x.C, 16);
  a.half = cols;
  a.n_gemm = mode == EX_JFWD ? 2 * cols : cols;
  if (a.n_gemm > 256) return set_err(ctx, MPI_ERR_UNSUPPORTED, "BF16 expansion: too many coils for one pass");
  int tcols = 32;
  while (tcols < a.n_gemm) tcols <<= 1;
  a.half_cols = tcols;     // accumulator buffer stride in TMEM columns
  a.tmem_cols = 2 * tcols;  // two accumulator buffers
  a.lo_cols = 0;
  a.nx = x.nx;
  a.ny = x.ny;
  a.centre = x.centre;
  a.scale = x.scale;
  a.alpha = x.alpha;
  a.dalpha = x.dalpha;
  a.p = x.p;
  a.dp = x.dp;
  a.w = x.w;
  a.out = x.out;
  a.vout = x.vout;
  a.err = ctx->dev_err;
  a.wait_cycles = ctx->wait_cycles;
  a.accumulate = x.accumulate;
  a.rows = x.rows;
  a.stall_after = -1;
  a.tuck_B = x.tuck_B;
  a.group_coils = 0;
  a.C_total = x.C;
  a.tuck_stride = x.tuck_stride;
  a.sc_L0 = x.sc.L0;
  a.sc_L1 = x.sc.L1;
  a.sc_hi = x.sc.s_hi;
  a.sc_mid = x.sc.s_mid;
  a.sc_col = x.sc.s_col;
  a.sc_im = x.sc.im;
  a.sc_col0 = 0;
  a.sc_bf16 = x.sc.bf16 ? 1 : 0;
  const size_t b_bytes = round_up(a.n_gemm * b->Kp * 2, 1024);
  // Two CTAs per SM (one's epilogue overlaps the other's loads) when each can
  // still keep four or more stages in flight within half of the SM's shared
  // memory, else one CTA with a deeper ring.
  const size_t fixed = 1024 + b_bytes + (2 * kMaxStages + 6) * 8 + 16;
  const size_t half_sm = 112 * 1024, whole_sm = 227 * 1024 - 128;
  int stages = half_sm > fixed ? (int)((half_sm - fixed) / kStageBytes) : 0;
  int per_sm = 2;
  if (stages < 4 || a.tmem_cols > 256) {  // two CTAs per SM must both hold their TMEM columns
    per_sm = 1;
    stages = whole_sm > fixed ? (int)((whole_sm - fixed) / kStageBytes) : 0;
  }
  stages = std::min(stages, kMaxStages);
  if (stages < 2) return set_err(ctx, MPI_ERR_UNSUPPORTED, "BF16 expansion: shared memory");
  const size_t smem = fixed + (size_t)stages * kStageBytes;
  const int n_tiles = (x.N + kTileM - 1) / kTileM;
  const int nrows = x.rows ? x.nrows : 1;
  const int per_row = x.rows && x.row_ctas > 0 ? x.row_ctas : std::max(per_sm * std::max(ctx->num_sms, 1) / nrows, 1);
  const dim3 grid((unsigned)std::min(n_tiles, per_row), (unsigned)nrows);
  const CUtensorMap& map = *(const CUtensorMap*)b->tmap;
  cudaError_t e = cudaSuccess;
#define MPI_TC_CASE(m)                                                                                        \
  case m:                                                                                                     \
    e = cudaFuncSetAttribute(k_expand_tc<m>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
    if (e != cudaSuccess) return cuda_check(ctx, e, "tc smem attribute");                                    \
    MPI_PROF(ctx, KF_EXPAND);                                                                                \
    launch_pdl(ctx, k_expand_tc<m>, dim3(grid), dim3(kThreads), smem, map, a, stages);                                           \
    break;
  switch (mode) {
    MPI_TC_CASE(EX_MAPS)
    MPI_TC_CASE(EX_FWD)
    MPI_TC_CASE(EX_JFWD)
    MPI_TC_CASE(EX_ADJ)
    MPI_TC_CASE(EX_JADJ)
    MPI_TC_CASE(EX_SCATTER)
    default:
      return set_err(ctx, MPI_ERR_ARG, "unknown expansion mode");
  }
#undef MPI_TC_CASE
  MPI_LAUNCH_CHECK(ctx, x.kname ? x.kname : "k_expand_tc");
  return MPI_OK;
}
