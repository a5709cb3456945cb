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
// thread.  The coefficient operand is written once per CTA straight into the
// swizzled shared-memory layout.  Persistent CTAs walk the pixel tiles.
// Every mbarrier wait is bounded (kWaitCycles); on a timeout the CTA records
// the error, drains what it issued (bounded) and frees its TMEM.
#include <cuda.h>

#include <algorithm>

#include "mpi_internal.h"
#include "ptx.cuh"

namespace {

constexpr int kTileM = 128;
constexpr int kKChunk = 64;                  // BF16 elements per 128-byte swizzle row
constexpr int kStageBytes = kTileM * 128;    // one 128 x 64 BF16 tile
constexpr int kStages = 4;
constexpr int kThreads = 192;

struct TcArgs {
  int N, q, C, KC, n_gemm, half, half_cols, tmem_cols;
  int nx, ny, centre;
  float scale;
  const float2* alpha;
  const float2* dalpha;
  const __nv_bfloat16* coef_img;
  const float2* p;
  const float2* dp;
  const float2* w;
  float2* out;
  float2* vout;
  int* err;
};

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzled layout: start address >> 4 (bits 0-13), leading byte offset 16 B
// (unused for this layout, bits 16-29), stride byte offset 1024 B between
// 8-row groups (bits 32-45), descriptor version 1 (bits 46-47), swizzle mode
// 2 = 128-byte (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(mpi_ptx::smem_addr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(mpi_ptx::smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mpi_ptx::smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* r) {
  uint32_t v[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(v[i]);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ float centre_sign(int n, int nx, int ny) {
  int x = n % nx;
  int t = n / nx;
  int y = t % ny;
  int z = t / ny;
  return ((x + y + z) & 1) ? -1.f : 1.f;
}

// Byte offset of element (row r, k) of a K-major operand stored as
// 64-element chunks of `rows` x 128 B with the 128-byte swizzle.
__device__ __forceinline__ uint32_t sw128_offset(int r, int k, int rows) {
  const int kc = k / kKChunk, kk = k % kKChunk;
  return (uint32_t)(kc * rows * 128 + r * 128 + ((((kk >> 3) ^ (r & 7))) << 4) + (kk & 7) * 2);
}

// The coefficient operand image, built once per call in global memory in the
// exact swizzled shared-memory layout: rows [0, 2C) from alpha, rows
// [half, half + 2C) from dalpha (Jacobian), zero elsewhere.
__global__ void k_build_coef(TcArgs a, int with_dalpha, __nv_bfloat16* __restrict__ img) {
  const int Kp = a.KC * kKChunk;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n_gemm * Kp) return;
  const int r = e / Kp, k = e % Kp;
  float v = 0.f;
  const float2* src = nullptr;
  int rr = r;
  if (r < 2 * a.C) {
    src = a.alpha;
  } else if (with_dalpha && r >= a.half && r < a.half + 2 * a.C) {
    src = a.dalpha;
    rr = r - a.half;
  }
  if (src && k < 2 * a.q) {
    const int c = rr >> 1, im_row = rr & 1;
    const int j = k < a.q ? k : k - a.q;
    const float2 al = src[(size_t)c * a.q + j];
    if (!im_row) v = k < a.q ? al.x : -al.y;  // row 2c: [Re a, -Im a]
    else v = k < a.q ? al.y : al.x;             // row 2c+1: [Im a, Re a]
  }
  img[sw128_offset(r, k, a.n_gemm) / 2] = __float2bfloat16_rn(v);
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) k_expand_tc(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int Kp = a.KC * kKChunk;
  const uint32_t b_bytes = (uint32_t)a.n_gemm * Kp * 2;
  unsigned char* sB = smem;
  unsigned char* sA = smem + ((b_bytes + 1023) & ~1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(sA + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;  // [2]: double-buffered accumulator
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint64_t* drain = acc_empty + 2;
  uint64_t* bfull = drain + 1;  // coefficient operand landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bfull + 1);
  __shared__ int s_failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    s_failed = 0;
    for (int s = 0; s < kStages; ++s) {
      mpi_ptx::mbar_init(&full[s], 1);
      mpi_ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mpi_ptx::mbar_init(&acc_full[b], 1);
      mpi_ptx::mbar_init(&acc_empty[b], 4);
    }
    mpi_ptx::mbar_init(drain, 1);
    mpi_ptx::mbar_init(bfull, 1);
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
    // ---------------- producer: the coefficient operand image, then TMA tiles of U
    mpi_ptx::mbar_arrive_expect_tx(bfull, b_bytes);
    mpi_ptx::bulk_g2s(sB, a.coef_img, b_bytes, bfull);
    long it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      for (int kc = 0; kc < a.KC; ++kc, ++it) {
        const int s = (int)(it % kStages);
        if (!mpi_ptx::mbar_wait(&empty[s], (uint32_t)(((it / kStages) & 1) ^ 1), a.err)) {
          ok = false;
          break;
        }
        mpi_ptx::mbar_arrive_expect_tx(&full[s], kStageBytes);
        tma_load_2d(sA + s * kStageBytes, &tmap, kc * kKChunk, t * kTileM, &full[s]);
      }
    }
    if (!ok) {
      s_failed = 1;
      // bounded wait for the fills still in flight
      for (long g = (it > kStages ? it - kStages : 0); g < it; ++g)
        mpi_ptx::mbar_wait(&full[g % kStages], (uint32_t)((g / kStages) & 1), nullptr);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_bf16(kTileM, a.n_gemm);
    const uint32_t b_base = mpi_ptx::smem_addr(sB);
    const uint32_t a_base = mpi_ptx::smem_addr(sA);
    long it = 0;
    int tc = 0;
    bool ok = mpi_ptx::mbar_wait(bfull, 0, a.err);
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      const uint32_t tacc = tmem + (uint32_t)(buf * a.half_cols);
      if (!mpi_ptx::mbar_wait(&acc_empty[buf], (uint32_t)(((tc >> 1) & 1) ^ 1), a.err)) {
        ok = false;
        break;
      }
      fence_after();
      for (int kc = 0; kc < a.KC; ++kc, ++it) {
        const int s = (int)(it % kStages);
        if (!mpi_ptx::mbar_wait(&full[s], (uint32_t)((it / kStages) & 1), a.err)) {
          ok = false;
          break;
        }
        fence_after();
#pragma unroll
        for (int ks = 0; ks < kKChunk / 16; ++ks) {
          const uint64_t ad = sdesc_sw128(a_base + s * kStageBytes + ks * 32);
          const uint64_t bd = sdesc_sw128(b_base + kc * a.n_gemm * 128 + ks * 32);
          mma_bf16(tacc, ad, bd, idesc, (kc | ks) != 0);
        }
        mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
      }
      if (ok) mma_commit(&acc_full[buf]);
    }
    // all MMAs issued by this thread have completed once `drain` fires
    mma_commit(drain);
    mpi_ptx::mbar_wait(drain, 0, a.err);
    if (!ok) s_failed = 1;
  } else if (warp >= 2) {
    // ---------------- epilogue: one pixel per thread
    const int quarter = warp & 3;  // TMEM lanes 32 * quarter ..
    const int row = quarter * 32 + lane;
    int tc = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      const bool got = mpi_ptx::mbar_wait(&acc_full[buf], (uint32_t)((tc >> 1) & 1), a.err);
      if (!__all_sync(0xffffffffu, got)) {  // warp-uniform decision before the .sync.aligned loads
        s_failed = 1;
        break;
      }
      fence_after();
      const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * a.half_cols);
      const int n = t * kTileM + row;
      const bool valid = n < a.N;
      const int nn = valid ? n : 0;
      const float sg = (a.centre ? centre_sign(nn, a.nx, a.ny) : 1.f) * a.scale;
      const float2 pimg = (MODE != EX_MAPS) ? a.p[nn] : make_float2(0.f, 0.f);
      const float2 dpi = (MODE == EX_JFWD) ? a.dp[nn] : make_float2(0.f, 0.f);
      float2 pacc = make_float2(0.f, 0.f);
      const int n_chunks = (2 * a.C + 15) / 16;
      for (int ch = 0; ch < n_chunks; ++ch) {
        // issue this chunk's per-coil loads before the accumulator reads
        float2 wv[8];
        if (MODE == EX_ADJ || MODE == EX_JADJ) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int c = min(ch * 8 + i, a.C - 1);
            wv[i] = a.w[(size_t)c * a.N + nn];
          }
        }
        float r[16];
        tmem_ld16(tbase + ch * 16, r);
        float rd[16];
        if (MODE == EX_JFWD) tmem_ld16(tbase + a.half + ch * 16, rd);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int c = ch * 8 + i;
          const bool cv = valid && c < a.C;
          const float2 s = make_float2(r[2 * i], r[2 * i + 1]);
          if (MODE == EX_MAPS) {
            if (cv) a.out[(size_t)c * a.N + n] = s;
          } else if (MODE == EX_FWD) {
            const float2 v = cmul(s, pimg);
            if (cv) a.out[(size_t)c * a.N + n] = make_float2(v.x * sg, v.y * sg);
          } else if (MODE == EX_JFWD) {
            const float2 ds = make_float2(rd[2 * i], rd[2 * i + 1]);
            const float2 v1 = cmul(s, dpi);
            const float2 v2 = cmul(ds, pimg);
            if (cv) a.out[(size_t)c * a.N + n] = make_float2((v1.x + v2.x) * sg, (v1.y + v2.y) * sg);
          } else {
            if (cv) {
              const float2 t2 = cmul_conj(s, wv[i]);
              pacc.x += t2.x;
              pacc.y += t2.y;
              if (MODE == EX_JADJ) {
                const float2 v = cmul_conj(pimg, wv[i]);
                a.vout[(size_t)c * a.N + n] = make_float2(v.x * sg, v.y * sg);
              }
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mpi_ptx::mbar_arrive(&acc_empty[buf]);
      if ((MODE == EX_ADJ || MODE == EX_JADJ) && valid) a.out[n] = make_float2(pacc.x * sg, pacc.y * sg);
    }
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

void tc_basis_release(mpi_basis* b) {
  delete (CUtensorMap*)b->tmap;
  b->tmap = nullptr;
}

mpi_status launch_expand_tc(mpi_ctx* ctx, const mpi_basis* b, int mode, const ExpandArgs& x) {
  if (!b->Ubf || !b->tmap) return set_err(ctx, MPI_ERR_UNSUPPORTED, "basis has no BF16 operand copy");
  if (x.N <= 0 || x.C <= 0) return MPI_OK;
  TcArgs a;
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
  const size_t b_bytes = round_up(a.n_gemm * b->Kp * 2, 1024);
  const size_t smem = 1024 + b_bytes + (size_t)kStages * kStageBytes + (2 * kStages + 6) * 8 + 16;
  if ((size_t)a.n_gemm * b->Kp * 2 > kCoefImgBytes) return set_err(ctx, MPI_ERR_UNSUPPORTED, "coefficient image");
  a.coef_img = (const __nv_bfloat16*)ctx->coef_img;
  MPI_PROF(ctx, KF_OTHER);
  k_build_coef<<<(a.n_gemm * b->Kp + 255) / 256, 256, 0, ctx->stream>>>(a, mode == EX_JFWD,
                                                                          (__nv_bfloat16*)ctx->coef_img);
  MPI_LAUNCH_CHECK(ctx, "k_build_coef");
  if (smem > 227 * 1024) return set_err(ctx, MPI_ERR_UNSUPPORTED, "BF16 expansion: shared memory");
  const int n_tiles = (x.N + kTileM - 1) / kTileM;
  // two CTAs per SM when shared memory allows, so that one's epilogue overlaps the other's loads
  const int per_sm = smem <= 110 * 1024 ? 2 : 1;
  const int grid = std::min(n_tiles, per_sm * std::max(ctx->num_sms, 1));
  const CUtensorMap& map = *(const CUtensorMap*)b->tmap;
  cudaError_t e = cudaSuccess;
#define MPI_TC_CASE(m)                                                                                        \
  case m:                                                                                                     \
    e = cudaFuncSetAttribute(k_expand_tc<m>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
    if (e != cudaSuccess) return cuda_check(ctx, e, "tc smem attribute");                                    \
    MPI_PROF(ctx, KF_EXPAND);                                                                                \
    k_expand_tc<m><<<grid, kThreads, smem, ctx->stream>>>(map, a);                                           \
    break;
  switch (mode) {
    MPI_TC_CASE(EX_MAPS)
    MPI_TC_CASE(EX_FWD)
    MPI_TC_CASE(EX_JFWD)
    MPI_TC_CASE(EX_ADJ)
    MPI_TC_CASE(EX_JADJ)
    default:
      return set_err(ctx, MPI_ERR_ARG, "unknown expansion mode");
  }
#undef MPI_TC_CASE
  MPI_LAUNCH_CHECK(ctx, "k_expand_tc");
  return MPI_OK;
}
