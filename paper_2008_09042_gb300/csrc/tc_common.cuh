// Shared pieces of the tensor-core expansion kernels (BF16 and 3xTF32):
// descriptors, TMA / tcgen05 wrappers and the per-pixel epilogue.
#pragma once

#include <cuda.h>

#include "mpi_internal.h"
#include "ptx.cuh"

namespace mpi_tc {

constexpr int kTileM = 128;
constexpr int kStageBytes = kTileM * 128;    // one 128 x 64 BF16 tile

struct TcArgs {
  int N, q, C, KC, n_gemm, half, half_cols, tmem_cols;
  int lo_cols;  // column offset of a second partial accumulator summed in the epilogue (0: none)
  int nx, ny, centre;
  float scale;
  const float2* alpha;
  const float2* dalpha;
  const void* coef_img;
  const float2* p;
  const float2* dp;
  const float2* w;
  float2* out;
  float2* vout;
  int* err;
};

// Position in a ring of `n` shared-memory stages: slot and the parity of the
// slot's current mbarrier phase.  Advanced one step at a time (no division on
// the issue path).
struct RingPos {
  int s = 0;
  uint32_t ph = 0;
  __device__ __forceinline__ void next(int n) {
    if (++s == n) {
      s = 0;
      ph ^= 1u;
    }
  }
};

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzled layout: start address >> 4 (bits 0-13), leading byte offset 16 B
// (unused for this layout, bits 16-29), stride byte offset 1024 B between
// 8-row groups (bits 32-45), descriptor version 1 (bits 46-47), swizzle mode
// 2 = 128-byte (bits 61-63).
static __device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
static __host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

static __device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(mpi_ptx::smem_addr(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(mpi_ptx::smem_addr(bar))
      : "memory");
}

// The MMA issue asm carries no memory clobber: the barrier waits, fences and
// commits around it (all volatile asm with memory clobbers) order it, and a
// clobber here would make the compiler reload state between back-to-back MMAs.
static __device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// As mma_bf16 with the accumulate flag fixed to 1.
static __device__ __forceinline__ void mma_bf16_acc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile("tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, 1;" ::"r"(tmem_d), "l"(adesc), "l"(bdesc),
               "r"(idesc));
}

static __device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   mpi_ptx::smem_addr(bar))
               : "memory");
}

static __device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
static __device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Start a load of 16 consecutive FP32 accumulator columns of this warp's 32 TMEM
// lanes; the registers are valid only after tmem_wait_ld() and reg_fence16().
static __device__ __forceinline__ void tmem_ld16_start(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
static __device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Ties the registers of a started load to a point after tmem_wait_ld(), so the
// compiler cannot move their first use ahead of the wait.
static __device__ __forceinline__ void reg_fence16(uint32_t (&v)[16]) {
  asm volatile(""
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                 "+r"(v[15]));
}

static __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
static __device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

static __device__ __forceinline__ float centre_sign(int n, int nx, int ny) {
  int x = n % nx;
  int t = n / nx;
  int y = t % ny;
  int z = t / ny;
  return ((x + y + z) & 1) ? -1.f : 1.f;
}

// Instruction descriptor, kind::tf32: as idesc_bf16 with A = B = TF32 (format 2).
static __host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row r, k) of a K-major operand with `esize`-byte
// elements, stored as chunks of 128-byte rows (`rows` rows per chunk) with the
// 128-byte swizzle (16-byte unit index XOR row mod 8).
static __host__ __device__ __forceinline__ uint32_t sw128_offset_e(int r, int k, int rows, int esize) {
  const int per_row = 128 / esize, per_unit = 16 / esize;
  const int kc = k / per_row, kk = k % per_row;
  return (uint32_t)(kc * rows * 128 + r * 128 + ((((kk / per_unit) ^ (r & 7))) << 4) + (kk % per_unit) * esize);
}

// Epilogue warps (4 of them, warp w owning TMEM lanes 32 (w % 4) ..): one pixel
// per thread, reading the double-buffered accumulator of each tile this CTA owns.
template <int MODE, bool SUM2 = false>
static __device__ __forceinline__ void tc_epilogue(const TcArgs& a, uint32_t tmem, int warp, int lane,
                                                   uint64_t* acc_full, uint64_t* acc_empty, int n_tiles,
                                                   int* s_failed) {
  {
    // ---------------- epilogue: one pixel per thread
    const int quarter = warp & 3;  // TMEM lanes 32 * quarter ..
    const int row = quarter * 32 + lane;
    int tc = 0;
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tc) {
      const int buf = tc & 1;
      const bool got = mpi_ptx::mbar_wait(&acc_full[buf], (uint32_t)((tc >> 1) & 1), a.err);
      if (!__all_sync(0xffffffffu, got)) {  // warp-uniform decision before the .sync.aligned loads
        *s_failed = 1;
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
        // accumulator columns of this chunk (and of the Jacobian's second block), plus
        // the second partial sums where the accumulation is split (a.lo_cols)
        uint32_t v[16], vd[16], w2[16], wd2[16];
        tmem_ld16_start(tbase + ch * 16, v);
        if (MODE == EX_JFWD) tmem_ld16_start(tbase + a.half + ch * 16, vd);
        if (SUM2) {
          tmem_ld16_start(tbase + a.lo_cols + ch * 16, w2);
          if (MODE == EX_JFWD) tmem_ld16_start(tbase + a.lo_cols + a.half + ch * 16, wd2);
        }
        tmem_wait_ld();
        reg_fence16(v);
        if (MODE == EX_JFWD) reg_fence16(vd);
        if (SUM2) {
          reg_fence16(w2);
          if (MODE == EX_JFWD) reg_fence16(wd2);
        }
        float r[16], rd[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          r[i] = __uint_as_float(v[i]) + (SUM2 ? __uint_as_float(w2[i]) : 0.f);
          if (MODE == EX_JFWD) rd[i] = __uint_as_float(vd[i]) + (SUM2 ? __uint_as_float(wd2[i]) : 0.f);
        }
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
}

}  // namespace mpi_tc
