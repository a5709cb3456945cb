// Shared pieces of the tensor-core expansion kernels (BF16 and 3xTF32):
// descriptors, TMA / tcgen05 wrappers and the per-pixel epilogue.
#pragma once

#include <cuda_bf16.h>

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
  const float2* p;
  const float2* dp;
  const float2* w;
  float2* out;
  float2* vout;
  int* err;
  int tuck_B;         // maps mode: output remap for a flattened Tucker operand (0: none)
  long tuck_stride;
  // Coil groups in one launch (3xTF32 kernel): CTA row blockIdx.y takes coils
  // [blockIdx.y group_coils, + group_coils) of C_total; 0 = one group.
  int group_coils;
  int C_total;
  // EX_SCATTER output map (see ScatterMap); sc_col0 = the launch row's first column pair
  int sc_L0, sc_L1, sc_im, sc_col0;
  long sc_hi, sc_mid, sc_col;
  int sc_bf16;            // EX_SCATTER: BF16 outputs (same element offsets)
  // K split (3xTF32 EX_SCATTER_ADD): grid row blockIdx.y takes K boxes
  // [y KC, (y + 1) KC) of ksplit parts and adds its partial products into the
  // (zeroed) output
  int ksplit;
  int k_off;              // global K index of the coefficient image's first column
  int accumulate;         // EX_FWD / EX_JFWD: add into out instead of storing
  const ExpandRow* rows;  // grouped launch: row blockIdx.y's pointers and coil count (nullptr: none)
  long long wait_cycles;  // bounded-wait limit (SM clock cycles)
  int stall_after;        // fault injection: the producer stops after this many stages (-1: off)
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

static __device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

// lo(x) = x - hi(x), rounded to the nearest TF32 value (ties away from zero)
// so that the tensor core reads it exactly.  An FP32 lo would be truncated by
// the tensor core, and the truncation of every lo towards zero biases a long
// sum of products; rounded, the error (at most 2^-11 of lo, 2^-22 of x) is
// unbiased.
static __device__ __forceinline__ float tf32_lo(float v) {
  const float lo = v - tf32_hi(v);
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(lo));
  return __uint_as_float(r);
}

// The coefficient operand, written straight into shared memory in the swizzled
// K-major layout by the four epilogue warps (etid = 0..127) while the first
// tiles of U are still in flight.  Per coil c, row 2c is [Re a_c, -Im a_c] and
// row 2c+1 is [Im a_c, Re a_c] over K = [0, q) | [q, 2q), so that accumulator
// columns 2c, 2c+1 hold Re and Im of s_c; rows [half, half + 2C) hold dalpha
// for the Jacobian; everything else is zero.  SPLIT (the 3xTF32 kernel): rows
// [0, n_gemm) hold hi of those values and rows [n_gemm, 2 n_gemm) their lo
// parts, as FP32; otherwise one block of BF16 rows.  Each step writes whole
// 16-byte swizzle units (4 FP32 or 8 BF16 consecutive K values of a row pair).
// Ends with the writes made visible to the tensor core and one arrival per
// warp on `ready`.
template <bool SPLIT>
static __device__ void build_coef_smem(const TcArgs& a, unsigned char* sB, int Kp, bool with_dalpha, int etid,
                                       uint64_t* ready) {
  constexpr int E = SPLIT ? 4 : 8;        // K values per 16-byte unit
  constexpr int esize = SPLIT ? 4 : 2;
  const int rows = SPLIT ? 2 * a.n_gemm : a.n_gemm;
  const int units = Kp / E;               // units along K per row
  const int per_blk = a.C * units;
  const int n_data = (with_dalpha ? 2 : 1) * per_blk;
  // zero rows: [2C, half) always, [half + 2C, n_gemm) for the Jacobian, [2C, n_gemm) otherwise
  const int z0 = with_dalpha ? a.half - 2 * a.C : a.n_gemm - 2 * a.C;
  const int z1 = with_dalpha ? a.n_gemm - a.half - 2 * a.C : 0;
  const int n_zero = (z0 + z1) * units;
  for (int task = etid; task < n_data + n_zero; task += 128) {
    if (task < n_data) {
      const int blk = task >= per_blk;
      const int t2 = task - blk * per_blk;
      const int c = t2 / units, u = t2 - c * units;
      const float2* src = (blk ? a.dalpha : a.alpha) + (size_t)c * a.q;
      const int r0 = (blk ? a.half : 0) + 2 * c, k0 = u * E;
      float re[E], im[E];  // rows r0 and r0 + 1
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int k = k0 + e + a.k_off;
        float2 al = make_float2(0.f, 0.f);
        if (k < 2 * a.q) al = src[k < a.q ? k : k - a.q];
        re[e] = k < a.q ? al.x : (k < 2 * a.q ? -al.y : 0.f);
        im[e] = k < a.q ? al.y : (k < 2 * a.q ? al.x : 0.f);
      }
      if (SPLIT) {
        float4 h0, h1, l0, l1;
        h0 = make_float4(tf32_hi(re[0]), tf32_hi(re[1]), tf32_hi(re[2]), tf32_hi(re[3]));
        h1 = make_float4(tf32_hi(im[0]), tf32_hi(im[1]), tf32_hi(im[2]), tf32_hi(im[3]));
        l0 = make_float4(tf32_lo(re[0]), tf32_lo(re[1]), tf32_lo(re[2]), tf32_lo(re[3]));
        l1 = make_float4(tf32_lo(im[0]), tf32_lo(im[1]), tf32_lo(im[2]), tf32_lo(im[3]));
        *reinterpret_cast<float4*>(sB + sw128_offset_e(r0, k0, rows, esize)) = h0;
        *reinterpret_cast<float4*>(sB + sw128_offset_e(r0 + 1, k0, rows, esize)) = h1;
        *reinterpret_cast<float4*>(sB + sw128_offset_e(r0 + a.n_gemm, k0, rows, esize)) = l0;
        *reinterpret_cast<float4*>(sB + sw128_offset_e(r0 + 1 + a.n_gemm, k0, rows, esize)) = l1;
      } else {
        uint4 v0, v1;
        __nv_bfloat162* p0 = reinterpret_cast<__nv_bfloat162*>(&v0);
        __nv_bfloat162* p1 = reinterpret_cast<__nv_bfloat162*>(&v1);
#pragma unroll
        for (int e = 0; e < E / 2; ++e) {
          p0[e] = __floats2bfloat162_rn(re[2 * e], re[2 * e + 1]);
          p1[e] = __floats2bfloat162_rn(im[2 * e], im[2 * e + 1]);
        }
        *reinterpret_cast<uint4*>(sB + sw128_offset_e(r0, k0, rows, esize)) = v0;
        *reinterpret_cast<uint4*>(sB + sw128_offset_e(r0 + 1, k0, rows, esize)) = v1;
      }
    } else {
      const int t2 = task - n_data;
      const int zr = t2 / units, u = t2 - zr * units;
      const int r = zr < z0 ? 2 * a.C + zr : a.half + 2 * a.C + (zr - z0);
      const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(sB + sw128_offset_e(r, u * E, rows, esize)) = zero;
      if (SPLIT) *reinterpret_cast<uint4*>(sB + sw128_offset_e(r + a.n_gemm, u * E, rows, esize)) = zero;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
  __syncwarp();
  if ((etid & 31) == 0) mpi_ptx::mbar_arrive(ready);
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
      const bool got = mpi_ptx::mbar_wait(&acc_full[buf], (uint32_t)((tc >> 1) & 1), a.err, a.wait_cycles);
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
      constexpr bool kScatter = MODE == EX_SCATTER || MODE == EX_SCATTER_ADD;
      const float2 pimg = (MODE != EX_MAPS && !kScatter) ? a.p[nn] : make_float2(0.f, 0.f);
      // maps mode: where coil c of pixel n goes ([C][N], or the Tucker remap)
      size_t maps_base = (size_t)n, maps_cstride = (size_t)a.N;
      if (MODE == EX_MAPS && a.tuck_B) {
        const long nb = nn / a.tuck_B;
        maps_base = (size_t)nb * a.tuck_stride + (size_t)(nn - nb * a.tuck_B);
        maps_cstride = (size_t)a.tuck_B;
      }
      const float2 dpi = (MODE == EX_JFWD) ? a.dp[nn] : make_float2(0.f, 0.f);
      // scatter mode: this row's part of the output address
      size_t sc_base = 0;
      if (kScatter) {
        const int lo = nn % a.sc_L0, q1 = nn / a.sc_L0;
        sc_base = (size_t)(q1 / a.sc_L1) * a.sc_hi + (size_t)(q1 % a.sc_L1) * a.sc_mid + lo +
                  (size_t)a.sc_col0 * a.sc_col;
      }
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
            if (cv) a.out[maps_base + (size_t)c * maps_cstride] = s;
          } else if (MODE == EX_SCATTER_ADD) {
            if (cv) {
              // partial sums of the K parts: added into a zeroed output; with two
              // parts (0 + a) + b = (0 + b) + a exactly, so the result does not
              // depend on which part lands first
              float* o = reinterpret_cast<float*>(a.out) + sc_base + (size_t)c * a.sc_col;
              atomicAdd(o, s.x);
              atomicAdd(o + a.sc_im, s.y);
            }
          } else if (MODE == EX_SCATTER) {
            if (cv && a.sc_bf16) {
              __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(a.out) + sc_base + (size_t)c * a.sc_col;
              o[0] = __float2bfloat16_rn(s.x);
              o[a.sc_im] = __float2bfloat16_rn(s.y);
            } else if (cv) {
              float* o = reinterpret_cast<float*>(a.out) + sc_base + (size_t)c * a.sc_col;
              o[0] = s.x;
              o[a.sc_im] = s.y;
            }
          } else if (MODE == EX_FWD) {
            const float2 v = cmul(s, pimg);
            if (cv) {
              float2* o = a.out + (size_t)c * a.N + n;
              float2 r2 = make_float2(v.x * sg, v.y * sg);
              if (a.accumulate) {
                r2.x += o->x;
                r2.y += o->y;
              }
              *o = r2;
            }
          } else if (MODE == EX_JFWD) {
            const float2 ds = make_float2(rd[2 * i], rd[2 * i + 1]);
            const float2 v1 = cmul(s, dpi);
            const float2 v2 = cmul(ds, pimg);
            if (cv) {
              float2* o = a.out + (size_t)c * a.N + n;
              float2 r2 = make_float2((v1.x + v2.x) * sg, (v1.y + v2.y) * sg);
              if (a.accumulate) {
                r2.x += o->x;
                r2.y += o->y;
              }
              *o = r2;
            }
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
