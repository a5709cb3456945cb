// FP32-accurate basis expansion on the tensor cores (3xTF32), the FP32 path's
// version of the dense contraction s_k = U alpha_k (Maxwell Regularization
// section; Eqs. 5 and 7 and the Jacobian-adjoint display after Eq. 7 for the
// fused epilogues).
//
// Every FP32 operand x is split as x = hi(x) + lo(x), hi(x) = x with its 13
// low mantissa bits cleared (exactly representable in TF32) and lo(x) = x - hi(x)
// (exact in FP32); then U A^T = U_hi A_hi + U_hi A_lo + U_lo A_hi up to a
// relative error of about 2^-20 (the dropped U_lo A_lo term and the TF32
// truncation of the lo parts), accumulated in FP32 in tensor memory.
//
// Same real-ified GEMM as the BF16 kernel: 128-pixel tiles of U are the A
// operand, the coefficient rows B, with a TMA ring (128-byte swizzle), one MMA
// thread, a double-buffered TMEM accumulator and four epilogue warps.  Per
// 8-element K step it issues two kind::tf32 MMAs:
//  - U_hi against the stacked rows [A_hi; A_lo] (N = 2 n), which writes U_hi A_hi
//    and U_hi A_lo into two column blocks that the epilogue adds.  U_hi is the
//    raw FP32 tile: the tensor core reads an FP32 operand of kind::tf32 as its
//    upper 19 bits, which is hi(x) exactly.  Each context measures that reading
//    when it is made (k_tf32_reading below) and runs these kernels only where
//    it holds.
//  - U_lo against A_hi (N = n) into the first block, with U_lo taken from tensor
//    memory: four converter warps read each landed tile from shared memory and
//    store lo(x) with tcgen05.st into a TMEM slot of the stage, so the split
//    costs no shared-memory writes and each ring stage is one 16 KB slot.
// A tcgen05.mma costs about the same to issue for any N up to 64, so stacking
// the coefficient rows saves a third of the instructions.  The stacked
// coefficient image is built once per call.  Every mbarrier wait is bounded.
// Operands whose K box count is odd end each tile with a one-box stage (a
// compile-time variant).  EX_SCATTER_ADD splits K over the grid rows: each
// row's coefficient image covers its part of K, and its partial products are
// added into the output, which the caller has cleared.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "mpi_internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace {

using namespace mpi_tc;

constexpr int kKChunk32 = 32;                     // FP32 elements per 128-byte swizzle row (one TMA box)
constexpr int kBoxBytes32 = kTileM * 128;          // one 128-pixel x 32-element box
constexpr int kBoxesPerStage = 2;                  // a ring stage holds 64 K elements
constexpr int kStageBytes32 = kBoxesPerStage * kBoxBytes32;
constexpr int kThreads32 = 320;   // warp 0 TMA, 1 MMA, 2-5 epilogue, 6-9 converters
constexpr size_t kSmemMax = 232448 - 128;  // 227 KB less room for the static shared word

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_tf32_acc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(tmem_d), "l"(adesc), "l"(bdesc),
               "r"(idesc));
}

// 32 consecutive 32-bit TMEM columns of this warp's 32 lanes, one row per thread.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
      "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
      "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}

// D += A B^T with A (128 x 8, TF32) read from tensor memory.
__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc) {
  asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;" ::"r"(tmem_d), "r"(tmem_a), "l"(bdesc),
               "r"(idesc));
}

// Roles: warp 0 lane 0 loads U tiles (TMA ring of `stages` 16 KB slots); warps
// 6-9 write each landed tile's lo part to the stage's TMEM slot (signalled on
// `conv`); warp 1 lane 0 issues the U_hi MMAs of a chunk once it has landed
// and the U_lo MMAs once its lo part is in TMEM, then commits the stage back to
// the producer (`empty`); warps 2-5 run the fused epilogue from a
// double-buffered accumulator.  A stage holds two 32-element boxes (64 K
// elements).  TMEM columns: [0, 2 half_cols) accumulators, then 64 columns of
// lo(U) per stage.
// ODD: the K box count is odd, so the last ring stage of each tile holds one box
// (a compile-time choice: with an even count the stage loop has no box test).
template <int MODE, bool ODD = false>
__global__ void __launch_bounds__(kThreads32, 1) k_expand_tf32x3(const __grid_constant__ CUtensorMap tmap, TcArgs a_in,
                                                                int stages) {
  // Coil groups: the CTAs of row blockIdx.y expand their group's coils.  The
  // rows of a launch stream the same basis tiles in the same order, so all but
  // one of them mostly find each tile in L2.
  TcArgs a = a_in;
  if (a.rows) {  // grouped launch: this row's slice
    const ExpandRow r = a.rows[blockIdx.y];
    a.alpha = r.alpha;
    a.p = r.p;
    a.w = r.w;
    a.out = r.out;
    a.C = r.C;
  }
  if (a.group_coils) {
    const int c0 = (int)blockIdx.y * a.group_coils;
    a.C = min(a.group_coils, a.C_total - c0);
    a.alpha += (size_t)c0 * a.q;
    if (a.dalpha) a.dalpha += (size_t)c0 * a.q;
    if (MODE == EX_SCATTER) a.sc_col0 = c0;
    else a.out += a.tuck_B ? (size_t)c0 * a.tuck_B : (size_t)c0 * a.N;
  }
  // K split: this row's boxes start at box kc0 of the operand rows
  int kc0 = 0;
  if (MODE == EX_SCATTER_ADD) {
    kc0 = (int)blockIdx.y * a.KC;
    a.k_off = kc0 * kKChunk32;
  }
  extern __shared__ unsigned char smem_raw[];
  // aligned by an offset from the shared array, so that accesses stay shared-memory ones
  unsigned char* smem = smem_raw + ((1024u - (mpi_ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  const int Kp = a.KC * kKChunk32;
  const uint32_t b_bytes = 2u * (uint32_t)a.n_gemm * Kp * 4;  // stacked [hi; lo] coefficient rows
  const uint32_t b_pad = (b_bytes + 1023) & ~1023u;
  unsigned char* sB = smem;
  unsigned char* sA = smem + b_pad;  // [stages] U tiles
  uint64_t* full = reinterpret_cast<uint64_t*>(sA + (size_t)stages * kStageBytes32);
  uint64_t* conv = full + stages;
  uint64_t* empty = conv + stages;
  uint64_t* acc_full = empty + stages;  // [2]
  uint64_t* acc_empty = acc_full + 2;   // [2]
  uint64_t* drain = acc_empty + 2;
  uint64_t* bfull = drain + 1;
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
      mpi_ptx::mbar_init(&conv[s], 4);
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
  const uint32_t tmem_lo = tmem + (uint32_t)(2 * a.half_cols);  // lo(U) slots, 32 columns per stage
  const int n_tiles = (a.N + kTileM - 1) / kTileM;
  // ring stages this CTA processes (its tiles x ceil(KC / 2)), numbered g = 0 .. G-1;
  // with an odd box count KC the last stage of each tile holds one box
  const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int G = my_tiles * ((a.KC + kBoxesPerStage - 1) / kBoxesPerStage);

  if (warp == 0 && lane == 0) {
    // ---------------- producer: TMA tiles of U
    RingPos r;
    int g = 0, kc = 0, t = (int)blockIdx.x;  // kc: first box of the stage
    for (; g < G; ++g) {
      // fault injection (a test of the timeout path): stop issuing copies, so
      // that every consumer's wait on the stages not loaded runs out
      if (a.stall_after >= 0 && g >= a.stall_after) break;
      if (!mpi_ptx::mbar_wait(&empty[r.s], r.ph ^ 1u, a.err, a.wait_cycles)) break;
      unsigned char* dst = sA + (size_t)r.s * kStageBytes32;
      const bool two = !ODD || kc + 1 < a.KC;
      mpi_ptx::mbar_arrive_expect_tx(&full[r.s], two ? kStageBytes32 : kBoxBytes32);
      tma_load_2d(dst, &tmap, (kc0 + kc) * kKChunk32, t * kTileM, &full[r.s]);
      if (two) tma_load_2d(dst + kBoxBytes32, &tmap, (kc0 + kc + 1) * kKChunk32, t * kTileM, &full[r.s]);
      r.next(stages);
      kc += kBoxesPerStage;
      if (kc >= a.KC) {
        kc = 0;
        t += (int)gridDim.x;
      }
    }
    if (g < G) {
      s_failed = 1;
      for (int h = (g > stages ? g - stages : 0); h < g; ++h)  // fills still in flight (bounded)
        mpi_ptx::mbar_wait(&full[h % stages], (uint32_t)((h / stages) & 1), nullptr, a.wait_cycles);
    }
  } else if (warp >= 6) {
    // ---------------- converters: lo(x) of tile row 32 (warp % 4) + lane into TMEM.
    // A stage's TMEM slot is free again once its tile has landed anew: the
    // producer reloads a stage only after the MMAs that read it have completed.
    const int row = (warp & 3) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    RingPos r;
    int kc = 0;  // first box of the stage (the last stage of a tile holds one box when KC is odd)
    for (int g = 0; g < G; ++g) {
      const bool got = mpi_ptx::mbar_wait(&full[r.s], r.ph, a.err, a.wait_cycles);
      if (!__all_sync(0xffffffffu, got)) {
        s_failed = 1;
        break;
      }
      const int nb = (!ODD || kc + 1 < a.KC) ? 2 : 1;
#pragma unroll
      for (int h = 0; h < kBoxesPerStage; ++h) {
        if (h >= nb) break;
        // the row's 32 FP32 values of box h: 16-byte unit j of a 128-byte row sits at unit j ^ (row % 8)
        const float4* x =
            reinterpret_cast<const float4*>(sA + (size_t)r.s * kStageBytes32 + h * kBoxBytes32 + row * 128);
        float lo[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 v = x[j ^ (row & 7)];
          lo[4 * j + 0] = tf32_lo(v.x);
          lo[4 * j + 1] = tf32_lo(v.y);
          lo[4 * j + 2] = tf32_lo(v.z);
          lo[4 * j + 3] = tf32_lo(v.w);
        }
        tmem_st32(tmem_lo + lane_base + (uint32_t)(r.s * 32 * kBoxesPerStage + 32 * h), lo);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      fence_before();
      __syncwarp();
      if (lane == 0) mpi_ptx::mbar_arrive(&conv[r.s]);
      r.next(stages);
      kc += kBoxesPerStage;
      if (kc >= a.KC) kc = 0;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: per 8-element K step, U_hi x [A_hi; A_lo] and U_lo x A_hi.
    // A descriptor of base + off is desc(base) + (off >> 4): the 14-bit start
    // address field holds every shared-memory address, so the sum never carries.
    const uint32_t idesc_hi = idesc_tf32(kTileM, 2 * a.n_gemm);
    const uint32_t idesc_lo = idesc_tf32(kTileM, a.n_gemm);
    const uint64_t a0 = sdesc_sw128(mpi_ptx::smem_addr(sA));
    const uint64_t b0 = sdesc_sw128(mpi_ptx::smem_addr(sB));
    const uint32_t b_chunk = (uint32_t)(2 * a.n_gemm * 128) >> 4;  // descriptor step per K chunk
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
      for (int kc = 0; kc < a.KC; kc += kBoxesPerStage) {
        const int s = r.s;
        if (!mpi_ptx::mbar_wait(&full[s], r.ph, a.err, a.wait_cycles)) {
          ok = false;
          break;
        }
        fence_after();
        const uint64_t ad = a0 + (uint32_t)(s * (kStageBytes32 >> 4));
        const uint64_t bd = b0 + (uint32_t)kc * b_chunk;
        constexpr uint32_t kBoxDesc = kBoxBytes32 >> 4;
        const bool two = !ODD || kc + 1 < a.KC;  // else this stage holds one box (the last of a tile, KC odd)
        mma_tf32(tacc, ad, bd, idesc_hi, kc != 0);
        mma_tf32_acc(tacc, ad + 2, bd + 2, idesc_hi);
        mma_tf32_acc(tacc, ad + 4, bd + 4, idesc_hi);
        mma_tf32_acc(tacc, ad + 6, bd + 6, idesc_hi);
        if (two) {
          mma_tf32_acc(tacc, ad + kBoxDesc, bd + b_chunk, idesc_hi);
          mma_tf32_acc(tacc, ad + kBoxDesc + 2, bd + b_chunk + 2, idesc_hi);
          mma_tf32_acc(tacc, ad + kBoxDesc + 4, bd + b_chunk + 4, idesc_hi);
          mma_tf32_acc(tacc, ad + kBoxDesc + 6, bd + b_chunk + 6, idesc_hi);
        }
        if (!mpi_ptx::mbar_wait(&conv[s], r.ph, a.err, a.wait_cycles)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t la = tmem_lo + (uint32_t)(s * 32 * kBoxesPerStage);  // K step ks at columns + 8 ks
        mma_tf32_tmem_a(tacc, la, bd, idesc_lo);
        mma_tf32_tmem_a(tacc, la + 8, bd + 2, idesc_lo);
        mma_tf32_tmem_a(tacc, la + 16, bd + 4, idesc_lo);
        mma_tf32_tmem_a(tacc, la + 24, bd + 6, idesc_lo);
        if (two) {
          mma_tf32_tmem_a(tacc, la + 32, bd + b_chunk, idesc_lo);
          mma_tf32_tmem_a(tacc, la + 40, bd + b_chunk + 2, idesc_lo);
          mma_tf32_tmem_a(tacc, la + 48, bd + b_chunk + 4, idesc_lo);
          mma_tf32_tmem_a(tacc, la + 56, bd + b_chunk + 6, idesc_lo);
        }
        mma_commit(&empty[s]);  // frees the stage (tile and TMEM slot) once these MMAs have read it
        r.next(stages);
      }
      if (ok) mma_commit(&acc_full[buf]);
    }
    mma_commit(drain);
    mpi_ptx::mbar_wait(drain, 0, a.err, a.wait_cycles);
    if (!ok) s_failed = 1;
  } else if (warp >= 2 && warp <= 5) {
    mpi_ptx::pdl_wait();  // alpha, p and w may come from the previous kernel
    build_coef_smem<true>(a, sB, Kp, MODE == EX_JFWD, tid - 64, bfull);
    tc_epilogue<MODE, true>(a, tmem, warp, lane, acc_full, acc_empty, n_tiles, &s_failed);
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// FP32 bit pattern of row r's test value in the operand-reading probe: the low
// 13 mantissa bits (the part a TF32 reading drops or rounds away) take
// half-way, just-above, just-below and scattered patterns, the sign alternates.
__host__ __device__ inline uint32_t tf32_probe_bits(int r) {
  constexpr uint32_t kLow[8] = {0x1000u, 0x1000u, 0x1FFFu, 0x0001u, 0x0FFFu, 0x1001u, 0x0800u, 0x17A5u};
  uint32_t hi = ((uint32_t)r * 2654435761u) >> 9;  // 23 scattered bits
  uint32_t low = r < 8 ? kLow[r] : (hi & 0x1FFFu);
  if (r == 1) hi |= 0x2000u;  // a tie whose kept part is odd (nearest-even rounds up, nearest-away too)
  if (r == 0) hi &= ~0x2000u; // a tie whose kept part is even (nearest-even keeps it)
  return ((uint32_t)(r & 1) << 31) | (127u << 23) | (hi & 0x7FE000u) | low;
}

// One kind::tf32 MMA, D = A B^T with A = 128 rows of one test value each (first
// K column; the other 31 zero) and B row 0 = e_0, so D[r][0] is exactly the
// value the tensor core took for A[r][0].  One CTA of 128 threads; the wait on
// the MMA's completion is bounded (on time-out the row reads NaN).
__global__ void __launch_bounds__(128, 1) k_tf32_reading(float* __restrict__ out, int* err, long long wait_cycles) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (mpi_ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = smem;                  // 128 rows x 32 FP32, 128-byte swizzle
  unsigned char* sB = smem + kTileM * 128;   // 16 rows x 32 FP32
  uint64_t* done = reinterpret_cast<uint64_t*>(sB + 16 * 128);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = 0; k < kKChunk32; ++k) {
    const float v = k == 0 ? __uint_as_float(tf32_probe_bits(tid)) : 0.f;
    *reinterpret_cast<float*>(sA + sw128_offset_e(tid, k, kTileM, 4)) = v;
  }
  for (int e = tid; e < 16 * kKChunk32; e += 128) {
    const int n = e / kKChunk32, k = e % kKChunk32;
    *reinterpret_cast<float*>(sB + sw128_offset_e(n, k, 16, 4)) = (n == 0 && k == 0) ? 1.f : 0.f;
  }
  mpi_ptx::fence_proxy_async();  // the tensor core reads what the threads wrote
  if (tid == 0) {
    mpi_ptx::mbar_init(done, 1);
    mpi_ptx::fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(mpi_ptx::smem_addr(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    mma_tf32(tmem, sdesc_sw128(mpi_ptx::smem_addr(sA)), sdesc_sw128(mpi_ptx::smem_addr(sB)), idesc_tf32(kTileM, 16), 0);
    mma_commit(done);
  }
  const bool ok = mpi_ptx::mbar_wait(done, 0, err, wait_cycles);
  fence_after();
  float r = __uint_as_float(0x7FC00000u);
  if (__all_sync(0xffffffffu, ok)) {
    uint32_t v[16];
    tmem_ld16_start(tmem + ((uint32_t)(warp * 32) << 16), v);
    tmem_wait_ld();
    reg_fence16(v);
    r = __uint_as_float(v[0]);
  }
  out[tid] = r;
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
  }
}

__global__ void k_basis_to_f32(const float2* __restrict__ U, int N, int q, int Kp, float* __restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)N * Kp) return;
  const int n = (int)(e / Kp), k = (int)(e % Kp);
  float v = 0.f;
  if (k < q) v = U[(size_t)k * N + n].x;
  else if (k < 2 * q) v = U[(size_t)(k - q) * N + n].y;
  out[e] = v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int round_up_i(int x, int m) { return (x + m - 1) / m * m; }

struct TfPlan {
  int n_gemm, half, half_cols, tmem_cols, stages;
  size_t b_bytes, smem;
};

constexpr int kMaxStages32 = 6;

// ksplit > 1: each CTA row takes 1/ksplit of the K boxes, so its coefficient
// image covers that part of K only.
bool plan_tf32(const mpi_basis* b, int mode, int C, TfPlan* p, int ksplit = 1) {
  const int cols = round_up_i(2 * C, 16);
  p->half = cols;
  p->n_gemm = mode == EX_JFWD ? 2 * cols : cols;
  if (2 * p->n_gemm > 256) return false;  // the stacked [hi; lo] rows form one MMA's N
  int acc_cols = 32;
  while (acc_cols < 2 * p->n_gemm) acc_cols <<= 1;
  p->half_cols = acc_cols;
  p->b_bytes = 2 * (size_t)p->n_gemm * (b->Kp32 / ksplit) * 4;
  // alignment slack + the stacked coefficient image + 3 barriers per stage and 6 more + TMEM slot
  const size_t fixed = 1024 + ((p->b_bytes + 1023) & ~(size_t)1023) + 8 * (3 * kMaxStages32 + 6) + 16;
  if (fixed + 2 * (size_t)kStageBytes32 > kSmemMax) return false;
  int stages = (int)std::min<size_t>(kMaxStages32, (kSmemMax - fixed) / kStageBytes32);
  // TMEM: two accumulators, then 64 columns of lo(U) per stage, within the SM's 512
  stages = std::min(stages, (512 - 2 * acc_cols) / (32 * kBoxesPerStage));
  if (stages < 2) return false;
  p->stages = stages;
  int tcols = 32;
  while (tcols < 2 * acc_cols + 32 * kBoxesPerStage * stages) tcols <<= 1;
  p->tmem_cols = tcols;
  p->smem = fixed + (size_t)stages * kStageBytes32;
  return true;
}

}  // namespace

mpi_status tf32_basis_prepare(mpi_ctx* ctx, mpi_basis* b) {
  const int Kp = round_up_i(2 * b->q, kKChunk32 * kBoxesPerStage);  // whole ring stages (an even box count)
  cudaError_t e = cudaMalloc(&b->Uf32, (size_t)b->N * Kp * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->Uf32 = nullptr;
    return set_err(ctx, MPI_ERR_OOM, "FP32 operand copy");
  }
  const size_t total = (size_t)b->N * Kp;
  MPI_PROF(ctx, KF_OTHER);
  k_basis_to_f32<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(b->U, b->N, b->q, Kp, b->Uf32);
  MPI_LAUNCH_CHECK(ctx, "k_basis_to_f32");
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
  }
  CUtensorMap* map = new CUtensorMap;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)b->N};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKChunk32, (cuuint32_t)kTileM};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = ((EncodeTiledFn)fn)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, b->Uf32, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    delete map;
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "tensor map encoding failed");
  }
  b->tmap32 = map;
  b->Kp32 = Kp;
  return MPI_OK;
}

bool tf32_encode_operand_map(void* map, void* ptr, long rows, int Kp) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKChunk32, (cuuint32_t)kTileM};
  const cuuint32_t estr[2] = {1, 1};
  return ((EncodeTiledFn)fn)((CUtensorMap*)map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tf32_encode_operand_map_k(void* map, void* ptr, long rows, int K) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  // K columns stored; boxes past K (up to the kernel's Kp) read as zeros
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kKChunk32, (cuuint32_t)kTileM};
  const cuuint32_t estr[2] = {1, 1};
  return ((EncodeTiledFn)fn)((CUtensorMap*)map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void tf32_basis_release(mpi_basis* b) {
  delete (CUtensorMap*)b->tmap32;
  b->tmap32 = nullptr;
}

bool tf32_ksplit_supported(const mpi_basis* b, int mode, int C, int ksplit) {
  TfPlan p;
  if (!b->ctx || !b->ctx->tf32x3 || mode != EX_SCATTER_ADD || ksplit < 2 || (b->Kp32 / kKChunk32) % ksplit)
    return false;
  return b->Uf32 && b->tmap32 && plan_tf32(b, mode, C, &p, ksplit);
}

bool tf32_supported(const mpi_basis* b, int mode, int C) {
  TfPlan p;
  // the 3xTF32 split is exact only where the probe found the truncating reading
  if (!b->ctx || !b->ctx->tf32x3) return false;
  return b->Uf32 && b->tmap32 && plan_tf32(b, mode, C, &p);
}

int tf32_reading_probe(mpi_ctx* ctx) {
  float* d = nullptr;
  if (cudaMalloc(&d, 128 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return MPI_TF32_READ_FAILED;
  }
  const size_t smem = kTileM * 128 + 16 * 128 + 64 + 1024;
  k_tf32_reading<<<1, 128, smem, ctx->stream>>>(d, ctx->dev_err, ctx->wait_cycles);
  cudaError_t e = cudaGetLastError();
  float h[128];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), ctx->stream);  // a timed-out wait
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MPI_TF32_READ_FAILED;
  }
  // compare each row with the candidate readings of its value (sign-magnitude
  // bits: rounding the magnitude is rounding the value symmetrically)
  bool trunc = true, even = true, away = true, full = true;
  for (int r = 0; r < 128; ++r) {
    const uint32_t x = tf32_probe_bits(r);
    uint32_t g;
    memcpy(&g, &h[r], 4);
    trunc &= g == (x & ~0x1FFFu);
    even &= g == ((x + 0x0FFFu + ((x >> 13) & 1u)) & ~0x1FFFu);
    away &= g == ((x + 0x1000u) & ~0x1FFFu);
    full &= g == x;
  }
  if (trunc) return MPI_TF32_READ_TRUNCATE;
  if (even) return MPI_TF32_READ_NEAREST_EVEN;
  if (away) return MPI_TF32_READ_NEAREST_AWAY;
  if (full) return MPI_TF32_READ_FULL;
  return MPI_TF32_READ_OTHER;
}

int tf32_group(const mpi_basis* b, int mode, int C) {
  if (tf32_supported(b, mode, C)) return C;
  // coils are independent in these modes, so they can run in groups whose
  // coefficient operand and accumulators fit; the adjoint modes sum over coils
  if (mode != EX_MAPS && mode != EX_FWD && mode != EX_JFWD && mode != EX_SCATTER) return 0;
  for (int g = C - 1; g >= 1; --g)
    if (tf32_supported(b, mode, g)) return g;
  return 0;
}

mpi_status launch_expand_tf32(mpi_ctx* ctx, const mpi_basis* b, int mode, const ExpandArgs& x, int group_coils) {
  TfPlan pl;
  const int Cg = group_coils > 0 ? std::min(group_coils, x.C) : x.C;  // coils per launch row
  const int groups = (x.C + Cg - 1) / Cg;
  const int ks = mode == EX_SCATTER_ADD ? x.ksplit : 1;
  if (mode == EX_SCATTER_ADD && (ks < 2 || groups > 1 || x.rows || (b->Kp32 / kKChunk32) % ks))
    return set_err(ctx, MPI_ERR_ARG, "3xTF32 K split: two or more parts of whole boxes, one coil group");
  if (!b->Uf32 || !b->tmap32 || !plan_tf32(b, mode, Cg, &pl, ks))
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "3xTF32 expansion unavailable for this shape");
  if (x.N <= 0 || x.C <= 0) return MPI_OK;
  TcArgs a{};  // every field not set below is zero (no K offset, no split)
  a.N = x.N;
  a.q = x.q;
  a.C = x.C;
  a.KC = b->Kp32 / kKChunk32 / ks;
  a.ksplit = ks;
  a.half = pl.half;
  a.n_gemm = pl.n_gemm;
  a.half_cols = pl.half_cols;
  a.tmem_cols = pl.tmem_cols;
  a.lo_cols = pl.n_gemm;
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
  a.stall_after = ctx->stall_after;
  a.tuck_B = x.tuck_B;
  a.tuck_stride = x.tuck_stride;
  a.sc_L0 = x.sc.L0;
  a.sc_L1 = x.sc.L1;
  a.sc_hi = x.sc.s_hi;
  a.sc_mid = x.sc.s_mid;
  a.sc_col = x.sc.s_col;
  a.sc_im = x.sc.im;
  a.sc_bf16 = x.sc.bf16 ? 1 : 0;
  a.sc_col0 = 0;
  a.group_coils = groups > 1 ? Cg : 0;
  a.C_total = x.C;
  if (groups > 1) a.C = Cg;
  const int n_tiles = (x.N + kTileM - 1) / kTileM;
  // one CTA per SM over all groups (or rows of a grouped launch, or K parts)
  const int nrows = x.rows ? x.nrows : (ks > 1 ? ks : groups);
  if (x.rows) a.group_coils = 0;
  const int per_row = x.rows && x.row_ctas > 0 ? x.row_ctas : std::max(std::max(ctx->num_sms, 1) / nrows, 1);
  const dim3 grid((unsigned)std::min(n_tiles, per_row), (unsigned)nrows);
  const CUtensorMap& map = *(const CUtensorMap*)b->tmap32;
  cudaError_t e = cudaSuccess;
  // an odd K box count occurs only for the chain's operand views (whole-box
  // padding); dense bases are padded to whole two-box stages
  const bool odd = a.KC % 2 != 0;
  if (odd && mode != EX_SCATTER && mode != EX_SCATTER_ADD)
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "3xTF32 expansion: odd K box count in this mode");
#define MPI_TF_LAUNCH(m, o)                                                                                   \
  do {                                                                                                        \
    e = cudaFuncSetAttribute(k_expand_tf32x3<m, o>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem); \
    if (e != cudaSuccess) return cuda_check(ctx, e, "tf32 smem attribute");                                  \
    MPI_PROF(ctx, KF_EXPAND);                                                                                \
    launch_pdl(ctx, k_expand_tf32x3<m, o>, grid, dim3(kThreads32), pl.smem, map, a, pl.stages);            \
  } while (0)
  switch (mode) {
    case EX_MAPS: MPI_TF_LAUNCH(EX_MAPS, false); break;
    case EX_FWD: MPI_TF_LAUNCH(EX_FWD, false); break;
    case EX_JFWD: MPI_TF_LAUNCH(EX_JFWD, false); break;
    case EX_ADJ: MPI_TF_LAUNCH(EX_ADJ, false); break;
    case EX_JADJ: MPI_TF_LAUNCH(EX_JADJ, false); break;
    case EX_SCATTER:
      if (odd) MPI_TF_LAUNCH(EX_SCATTER, true);
      else MPI_TF_LAUNCH(EX_SCATTER, false);
      break;
    case EX_SCATTER_ADD:
      if (odd) MPI_TF_LAUNCH(EX_SCATTER_ADD, true);
      else MPI_TF_LAUNCH(EX_SCATTER_ADD, false);
      break;
    default:
      return set_err(ctx, MPI_ERR_ARG, "unknown expansion mode");
  }
#undef MPI_TF_LAUNCH
  MPI_LAUNCH_CHECK(ctx, x.kname ? x.kname : "k_expand_tf32x3");
  return MPI_OK;
}
