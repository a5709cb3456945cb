// The x1 mode product of a Tucker-factored basis ("A Compression Scheme for
// Maxwell Basis", the contraction printed under Eq. 19) on the tensor cores,
// fused with the operator steps around it on a 3D Cartesian grid:
//
//   forward  (Eq. 5):  v_c[z][b] = sign(z, b) scale p[z][b] sum_a U1[z][a] T_c[a][b],
//                      then the DFT of v_c along z, written as vhat_c[kz][b];
//   adjoint:           w_c = the inverse DFT along z of wk_c[kz][b] (the per-coil
//                      data after the inverse passes along x and y), then
//                      x[z][b] = sign(z, b) scale sum_c conj(s_c[z][b]) w_c[z][b],
//                      s_c[z][b] = sum_a U1[z][a] T_c[a][b],
//
// with T_c = G alpha_c x3 U3 x2 U2 (the core contraction and the other two mode
// products, made before this kernel) and b = (y, x) the position in a z-plane.
// The coil maps are never stored, and neither pass along z is a separate kernel.
//
// GEMM: the flattened operand rows are the positions (c, b) (K = [Re T | Im T]
// over a), the coefficient rows are U1's rows real-ified as in the dense
// expansion, so accumulator columns 2z, 2z + 1 of row (c, b) hold Re and Im of
// s_c[z][b].  FP32: 3xTF32 (raw tile as hi, lo(T) staged in tensor memory by
// four converter warps, hi and lo coefficient rows as two MMAs into one
// accumulator); BF16: one kind::f16 MMA per K step.
//
// A CTA owns one block of 128 positions and runs through the coils (a 128-row
// tile per coil), so the data that every coil of the block shares stays in
// shared memory: the image block (forward) or the coil-sum accumulator
// (adjoint), [N1][128] complex.  The DFT of length N1 = 8 R along z is done per
// position (one thread) through tensor memory: for each j1 < 8 the R values
// z = j1 + 8 j2 are transformed in registers (R-point DFT), twiddled by
// w_N1^(j1 k2) and written back to the same columns; after a barrier of the
// epilogue warps each k2 < R reads its 8 values (16 consecutive columns) and
// takes the 8-point DFT, giving index k2 + R k1.  The inverse is the forward
// on conjugated data.  The j1 and k2 work is split over the two epilogue warps
// of each lane quarter.  Every mbarrier wait is bounded; an epilogue decision
// that depends on a wait is made uniform over the epilogue warps with a
// reducing barrier.
#include <cuda.h>

#include <algorithm>

#include "mpi_internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"
#include "dft_reg.cuh"

namespace {

using namespace mpi_tc;
using namespace mpi_dft;

constexpr int kTxFwd = 0;  // forward with the DFT along z
constexpr int kTxAdj = 1;  // adjoint, summed over coils
constexpr int kEpi0 = 6;   // first epilogue warp
constexpr int kKp = 64;    // operand K: 2 r1 <= 64
constexpr int kBox32 = kTileM * 128;  // 128 rows x 32 FP32
constexpr size_t kSmemCap = 232448 - 1024;

struct TxArgs {
  int rows;      // C B operand rows
  int B;         // positions per z-plane (n2 n3), a multiple of 128
  int C;         // coils
  int cgroups;   // forward: coil groups per position block (grid.y); coil c goes to group c % cgroups
  int nx, ny;    // the position b = y nx + x, for the centring sign
  int centre;
  float scale;
  const float2* p;   // image [N1][B]
  const float2* w;   // adjoint input [C][N1][B]
  float2* out;       // forward: vhat [C][N1][B]; adjoint: image [N1][B]
  int accumulate;    // forward: add into out instead of storing
  const float2* wk;  // adjoint input: per-coil data along kz [C][N1][B]
  const float2* tw;  // exp(-2 pi i m / N1), m < N1
  int* err;
  long long wait_cycles;  // bounded-wait limit (SM clock cycles)
  int tmem_cols;
  int stages;
  TcArgs coef;       // coefficient builder: C = N1 rows of U1, q = r1, alpha = U1
};

// ------------------------------------------------------------------ helpers

// Two consecutive 32-bit TMEM columns of this warp's lanes (one complex value).
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float2& v) {
  uint32_t a, b;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "r"(taddr));
  v = make_float2(__uint_as_float(a), __uint_as_float(b));
}
__device__ __forceinline__ void tmem_st2(uint32_t taddr, float2 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(__float_as_uint(v.x)),
               "r"(__float_as_uint(v.y))
               : "memory");
}
__device__ __forceinline__ void fence_reg2(float2& v) { asm volatile("" : "+f"(v.x), "+f"(v.y)); }

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

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc) {
  asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;" ::"r"(d), "r"(a), "l"(b), "r"(idesc));
}

// Barrier over the `n` epilogue threads (named barrier 1) that also returns
// whether any of them passed `flag` != 0.
__device__ __forceinline__ bool epi_bar_any(int flag, int n) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"(flag), "r"(n)
      : "memory");
  return out != 0;
}

// Barrier over the two epilogue warps of TMEM lane quarter `qd` (named barrier
// 2 + qd, 64 threads), returning whether either passed `flag` != 0.  Those two
// warps share the quarter's TMEM lanes (the DFT scratch columns) and nothing
// else, so the adjoint synchronises them alone.
__device__ __forceinline__ bool quarter_bar_any(int flag, int qd) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, 64, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"(flag), "r"(2 + qd)
      : "memory");
  return out != 0;
}

// Bring 256 bytes at `p` (256-byte aligned) into L2, asynchronously.
__device__ __forceinline__ void l2_prefetch_256(const void* p) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], 256;" ::"l"(p) : "memory");
}

__device__ __forceinline__ float pos_sign(int z, int b, int nx) {
  return ((z + b % nx + b / nx) & 1) ? -1.f : 1.f;
}

// ------------------------------------------------------------------- kernel

constexpr int kNSub = 2;                  // epilogue warps per lane quarter
constexpr int kNEpi = 4 * kNSub;          // epilogue warps
constexpr int kTxThreads = (kEpi0 + kNEpi) * 32;

template <int PREC, int N1>
struct TxShape {
  static constexpr bool TF = PREC == 0;
  static constexpr int NG = 2 * N1;  // accumulator columns
  static constexpr int STAGE = TF ? 2 * kBox32 : kTileM * 128;
  static constexpr uint32_t B_BYTES = TF ? 2u * NG * kKp * 4 : (uint32_t)NG * kKp * 2;
  static constexpr uint32_t B_PAD = (B_BYTES + 1023) & ~1023u;
  static constexpr uint32_t X_BYTES = (uint32_t)N1 * kTileM * 8;  // [N1][128] complex
};

template <int PREC, int MODE, int N1>
__global__ void __launch_bounds__(kTxThreads, 1) k_tucker_x1(const __grid_constant__ CUtensorMap tmap, TxArgs a) {
  using S = TxShape<PREC, N1>;
  constexpr bool TF = S::TF;
  constexpr int NG = S::NG;
  constexpr int R = N1 / 8;  // the DFT along z is 8 x R
  constexpr int STAGE = S::STAGE;
  extern __shared__ unsigned char smem_raw[];
  // aligned by an offset from the shared array, so that accesses stay shared-memory ones
  unsigned char* smem = smem_raw + ((1024u - (mpi_ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  const int stages = a.stages;
  unsigned char* sB = smem;
  float2* sX = reinterpret_cast<float2*>(smem + S::B_PAD);  // image block or coil-sum accumulator
  unsigned char* sA = smem + S::B_PAD + S::X_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sA + (size_t)stages * STAGE);
  uint64_t* conv = full + stages;
  uint64_t* empty = conv + stages;
  uint64_t* acc_full = empty + stages;  // [2]
  uint64_t* acc_empty = acc_full + 2;   // [2]
  uint64_t* drain = acc_empty + 2;
  uint64_t* bfull = drain + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bfull + 1);
  __shared__ float2 s_tw[N1];  // w_N1^(j1 k2) at [j1 R + k2]
  __shared__ int s_failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the operand and the per-coil data are written by the previous kernels
  mpi_ptx::pdl_wait();
  mpi_ptx::pdl_trigger();
  // forward: double-buffered accumulator; adjoint: one accumulator plus a
  // scratch block for the inverse DFT along z
  constexpr int NACC = MODE == kTxFwd ? 2 : 1;
  if (tid == 0) {
    s_failed = 0;
    for (int s = 0; s < stages; ++s) {
      mpi_ptx::mbar_init(&full[s], 1);
      mpi_ptx::mbar_init(&conv[s], 4);
      mpi_ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mpi_ptx::mbar_init(&acc_full[b], 1);
      // forward: the 4 warps of the buffer's parity release it; adjoint: all
      mpi_ptx::mbar_init(&acc_empty[b], MODE == kTxFwd ? 4 : kNEpi);
    }
    mpi_ptx::mbar_init(drain, 1);
    mpi_ptx::mbar_init(bfull, 4);
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
  const uint32_t tmem_scr = tmem + (uint32_t)NG;           // adjoint: DFT scratch
  const uint32_t tmem_lo = tmem + 2u * NG;                 // lo(T) slots: 64 columns per stage (FP32)
  // this CTA: position block blockIdx.x, coils blockIdx.y, blockIdx.y + gridDim.y, ...
  const int nb = a.B / kTileM;
  const int my_tiles = (int)blockIdx.y < a.C ? (a.C - 1 - (int)blockIdx.y) / (int)gridDim.y + 1 : 0;
  auto tile_row0 = [&](int k) -> int { return ((int)blockIdx.y + k * (int)gridDim.y) * a.B + (int)blockIdx.x * kTileM; };
  (void)nb;

  if (warp == 0 && lane == 0) {
    // ---------------- producer: one stage (the whole K = 64) per tile
    RingPos r;
    int g = 0;
    for (; g < my_tiles; ++g) {
      if (!mpi_ptx::mbar_wait(&empty[r.s], r.ph ^ 1u, a.err, a.wait_cycles)) break;
      unsigned char* dst = sA + (size_t)r.s * STAGE;
      mpi_ptx::mbar_arrive_expect_tx(&full[r.s], STAGE);
      tma_load_2d(dst, &tmap, 0, tile_row0(g), &full[r.s]);
      if (TF) tma_load_2d(dst + kBox32, &tmap, 32, tile_row0(g), &full[r.s]);
      r.next(stages);
    }
    if (g < my_tiles) {
      s_failed = 1;
      for (int h = (g > stages ? g - stages : 0); h < g; ++h)  // fills still in flight (bounded)
        mpi_ptx::mbar_wait(&full[h % stages], (uint32_t)((h / stages) & 1), nullptr, a.wait_cycles);
    }
  } else if (TF && warp >= 2 && warp <= 5) {
    // ---------------- converters: lo(x) of tile row 32 (warp % 4) + lane into TMEM
    const int row = (warp & 3) * 32 + lane;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    RingPos r;
    for (int g = 0; g < my_tiles; ++g) {
      const bool got = mpi_ptx::mbar_wait(&full[r.s], r.ph, a.err, a.wait_cycles);
      if (!__all_sync(0xffffffffu, got)) {
        s_failed = 1;
        break;
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4* x = reinterpret_cast<const float4*>(sA + (size_t)r.s * STAGE + h * kBox32 + row * 128);
        float lo[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 v = x[j ^ (row & 7)];
          lo[4 * j + 0] = tf32_lo(v.x);
          lo[4 * j + 1] = tf32_lo(v.y);
          lo[4 * j + 2] = tf32_lo(v.z);
          lo[4 * j + 3] = tf32_lo(v.w);
        }
        tmem_st32(tmem_lo + lane_base + (uint32_t)(r.s * 64 + 32 * h), lo);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      fence_before();
      __syncwarp();
      if (lane == 0) mpi_ptx::mbar_arrive(&conv[r.s]);
      r.next(stages);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint64_t a0 = sdesc_sw128(mpi_ptx::smem_addr(sA));
    const uint64_t b0 = sdesc_sw128(mpi_ptx::smem_addr(sB));
    RingPos r;
    bool ok = mpi_ptx::mbar_wait(bfull, 0, a.err, a.wait_cycles);
    for (int tc = 0; tc < my_tiles && ok; ++tc) {
      const int buf = NACC == 2 ? (tc & 1) : 0;
      const uint32_t par = NACC == 2 ? (uint32_t)((tc >> 1) & 1) : (uint32_t)(tc & 1);
      const uint32_t tacc = tmem + (uint32_t)(buf * NG);
      if (!mpi_ptx::mbar_wait(&acc_empty[buf], par ^ 1u, a.err, a.wait_cycles)) {
        ok = false;
        break;
      }
      fence_after();
      const int s = r.s;
      if (!mpi_ptx::mbar_wait(&full[s], r.ph, a.err, a.wait_cycles)) {
        ok = false;
        break;
      }
      fence_after();
      const uint64_t ad = a0 + (uint32_t)(s * (STAGE >> 4));
      if (TF) {
        const uint32_t idesc = idesc_tf32(kTileM, NG);
        constexpr uint32_t b_chunk = (uint32_t)(2 * NG * 128) >> 4;  // [hi; lo] rows per 32-element K chunk
        constexpr uint32_t lo_off = (uint32_t)(NG * 128) >> 4;
        constexpr uint32_t box = kBox32 >> 4;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t adk = ad + h * box + 2 * ks, bdk = b0 + h * b_chunk + 2 * ks;
            mma_tf32(tacc, adk, bdk, idesc, (h | ks) != 0);
            mma_tf32(tacc, adk, bdk + lo_off, idesc, 1);
          }
        if (!mpi_ptx::mbar_wait(&conv[s], r.ph, a.err, a.wait_cycles)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t la = tmem_lo + (uint32_t)(s * 64);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            mma_tf32_tmem_a(tacc, la + 32 * h + 8 * ks, b0 + h * b_chunk + 2 * ks, idesc);
      } else {
        const uint32_t idesc = idesc_bf16(kTileM, NG);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) mma_bf16(tacc, ad + 2 * ks, b0 + 2 * ks, idesc, ks != 0);
      }
      mma_commit(&empty[s]);
      mma_commit(&acc_full[buf]);
      r.next(stages);
    }
    mma_commit(drain);
    mpi_ptx::mbar_wait(drain, 0, a.err, a.wait_cycles);
    if (!ok) s_failed = 1;
  } else if (warp >= kEpi0) {
    // ---------------- epilogue: 2 warps per lane quarter (sub 0, 1)
    const int e = warp - kEpi0;
    const int qd = warp & 3, sub = e >> 2;
    const int row = qd * 32 + lane;
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    constexpr int NT = kNEpi * 32;
    const int et = e * 32 + lane;  // 0 .. NT - 1
    const int b = (int)blockIdx.x * kTileM + row;
    if (e < 4) build_coef_smem<TF>(a.coef, sB, kKp, false, et, bfull);
    for (int i = et; i < N1; i += NT) s_tw[i] = a.tw[((i / R) * (i % R)) % N1];
    // forward: this block's image values with the centring sign and the scale;
    // adjoint: a zeroed accumulator ([z][position])
    for (int i = et; i < N1 * kTileM; i += NT) {
      const int z = i / kTileM, pos = i - z * kTileM;
      const int bb = (int)blockIdx.x * kTileM + pos;
      if (MODE == kTxFwd) {
        const float sg = (a.centre ? pos_sign(z, bb, a.nx) : 1.f) * a.scale;
        sX[i] = cscale(a.p[(size_t)z * a.B + bb], sg);
      } else {
        sX[i] = make_float2(0.f, 0.f);
      }
    }
    epi_bar_any(0, NT);
    constexpr int J1_PER = 8 / kNSub, K2_PER = (R + kNSub - 1) / kNSub;
    const int j1_lo = sub * J1_PER, k2_lo = sub * K2_PER, k2_hi = min(R, (sub + 1) * K2_PER);
    bool failed = false;
    // adjoint: the per-coil data of the current j1, loaded one step ahead
    float2 nxt[R];
    if (MODE == kTxAdj && my_tiles > 0) {
      const float2* wk0 = a.wk + (size_t)blockIdx.y * N1 * a.B + b;
#pragma unroll
      for (int j2 = 0; j2 < R; ++j2) nxt[j2] = wk0[(size_t)(j1_lo + 8 * j2) * a.B];
    }
    for (int tc = 0; tc < my_tiles; ++tc) {
      const int c = (int)blockIdx.y + tc * (int)gridDim.y;
      const int buf = NACC == 2 ? (tc & 1) : 0;
      const uint32_t par = NACC == 2 ? (uint32_t)((tc >> 1) & 1) : (uint32_t)(tc & 1);
      const uint32_t tacc = tmem + lane_base + (uint32_t)(buf * NG);
      if (MODE == kTxFwd) {
        // the two warps of a lane quarter take alternate tiles (sub = buffer =
        // tile parity) and each runs the whole DFT of its 32 positions
        if ((tc & 1) != sub) continue;
        if (a.accumulate) {
          // the read-modify-write of the output: bring this warp's block of the
          // tile after next (its next one) into L2 now, and of this one if first
          for (int k = (tc == sub ? tc : tc + 2); k <= tc + 2 && k < my_tiles; k += 2) {
            const int ck = (int)blockIdx.y + k * (int)gridDim.y;
            const float2* blk = a.out + (size_t)ck * N1 * a.B + (size_t)blockIdx.x * kTileM + qd * 32;
            for (int z = lane; z < N1; z += 32) l2_prefetch_256(blk + (size_t)z * a.B);
          }
        }
        const bool got = mpi_ptx::mbar_wait(&acc_full[buf], par, a.err, a.wait_cycles);
        if (!__all_sync(0xffffffffu, got)) {
          failed = true;
          break;
        }
        fence_after();
        float2* o = a.out + (size_t)c * N1 * a.B + b;
        float2 pn[8];
        if (a.accumulate) {
#pragma unroll
          for (int k1 = 0; k1 < 8; ++k1) pn[k1] = o[(size_t)(R * k1) * a.B];
        }
        // stage 1: v = s p (sign and scale folded into the staged image) over
        // z = j1 + 8 j2, R-point DFT, twiddle, in place; two j1 per round
        for (int j1 = 0; j1 < 8; j1 += 2) {
          float2 v[2][R];
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int j2 = 0; j2 < R; ++j2) tmem_ld2(tacc + 2u * (j1 + h + 8 * j2), v[h][j2]);
          tmem_wait_ld();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int j2 = 0; j2 < R; ++j2) {
              fence_reg2(v[h][j2]);
              v[h][j2] = cmulf(v[h][j2], sX[(j1 + h + 8 * j2) * kTileM + row]);
            }
            dft_r<R>(v[h]);
#pragma unroll
            for (int k2 = 1; k2 < R; ++k2) v[h][k2] = cmulf(v[h][k2], s_tw[(j1 + h) * R + k2]);
#pragma unroll
            for (int k2 = 0; k2 < R; ++k2) tmem_st2(tacc + 2u * (j1 + h + 8 * k2), v[h][k2]);
          }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        // stage 2: 8-point DFTs over j1 for each k2; output kz = k2 + R k1.
        // Accumulating, the output values of k2 + 1 are loaded while k2 is
        // transformed (those of k2 = 0 were loaded before stage 1).
        for (int k2 = 0; k2 < R; ++k2) {
          float2 prev[8];
          if (a.accumulate) {
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) prev[k1] = pn[k1];
            if (k2 + 1 < R) {
#pragma unroll
              for (int k1 = 0; k1 < 8; ++k1) pn[k1] = o[(size_t)(k2 + 1 + R * k1) * a.B];
            }
          }
          uint32_t raw[16];
          tmem_ld16_start(tacc + 16u * k2, raw);
          tmem_wait_ld();
          reg_fence16(raw);
          float2 u[8];
#pragma unroll
          for (int j1 = 0; j1 < 8; ++j1)
            u[j1] = make_float2(__uint_as_float(raw[2 * j1]), __uint_as_float(raw[2 * j1 + 1]));
          dft8(u);
          if (a.accumulate) {
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1)
              o[(size_t)(k2 + R * k1) * a.B] = make_float2(prev[k1].x + u[k1].x, prev[k1].y + u[k1].y);
          } else {
#pragma unroll
            for (int k1 = 0; k1 < 8; ++k1) o[(size_t)(k2 + R * k1) * a.B] = u[k1];
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mpi_ptx::mbar_arrive(&acc_empty[buf]);
      } else {
        // stage 1 (no accumulator needed): the inverse DFT along z of wk_c,
        // first half: conjugated inputs kz = j1 + 8 j2, R-point DFT, twiddle,
        // into the scratch columns j1 + 8 k2.  The next j1's loads are issued
        // before the current one is transformed.
        // (The first j1's values were loaded before this tile: by the previous
        // tile's last j1, or before the tile loop for the first tile.)
        const float2* wk = a.wk + (size_t)c * N1 * a.B + b;
        for (int j1 = j1_lo; j1 < j1_lo + J1_PER; ++j1) {
          float2 v[R];
#pragma unroll
          for (int j2 = 0; j2 < R; ++j2) v[j2] = make_float2(nxt[j2].x, -nxt[j2].y);
          if (j1 + 1 < j1_lo + J1_PER) {
#pragma unroll
            for (int j2 = 0; j2 < R; ++j2) nxt[j2] = wk[(size_t)(j1 + 1 + 8 * j2) * a.B];
          } else if (tc + 1 < my_tiles) {
            // the next tile's (coil's) first j1, in flight through this tile's stage 2
            const float2* wn = wk + (size_t)gridDim.y * N1 * a.B;
#pragma unroll
            for (int j2 = 0; j2 < R; ++j2) nxt[j2] = wn[(size_t)(j1_lo + 8 * j2) * a.B];
          }
          dft_r<R>(v);
#pragma unroll
          for (int k2 = 1; k2 < R; ++k2) v[k2] = cmulf(v[k2], s_tw[j1 * R + k2]);
#pragma unroll
          for (int k2 = 0; k2 < R; ++k2) tmem_st2(tmem_scr + lane_base + 2u * (j1 + 8 * k2), v[k2]);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        fence_before();
        const bool got = mpi_ptx::mbar_wait(&acc_full[buf], par, a.err, a.wait_cycles);
        if (quarter_bar_any(!got, qd)) {  // the quarter's scratch is complete (or a wait ran out)
          failed = true;
          break;
        }
        fence_after();
        // stage 2: 8-point DFTs over j1, conjugated back: w_c[z], z = k2 + R k1;
        // then the accumulator's conj(s_c[z]) times w_c[z] into the coil sum
        for (int k2 = k2_lo; k2 < k2_hi; ++k2) {
          uint32_t raw[16];
          float2 sv[8];
          tmem_ld16_start(tmem_scr + lane_base + 16u * k2, raw);
#pragma unroll
          for (int k1 = 0; k1 < 8; ++k1) tmem_ld2(tacc + 2u * (k2 + R * k1), sv[k1]);
          tmem_wait_ld();
          reg_fence16(raw);
          float2 u[8];
#pragma unroll
          for (int j1 = 0; j1 < 8; ++j1)
            u[j1] = make_float2(__uint_as_float(raw[2 * j1]), __uint_as_float(raw[2 * j1 + 1]));
          dft8(u);
#pragma unroll
          for (int k1 = 0; k1 < 8; ++k1) {
            fence_reg2(sv[k1]);
            const float2 wz = make_float2(u[k1].x, -u[k1].y);
            float2& acc = sX[(k2 + R * k1) * kTileM + row];
            acc.x += sv[k1].x * wz.x + sv[k1].y * wz.y;
            acc.y += sv[k1].x * wz.y - sv[k1].y * wz.x;
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mpi_ptx::mbar_arrive(&acc_empty[buf]);
        // the quarter's scratch columns are rewritten by the next tile's first stage
        quarter_bar_any(0, qd);
        fence_after();
      }
    }
    if (failed) s_failed = 1;
    // every epilogue thread arrives here, having finished its tiles or given up
    // (the quarters decide separately), so the image is written only if none failed
    if (MODE == kTxAdj && my_tiles > 0 && !epi_bar_any(failed, NT)) {
      // the coil sum of this position block: the image, with sign and scale
      for (int i = et; i < N1 * kTileM; i += NT) {
        const int z = i / kTileM, pos = i - z * kTileM;
        const int bb = (int)blockIdx.x * kTileM + pos;
        const float sg = (a.centre ? pos_sign(z, bb, a.nx) : 1.f) * a.scale;
        a.out[(size_t)z * a.B + bb] = cscale(sX[i], sg);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

template <int PREC, int N1>
size_t tx_smem(int stages) {
  using S = TxShape<PREC, N1>;
  return 1024 + S::B_PAD + S::X_BYTES + (size_t)stages * S::STAGE + 8 * (3 * stages + 6) + 16;
}

template <int PREC, int MODE, int N1>
mpi_status tx_launch(mpi_ctx* ctx, const CUtensorMap* map, TxArgs& a, dim3 grid) {
  using S = TxShape<PREC, N1>;
  int stages = 4;
  while (stages > 1 && tx_smem<PREC, N1>(stages) > kSmemCap) --stages;
  if (tx_smem<PREC, N1>(stages) > kSmemCap) return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker x1 kernel: shared memory");
  // tensor memory: accumulators (two forward, one adjoint), the adjoint's DFT
  // scratch, the lo(T) slots of the FP32 kernel
  auto cols_for = [&](int st) {
    return (MODE == kTxFwd ? 2 * S::NG : 2 * S::NG) + (PREC == 0 ? 64 * st : 0);
  };
  while (stages > 1 && cols_for(stages) > 512) --stages;
  if (cols_for(stages) > 512) return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker x1 kernel: tensor memory");
  int tcols = 32;
  while (tcols < cols_for(stages)) tcols <<= 1;
  a.tmem_cols = tcols;
  a.stages = stages;
  const size_t smem = tx_smem<PREC, N1>(stages);
  auto kern = k_tucker_x1<PREC, MODE, N1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "Tucker x1 smem attribute");
  MPI_PROF(ctx, KF_EXPAND);
  launch_pdl(ctx, kern, grid, dim3(kTxThreads), smem, *map, a);
  MPI_LAUNCH_CHECK(ctx, MODE == kTxFwd ? (PREC == 0 ? "k_tucker_x1<tf32x3,fwd+dft_z>" : "k_tucker_x1<bf16,fwd+dft_z>")
                                       : (PREC == 0 ? "k_tucker_x1<tf32x3,idft_z+adj>" : "k_tucker_x1<bf16,idft_z+adj>"));
  return MPI_OK;
}

}  // namespace

bool tucker_x1_fused_supported(const mpi_basis* b, const mpi_plan* plan, int C, mpi_precision prec) {
  if (!b->tucker || !plan || plan->kind != MPI_TRAJ_CARTESIAN || plan->ndim != 3) return false;
  if (prec != MPI_PREC_FP32 && prec != MPI_PREC_BF16) return false;
  const int n1 = b->n[0];
  if (!(n1 == 64 || n1 == 96 || (n1 == 128 && prec == MPI_PREC_BF16))) return false;
  if (2 * b->r[0] > kKp) return false;
  const long B = (long)b->n[1] * b->n[2];
  if (B % kTileM || (long)C * B > 0x7fffffffL || C > 65535) return false;
  if (B / kTileM > 0x7fffffffL) return false;
  return plan->nz == b->n[0] && plan->ny == b->n[1] && plan->nx == b->n[2];
}

// x1 product fused with the forward's point-wise step and the DFT along z
// (forward: out = vhat [C][n1][n2 n3]), or with the inverse DFT along z of `wk`
// and the adjoint's coil sum (adjoint: out = image [N]).  `map` is the tensor
// map of the flattened operand [C B][64] (FP32 or BF16, from k_x1_operand).
// `accumulate` (forward): add the result into out.
mpi_status tucker_x1_fused_launch(mpi_ctx* ctx, const mpi_basis* b, const mpi_plan* plan, bool adjoint, int C,
                                  const void* map, const float2* p, const float2* wk, float2* out, float scale,
                                  mpi_precision prec, bool accumulate) {
  TxArgs a;
  a.accumulate = !adjoint && accumulate;
  const long B = (long)b->n[1] * b->n[2];
  a.rows = (int)(C * B);
  a.B = (int)B;
  a.C = C;
  a.nx = plan->nx;
  a.ny = plan->ny;
  a.centre = 1;
  a.scale = scale;
  a.p = p;
  a.w = nullptr;
  a.wk = wk;
  a.out = out;
  a.tw = twiddle_table(ctx, b->n[0]);
  a.err = ctx->dev_err;
  a.wait_cycles = ctx->wait_cycles;
  if (!a.tw) return set_err(ctx, MPI_ERR_SHAPE, "Tucker x1: no twiddle table for n1");
  TcArgs& cf = a.coef;
  cf = TcArgs{};
  cf.C = b->n[0];
  cf.q = b->r[0];
  cf.n_gemm = 2 * b->n[0];
  cf.half = cf.n_gemm;
  cf.alpha = b->F[0];
  // one CTA per 128-position block; the forward splits the coils into groups
  // when there are fewer blocks than SMs (the adjoint's coil sum stays in one CTA)
  const int nb = (int)(B / kTileM);
  int groups = 1;
  if (!adjoint) groups = std::max(1, std::min(C, std::max(ctx->num_sms, 1) / nb));
  a.cgroups = groups;
  const dim3 grid((unsigned)nb, (unsigned)groups);
  const CUtensorMap* m = (const CUtensorMap*)map;
  const bool bf = prec == MPI_PREC_BF16;
#define MPI_TX(P, M, N)                                   \
  if (b->n[0] == N) return tx_launch<P, M, N>(ctx, m, a, grid);
  if (!adjoint && !bf) { MPI_TX(0, kTxFwd, 64) MPI_TX(0, kTxFwd, 96) }
  if (!adjoint && bf) { MPI_TX(1, kTxFwd, 64) MPI_TX(1, kTxFwd, 96) MPI_TX(1, kTxFwd, 128) }
  if (adjoint && !bf) { MPI_TX(0, kTxAdj, 64) MPI_TX(0, kTxAdj, 96) }
  if (adjoint && bf) { MPI_TX(1, kTxAdj, 64) MPI_TX(1, kTxAdj, 96) MPI_TX(1, kTxAdj, 128) }
#undef MPI_TX
  return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker x1: unsupported n1");
}
