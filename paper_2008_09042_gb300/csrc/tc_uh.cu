// The coefficient block of the Jacobian adjoint on the tensor cores:
// dalpha_c = U^H v_c for every coil c, where v_c = conj(p) (F_s^H r_c) has
// been formed by the image-block pass (the Jacobian-adjoint display after
// Eq. 7).  The Tucker form's adjoint ends with the same contraction against
// its core (Eq. S3).
//
// Real form.  U is stored [q][N] complex, so row k of its FP32 view [q][2N]
// is (Re U[0,k], Im U[0,k], Re U[1,k], Im U[1,k], ...).  With two real
// right-hand sides per coil over the same 2N interleaved values,
//     b_c  = (Re v[0],  Im v[0], Re v[1],  Im v[1], ...)   (v_c as stored)
//     b'_c = (Im v[0], -Re v[0], Im v[1], -Re v[1], ...)   (-i v_c)
// the dot products are <row k, b_c> = Re (U^H v_c)_k and
// <row k, b'_c> = Im (U^H v_c)_k.  So D = U_view [b; b']^T (M = k, N = 2C,
// K = 2N) is the result itself, and the FP32 path reads the basis in place.
//
// The K extent (all pixels) is split over the CTAs: CTA (x, y) takes M block
// y (128 basis indices) and a contiguous range of 32- or 64-pixel stages,
// accumulates them in tensor memory and writes its partial tile; k_uh_reduce
// sums the partial tiles in a fixed order (bit-reproducible).
//
// FP32 (3xTF32): the B stage rows are [b, b', lo(b), lo(b')] (Cp rows each,
// Cp = C rounded up to 8).  One MMA takes the raw U tile (read by kind::tf32
// as hi(U)) against all four blocks, a second takes lo(U) from tensor memory
// against [b, b']; the epilogue adds the hi x lo block to the first.  TMA
// brings U and b; four converter warps write b', the lo parts and lo(U).
// BF16: U comes from a BF16 copy of the same view, b is loaded as FP32 and the
// converter warps write the BF16 rows [b, b']; one MMA per K step.
// Every mbarrier wait is bounded; on a timeout the CTA records the error,
// waits (bounded) for its copies in flight and frees its TMEM.
#include <cuda.h>

#include <algorithm>

#include "mpi_internal.h"
#include "ptx.cuh"
#include "tc_common.cuh"

namespace {

using namespace mpi_tc;

constexpr int kUhThreads = 192;  // warp 0 TMA, warp 1 MMA + TMEM, warps 2-5 converters + epilogue
constexpr int kBoxes = 2;        // A boxes (128 rows x 128 bytes) per ring stage
constexpr int kABox = 128 * 128;
constexpr int kMaxStagesUh = 8;
constexpr int kMaxCp = 64;       // 4 Cp rows form one MMA's N (<= 256)
constexpr size_t kSmemMaxUh = 232448 - 128;

template <bool BF>
struct UhCfg {
  static constexpr int kElems = BF ? 64 : 32;        // A elements per 128-byte row
  static constexpr int kBoxPix = kElems / 2;          // pixels per A box
  static constexpr int kStagePix = kBoxes * kBoxPix;  // pixels per ring stage
  static constexpr int kBRows = BF ? 2 : 4;           // B row blocks of Cp rows
};

struct UhArgs {
  int q, Cp, n_mblk, T, S, stages, lo_base, tmem_cols;
  float* part;  // [S][n_mblk][2 Cp][128]: column-major partial tiles
  int* err;
  long long wait_cycles;
};

__device__ __forceinline__ void mma_tf32_uh(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// D += A B^T with A (128 x 8 TF32) in tensor memory.
__device__ __forceinline__ void mma_tf32_uh_tmem(uint32_t d, uint32_t ta, uint64_t bd, uint32_t idesc) {
  asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;" ::"r"(d), "r"(ta), "l"(bd), "r"(idesc));
}

__device__ __forceinline__ void tmem_st32_uh(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
      "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
      "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}

__device__ __forceinline__ float4 lo4(float4 x) {
  return make_float4(tf32_lo(x.x), tf32_lo(x.y), tf32_lo(x.z), tf32_lo(x.w));
}
// -i (a + i b) = b - i a on each of the two complex values of a 16-byte unit
__device__ __forceinline__ float4 mul_mi4(float4 x) { return make_float4(x.y, -x.x, x.w, -x.z); }

template <bool BF>
__global__ void __launch_bounds__(kUhThreads, 1) k_uh_tc(const __grid_constant__ CUtensorMap umap,
                                                         const __grid_constant__ CUtensorMap vmap, UhArgs a) {
  using Cfg = UhCfg<BF>;
  extern __shared__ unsigned char smem_raw[];
  // aligned by an offset from the shared array, so that accesses stay shared-memory ones
  unsigned char* smem = smem_raw + ((1024u - (mpi_ptx::smem_addr(smem_raw) & 1023u)) & 1023u);
  const int Cp = a.Cp, stages = a.stages;
  const uint32_t a_stage = kBoxes * kABox;
  const uint32_t b_box = (uint32_t)Cfg::kBRows * Cp * 128;
  const uint32_t v_box = BF ? 2u * Cp * 128 : 0u;  // FP32 staging of b (two 32-float boxes per A box)
  const uint32_t stage_bytes = a_stage + kBoxes * (b_box + v_box);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)stages * stage_bytes);
  uint64_t* conv = full + stages;
  uint64_t* empty = conv + stages;
  uint64_t* acc_full = empty + stages;
  uint64_t* drain = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  __shared__ int s_failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  mpi_ptx::pdl_trigger();
  if (tid == 0) {
    s_failed = 0;
    for (int s = 0; s < stages; ++s) {
      mpi_ptx::mbar_init(&full[s], 1);
      mpi_ptx::mbar_init(&conv[s], 4);
      mpi_ptx::mbar_init(&empty[s], 1);
    }
    mpi_ptx::mbar_init(acc_full, 1);
    mpi_ptx::mbar_init(drain, 1);
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
  const int mb = (int)blockIdx.y, split = (int)blockIdx.x;
  // this CTA's stages [g0, g1) along the pixels (g1 > g0: the host keeps S <= T)
  const int g0 = (int)((long long)a.T * split / a.S);
  const int G = (int)((long long)a.T * (split + 1) / a.S) - g0;
  const uint32_t tx = a_stage + kBoxes * (BF ? 2u * Cp * 128 : (uint32_t)Cp * 128);

  if (warp == 0 && lane == 0) {
    // ---------------- producer: U tiles and the stored right-hand sides b
    mpi_ptx::pdl_wait();  // v comes from the previous kernel
    RingPos r;
    int g = 0;
    for (; g < G; ++g) {
      if (!mpi_ptx::mbar_wait(&empty[r.s], r.ph ^ 1u, a.err, a.wait_cycles)) break;
      unsigned char* st = smem + (size_t)r.s * stage_bytes;
      mpi_ptx::mbar_arrive_expect_tx(&full[r.s], tx);
      const int p0 = (g0 + g) * Cfg::kStagePix;
#pragma unroll
      for (int h = 0; h < kBoxes; ++h) {
        const int x = 2 * (p0 + h * Cfg::kBoxPix);  // element index in the interleaved view
        tma_load_2d(st + h * kABox, &umap, x, mb * kTileM, &full[r.s]);
        if (BF) {
          unsigned char* vb = st + a_stage + kBoxes * b_box + h * v_box;
          tma_load_2d(vb, &vmap, x, 0, &full[r.s]);
          tma_load_2d(vb + Cp * 128, &vmap, x + 32, 0, &full[r.s]);
        } else {
          tma_load_2d(st + a_stage + h * b_box, &vmap, x, 0, &full[r.s]);
        }
      }
      r.next(stages);
    }
    if (g < G) {
      s_failed = 1;
      for (int h = (g > stages ? g - stages : 0); h < g; ++h)  // fills still in flight (bounded)
        mpi_ptx::mbar_wait(&full[h % stages], (uint32_t)((h / stages) & 1), nullptr, a.wait_cycles);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc_hi = BF ? idesc_bf16(kTileM, 2 * Cp) : idesc_tf32(kTileM, 4 * Cp);
    const uint32_t idesc_lo = idesc_tf32(kTileM, 2 * Cp);
    const uint64_t d0 = sdesc_sw128(mpi_ptx::smem_addr(smem));
    RingPos r;
    bool ok = true;
    for (int g = 0; g < G; ++g) {
      const int s = r.s;
      if (!mpi_ptx::mbar_wait(&full[s], r.ph, a.err, a.wait_cycles) ||
          !mpi_ptx::mbar_wait(&conv[s], r.ph, a.err, a.wait_cycles)) {
        ok = false;
        break;
      }
      fence_after();
      const uint64_t sd = d0 + (uint32_t)((s * stage_bytes) >> 4);
#pragma unroll
      for (int h = 0; h < kBoxes; ++h) {
        const uint64_t ad = sd + (uint32_t)((h * kABox) >> 4);
        const uint64_t bd = sd + (uint32_t)((a_stage + h * b_box) >> 4);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {  // 4 K steps of 32 bytes per 128-byte row
          const uint32_t acc = (g | h | ks) != 0;
          if (BF) {
            mma_bf16(tmem, ad + 2 * ks, bd + 2 * ks, idesc_hi, acc);
          } else {
            mma_tf32_uh(tmem, ad + 2 * ks, bd + 2 * ks, idesc_hi, acc);
            mma_tf32_uh_tmem(tmem, tmem + (uint32_t)(a.lo_base + s * 64 + 32 * h + 8 * ks), bd + 2 * ks, idesc_lo);
          }
        }
      }
      mma_commit(&empty[s]);  // frees the stage (and its lo(U) slot) once these MMAs have read it
      r.next(stages);
    }
    if (ok) mma_commit(acc_full);
    mma_commit(drain);
    mpi_ptx::mbar_wait(drain, 0, a.err, a.wait_cycles);
    if (!ok) s_failed = 1;
  } else if (warp >= 2) {
    // ---------------- converters, then the epilogue
    mpi_ptx::pdl_wait();
    const int etid = tid - 64;
    const int row = (warp & 3) * 32 + lane;  // this warp's TMEM lanes: 32 (warp % 4) ..
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    RingPos r;
    bool ok = true;
    for (int g = 0; g < G; ++g) {
      const bool got = mpi_ptx::mbar_wait(&full[r.s], r.ph, a.err, a.wait_cycles);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      unsigned char* st = smem + (size_t)r.s * stage_bytes;
      if (!BF) {
        // lo(U) of tile row `row` into the stage's TMEM slot
#pragma unroll
        for (int h = 0; h < kBoxes; ++h) {
          const float4* x = reinterpret_cast<const float4*>(st + h * kABox + row * 128);
          float lo[32];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 v = lo4(x[j ^ (row & 7)]);
            lo[4 * j + 0] = v.x;
            lo[4 * j + 1] = v.y;
            lo[4 * j + 2] = v.z;
            lo[4 * j + 3] = v.w;
          }
          tmem_st32_uh(tmem + lane_base + (uint32_t)(a.lo_base + r.s * 64 + 32 * h), lo);
        }
        // B rows b', lo(b), lo(b'): the same 16-byte unit position as the b unit
        // (row offsets are multiples of 8, so the swizzle pattern repeats)
        for (int u = etid; u < kBoxes * Cp * 8; u += 128) {
          const int h = u / (Cp * 8), rem = u - h * Cp * 8;
          const int rr = rem >> 3, j = rem & 7;
          unsigned char* bb = st + a_stage + h * b_box + rr * 128 + ((j ^ (rr & 7)) << 4);
          const float4 x = *reinterpret_cast<const float4*>(bb);
          const float4 y = mul_mi4(x);
          *reinterpret_cast<float4*>(bb + Cp * 128) = y;
          *reinterpret_cast<float4*>(bb + 2 * Cp * 128) = lo4(x);
          *reinterpret_cast<float4*>(bb + 3 * Cp * 128) = lo4(y);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      } else {
        // BF16 rows [b, b'] from the FP32 staging: BF16 unit j of a row holds
        // pixels 4j .. 4j+3 of the A box, FP32 units 2 (j % 4) and 2 (j % 4) + 1
        // of staging box j / 4
        for (int u = etid; u < kBoxes * Cp * 8; u += 128) {
          const int h = u / (Cp * 8), rem = u - h * Cp * 8;
          const int rr = rem >> 3, j = rem & 7;
          const unsigned char* vb = st + a_stage + kBoxes * b_box + h * v_box + (j >> 2) * Cp * 128 + rr * 128;
          const int u0 = 2 * (j & 3);
          const float4 x0 = *reinterpret_cast<const float4*>(vb + ((u0 ^ (rr & 7)) << 4));
          const float4 x1 = *reinterpret_cast<const float4*>(vb + (((u0 + 1) ^ (rr & 7)) << 4));
          const float4 y0 = mul_mi4(x0), y1 = mul_mi4(x1);
          uint4 pb, pm;
          __nv_bfloat162* b2 = reinterpret_cast<__nv_bfloat162*>(&pb);
          __nv_bfloat162* m2 = reinterpret_cast<__nv_bfloat162*>(&pm);
          b2[0] = __floats2bfloat162_rn(x0.x, x0.y);
          b2[1] = __floats2bfloat162_rn(x0.z, x0.w);
          b2[2] = __floats2bfloat162_rn(x1.x, x1.y);
          b2[3] = __floats2bfloat162_rn(x1.z, x1.w);
          m2[0] = __floats2bfloat162_rn(y0.x, y0.y);
          m2[1] = __floats2bfloat162_rn(y0.z, y0.w);
          m2[2] = __floats2bfloat162_rn(y1.x, y1.y);
          m2[3] = __floats2bfloat162_rn(y1.z, y1.w);
          unsigned char* bb = st + a_stage + h * b_box + rr * 128 + ((j ^ (rr & 7)) << 4);
          *reinterpret_cast<uint4*>(bb) = pb;
          *reinterpret_cast<uint4*>(bb + Cp * 128) = pm;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
      fence_before();
      __syncwarp();
      if (lane == 0) mpi_ptx::mbar_arrive(&conv[r.s]);
      r.next(stages);
    }
    // epilogue: this thread's accumulator row is basis index k = 128 mb + row
    const bool got = ok && mpi_ptx::mbar_wait(acc_full, 0, a.err, a.wait_cycles);
    if (!__all_sync(0xffffffffu, got)) {
      s_failed = 1;
    } else {
      fence_after();
      const int k = mb * kTileM + row;
      // column j of the tile at dst[j * 128]: a warp stores 32 consecutive rows
      float* dst = a.part + ((size_t)split * a.n_mblk + mb) * (size_t)(2 * Cp) * kTileM + row;
      const uint32_t trow = tmem + lane_base;
      for (int c0 = 0; c0 < 2 * Cp; c0 += 16) {
        uint32_t v[16], w[16];
        tmem_ld16_start(trow + (uint32_t)c0, v);
        if (!BF) tmem_ld16_start(trow + (uint32_t)(2 * Cp + c0), w);
        tmem_wait_ld();
        reg_fence16(v);
        if (!BF) reg_fence16(w);
        if (k < a.q) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            dst[(size_t)(c0 + i) * kTileM] = __uint_as_float(v[i]) + (BF ? 0.f : __uint_as_float(w[i]));
        }
      }
    }
    if (!ok) s_failed = 1;
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// dalpha[c][k] = sum over the splits, in a fixed order, of the partial tiles'
// columns c (real part) and Cp + c (imaginary part) at row k.  Block = 32 rows
// (one per lane) x 32 split groups; group g sums splits g, g + 32, ... (coalesced
// 128-byte reads of a column), then group 0 adds the group sums in order.
constexpr int kRedGroups = 32;

__global__ void __launch_bounds__(32 * kRedGroups) k_uh_reduce(const float* __restrict__ part, int S, int n_mblk,
                                                               int Cp, int q, float2* __restrict__ dalpha) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  __shared__ float2 s_sum[kRedGroups][32];
  const int c = blockIdx.y;
  const int k = blockIdx.x * 32 + (threadIdx.x & 31);
  const int grp = threadIdx.x >> 5;
  const int mb = k / kTileM, row = k % kTileM;
  float re = 0.f, im = 0.f;
  if (k < q) {
    const size_t tile = (size_t)2 * Cp * kTileM;
    const float* p = part + (size_t)mb * tile + (size_t)c * kTileM + row;
    const size_t step = (size_t)n_mblk * tile;
#pragma unroll 4
    for (int s = grp; s < S; s += kRedGroups) {
      re += p[(size_t)s * step];
      im += p[(size_t)s * step + (size_t)Cp * kTileM];
    }
  }
  s_sum[grp][threadIdx.x & 31] = make_float2(re, im);
  __syncthreads();
  if (grp == 0 && k < q) {
    float2 t = s_sum[0][threadIdx.x];
#pragma unroll
    for (int g = 1; g < kRedGroups; ++g) {
      t.x += s_sum[g][threadIdx.x].x;
      t.y += s_sum[g][threadIdx.x].y;
    }
    dalpha[(size_t)c * q + k] = t;
  }
}

// BF16 copy of the interleaved view: out[k][2n + t] = (Re, Im)[t] of U[k][n].
__global__ void k_basis_to_bf16_view(const float2* __restrict__ U, size_t total, __nv_bfloat162* __restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const float2 u = U[e];
  out[e] = __floats2bfloat162_rn(u.x, u.y);
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (fn) return fn;
  void* p = nullptr;
  cudaDriverEntryPointQueryResult qr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return nullptr;
  }
  fn = (EncodeFn)p;
  return fn;
}

// 2D row-major tensor [rows][cols] of `esize`-byte elements, 128-byte swizzle,
// box {128 bytes, box_rows}; out-of-range rows and columns read as zeros.
bool encode_rows(CUtensorMap* m, void* ptr, bool bf16, long cols, long rows, int box_rows) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  const int esize = bf16 ? 2 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * esize};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct UhPlan {
  int Cp, stages, lo_base, tmem_cols, n_mblk, T, S;
  size_t smem;
};

bool plan_uh(const mpi_ctx* ctx, bool bf, int N, int q, int Cg, UhPlan* p) {
  p->Cp = (Cg + 7) / 8 * 8;
  if (p->Cp > kMaxCp) return false;
  const int nD = (bf ? 2 : 4) * p->Cp;  // accumulator columns
  const size_t b_box = (size_t)(bf ? 2 : 4) * p->Cp * 128;
  const size_t v_box = bf ? (size_t)2 * p->Cp * 128 : 0;
  const size_t stage = (size_t)kBoxes * kABox + kBoxes * (b_box + v_box);
  const size_t fixed = 1024 + 8 * (3 * kMaxStagesUh + 2) + 16;
  int stages = (int)std::min<size_t>(kMaxStagesUh, (kSmemMaxUh - fixed) / stage);
  p->lo_base = bf ? 0 : (nD + 63) / 64 * 64;
  if (!bf) stages = std::min(stages, (512 - p->lo_base) / 64);  // one 64-column lo(U) slot per stage
  if (stages < 2) return false;
  p->stages = stages;
  const int used = bf ? nD : p->lo_base + 64 * stages;
  int tcols = 32;
  while (tcols < used) tcols <<= 1;
  p->tmem_cols = tcols;
  p->smem = fixed + (size_t)stages * stage;
  p->n_mblk = (q + kTileM - 1) / kTileM;
  const int stage_pix = bf ? UhCfg<true>::kStagePix : UhCfg<false>::kStagePix;
  p->T = (N + stage_pix - 1) / stage_pix;
  p->S = std::max(1, std::min(std::max(ctx->num_sms, 1) / p->n_mblk, p->T));
  return true;
}

}  // namespace

mpi_status uh_tc_prepare(mpi_ctx* ctx, mpi_basis* b) {
  if (b->N % 4) return MPI_OK;  // the views need 16-byte row strides
  CUtensorMap* m = new CUtensorMap;
  if (!encode_rows(m, b->U, false, 2L * b->N, b->q, kTileM)) {
    delete m;
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "tensor map of the basis view");
  }
  b->umap32 = m;
  if (!b->Ubf) return MPI_OK;  // the BF16 path is off for this basis
  const size_t total = (size_t)b->N * b->q;
  cudaError_t e = cudaMalloc(&b->Uview_bf, total * sizeof(__nv_bfloat162));
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->Uview_bf = nullptr;
    return set_err(ctx, MPI_ERR_OOM, "BF16 basis view");
  }
  MPI_PROF(ctx, KF_OTHER);
  k_basis_to_bf16_view<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(
      b->U, total, reinterpret_cast<__nv_bfloat162*>(b->Uview_bf));
  MPI_LAUNCH_CHECK(ctx, "k_basis_to_bf16_view");
  CUtensorMap* mb = new CUtensorMap;
  if (!encode_rows(mb, b->Uview_bf, true, 2L * b->N, b->q, kTileM)) {
    delete mb;
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "tensor map of the BF16 basis view");
  }
  b->umap_bf = mb;
  return MPI_OK;
}

void uh_tc_release(mpi_basis* b) {
  delete (CUtensorMap*)b->umap32;
  delete (CUtensorMap*)b->umap_bf;
  b->umap32 = b->umap_bf = nullptr;
  if (b->Uview_bf) cudaFree(b->Uview_bf);
  b->Uview_bf = nullptr;
}

bool uh_tc_supported(const mpi_basis* b, mpi_precision prec) {
  if (prec == MPI_PREC_FP32) return b->umap32 != nullptr && b->ctx && b->ctx->tf32x3;  // 3xTF32 split
  if (prec == MPI_PREC_BF16) return b->umap_bf != nullptr;
  return false;
}

size_t uh_tc_partial_elems(const mpi_ctx* ctx, int N, int q, int C) {
  // float2 elements: the largest split count times the partial tile (per coil group of <= 64)
  const int Cp = (std::min(C, kMaxCp) + 7) / 8 * 8;
  const int n_mblk = (q + kTileM - 1) / kTileM;
  (void)N;
  return (size_t)std::max(ctx->num_sms, 1) * kTileM * Cp + (size_t)n_mblk * kTileM * Cp;
}

mpi_status launch_uh_tc(mpi_ctx* ctx, const mpi_basis* b, const float2* V, int C, float2* dalpha,
                        float2* partials, size_t partial_cap, mpi_precision prec) {
  if (C <= 0) return MPI_OK;
  const bool bf = prec == MPI_PREC_BF16;
  if (!uh_tc_supported(b, prec)) return set_err(ctx, MPI_ERR_UNSUPPORTED, "tensor-core U^H V unavailable");
  for (int c0 = 0; c0 < C; c0 += kMaxCp) {
    const int Cg = std::min(kMaxCp, C - c0);
    UhPlan pl;
    if (!plan_uh(ctx, bf, b->N, b->q, Cg, &pl)) return set_err(ctx, MPI_ERR_UNSUPPORTED, "U^H V plan");
    // partial tiles (float4 stores): the buffer rounded up to 16 bytes
    float* part = reinterpret_cast<float*>(((uintptr_t)partials + 15) & ~(uintptr_t)15);
    if ((size_t)pl.S * pl.n_mblk * kTileM * pl.Cp + 1 > partial_cap) return set_err(ctx, MPI_ERR_OOM, "U^H V partials");
    CUtensorMap vmap;
    if (!encode_rows(&vmap, const_cast<float2*>(V + (size_t)c0 * b->N), false, 2L * b->N, Cg, pl.Cp))
      return set_err(ctx, MPI_ERR_UNSUPPORTED, "tensor map of the right-hand sides");
    UhArgs a;
    a.q = b->q;
    a.Cp = pl.Cp;
    a.n_mblk = pl.n_mblk;
    a.T = pl.T;
    a.S = pl.S;
    a.stages = pl.stages;
    a.lo_base = pl.lo_base;
    a.tmem_cols = pl.tmem_cols;
    a.part = part;
    a.err = ctx->dev_err;
    a.wait_cycles = ctx->wait_cycles;
    const dim3 grid((unsigned)pl.S, (unsigned)pl.n_mblk);
    const CUtensorMap& um = *(const CUtensorMap*)(bf ? b->umap_bf : b->umap32);
    cudaError_t e;
    if (bf) {
      e = cudaFuncSetAttribute(k_uh_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
      if (e != cudaSuccess) return cuda_check(ctx, e, "uh smem attribute");
      MPI_PROF(ctx, KF_UHV);
      launch_pdl(ctx, k_uh_tc<true>, grid, dim3(kUhThreads), pl.smem, um, vmap, a);
      MPI_LAUNCH_CHECK(ctx, "k_uh_tc<bf16>");
    } else {
      e = cudaFuncSetAttribute(k_uh_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
      if (e != cudaSuccess) return cuda_check(ctx, e, "uh smem attribute");
      MPI_PROF(ctx, KF_UHV);
      launch_pdl(ctx, k_uh_tc<false>, grid, dim3(kUhThreads), pl.smem, um, vmap, a);
      MPI_LAUNCH_CHECK(ctx, "k_uh_tc<tf32x3>");
    }
    MPI_PROF(ctx, KF_UHV);
    launch_pdl(ctx, k_uh_reduce, dim3((unsigned)((b->q + 31) / 32), (unsigned)Cg), dim3(32 * kRedGroups), 0,
               (const float*)part, pl.S, pl.n_mblk, pl.Cp, b->q, dalpha + (size_t)c0 * b->q);
    MPI_LAUNCH_CHECK(ctx, "k_uh_reduce");
  }
  return MPI_OK;
}
