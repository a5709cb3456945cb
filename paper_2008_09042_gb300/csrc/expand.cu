// Basis expansion s_k = U alpha_k (Eq. 5) fused with the point-wise products of
// the operator (Eq. 5 forward, Eq. 7 Jacobian, the Jacobian-adjoint display after
// Eq. 7) and the U^H contraction of the coefficient block.
//
// FP32 CUDA-core path.  U is [q][N] (basis vector contiguous), so one thread per
// pixel reads U[j][n] fully coalesced for every j, while the coefficients of a
// block of coils sit in shared memory and are read as warp-wide broadcasts.
#include <algorithm>

#include "mpi_internal.h"
#include "ptx.cuh"

namespace {

__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// (-1)^(x + y + z) for raster index n of an (nz, ny, nx) grid.
__device__ __forceinline__ float centre_sign(int n, int nx, int ny) {
  int x = n % nx;
  int t = n / nx;
  int y = t % ny;
  int z = t / ny;
  return ((x + y + z) & 1) ? -1.f : 1.f;
}

constexpr int kExpandMaxThreads = 512;
constexpr int kPrefetch = 8;  // basis rows of U kept in flight per thread

// One thread per pixel, grid sized so that every SM gets the same number of
// pixels.  All coils' coefficients sit in shared memory as [q_pad][c_pad]
// (zero padded), read as warp-wide broadcasts, CB coils per pass.  U[j][n] is
// prefetched kPrefetch rows ahead into registers so that each thread keeps
// that many independent loads in flight while it does the FFMAs of the
// previous rows.  Forward-type modes (MAPS, FWD, JFWD) split coil blocks over
// blockIdx.y (the CTAs of one pixel range run together, so the second read of
// U hits L2); adjoint-type modes (ADJ, JADJ) loop over all coil blocks to sum
// over coils.
template <int MODE, int CB>
__global__ void __launch_bounds__(kExpandMaxThreads) k_expand(ExpandArgs a, int q_pad, int c_pad) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  extern __shared__ float4 smem4[];
  float2* sA = reinterpret_cast<float2*>(smem4);  // [q_pad][c_pad]
  float2* sD = sA + (size_t)q_pad * c_pad;         // [q_pad][c_pad], Jacobian only
  const int tid = threadIdx.x;
  constexpr bool kAdjLike = (MODE == EX_ADJ || MODE == EX_JADJ);
  for (int e = tid; e < q_pad * c_pad; e += blockDim.x) {
    const int j = e / c_pad, c = e % c_pad;
    const bool ok = c < a.C && j < a.q;
    sA[e] = ok ? a.alpha[(size_t)c * a.q + j] : make_float2(0.f, 0.f);
    if (MODE == EX_JFWD) sD[e] = ok ? a.dalpha[(size_t)c * a.q + j] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int cb_begin = kAdjLike ? 0 : blockIdx.y * CB;
  const int cb_end = kAdjLike ? a.C : min(a.C, cb_begin + CB);

  for (int n = blockIdx.x * blockDim.x + tid; n < a.N; n += gridDim.x * blockDim.x) {
    const float sg = (a.centre ? centre_sign(n, a.nx, a.ny) : 1.f) * a.scale;
    const float2 pimg = (MODE != EX_MAPS) ? a.p[n] : make_float2(0.f, 0.f);
    float2 pacc = make_float2(0.f, 0.f);
    const float2* Up = a.U + n;
    for (int c0 = cb_begin; c0 < cb_end; c0 += CB) {
      float2 acc[CB];
      float2 dacc[MODE == EX_JFWD ? CB : 1];
#pragma unroll
      for (int c = 0; c < CB; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < (MODE == EX_JFWD ? CB : 1); ++c) dacc[c] = make_float2(0.f, 0.f);

      float2 ubuf[kPrefetch];
#pragma unroll
      for (int t = 0; t < kPrefetch; ++t)
        ubuf[t] = t < a.q ? __ldg(Up + (size_t)t * a.N) : make_float2(0.f, 0.f);
      for (int j0 = 0; j0 < q_pad; j0 += kPrefetch) {
        float2 nbuf[kPrefetch];
#pragma unroll
        for (int t = 0; t < kPrefetch; ++t) {
          const int jn = j0 + kPrefetch + t;
          nbuf[t] = jn < a.q ? __ldg(Up + (size_t)jn * a.N) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < kPrefetch; ++t) {
          const float2 u = ubuf[t];
          const float4* ap = reinterpret_cast<const float4*>(sA + (size_t)(j0 + t) * c_pad + c0);
#pragma unroll
          for (int c2 = 0; c2 < CB / 2; ++c2) {
            const float4 av = ap[c2];
            cfma(acc[2 * c2], u, make_float2(av.x, av.y));
            cfma(acc[2 * c2 + 1], u, make_float2(av.z, av.w));
          }
          if (MODE == EX_JFWD) {
            const float4* dpp = reinterpret_cast<const float4*>(sD + (size_t)(j0 + t) * c_pad + c0);
#pragma unroll
            for (int c2 = 0; c2 < CB / 2; ++c2) {
              const float4 dv = dpp[c2];
              cfma(dacc[2 * c2], u, make_float2(dv.x, dv.y));
              cfma(dacc[2 * c2 + 1], u, make_float2(dv.z, dv.w));
            }
          }
        }
#pragma unroll
        for (int t = 0; t < kPrefetch; ++t) ubuf[t] = nbuf[t];
      }

      if (MODE == EX_MAPS) {
#pragma unroll
        for (int c = 0; c < CB; ++c)
          if (c0 + c < a.C) a.out[(size_t)(c0 + c) * a.N + n] = acc[c];
      } else if (MODE == EX_FWD) {
#pragma unroll
        for (int c = 0; c < CB; ++c)
          if (c0 + c < a.C) {
            float2* o = a.out + (size_t)(c0 + c) * a.N + n;
            float2 v = cscale(cmul(acc[c], pimg), sg);
            if (a.accumulate) {
              v.x += o->x;
              v.y += o->y;
            }
            *o = v;
          }
      } else if (MODE == EX_JFWD) {
        const float2 dpi = a.dp[n];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          if (c0 + c < a.C) {
            float2 v = cmul(acc[c], dpi);
            const float2 t = cmul(dacc[c], pimg);
            v.x += t.x;
            v.y += t.y;
            float2* o = a.out + (size_t)(c0 + c) * a.N + n;
            v = cscale(v, sg);
            if (a.accumulate) {
              v.x += o->x;
              v.y += o->y;
            }
            *o = v;
          }
        }
      } else {  // ADJ / JADJ
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          if (c0 + c < a.C) {
            const float2 wv = a.w[(size_t)(c0 + c) * a.N + n];
            cfma_conj(pacc, acc[c], wv);
            if (MODE == EX_JADJ)
              a.vout[(size_t)(c0 + c) * a.N + n] = cscale(cmul_conj(pimg, wv), sg);
          }
        }
      }
    }
    if (kAdjLike) a.out[n] = cscale(pacc, sg);
  }
}

template <int MODE, int CB>
mpi_status launch_mode(mpi_ctx* ctx, const ExpandArgs& a) {
  const int q_pad = ((a.q + kPrefetch - 1) / kPrefetch) * kPrefetch;
  const int c_pad = ((a.C + CB - 1) / CB) * CB;
  const size_t smem = (size_t)q_pad * c_pad * sizeof(float2) * (MODE == EX_JFWD ? 2 : 1);
  if (smem > 200 * 1024) return set_err(ctx, MPI_ERR_UNSUPPORTED, "coefficient block too large for shared memory");
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_expand<MODE, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_check(ctx, e, "expand smem attribute");
  }
  // every SM gets the same number of pixels: grid = k * SMs CTAs of a warp multiple
  const long sms = std::max(ctx->num_sms, 1);
  const long k = std::max(1L, ((long)a.N + sms * kExpandMaxThreads - 1) / (sms * kExpandMaxThreads));
  const long grid = sms * k;
  const int block = std::max(32, (int)(32 * (((long)a.N + grid * 32 - 1) / (grid * 32))));
  const bool adj_like = (MODE == EX_ADJ || MODE == EX_JADJ);
  const int gy = adj_like ? 1 : (a.C + CB - 1) / CB;
  const long gx = std::min(grid, ((long)a.N + block - 1) / block);
  MPI_PROF(ctx, KF_EXPAND);
  launch_pdl(ctx, k_expand<MODE, CB>, dim3((unsigned)gx, gy), dim3(block), smem, a, q_pad, c_pad);
  MPI_LAUNCH_CHECK(ctx, a.kname ? a.kname : "k_expand");
  return MPI_OK;
}

// ---------------------------------------------------------------- U^H V

constexpr int kUhvThreads = 256;
constexpr int kUhvP = 64;  // pixels per staged chunk

// Split-K over pixels: every CTA walks chunks blockIdx.x, blockIdx.x + gridDim.x,
// ... and keeps its share of the (C x q) outputs in registers.  Thread t owns
// basis index j = t % q and coils [cs*CT, cs*CT + CT) with cs = t / q + cgroup
// offset.  sU rows are padded to P + 1 so that lanes with consecutive j hit
// distinct banks.
template <int CT>
__global__ void __launch_bounds__(kUhvThreads) k_uh_v(const float2* __restrict__ U, int N, int q,
                                                      const float2* __restrict__ V, int C, int c_begin,
                                                      int c_count, float2* __restrict__ partials) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  extern __shared__ float4 smem4[];
  float2* sU = reinterpret_cast<float2*>(smem4);  // [q][P + 1]
  float2* sV = sU + q * (kUhvP + 1);               // [P][c_count_pad]
  const int cpad = ((c_count + CT - 1) / CT) * CT;
  const int tid = threadIdx.x;
  const int groups = kUhvThreads / q;  // >= 1 (q <= 256)
  const int j = tid % q;
  const int cs = tid / q;
  const bool owner = (tid < groups * q);
  float2 acc[CT];
#pragma unroll
  for (int k = 0; k < CT; ++k) acc[k] = make_float2(0.f, 0.f);
  const int n_chunks = (N + kUhvP - 1) / kUhvP;

  for (int ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const int n0 = ch * kUhvP;
    const int cnt = min(kUhvP, N - n0);
    __syncthreads();
    for (int e = tid; e < q * kUhvP; e += kUhvThreads) {
      const int jj = e / kUhvP, i = e % kUhvP;
      sU[jj * (kUhvP + 1) + i] = (i < cnt) ? __ldg(U + (size_t)jj * N + n0 + i) : make_float2(0.f, 0.f);
    }
    for (int e = tid; e < cpad * kUhvP; e += kUhvThreads) {
      const int c = e / kUhvP, i = e % kUhvP;
      sV[i * cpad + c] = (i < cnt && c < c_count) ? __ldg(V + (size_t)(c_begin + c) * N + n0 + i)
                                                  : make_float2(0.f, 0.f);
    }
    __syncthreads();
    if (owner) {
      // this thread's coil slots: cs, cs + groups, ... (CT of them)
      for (int i = 0; i < kUhvP; ++i) {
        const float2 u = sU[j * (kUhvP + 1) + i];
#pragma unroll
        for (int k = 0; k < CT; ++k) {
          const int c = cs + k * groups;
          if (c < cpad) cfma_conj(acc[k], u, sV[i * cpad + c]);
        }
      }
    }
  }
  if (owner) {
#pragma unroll
    for (int k = 0; k < CT; ++k) {
      const int c = cs + k * groups;
      if (c < c_count) partials[((size_t)blockIdx.x * C + c_begin + c) * q + j] = acc[k];
    }
  }
}

__global__ void k_reduce_partials(const float2* __restrict__ partials, int nblk, int CQ,
                                  float2* __restrict__ out) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= CQ) return;
  float2 s = make_float2(0.f, 0.f);
  for (int b = 0; b < nblk; ++b) {
    const float2 v = partials[(size_t)b * CQ + e];
    s.x += v.x;
    s.y += v.y;
  }
  out[e] = s;
}

int uhv_blocks(const mpi_ctx* ctx, int N) {
  const int n_chunks = (N + kUhvP - 1) / kUhvP;
  return std::max(1, std::min(n_chunks, 2 * std::max(ctx->num_sms, 1)));
}

}  // namespace

mpi_status launch_expand(mpi_ctx* ctx, int mode, const ExpandArgs& a) {
  if (a.N <= 0 || a.C <= 0) return MPI_OK;
  switch (mode) {
    case EX_MAPS: return launch_mode<EX_MAPS, 8>(ctx, a);
    case EX_FWD: return launch_mode<EX_FWD, 8>(ctx, a);
    case EX_JFWD: return launch_mode<EX_JFWD, 8>(ctx, a);
    case EX_ADJ: return launch_mode<EX_ADJ, 16>(ctx, a);
    case EX_JADJ: return launch_mode<EX_JADJ, 16>(ctx, a);
    default: return set_err(ctx, MPI_ERR_ARG, "unknown expansion mode");
  }
}

size_t uh_v_partial_elems(const mpi_ctx* ctx, int N, int q, int C) {
  return (size_t)uhv_blocks(ctx, N) * (size_t)C * (size_t)q;
}

mpi_status launch_uh_v(mpi_ctx* ctx, const float2* U, int N, int q, const float2* V, int C,
                       float2* dalpha, float2* partials, size_t partial_cap_elems) {
  if (C <= 0) return MPI_OK;
  if (q > kUhvThreads) return set_err(ctx, MPI_ERR_UNSUPPORTED, "dense basis with q > 256");
  const int nblk = uhv_blocks(ctx, N);
  if ((size_t)nblk * C * q > partial_cap_elems) return set_err(ctx, MPI_ERR_OOM, "U^H V partials");
  const int groups = kUhvThreads / q;
  constexpr int CT = 8;
  const int per_launch = CT * groups;  // coils one launch covers
  for (int c_begin = 0; c_begin < C; c_begin += per_launch) {
    const int c_count = std::min(per_launch, C - c_begin);
    const int cpad = ((c_count + CT - 1) / CT) * CT;
    const size_t smem = ((size_t)q * (kUhvP + 1) + (size_t)kUhvP * cpad) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_uh_v<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_check(ctx, e, "uh_v smem attribute");
    MPI_PROF(ctx, KF_UHV);
  launch_pdl(ctx, k_uh_v<CT>, dim3(nblk), dim3(kUhvThreads), smem, U, N, q, V, C, c_begin, c_count, partials);
    MPI_LAUNCH_CHECK(ctx, "k_uh_v");
  }
  const int CQ = C * q;
  MPI_PROF(ctx, KF_UHV);
  launch_pdl(ctx, k_reduce_partials, dim3((CQ + 255) / 256), dim3(256), 0, partials, nblk, CQ, dalpha);
  MPI_LAUNCH_CHECK(ctx, "k_reduce_partials");
  return MPI_OK;
}
