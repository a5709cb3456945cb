// Tucker-factored Maxwell basis for 3D volumes ("A Compression Scheme for
// Maxwell Basis", Eqs. 19-21): the basis tensor is G x1 U1 x2 U2 x3 U3 with a
// core G of shape (r1, r2, r3, q) shared by the q columns and factors
// U_k in C^{n_k x r_k}.  A coil map is
//   s_c = (G x4 alpha_c^T) x1 U1 x2 U2 x3 U3,
// computed here as
//   1. the core contraction g_c = G alpha_c, exactly the dense basis expansion
//      with the core as an (r1 r2 r3) x q basis (FP32 FFMA or BF16 tcgen05 kernels);
//   2. three mode products (the contraction printed under Eq. 19), last mode
//      first (x3 U3, then x2 U2, then x1 U1), which keeps the intermediate
//      tensors smallest;
// and the adjoint U^H v runs the conjugate-transposed mode products in the
// reverse order followed by the core's U^H V contraction.  FP32: the whole
// chain, and the Jacobian-adjoint's conjugate chain, on the 3xTF32 tensor-core
// kernel, each product written by its scatter epilogue in the K-major rows the
// next one streams (tucker_chain_tc, tucker_jadj_alpha); the core contraction
// over all coils in one launch with K split in two, its halves adding their
// partial products into the cleared g; the x1 product fused with the operator
// steps around it (tc_tucker.cu).  BF16: the same chain with the core
// contraction on the BF16 kernel and the x1 operand written as BF16 rows.  The
// shapes those kernels do not take, and FP32 where the 3xTF32 kernels are off:
// the x3 and x2 products (and the conjugate ones) as FP32 complex on the CUDA
// cores (k_mode_last, k_mode_b), the x1 product on the
// tensor-core expansion kernels (over all coils a dense expansion whose basis
// rows are the positions (c, y, x) of T2 with K = r1 and whose coefficient rows
// are the rows of U1) or, forward only, on the CUDA cores fused with the
// point-wise step.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "dft_reg.cuh"
#include "mpi_internal.h"
#include "ptx.cuh"

namespace {

__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

constexpr int kPB = 8;   // contracted elements loaded per batch
constexpr int kMaxP = 256;  // longest contracted length of the CUDA-core mode products (factor length or rank)
constexpr int kIB1 = 16; // outputs along i per thread of the CUDA-core x1 forward

// Clears n floats at x (16-byte aligned), after the previous kernel in the
// stream has completed (programmatic launch: the next kernel may start early
// and waits for this one before its first dependent access).
__global__ void k_zero_f32(float* __restrict__ x, size_t n) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const size_t n4 = n / 4, stride = (size_t)gridDim.x * blockDim.x;
  float4* x4 = reinterpret_cast<float4*>(x);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
    x4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (size_t i = 4 * n4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) x[i] = 0.f;
}

// Y[r][i][b] = sum_p X[r][p][b] M(i, p), with M(i, p) = F[i][p] (forward, F is I x P)
// or conj(F[p][i]) (adjoint, F is P x I).  Threads run along b (coalesced);
// each thread keeps kIB outputs along i in registers; M is staged in shared
// memory as [P][kIB] for the CTA's i-block.  The i-block is the fastest grid
// index, so the CTAs that read the same X tile run together and all but the
// first find it in L2.
template <bool ADJ, int kIB, int MAXP>
__global__ void __launch_bounds__(256) k_mode_b(const float2* __restrict__ X, const float2* __restrict__ F, int R,
                                                int P, int I, long B, float2* __restrict__ Y) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  __shared__ float2 sM[(MAXP + kPB) * kIB];  // rows beyond P are zero (the last load batch)
  const int i0 = blockIdx.x * kIB;
  for (int e = P * kIB + threadIdx.x; e < ((P + kPB - 1) / kPB) * kPB * kIB; e += blockDim.x)
    sM[e] = make_float2(0.f, 0.f);
  for (int e = threadIdx.x; e < P * kIB; e += blockDim.x) {
    const int p = e / kIB, ii = e % kIB;
    const int i = i0 + ii;
    float2 m = make_float2(0.f, 0.f);
    if (i < I) {
      if (ADJ) {
        const float2 f = F[(size_t)p * I + i];
        m = make_float2(f.x, -f.y);
      } else {
        m = F[(size_t)i * P + p];
      }
    }
    sM[e] = m;
  }
  __syncthreads();
  const long b = (long)blockIdx.y * blockDim.x + threadIdx.x;
  const int r = blockIdx.z;  // blockDim.x is B rounded to a warp multiple, at most 256
  if (b >= B || r >= R) return;
  float2 acc[kIB];
#pragma unroll
  for (int ii = 0; ii < kIB; ++ii) acc[ii] = make_float2(0.f, 0.f);
  const float2* x = X + (size_t)r * P * B + b;
  for (int p0 = 0; p0 < P; p0 += kPB) {
    float2 xv[kPB];  // the batch's loads are all issued before the first is used
#pragma unroll
    for (int u = 0; u < kPB; ++u) xv[u] = p0 + u < P ? x[(size_t)(p0 + u) * B] : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kPB; ++u) {
      const float4* mp = reinterpret_cast<const float4*>(sM + (p0 + u) * kIB);
#pragma unroll
      for (int i2 = 0; i2 < kIB / 2; ++i2) {
        const float4 m = mp[i2];
        cfma(acc[2 * i2], xv[u], make_float2(m.x, m.y));
        cfma(acc[2 * i2 + 1], xv[u], make_float2(m.z, m.w));
      }
    }
  }
  float2* y = Y + (size_t)r * I * B + b;
#pragma unroll
  for (int ii = 0; ii < kIB; ++ii)
    if (i0 + ii < I) y[(size_t)(i0 + ii) * B] = acc[ii];
}

// Same contraction with B = 1 (last mode): Y[r][i] = sum_p X[r][p] M(i, p).
// A CTA of 256 threads takes 64 rows r and every i: M is staged in shared
// memory as [p][i] (so a warp's lanes read consecutive i), the CTA's X rows as
// [r][p]; each thread accumulates 8 rows (warp-uniform, shared-memory
// broadcasts) x 4 values of i (i = lane + 32 k) in registers.
constexpr int kLastRows = 64;
template <bool ADJ>
__global__ void __launch_bounds__(256) k_mode_last(const float2* __restrict__ X, const float2* __restrict__ F, int R,
                                                   int P, int I, float2* __restrict__ Y) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  extern __shared__ float2 sh[];
  float2* sM = sh;                           // [P][I]
  float2* sX = sh + (size_t)P * I;           // [kLastRows][P]
  const int r0 = blockIdx.x * kLastRows;
  // F is read in its own memory order (coalesced); forward F is [I][P], adjoint [P][I]
  for (int e = threadIdx.x; e < P * I; e += blockDim.x) {
    const float2 f = F[e];
    if (ADJ) {
      sM[e] = make_float2(f.x, -f.y);  // e = p I + i
    } else {
      const int i = e / P, p = e - i * P;
      sM[p * I + i] = f;
    }
  }
  for (int e = threadIdx.x; e < kLastRows * P; e += blockDim.x) {
    const int rr = e / P;
    sX[e] = (r0 + rr < R) ? X[(size_t)r0 * P + e] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;  // rows rg * 8 .. rg * 8 + 7
  for (int i0 = 0; i0 < I; i0 += 128) {
    float2 acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[j][k] = make_float2(0.f, 0.f);
    for (int p = 0; p < P; ++p) {
      float2 m[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + lane + 32 * k;
        m[k] = i < I ? sM[p * I + i] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 x = sX[(rg * 8 + j) * P + p];
#pragma unroll
        for (int k = 0; k < 4; ++k) cfma(acc[j][k], x, m[k]);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = r0 + rg * 8 + j;
      if (r >= R) continue;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + lane + 32 * k;
        if (i < I) Y[(size_t)r * I + i] = acc[j][k];
      }
    }
  }
}

float centre_sign_host(int) { return 1.f; }

__device__ __forceinline__ float centre_sign(long n, int nx, int ny) {
  const int x = (int)(n % nx);
  const long t = n / nx;
  const int y = (int)(t % ny);
  const int z = (int)(t / ny);
  return ((x + y + z) & 1) ? -1.f : 1.f;
}

// Point-wise operator epilogues from materialised maps S (and dS) [C][N].
template <int MODE>
__global__ void k_pointwise(ExpandArgs a, const float2* __restrict__ S, const float2* __restrict__ dS) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  for (long n = (long)blockIdx.x * blockDim.x + threadIdx.x; n < a.N; n += (long)gridDim.x * blockDim.x) {
    const float sg = (a.centre ? centre_sign(n, a.nx, a.ny) : 1.f) * a.scale;
    const float2 pv = a.p[n];
    if (MODE == EX_FWD) {
      for (int c = 0; c < a.C; ++c) {
        const float2 v = cmul(S[(size_t)c * a.N + n], pv);
        a.out[(size_t)c * a.N + n] = make_float2(v.x * sg, v.y * sg);
      }
    } else if (MODE == EX_JFWD) {
      const float2 dpv = a.dp[n];
      for (int c = 0; c < a.C; ++c) {
        const float2 v1 = cmul(S[(size_t)c * a.N + n], dpv);
        const float2 v2 = cmul(dS[(size_t)c * a.N + n], pv);
        a.out[(size_t)c * a.N + n] = make_float2((v1.x + v2.x) * sg, (v1.y + v2.y) * sg);
      }
    } else {
      float2 acc = make_float2(0.f, 0.f);
      for (int c = 0; c < a.C; ++c) {
        const float2 wv = a.w[(size_t)c * a.N + n];
        const float2 t = cmul_conj(S[(size_t)c * a.N + n], wv);
        acc.x += t.x;
        acc.y += t.y;
        if (MODE == EX_JADJ) {
          const float2 v = cmul_conj(pv, wv);
          a.vout[(size_t)c * a.N + n] = make_float2(v.x * sg, v.y * sg);
        }
      }
      a.out[n] = make_float2(acc.x * sg, acc.y * sg);
    }
  }
}

// The x1 mode product fused with the forward operator's point-wise step:
// v_c[n] = sign(n) scale * p[n] * sum_p X[c][p][b] F[i][p], with i the slowest
// image axis and b = (y, x), so that voxel n = i B + b.  Same tiling as
// k_mode_b (threads along b, kIB outputs along i per thread, one coil per
// grid z), so the per-coil maps are never stored.
__global__ void __launch_bounds__(256) k_mode1_fwd(const float2* __restrict__ X, const float2* __restrict__ F, int P,
                                                   int I, long B, ExpandArgs a) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  __shared__ float2 sM[(128 + kPB) * kIB1];  // M(i, p) = F[i][p] of the i-block (P = r1 <= 128); rows beyond P are zero
  const int i0 = blockIdx.x * kIB1;
  for (int e = P * kIB1 + threadIdx.x; e < ((P + kPB - 1) / kPB) * kPB * kIB1; e += blockDim.x)
    sM[e] = make_float2(0.f, 0.f);
  for (int e = threadIdx.x; e < P * kIB1; e += blockDim.x) {
    const int p = e / kIB1, ii = e % kIB1;
    sM[e] = i0 + ii < I ? F[(size_t)(i0 + ii) * P + p] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const long b = (long)blockIdx.y * blockDim.x + threadIdx.x;
  const int c = blockIdx.z;
  if (b >= B || c >= a.C) return;
  // the image values this thread multiplies, loaded before the contraction so
  // that their latency overlaps it
  float2 pv[kIB1];
#pragma unroll
  for (int ii = 0; ii < kIB1; ++ii) pv[ii] = i0 + ii < I ? a.p[(size_t)(i0 + ii) * B + b] : make_float2(0.f, 0.f);
  float2 acc[kIB1];
#pragma unroll
  for (int ii = 0; ii < kIB1; ++ii) acc[ii] = make_float2(0.f, 0.f);
  const float2* x = X + (size_t)c * P * B + b;
  for (int p0 = 0; p0 < P; p0 += kPB) {
    float2 xv[kPB];
#pragma unroll
    for (int u = 0; u < kPB; ++u) xv[u] = p0 + u < P ? x[(size_t)(p0 + u) * B] : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kPB; ++u) {
      const float4* mp = reinterpret_cast<const float4*>(sM + (p0 + u) * kIB1);
#pragma unroll
      for (int i2 = 0; i2 < kIB1 / 2; ++i2) {
        const float4 m = mp[i2];
        cfma(acc[2 * i2], xv[u], make_float2(m.x, m.y));
        cfma(acc[2 * i2 + 1], xv[u], make_float2(m.z, m.w));
      }
    }
  }
  // centring sign (-1)^(x + y + z) with z = i and b = y nx + x
  const int sb = (int)((b % a.nx) + (b / a.nx)) & 1;
#pragma unroll
  for (int ii = 0; ii < kIB1; ++ii) {
    const int i = i0 + ii;
    if (i >= I) continue;
    const size_t n = (size_t)i * B + b;
    const float sg = (a.centre && ((sb + i) & 1) ? -1.f : 1.f) * a.scale;
    const float2 v = cmul(acc[ii], pv[ii]);
    a.out[(size_t)c * a.N + n] = make_float2(v.x * sg, v.y * sg);
  }
}

// The x1 product's operand for the tensor-core expansion kernels: t2
// [C][r1][B] (complex) rewritten as K-major rows op[(c B + b)][k], k < r1 the
// real part of t2[c][k][b], r1 <= k < 2 r1 the imaginary part, zero up to Kp.
// A CTA transposes a 32-position block of one coil through shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_x1_operand(const float2* __restrict__ t2, int r1, long B, int Kp,
                                                    T* __restrict__ op) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  __shared__ float2 tile[128][33];  // [k][position], padded against bank conflicts
  const int c = blockIdx.y;
  const long b0 = (long)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32 threads
  for (int k = ty; k < r1; k += 8)
    tile[k][tx] = b0 + tx < B ? t2[((size_t)c * r1 + k) * B + b0 + tx] : make_float2(0.f, 0.f);
  __syncthreads();
  // each warp writes whole rows: position b0 + j, elements k = lane, lane + 32, ...
  for (int j = ty; j < 32 && b0 + j < B; j += 8) {
    T* row = op + ((size_t)c * B + b0 + j) * Kp;
    for (int k = tx; k < Kp; k += 32) {
      const float v = k < r1 ? tile[k][j].x : (k < 2 * r1 ? tile[k - r1][j].y : 0.f);
      if constexpr (sizeof(T) == 2) row[k] = __float2bfloat16_rn(v);
      else row[k] = v;
    }
  }
}

mpi_status mode_b(mpi_ctx* ctx, bool adj, const float2* X, const float2* F, int R, int P, int I, long B, float2* Y) {
  if (P > kMaxP) return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker mode product: contracted length > 256");
  const int block = (int)std::min<long>(256, (B + 31) / 32 * 32);  // no idle lanes when B = 128
  // 16 outputs along i per thread (32 measured slower: fewer resident warps)
  const int ib = 16;
  const dim3 grid((unsigned)((I + ib - 1) / ib), (unsigned)((B + block - 1) / block), (unsigned)R);
  if (R > 65535 || grid.y > 65535) return set_err(ctx, MPI_ERR_SHAPE, "Tucker mode product grid");
  MPI_PROF(ctx, KF_EXPAND);
  // contracted lengths above 128 (the adjoint products of factors longer than
  // 128) take a kernel with a larger staging buffer
  if (P > 128) {
    if (adj) launch_pdl(ctx, k_mode_b<true, 16, kMaxP>, grid, dim3(block), 0, X, F, R, P, I, B, Y);
    else launch_pdl(ctx, k_mode_b<false, 16, kMaxP>, grid, dim3(block), 0, X, F, R, P, I, B, Y);
  } else {
    if (adj) launch_pdl(ctx, k_mode_b<true, 16, 128>, grid, dim3(block), 0, X, F, R, P, I, B, Y);
    else launch_pdl(ctx, k_mode_b<false, 16, 128>, grid, dim3(block), 0, X, F, R, P, I, B, Y);
  }
  MPI_LAUNCH_CHECK(ctx, "k_mode_b");
  return MPI_OK;
}

mpi_status mode_last(mpi_ctx* ctx, bool adj, const float2* X, const float2* F, int R, int P, int I, float2* Y) {
  const unsigned grid = (unsigned)((R + kLastRows - 1) / kLastRows);
  const size_t smem = ((size_t)P * I + (size_t)kLastRows * P) * sizeof(float2);
  if (smem > 232448 - 1024) return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker last-mode product: factor too large");
  cudaError_t e = adj ? cudaFuncSetAttribute(k_mode_last<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                      : cudaFuncSetAttribute(k_mode_last<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_check(ctx, e, "k_mode_last smem attribute");
  MPI_PROF(ctx, KF_EXPAND);
  if (adj) launch_pdl(ctx, k_mode_last<true>, dim3(grid), dim3(256), smem, X, F, R, P, I, Y);
  else launch_pdl(ctx, k_mode_last<false>, dim3(grid), dim3(256), smem, X, F, R, P, I, Y);
  MPI_LAUNCH_CHECK(ctx, "k_mode_last");
  return MPI_OK;
}

}  // namespace

namespace {
int x1_kp(const mpi_basis* b) { return (2 * b->r[0] + 63) / 64 * 64; }
size_t x1_op_offset(const mpi_basis* b, int C) {  // float2 elements before the x1 operand, 256-byte aligned
  const size_t R = (size_t)b->r[0] * b->r[1] * b->r[2];
  const size_t t1 = (size_t)b->r[0] * b->r[1] * b->n[2];
  const size_t t2 = (size_t)b->r[0] * b->n[1] * b->n[2];
  return ((size_t)C * (R + t1 + t2) + 31) / 32 * 32;
}
}  // namespace

size_t tucker_work_elems(const mpi_basis* b, int C) {
  if (!b->tucker) return 0;
  // core and mode-product intermediates, then the x1 operand (FP32, Kp floats per position)
  return x1_op_offset(b, C) + (size_t)C * b->n[1] * b->n[2] * (x1_kp(b) / 2) + 32;
}

namespace {

// The core contraction and the x3, x2 mode products: t2 [C][r1][n2][n3] in `tmp`
// (after g [C][R] and t1 [C][r1][r2][n3]); returns t2.
mpi_status tucker_t2(mpi_ctx* ctx, const mpi_basis* b, const float2* alpha, int C, float2* tmp, mpi_precision prec,
                     float2** t2_out) {
  const int n2 = b->n[1], n3 = b->n[2];
  const int r1 = b->r[0], r2 = b->r[1], r3 = b->r[2];
  const long R = (long)r1 * r2 * r3;
  float2* g = tmp;                                  // [C][r1][r2][r3]
  float2* t1 = g + (size_t)C * R;                   // [C][r1][r2][n3]
  float2* t2 = t1 + (size_t)C * r1 * r2 * n3;       // [C][r1][n2][n3]
  ExpandArgs a;
  a.U = b->core->U;
  a.N = b->core->N;
  a.q = b->q;
  a.C = C;
  a.alpha = alpha;
  a.out = g;
  a.kname = prec == MPI_PREC_BF16 ? "k_expand_tc<tucker core>" : "k_expand_tf32x3<tucker core>";
  mpi_status st = expand(ctx, b->core, EX_MAPS, a, prec);
  if (st) return st;
  if ((st = mode_last(ctx, false, g, b->F[2], C * r1 * r2, r3, n3, t1))) return st;
  if ((st = mode_b(ctx, false, t1, b->F[1], C * r1, r2, n2, n3, t2))) return st;
  *t2_out = t2;
  return MPI_OK;
}

}  // namespace

namespace {

// A basis view over the flattened x1 operand: N' = C B rows (coil-major), q = r1,
// with the operand in the layout of the tensor-core kernels' own basis copies.
void x1_view(const mpi_basis* b, int C, mpi_precision prec, void* op, void* map, mpi_basis* fb) {
  fb->ctx = b->ctx;
  fb->device = b->device;
  fb->N = C * b->n[1] * b->n[2];
  fb->q = b->r[0];
  if (prec == MPI_PREC_BF16) {
    fb->Ubf = (__nv_bfloat16*)op;
    fb->Kp = x1_kp(b);
    fb->tmap = map;
  } else {
    fb->Uf32 = (float*)op;
    fb->Kp32 = x1_kp(b);
    fb->tmap32 = map;
  }
}

}  // namespace

bool tucker_x1_on_tensor_cores(const mpi_basis* b, int C, mpi_precision prec) {
  if (prec != MPI_PREC_FP32 && prec != MPI_PREC_BF16) return false;
  const long rows = (long)C * b->n[1] * b->n[2];
  if (rows > 0x7fffffffL - 128 || b->n[0] > 128) return false;  // one MMA holds 2 n1 <= 256 coefficient rows
  if (prec == MPI_PREC_BF16) return true;
  mpi_basis fb;  // shape-only view: the 3xTF32 kernel must take the n1 coefficient rows in coil groups
  x1_view(b, C, prec, (void*)256, (void*)256, &fb);
  const bool ok = tf32_group(&fb, EX_MAPS, b->n[0]) > 0;
  fb.Uf32 = nullptr;
  fb.tmap32 = nullptr;
  return ok;
}

namespace {

template <typename T>
T* align256(void* p) {
  return (T*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
}

// A 3xTF32 "basis" over an FP32 operand of `rows` rows of K = 2 q values
// (real parts, then imaginary parts), read as round_up(K, 32) columns (whole
// 32-value boxes; an odd box count ends each tile with a one-box stage).
void operand_view(const mpi_basis* b, void* ptr, void* map, long rows, int q, mpi_basis* v) {
  v->ctx = b->ctx;
  v->device = b->device;
  v->N = (int)rows;
  v->q = q;
  v->Uf32 = (float*)ptr;
  v->Kp32 = (2 * q + 31) / 32 * 32;
  v->tmap32 = map;
}

// Tensor map cache of the chain's operands (re-encoded when the address or
// the row count changes).
// Slots 0-2: the forward chain's operands; 3-5: the conjugate chain's; 6: the
// BF16 x1 operand the chain writes for the BF16 x1 kernel.
constexpr int kChainSlots = 7;
constexpr int kSlotX1Bf16 = 6;
struct ChainMaps {
  CUtensorMap m[kChainSlots];
  const void* ptr[kChainSlots] = {};
  long rows[kChainSlots] = {};
};

bool chain_map(mpi_basis* b, int i, void* ptr, long rows, int K, void** out) {
  if (!b->chain_maps) b->chain_maps = new ChainMaps;
  ChainMaps* cm = (ChainMaps*)b->chain_maps;
  if (cm->ptr[i] != ptr || cm->rows[i] != rows) {
    const bool ok = i == kSlotX1Bf16 ? tc_encode_operand_map_k(&cm->m[i], ptr, rows, K)
                                     : tf32_encode_operand_map_k(&cm->m[i], ptr, rows, K);
    if (!ok) {
      cm->ptr[i] = nullptr;
      return false;
    }
    cm->ptr[i] = ptr;
    cm->rows[i] = rows;
  }
  *out = &cm->m[i];
  return true;
}

}  // namespace

void tucker_chain_release(mpi_basis* b) {
  delete (ChainMaps*)b->chain_maps;
  b->chain_maps = nullptr;
}

// Whether the FP32 mode-product chain runs on the tensor cores: even ranks (the
// operands' rows are whole 16-byte units), 2 r_k <= 128, and factor lengths
// the 3xTF32 kernel takes in coil groups.
bool tucker_chain_on_tensor_cores(const mpi_basis* b, int C) {
  for (int k = 0; k < 3; ++k)
    if (b->r[k] % 2 || 2 * b->r[k] > 128) return false;
  const long rows3 = (long)C * b->r[0] * b->r[1], rows2 = (long)C * b->n[2] * b->r[0];
  if (rows2 > 0x7fffffffL - 128 || (long)C * b->n[1] * b->n[2] > 0x7fffffffL - 128) return false;
  mpi_basis v3, v2;  // shape-only views
  operand_view(b, (void*)256, (void*)256, rows3, b->r[2], &v3);
  operand_view(b, (void*)256, (void*)256, rows2, b->r[1], &v2);
  const bool ok = tf32_group(&v3, EX_SCATTER, b->n[2]) > 0 && tf32_group(&v2, EX_SCATTER, b->n[1]) > 0 &&
                  tf32_group(b->core, EX_SCATTER, C) > 0;
  v3.Uf32 = v2.Uf32 = nullptr;
  v3.tmap32 = v2.tmap32 = nullptr;
  return ok;
}

// BF16 form of the chain: the BF16 core contraction's coefficient rows fit one
// MMA (2 C <= 256), the core has its BF16 copy, and the BF16 x1 operand rows
// (2 r1 values) are whole 16-byte units.
static bool tucker_chain_bf16_ok(const mpi_basis* b, int C) {
  return C <= 128 && b->core && b->core->Ubf && b->core->tmap && (2 * b->r[0]) % 8 == 0;
}

namespace {

// The chain on the tensor cores, every product written by a scatter epilogue
// straight into the real-ified K-major rows the next one streams.  FP32: all
// three products on the 3xTF32 kernel.  BF16: the core contraction on the BF16
// kernel (BF16 core and coefficients, FP32 output rows), x3 and x2 on the
// 3xTF32 kernel, x2 writing the x1 operand as BF16 rows for the BF16 x1 kernel
// (so the only BF16 roundings are those of the BF16 path's core, coefficients,
// x1 operand and U1):
//   g  = G alpha_c            rows (c, a, b) x [Re g(d) | Im g(d)]       (K = 2 r3)
//   t1 = g x3 U3              rows (c, x, a) x [Re t1(b) | Im t1(b)]     (K = 2 r2)
//   op = t1 x2 U2             rows (c, y, x) x [Re t2(a) | Im t2(a)]     (K = 2 r1)
// (a, b, d index the ranks r1, r2, r3; z, y, x the grid n1, n2, n3).  Each
// factor's rows are the coefficient rows of its product.
mpi_status tucker_chain_tc(mpi_ctx* ctx, const mpi_basis* b, const float2* alpha, int C, float2* tmp,
                           mpi_precision prec, void** op_out, void** map_out) {
  const bool bf = prec == MPI_PREC_BF16;
  const int n2 = b->n[1], n3 = b->n[2];
  const int r1 = b->r[0], r2 = b->r[1], r3 = b->r[2];
  const long R = (long)r1 * r2 * r3;
  mpi_basis* mb = const_cast<mpi_basis*>(b);
  float* g = align256<float>(tmp);
  float* t1 = align256<float>(g + (size_t)C * R * 2);
  float* op = align256<float>(tmp + x1_op_offset(b, C));
  const long rows3 = (long)C * r1 * r2, rows2 = (long)C * n3 * r1, rows1 = (long)C * n2 * n3;
  void *m3 = nullptr, *m2 = nullptr, *m1 = nullptr;
  if (!chain_map(mb, 0, g, rows3, 2 * r3, &m3) || !chain_map(mb, 1, t1, rows2, 2 * r2, &m2) ||
      !chain_map(mb, bf ? kSlotX1Bf16 : 2, op, rows1, 2 * r1, &m1))
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker chain tensor maps");
  // the core contraction: rows (a, b, d) of the core, column pairs = coils
  ExpandArgs a;
  a.U = b->core->U;
  a.N = b->core->N;
  a.q = b->q;
  a.C = C;
  a.alpha = alpha;
  a.out = (float2*)g;
  a.sc.L0 = r3;
  a.sc.L1 = 1 << 30;
  a.sc.s_mid = 2L * r3;
  a.sc.s_col = R / r3 * 2L * r3;
  a.sc.im = r3;
  a.kname = bf ? "k_expand_tc<tucker core>" : "k_expand_tf32x3<tucker core>";
  mpi_status st;
  if (!bf && tf32_ksplit_supported(b->core, EX_SCATTER_ADD, C, 2)) {
    // all coils in one launch with K split in two (the real and the imaginary
    // halves of the core rows), so the core streams through the SMs once: each
    // half's CTAs add their partial products into g, cleared just before (both
    // launches programmatic: the expansion streams the core while the clear
    // runs, and its epilogue waits for the clear)
    const size_t n = (size_t)C * R * 2;
    MPI_PROF(ctx, KF_EXPAND);
    launch_pdl(ctx, k_zero_f32, dim3((unsigned)std::max(1, 4 * ctx->num_sms)), dim3(256), 0, g, n);
    MPI_LAUNCH_CHECK(ctx, "k_zero_f32");
    a.ksplit = 2;
    st = launch_expand_tf32(ctx, b->core, EX_SCATTER_ADD, a);
  } else {
    st = expand(ctx, b->core, EX_SCATTER, a, bf ? MPI_PREC_BF16 : MPI_PREC_FP32);
  }
  if (st) return st;
  // x3: rows (c, a, b) with K = d, column pairs = x; out rows (c, x, a)
  // (these kernels stream operands written by the kernel before: plain stream order)
  const bool pdl = ctx->pdl;
  ctx->pdl = false;
  mpi_basis v;
  operand_view(b, g, m3, rows3, r3, &v);
  ExpandArgs a3;
  a3.N = (int)rows3;
  a3.q = r3;
  a3.C = n3;
  a3.alpha = b->F[2];
  a3.out = (float2*)t1;
  a3.sc.L0 = r2;
  a3.sc.L1 = r1;
  a3.sc.s_hi = (long)n3 * r1 * 2 * r2;
  a3.sc.s_mid = 2L * r2;
  a3.sc.s_col = (long)r1 * 2 * r2;
  a3.sc.im = r2;
  a3.kname = "k_expand_tf32x3<tucker x3>";
  st = expand(ctx, &v, EX_SCATTER, a3, MPI_PREC_FP32);
  // x2: rows (c, x, a) with K = b, column pairs = y; out rows (c, y, x)
  if (!st) {
    operand_view(b, t1, m2, rows2, r2, &v);
    ExpandArgs a2;
    a2.N = (int)rows2;
    a2.q = r2;
    a2.C = n2;
    a2.alpha = b->F[1];
    a2.out = (float2*)op;
    a2.sc.L0 = r1;
    a2.sc.L1 = n3;
    a2.sc.s_hi = (long)n2 * n3 * 2 * r1;
    a2.sc.s_mid = 2L * r1;
    a2.sc.s_col = (long)n3 * 2 * r1;
    a2.sc.im = r1;
    a2.sc.bf16 = bf;
    a2.kname = "k_expand_tf32x3<tucker x2>";
    st = expand(ctx, &v, EX_SCATTER, a2, MPI_PREC_FP32);
  }
  ctx->pdl = pdl;
  v.Uf32 = nullptr;
  v.tmap32 = nullptr;
  if (st) return st;
  *op_out = op;
  *map_out = m1;
  return MPI_OK;
}

}  // namespace

// The flattened x1 operand of alpha's coil maps: the core contraction, the x3
// and x2 mode products and the rewrite of T2 [C][r1][n2 n3] as K-major rows
// [(c, b)][Kp] (FP32 or BF16) at a 256-byte aligned place in `tmp`; returns the
// operand and its tensor map (re-encoded only when the workspace, C or the
// precision change).  FP32 with even ranks: the whole chain on the tensor cores
// (tucker_chain_tc), rows of 2 r1 values; BF16 likewise where 2 r1 is a
// multiple of 8 and the coils fit one BF16 core contraction (BF16 rows).
mpi_status tucker_x1_operand(mpi_ctx* ctx, const mpi_basis* b, const float2* alpha, int C, float2* tmp,
                             mpi_precision prec, void** op_out, void** map_out) {
  if ((prec == MPI_PREC_FP32 || (prec == MPI_PREC_BF16 && tucker_chain_bf16_ok(b, C))) &&
      tucker_chain_on_tensor_cores(b, C))
    return tucker_chain_tc(ctx, b, alpha, C, tmp, prec, op_out, map_out);
  float2* t2 = nullptr;
  mpi_status st = tucker_t2(ctx, b, alpha, C, tmp, prec, &t2);
  if (st) return st;
  const long B = (long)b->n[1] * b->n[2];
  const int Kp = x1_kp(b);
  void* op = (void*)(((uintptr_t)(tmp + x1_op_offset(b, C)) + 255) & ~(uintptr_t)255);  // TMA wants 16-byte alignment
  const dim3 grid((unsigned)((B + 31) / 32), (unsigned)C);
  MPI_PROF(ctx, KF_EXPAND);
  if (prec == MPI_PREC_BF16)
    launch_pdl(ctx, k_x1_operand<__nv_bfloat16>, grid, dim3(256), 0, (const float2*)t2, b->r[0], B, Kp,
               (__nv_bfloat16*)op);
  else
    launch_pdl(ctx, k_x1_operand<float>, grid, dim3(256), 0, (const float2*)t2, b->r[0], B, Kp, (float*)op);
  MPI_LAUNCH_CHECK(ctx, "k_x1_operand");
  mpi_basis* mb = const_cast<mpi_basis*>(b);
  if (!mb->op_map) mb->op_map = new CUtensorMap;
  if (mb->op_map_ptr != op || mb->op_map_C != C || mb->op_map_prec != (int)prec) {
    const bool ok = prec == MPI_PREC_BF16 ? tc_encode_operand_map(mb->op_map, op, (long)C * B, Kp)
                                          : tf32_encode_operand_map(mb->op_map, op, (long)C * B, Kp);
    if (!ok) {
      mb->op_map_ptr = nullptr;
      return set_err(ctx, MPI_ERR_UNSUPPORTED, "x1 operand tensor map");
    }
    mb->op_map_ptr = op;
    mb->op_map_C = C;
    mb->op_map_prec = (int)prec;
  }
  *op_out = op;
  *map_out = mb->op_map;
  return MPI_OK;
}

// maps[c] = s_c for all coils (C x N), through the core contraction and the
// three mode products; `tmp` holds tucker_work_elems(b, C) elements.  The x1
// product runs on the tensor-core expansion kernels where it can (per coil it
// is a dense expansion with T2_c^T as the basis and the rows of U1 as the
// coefficients), else on the CUDA cores.
mpi_status tucker_maps(mpi_ctx* ctx, const mpi_basis* b, const float2* alpha, int C, float2* maps, float2* tmp,
                       mpi_precision prec) {
  const long B = (long)b->n[1] * b->n[2];
  if (!tucker_x1_on_tensor_cores(b, C, prec)) {
    float2* t2 = nullptr;
    mpi_status st = tucker_t2(ctx, b, alpha, C, tmp, prec, &t2);
    if (st) return st;
    return mode_b(ctx, false, t2, b->F[0], C, b->r[0], b->n[0], B, maps);
  }
  void* op = nullptr;
  void* map = nullptr;
  mpi_status st = tucker_x1_operand(ctx, b, alpha, C, tmp, prec, &op, &map);
  if (st) return st;
  mpi_basis fb;
  x1_view(b, C, prec, op, map, &fb);
  ExpandArgs a;
  a.N = fb.N;
  a.q = b->r[0];
  a.C = b->n[0];
  a.alpha = b->F[0];  // U1 [n1][r1]: row i is coefficient row i
  a.out = maps;
  a.tuck_B = (int)B;
  a.tuck_stride = (long)b->n[0] * B;
  a.kname = prec == MPI_PREC_BF16 ? "k_expand_tc<tucker x1>" : "k_expand_tf32x3<tucker x1>";
  // The tensor-core kernels start streaming their basis before waiting on the
  // previous kernel; this basis is the operand just written, so launch them in
  // plain stream order.
  const bool pdl = ctx->pdl;
  ctx->pdl = false;
  st = expand(ctx, &fb, EX_MAPS, a, prec);
  ctx->pdl = pdl;
  fb.Ubf = nullptr;  // the view owns nothing
  fb.Uf32 = nullptr;
  fb.tmap = nullptr;
  fb.tmap32 = nullptr;
  return st;
}

bool tucker_fusable(int mode) { return mode == EX_FWD; }

// The forward pass straight from alpha: core contraction, x3, x2, then the x1
// product fused with the point-wise step.
mpi_status tucker_fused(mpi_ctx* ctx, const mpi_basis* b, int mode, const ExpandArgs& a, float2* tmp,
                        mpi_precision prec) {
  if (!tucker_fusable(mode)) return set_err(ctx, MPI_ERR_ARG, "fused Tucker pass: mode");
  float2* t2 = nullptr;
  mpi_status st = tucker_t2(ctx, b, a.alpha, a.C, tmp, prec, &t2);
  if (st) return st;
  const int P = b->r[0], I = b->n[0];
  const long B = (long)b->n[1] * b->n[2];
  if (P > 128) return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker mode product: rank > 128");
  const int block = (int)std::min<long>(256, (B + 31) / 32 * 32);
  const dim3 grid((unsigned)((I + kIB1 - 1) / kIB1), (unsigned)((B + block - 1) / block), (unsigned)a.C);
  if (grid.y > 65535 || a.C > 65535) return set_err(ctx, MPI_ERR_SHAPE, "Tucker mode product grid");
  MPI_PROF(ctx, KF_EXPAND);
  launch_pdl(ctx, k_mode1_fwd, grid, dim3(block), 0, t2, b->F[0], P, I, B, a);
  MPI_LAUNCH_CHECK(ctx, "k_mode1_fwd");
  return MPI_OK;
}

// dalpha[c] = U^H v_c (C x q): conjugate-transposed mode products, then the core's U^H V.
mpi_status tucker_adjoint(mpi_ctx* ctx, const mpi_basis* b, const float2* V, int C, float2* dalpha, float2* tmp,
                          float2* partials, size_t partial_cap, mpi_precision prec) {
  const int n1 = b->n[0], n2 = b->n[1], n3 = b->n[2];
  const int r1 = b->r[0], r2 = b->r[1], r3 = b->r[2];
  const long R = (long)r1 * r2 * r3;
  float2* g = tmp;                             // [C][r1][r2][r3]
  float2* t1 = g + (size_t)C * R;              // [C][r1][r2][n3]
  float2* t2 = t1 + (size_t)C * r1 * r2 * n3;  // [C][r1][n2][n3]
  mpi_status st;
  if ((st = mode_b(ctx, true, V, b->F[0], C, n1, r1, (long)n2 * n3, t2))) return st;
  if ((st = mode_b(ctx, true, t2, b->F[1], C * r1, n2, r2, n3, t1))) return st;
  if ((st = mode_last(ctx, true, t1, b->F[2], C * r1 * r2, n3, r3, g))) return st;
  return uh_v(ctx, b->core, g, C, dalpha, partials, partial_cap, prec);
}

// ------------------------------------------- Jacobian-adjoint on the tensor cores
//
// The coefficient block of the Jacobian-adjoint (the display after Eq. 7),
// dalpha_c = U^H v_c with v_c = conj(p) (.) F^H r_c, through the Tucker factors
// ("A Compression Scheme for Maxwell Basis", Eq. 19 read backwards): the
// conjugate mode products x1^H, x2^H, x3^H on the 3xTF32 kernel, each
// written by its scatter epilogue into the next one's K-major rows, then the
// core's conjugate contraction.  v_c itself is formed from the per-coil data
// after the passes along x and y: the inverse DFT along z and the point-wise
// step, written straight as the x1^H operand.

namespace {

// Fh[k] = U_k^H [r_k][n_k]: the coefficient rows of the conjugate products.
__global__ void k_conj_transpose(const float2* __restrict__ F, int n, int r, float2* __restrict__ Fh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * r) return;
  const int row = i / n, col = i - row * n;  // Fh[row][col] = conj(F[col][row])
  const float2 v = F[(size_t)col * r + row];
  Fh[i] = make_float2(v.x, -v.y);
}

// The x1^H operand: per coil c and 32 consecutive positions b = y n3 + x of a
// z-plane, the inverse DFT along z of wk_c[kz][b] (two steps, N1 = 8 R: DFT8
// over kz = r + R m, twiddle, R-point DFT; output z = k1 + 8 k2, conjugation on
// both sides), then v = conj(p) w sign(z, y, x) scale, stored as row (c, x, y)
// of [Re v(z), z < N1 | Im v(z), z < N1] (FP32).
template <int N1>
__global__ void __launch_bounds__(256) k_jadj_operand(const float2* __restrict__ wk, const float2* __restrict__ p,
                                                      const float2* __restrict__ tw_g, int B, int nx, int ny,
                                                      float scale, float* __restrict__ out) {
  constexpr int R = N1 / 8, P = 32, NT = 256, OS = 2 * N1 + 1;
  constexpr int T_FLOATS = 2 * N1 * P, O_FLOATS = P * OS;
  __shared__ float smf[T_FLOATS > O_FLOATS ? T_FLOATS : O_FLOATS];
  __shared__ float2 tw[N1];
  float2* T = reinterpret_cast<float2*>(smf);  // [N1][P]
  float* O = smf;                              // [P][OS], after the transform
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const int tid = threadIdx.x, c = blockIdx.y, b0 = blockIdx.x * P;
  for (int i = tid; i < N1; i += NT) tw[i] = tw_g[i];
  const float2* src = wk + (size_t)c * N1 * B + b0;
  constexpr int LD = N1 * P / NT;  // loads per thread, all issued before the first is used
  static_assert(N1 * P % NT == 0, "load split");
  float2 ld[LD];
#pragma unroll
  for (int u = 0; u < LD; ++u) {
    const int i = tid + u * NT, kz = i / P, pos = i - kz * P;
    ld[u] = src[(size_t)kz * B + pos];
  }
#pragma unroll
  for (int u = 0; u < LD; ++u) T[tid + u * NT] = make_float2(ld[u].x, -ld[u].y);
  __syncthreads();
  for (int it = tid; it < P * R; it += NT) {
    const int pos = it % P, r = it / P;
    float2 v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = T[(r + R * m) * P + pos];
    mpi_dft::dft8(v);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) v[k1] = mpi_dft::cmulf(v[k1], tw[r * k1]);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) T[(r + R * k1) * P + pos] = v[k1];
  }
  __syncthreads();
  // one item per thread: (pos, k1), P x 8 = NT
  const int pos = tid % P, k1 = tid / P;
  const int b = b0 + pos;
  float2 u[R];
#pragma unroll
  for (int r = 0; r < R; ++r) u[r] = T[(R * k1 + r) * P + pos];
  mpi_dft::dft_r<R>(u);
  float2 pv[R];
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) pv[k2] = p[(size_t)(k1 + 8 * k2) * B + b];
  __syncthreads();  // T is reused as O below
  const int x = b % nx, y = b / nx;
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) {
    const int z = k1 + 8 * k2;
    const float2 w = make_float2(u[k2].x, -u[k2].y);
    const float sg = ((x + y + z) & 1) ? -scale : scale;
    // conj(p) w
    const float re = pv[k2].x * w.x + pv[k2].y * w.y, im = pv[k2].x * w.y - pv[k2].y * w.x;
    O[pos * OS + z] = re * sg;
    O[pos * OS + N1 + z] = im * sg;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  for (int q = warp; q < P; q += NT / 32) {
    const int bq = b0 + q, xq = bq % nx, yq = bq / nx;
    float* dst = out + ((size_t)c * B + (size_t)xq * ny + yq) * (2 * N1);
    for (int i = lane; i < 2 * N1; i += 32) dst[i] = O[q * OS + i];
  }
}

}  // namespace

mpi_status tucker_conj_factors(mpi_ctx* ctx, mpi_basis* b) {
  for (int k = 0; k < 3; ++k) {
    const int n = b->n[k], r = b->r[k];
    cudaError_t e = cudaMalloc(&b->Fh[k], (size_t)n * r * sizeof(float2));
    if (e != cudaSuccess) return cuda_check(ctx, e, "Tucker conjugate factors");
    MPI_PROF(ctx, KF_OTHER);
    k_conj_transpose<<<(n * r + 255) / 256, 256, 0, ctx->stream>>>(b->F[k], n, r, b->Fh[k]);
    MPI_LAUNCH_CHECK(ctx, "k_conj_transpose");
  }
  return MPI_OK;
}

namespace {

mpi_basis conj_view(const mpi_basis* b, int i, void* ptr, long rows, int n, bool* ok) {
  mpi_basis v;
  void* m = nullptr;
  *ok = chain_map(const_cast<mpi_basis*>(b), 3 + i, ptr, rows, 2 * n, &m);
  operand_view(b, ptr, m, rows, n, &v);
  return v;
}

bool conj_chain_shapes(const mpi_basis* b, int C) {
  const int n1 = b->n[0], n2 = b->n[1], n3 = b->n[2], r1 = b->r[0], r2 = b->r[1];
  const long rows1 = (long)C * n2 * n3, rows2 = (long)C * r1 * n3, rows3 = (long)C * r1 * r2;
  if (rows1 > 0x7fffffffL - 128) return false;
  for (int k = 0; k < 3; ++k)
    if (b->n[k] % 2 || b->n[k] > 256) return false;
  mpi_basis v1, v2, v3;  // shape-only views
  operand_view(b, (void*)256, (void*)256, rows1, n1, &v1);
  operand_view(b, (void*)256, (void*)256, rows2, n2, &v2);
  operand_view(b, (void*)256, (void*)256, rows3, n3, &v3);
  return tf32_group(&v1, EX_SCATTER, b->r[0]) > 0 && tf32_group(&v2, EX_SCATTER, b->r[1]) > 0 &&
         tf32_group(&v3, EX_SCATTER, b->r[2]) > 0;
}

}  // namespace

// FP32 and BF16 (the coefficient block then runs on the 3xTF32 kernels too,
// more accurate than BF16 operands and faster than the CUDA-core products).
bool tucker_jadj_tc_supported(const mpi_basis* b, const mpi_plan* plan, int C, mpi_precision prec) {
  if ((prec != MPI_PREC_FP32 && prec != MPI_PREC_BF16) || !b->tucker || !b->Fh[0]) return false;
  if (!tucker_x1_fused_supported(b, plan, C, prec) || !tucker_chain_on_tensor_cores(b, C)) return false;
  if (b->n[0] != 64 && b->n[0] != 96 && b->n[0] != 128) return false;
  const long B = (long)b->n[1] * b->n[2];
  if (B % 32) return false;
  return conj_chain_shapes(b, C);
}

// dalpha_c = U^H (conj(p) (.) w_c), w_c the inverse DFT along z of wk_c [C][n1][B]
// (the per-coil data after the inverse passes along x and y).  `opbuf` holds
// C n1 B complex elements (the x1^H operand); `tmp` the Tucker workspace.
mpi_status tucker_jadj_alpha(mpi_ctx* ctx, const mpi_basis* b, const mpi_plan* plan, const float2* wk,
                             const float2* p, float scale, int C, float2* opbuf, float2* dalpha, float2* tmp,
                             float2* partials, size_t partial_cap) {
  const int n1 = b->n[0], n2 = b->n[1], n3 = b->n[2];
  const int r1 = b->r[0], r2 = b->r[1], r3 = b->r[2];
  const long B = (long)n2 * n3, R = (long)r1 * r2 * r3;
  const float2* tw = twiddle_table(ctx, n1);
  if (!tw) return set_err(ctx, MPI_ERR_SHAPE, "Jacobian-adjoint: no twiddle table for n1");
  float* op1 = (float*)opbuf;                                   // rows (c, x, y), K = 2 n1
  float* op2 = align256<float>(tmp);                            // rows (c, a, x), K = 2 n2
  float* op3 = align256<float>(op2 + (size_t)C * r1 * n3 * n2 * 2);  // rows (c, a, b), K = 2 n3
  float* g = align256<float>(op3 + (size_t)C * r1 * r2 * n3 * 2);    // [C][R] complex
  const dim3 grid((unsigned)(B / 32), (unsigned)C);
  MPI_PROF(ctx, KF_EXPAND);
  if (n1 == 64)
    launch_pdl(ctx, k_jadj_operand<64>, grid, dim3(256), 0, wk, p, tw, (int)B, plan->nx, plan->ny, scale, op1);
  else if (n1 == 96)
    launch_pdl(ctx, k_jadj_operand<96>, grid, dim3(256), 0, wk, p, tw, (int)B, plan->nx, plan->ny, scale, op1);
  else
    launch_pdl(ctx, k_jadj_operand<128>, grid, dim3(256), 0, wk, p, tw, (int)B, plan->nx, plan->ny, scale, op1);
  MPI_LAUNCH_CHECK(ctx, "k_jadj_operand");
  bool ok1, ok2, ok3;
  mpi_basis v1 = conj_view(b, 0, op1, (long)C * B, n1, &ok1);
  mpi_basis v2 = conj_view(b, 1, op2, (long)C * r1 * n3, n2, &ok2);
  mpi_basis v3 = conj_view(b, 2, op3, (long)C * r1 * r2, n3, &ok3);
  mpi_status st = MPI_OK;
  if (!ok1 || !ok2 || !ok3) st = set_err(ctx, MPI_ERR_UNSUPPORTED, "Jacobian-adjoint chain tensor maps");
  // these kernels stream operands written by the kernel before: plain stream order
  const bool pdl = ctx->pdl;
  ctx->pdl = false;
  if (!st) {  // x1^H: rows (c, x, y), K = z, column pairs a; out rows (c, a, x) with K = y
    ExpandArgs a;
    a.N = (int)(C * B);
    a.q = n1;
    a.C = r1;
    a.alpha = b->Fh[0];
    a.out = (float2*)op2;
    a.sc.L0 = n2;
    a.sc.L1 = n3;
    a.sc.s_hi = (long)r1 * n3 * 2 * n2;
    a.sc.s_mid = 2L * n2;
    a.sc.s_col = (long)n3 * 2 * n2;
    a.sc.im = n2;
    a.kname = "k_expand_tf32x3<tucker x1h>";
    st = expand(ctx, &v1, EX_SCATTER, a, MPI_PREC_FP32);
  }
  if (!st) {  // x2^H: rows (c, a, x), K = y, column pairs b; out rows (c, a, b) with K = x
    ExpandArgs a;
    a.N = (int)((long)C * r1 * n3);
    a.q = n2;
    a.C = r2;
    a.alpha = b->Fh[1];
    a.out = (float2*)op3;
    a.sc.L0 = n3;
    a.sc.L1 = r1;
    a.sc.s_hi = (long)r1 * r2 * 2 * n3;
    a.sc.s_mid = (long)r2 * 2 * n3;
    a.sc.s_col = 2L * n3;
    a.sc.im = n3;
    a.kname = "k_expand_tf32x3<tucker x2h>";
    st = expand(ctx, &v2, EX_SCATTER, a, MPI_PREC_FP32);
  }
  if (!st) {  // x3^H: rows (c, a, b), K = x, column pairs d; out g [C][R] complex
    ExpandArgs a;
    a.N = (int)((long)C * r1 * r2);
    a.q = n3;
    a.C = r3;
    a.alpha = b->Fh[2];
    a.out = (float2*)g;
    a.sc.L0 = 1;
    a.sc.L1 = 1 << 30;
    a.sc.s_mid = 2L * r3;
    a.sc.s_col = 2;
    a.sc.im = 1;
    a.kname = "k_expand_tf32x3<tucker x3h>";
    st = expand(ctx, &v3, EX_SCATTER, a, MPI_PREC_FP32);
  }
  ctx->pdl = pdl;
  v1.Uf32 = v2.Uf32 = v3.Uf32 = nullptr;  // views own nothing
  v1.tmap32 = v2.tmap32 = v3.tmap32 = nullptr;
  if (st) return st;
  (void)R;
  return uh_v(ctx, b->core, (const float2*)g, C, dalpha, partials, partial_cap, MPI_PREC_FP32);
}

mpi_status launch_pointwise(mpi_ctx* ctx, int mode, const ExpandArgs& a, const float2* S, const float2* dS) {
  const long blocks = std::min(((long)a.N + 255) / 256, 8L * std::max(ctx->num_sms, 1));
  MPI_PROF(ctx, KF_EXPAND);
  const char* name = "k_pointwise";
  switch (mode) {
    case EX_FWD:
      launch_pdl(ctx, k_pointwise<EX_FWD>, dim3((unsigned)blocks), dim3(256), 0, a, S, dS);
      name = "k_pointwise<fwd>";
      break;
    case EX_JFWD:
      launch_pdl(ctx, k_pointwise<EX_JFWD>, dim3((unsigned)blocks), dim3(256), 0, a, S, dS);
      name = "k_pointwise<jfwd>";
      break;
    case EX_ADJ:
      launch_pdl(ctx, k_pointwise<EX_ADJ>, dim3((unsigned)blocks), dim3(256), 0, a, S, dS);
      name = "k_pointwise<adj>";
      break;
    case EX_JADJ:
      launch_pdl(ctx, k_pointwise<EX_JADJ>, dim3((unsigned)blocks), dim3(256), 0, a, S, dS);
      name = "k_pointwise<jadj>";
      break;
    default: return set_err(ctx, MPI_ERR_ARG, "pointwise mode");
  }
  MPI_LAUNCH_CHECK(ctx, name);
  return MPI_OK;
}

// The HOSVD core of a dense tensor: conjugate-transposed mode products, mode 1
// first (the same products as the adjoint chain above).
mpi_status tucker_project(mpi_ctx* ctx, const float2* T, int q, const int n[3], const int r[3], const float2* F0,
                          const float2* F1, const float2* F2, float2* core, float2* tmp) {
  float2* t2 = tmp;                                           // [q][r1][n2][n3]
  float2* t1 = t2 + (size_t)q * r[0] * n[1] * n[2];           // [q][r1][r2][n3]
  mpi_status st;
  if ((st = mode_b(ctx, true, T, F0, q, n[0], r[0], (long)n[1] * n[2], t2))) return st;
  if ((st = mode_b(ctx, true, t2, F1, q * r[0], n[1], r[1], n[2], t1))) return st;
  return mode_last(ctx, true, t1, F2, q * r[0] * r[1], n[2], r[2], core);
}
