// Radial F_s: Kaiser-Bessel gridding NUFFT of the non-uniform DFT
//   y_m = N^{-1/2} sum_j v_j exp(-i k_m . (j - n/2)),  k in rad/pixel,
// the operator the paper takes as given for non-Cartesian data (Results,
// "2D synthetic radial sequences").  Steps (forward):
//   1. scale by 1/Phi(t) per axis (deapodisation, t = j - n/2) and 1/n, zero-pad
//      centred into a G x G grid (G = sigma n) with the image-side sign (-1)^g;
//   2. plain FFT along y then x (the k-side sign (-1)^g is applied at read time,
//      so the two signs make the centred DFT of the grid);
//   3. interpolate at kappa = k G / (2 pi) with the separable kernel
//      phi(u) = I0(beta sqrt(1 - (2u/W)^2)) / I0(beta) over the W grid points
//      floor(kappa) - W/2 + 1 ... floor(kappa) + W/2 (periodic).
// The adjoint runs the transposed steps: spread (float2 atomics), inverse FFTs,
// crop with the sign and deapodisation.
// beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8) (Beatty et al. 2005);
// Phi(t) = W sinh(z) / (z I0(beta)), z = sqrt(beta^2 - (pi W t / G)^2).
// Grid positions, start taps and weights are computed once per plan in FP64.
#include <math.h>

#include <algorithm>

#include "mpi_internal.h"
#include "ptx.cuh"

namespace {

// I0(x) by its power series sum_k (x^2/4)^k / (k!)^2 (all terms positive).
__device__ double bessel_i0(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 200; ++k) {
    term *= q / ((double)k * (double)k);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  return sum;
}

__global__ void k_nufft_setup(const float* __restrict__ traj, int M, int G, int W, double beta,
                              double kscale, int32_t* __restrict__ gstart, float* __restrict__ gw) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // (m, axis)
  if (e >= 2 * M) return;
  const double kap = (double)traj[e] * kscale;
  const double fl = floor(kap);
  const long start = (long)fl - W / 2 + 1;  // centred index of the first tap
  long g = (start + G / 2) % G;
  if (g < 0) g += G;
  gstart[e] = (int32_t)g;
  const double i0b = bessel_i0(beta);
  for (int a = 0; a < W; ++a) {
    const double u = kap - (double)(start + a);
    const double r = 1.0 - (2.0 * u / W) * (2.0 * u / W);
    gw[(size_t)e * W + a] = r >= 0.0 ? (float)(bessel_i0(beta * sqrt(r)) / i0b) : 0.f;
  }
}

__global__ void k_nufft_deap(int n, int G, int W, double beta, float* __restrict__ deap) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double t = (double)(j - n / 2);
  const double x = M_PI * W * t / G;
  const double z2 = beta * beta - x * x;
  double phi;
  if (z2 > 0) {
    const double z = sqrt(z2);
    phi = sinh(z) / z;
  } else if (z2 < 0) {
    const double z = sqrt(-z2);
    phi = sin(z) / z;
  } else {
    phi = 1.0;
  }
  phi = W * phi / bessel_i0(beta);
  deap[j] = (float)(1.0 / phi);
}

// grid[c] = 0 outside the centred n x n window; inside,
// v[c][y][x] * deap[y] * deap[x] * (-1)^(gx + gy) / n with (gy, gx) = (o + y, o + x).
__global__ void k_nufft_pad(const float2* __restrict__ v, int C, int n, int G, const float* __restrict__ deap,
                            float2* __restrict__ grid) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t GG = (size_t)G * G;
  if (e >= (size_t)C * GG) return;
  const int c = (int)(e / GG);
  const int g = (int)(e % GG);
  const int gy = g / G, gx = g % G;
  const int o = G / 2 - n / 2;
  const int y = gy - o, x = gx - o;
  float2 out = make_float2(0.f, 0.f);
  if (y >= 0 && y < n && x >= 0 && x < n) {
    const float2 val = v[(size_t)c * n * n + (size_t)y * n + x];
    float s = deap[y] * deap[x] / (float)n;
    if ((gx + gy) & 1) s = -s;
    out = make_float2(val.x * s, val.y * s);
  }
  grid[e] = out;
}

template <int W>
__global__ void k_nufft_interp(const float2* __restrict__ grid, int C, int G, int M,
                               const int32_t* __restrict__ gstart, const float* __restrict__ gw,
                               float ksign, float2* __restrict__ y) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)C * M) return;
  const int c = (int)(e / M), m = (int)(e % M);
  const int sx = gstart[2 * m], sy = gstart[2 * m + 1];
  float wx[W], wy[W];
#pragma unroll
  for (int a = 0; a < W; ++a) {
    wx[a] = gw[(size_t)(2 * m) * W + a];
    wy[a] = gw[(size_t)(2 * m + 1) * W + a];
  }
  const float2* gc = grid + (size_t)c * G * G;
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int a = 0; a < W; ++a) {
    int gy = sy + a;
    if (gy >= G) gy -= G;
    float2 racc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < W; ++b) {
      int gx = sx + b;
      if (gx >= G) gx -= G;
      const float2 g = gc[(size_t)gy * G + gx];
      const float w = ((gx + gy) & 1) ? -wx[b] : wx[b];
      racc.x = fmaf(w, g.x, racc.x);
      racc.y = fmaf(w, g.y, racc.y);
    }
    acc.x = fmaf(wy[a], racc.x, acc.x);
    acc.y = fmaf(wy[a], racc.y, acc.y);
  }
  y[e] = make_float2(acc.x * ksign, acc.y * ksign);
}

template <int W>
__global__ void k_nufft_spread(const float2* __restrict__ y, int C, int G, int M,
                               const int32_t* __restrict__ gstart, const float* __restrict__ gw,
                               float ksign, float2* __restrict__ grid) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)C * M) return;
  const int c = (int)(e / M), m = (int)(e % M);
  const int sx = gstart[2 * m], sy = gstart[2 * m + 1];
  float wx[W], wy[W];
#pragma unroll
  for (int a = 0; a < W; ++a) {
    wx[a] = gw[(size_t)(2 * m) * W + a];
    wy[a] = gw[(size_t)(2 * m + 1) * W + a];
  }
  const float2 yv = y[e];
  const float2 v = make_float2(yv.x * ksign, yv.y * ksign);
  float2* gc = grid + (size_t)c * G * G;
#pragma unroll
  for (int a = 0; a < W; ++a) {
    int gy = sy + a;
    if (gy >= G) gy -= G;
    const float2 va = make_float2(v.x * wy[a], v.y * wy[a]);
#pragma unroll
    for (int b = 0; b < W; ++b) {
      int gx = sx + b;
      if (gx >= G) gx -= G;
      const float w = ((gx + gy) & 1) ? -wx[b] : wx[b];
      atomicAdd(gc + (size_t)gy * G + gx, make_float2(va.x * w, va.y * w));
    }
  }
}

__global__ void k_nufft_crop(const float2* __restrict__ grid, int C, int n, int G, const float* __restrict__ deap,
                             float2* __restrict__ out) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nn = (size_t)n * n;
  if (e >= (size_t)C * nn) return;
  const int c = (int)(e / nn);
  const int j = (int)(e % nn);
  const int y = j / n, x = j % n;
  const int o = G / 2 - n / 2;
  const int gy = o + y, gx = o + x;
  const float2 g = grid[(size_t)c * G * G + (size_t)gy * G + gx];
  float s = deap[y] * deap[x] / (float)n;
  if ((gx + gy) & 1) s = -s;
  out[e] = make_float2(g.x * s, g.y * s);
}

float axis_sign(int n) { return ((n / 2) & 1) ? -1.f : 1.f; }

unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

mpi_status launch_fft_rows_inplace(mpi_ctx* ctx, float2* data, long n_rows, int L, bool inverse);

mpi_status nufft_plan_init(mpi_ctx* ctx, mpi_plan* plan, const float* traj_host) {
  const int M = plan->M, W = plan->W, G = plan->G, n = plan->nx;
  const double sigma = (double)G / n;
  const double beta = M_PI * sqrt((W / sigma) * (W / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
  cudaError_t e = cudaMalloc(&plan->deap, (size_t)n * sizeof(float));
  if (e != cudaSuccess) return cuda_check(ctx, e, "nufft plan alloc");
  if (M > 0) {
    e = cudaMalloc(&plan->traj, (size_t)M * 2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&plan->gstart, (size_t)M * 2 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&plan->gw, (size_t)M * 2 * W * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpy(plan->traj, traj_host, (size_t)M * 2 * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_check(ctx, e, "nufft plan alloc");
    const double kscale = (double)G / (2.0 * M_PI);
    MPI_PROF(ctx, KF_NUFFT);
    k_nufft_setup<<<blocks_for((size_t)2 * M, 256), 256, 0, ctx->stream>>>(plan->traj, M, G, W, beta, kscale,
                                                                          plan->gstart, plan->gw);
    MPI_LAUNCH_CHECK(ctx, "k_nufft_setup");
  }
  MPI_PROF(ctx, KF_NUFFT);
  k_nufft_deap<<<blocks_for(n, 256), 256, 0, ctx->stream>>>(n, G, W, beta, plan->deap);
  MPI_LAUNCH_CHECK(ctx, "k_nufft_deap");
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "nufft plan setup");
}

mpi_status nufft_forward(mpi_ctx* ctx, const mpi_plan* plan, const float2* v, int C, float2* y, float2* grid) {
  const int n = plan->nx, G = plan->G, M = plan->M;
  const size_t total = (size_t)C * G * G;
  MPI_PROF(ctx, KF_NUFFT);
  launch_pdl(ctx, k_nufft_pad, dim3(blocks_for(total, 256)), dim3(256), 0, v, C, n, G, plan->deap, grid);
  MPI_LAUNCH_CHECK(ctx, "k_nufft_pad");
  mpi_status st = launch_fft_cols(ctx, grid, C, 1, G, G, false);
  if (st) return st;
  st = launch_fft_rows_inplace(ctx, grid, (long)C * G, G, false);
  if (st) return st;
  if (M == 0) return MPI_OK;
  const float ks = axis_sign(G) * axis_sign(G);
  const size_t cm = (size_t)C * M;
  MPI_PROF(ctx, KF_NUFFT);
  switch (plan->W) {
#define MPI_W_CASE(w)                                                                                \
  case w:                                                                                            \
    launch_pdl(ctx, k_nufft_interp<w>, dim3(blocks_for(cm, 256)), dim3(256), 0, grid, C, G, M,          \
               plan->gstart, plan->gw, ks, y);                                                     \
    break;
    MPI_W_CASE(2) MPI_W_CASE(3) MPI_W_CASE(4) MPI_W_CASE(5) MPI_W_CASE(6) MPI_W_CASE(7) MPI_W_CASE(8)
#undef MPI_W_CASE
    default:
      return set_err(ctx, MPI_ERR_ARG, "kernel width");
  }
  MPI_LAUNCH_CHECK(ctx, "k_nufft_interp");
  return MPI_OK;
}

mpi_status nufft_adjoint(mpi_ctx* ctx, const mpi_plan* plan, const float2* y, int C, float2* out, float2* grid) {
  const int n = plan->nx, G = plan->G, M = plan->M;
  const size_t total = (size_t)C * G * G;
  cudaError_t e = cudaMemsetAsync(grid, 0, total * sizeof(float2), ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "grid clear");
  if (M > 0) {
    const float ks = axis_sign(G) * axis_sign(G);
    const size_t cm = (size_t)C * M;
    MPI_PROF(ctx, KF_NUFFT);
  switch (plan->W) {
#define MPI_W_CASE(w)                                                                                \
  case w:                                                                                            \
    launch_pdl(ctx, k_nufft_spread<w>, dim3(blocks_for(cm, 256)), dim3(256), 0, y, C, G, M,             \
               plan->gstart, plan->gw, ks, grid);                                                  \
    break;
      MPI_W_CASE(2) MPI_W_CASE(3) MPI_W_CASE(4) MPI_W_CASE(5) MPI_W_CASE(6) MPI_W_CASE(7) MPI_W_CASE(8)
#undef MPI_W_CASE
      default:
        return set_err(ctx, MPI_ERR_ARG, "kernel width");
    }
    MPI_LAUNCH_CHECK(ctx, "k_nufft_spread");
  }
  mpi_status st = launch_fft_rows_inplace(ctx, grid, (long)C * G, G, true);
  if (st) return st;
  st = launch_fft_cols(ctx, grid, C, 1, G, G, true);
  if (st) return st;
  MPI_PROF(ctx, KF_NUFFT);
  launch_pdl(ctx, k_nufft_crop, dim3(blocks_for((size_t)C * n * n, 256)), dim3(256), 0, grid, C, n, G,
             plan->deap, out);
  MPI_LAUNCH_CHECK(ctx, "k_nufft_crop");
  return MPI_OK;
}
