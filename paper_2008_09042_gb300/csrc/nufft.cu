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
//      floor(kappa) - W/2 + 1 ... floor(kappa) + W/2 (periodic), reading the
//      grid through shared-memory tiles (samples binned by first-tap tile).
// The adjoint runs the transposed steps: spread, inverse FFTs, crop with the
// sign and deapodisation (the zero-padding of step 1 and the crop are folded
// into the FFT pass along y).  Spreading is output-driven: each grid cell sums the
// samples whose W x W footprint covers it, found through a per-plan CSR of the
// samples by first-tap cell, so no cell is written twice and no atomics run.
// beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8) (Beatty et al. 2005);
// Phi(t) = W sinh(z) / (z I0(beta)), z = sqrt(beta^2 - (pi W t / G)^2).
// Grid positions, start taps and weights are computed once per plan in FP64.
#include <math.h>

#include <algorithm>
#include <vector>

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

constexpr int kInterpTile = 32;    // first-tap tile of the shared-memory interpolation
constexpr int kInterpChunk = 256;  // samples per interpolation work item (one per thread)

// Interpolation through shared memory: CTA (item, coil) takes a chunk of at
// most kInterpChunk of the samples whose first tap lies in one 32 x 32 tile
// (the plan's tile-sorted list).  Each thread loads its sample's first tap
// and weights (before waiting on the kernel that writes the grid), the CTA
// copies the grid cells the chunk reads, (32 + W - 1)^2 from the tile's corner
// (periodic), into shared memory with coalesced loads, and each thread forms
// its sample's W x W sum there.
template <int W>
__global__ void __launch_bounds__(kInterpChunk) k_nufft_interp_tiled(const float2* __restrict__ grid, int C, int G,
                                                                     int M, const int32_t* __restrict__ gstart,
                                                                     const float* __restrict__ gw, float ksign,
                                                                     const int32_t* __restrict__ items,
                                                                     const int32_t* __restrict__ samples,
                                                                     float2* __restrict__ y) {
  mpi_ptx::pdl_trigger();
  constexpr int TT = kInterpTile + W - 1;
  __shared__ float2 tile[TT * TT];
  const int it = blockIdx.x, c = blockIdx.y;
  const int t = items[3 * it], s0 = items[3 * it + 1], cnt = items[3 * it + 2];
  const int tpr = (G + kInterpTile - 1) / kInterpTile;
  const int oy = (t / tpr) * kInterpTile, ox = (t % tpr) * kInterpTile;
  const bool active = (int)threadIdx.x < cnt;
  const int m = samples[s0 + (active ? (int)threadIdx.x : 0)];
  const int sx = gstart[2 * m], sy = gstart[2 * m + 1];
  float wx[W], wy[W];
#pragma unroll
  for (int a = 0; a < W; ++a) {
    wx[a] = gw[(size_t)(2 * m) * W + a];
    wy[a] = gw[(size_t)(2 * m + 1) * W + a];
  }
  mpi_ptx::pdl_wait();
  const float2* gc = grid + (size_t)c * G * G;
  for (int e = threadIdx.x; e < TT * TT; e += blockDim.x) {
    const int r = e / TT, q = e % TT;
    tile[e] = gc[(size_t)((oy + r) % G) * G + (ox + q) % G];
  }
  __syncthreads();
  if (!active) return;
  const float2* tp = tile + (sy - oy) * TT + (sx - ox);
  const bool odd = (sx + sy) & 1;  // (-1)^(gx + gy); G is even, so wrapping keeps the parity
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int a = 0; a < W; ++a) {
    float2 racc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const float2 g = tp[a * TT + b];
      const float w = (((a + b) & 1) != odd) ? -wx[b] : wx[b];
      racc.x = fmaf(w, g.x, racc.x);
      racc.y = fmaf(w, g.y, racc.y);
    }
    acc.x = fmaf(wy[a], racc.x, acc.x);
    acc.y = fmaf(wy[a], racc.y, acc.y);
  }
  y[(size_t)c * M + m] = make_float2(acc.x * ksign, acc.y * ksign);
}

constexpr int kSpreadCoils = 4;   // coils a spreading thread accumulates (one group of four)
constexpr int kSpreadDense = 24;  // cells with more samples in their window go to the warp kernel

int spread_coils_padded(int C) { return (C + 3) / 4 * 4; }

// ys[cell_rank[m]][c] = ksign * y[c][m] for c < C, zero for C <= c < Cp (C
// padded to a multiple of four): the samples in first-tap-cell order, the
// coils of one sample contiguous.  Reads follow y's layout; writes scatter.
__global__ void k_nufft_sort_y(const float2* __restrict__ y, int C, int Cp, int M,
                               const int32_t* __restrict__ cell_rank, float ksign, float2* __restrict__ ys) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)Cp * M) return;
  const int c = (int)(e / M), m = (int)(e % M);
  float2 v = make_float2(0.f, 0.f);
  if (c < C) {
    const float2 t = y[e];
    v = make_float2(t.x * ksign, t.y * ksign);
  }
  ys[(size_t)cell_rank[m] * Cp + c] = v;
}

// The samples that reach grid cell (gy, gx) from first-tap row sy = gy - a:
// first taps (sy, gx - b), b = 0 .. W-1, one CSR range [r[0], r[1]) and, when
// the window wraps past column 0 (G >= 2W: once at most), a second [r[2], r[3]).
template <int W>
__device__ __forceinline__ void spread_row_ranges(const int32_t* __restrict__ rp, int gx, int G, int r[4]) {
  const int lo = gx - (W - 1);
  r[1] = rp[gx + 1];
  if (lo >= 0) {
    r[0] = rp[lo];
    r[2] = r[3] = 0;
  } else {
    r[0] = rp[0];
    r[2] = rp[G + lo];
    r[3] = rp[G];
  }
}

// One sample's term: weight phi_x(b) phi_y(a) with b = gx - sx (mod G) read
// from the sample's own first tap, times four coils of ys.
template <int W>
__device__ __forceinline__ void spread_term(const float* __restrict__ cell_w, const int32_t* __restrict__ cell_sx,
                                            const float4* __restrict__ yc, int ystride, int k, int gx, int a,
                                            int G, float acc[8]) {
  int b = gx - cell_sx[k];
  if (b < 0) b += G;
  const float w = cell_w[k * 2 * W + b] * cell_w[k * 2 * W + W + a];
  const float4 u = yc[k * ystride], v = yc[k * ystride + 1];
  acc[0] = fmaf(w, u.x, acc[0]);
  acc[1] = fmaf(w, u.y, acc[1]);
  acc[2] = fmaf(w, u.z, acc[2]);
  acc[3] = fmaf(w, u.w, acc[3]);
  acc[4] = fmaf(w, v.x, acc[4]);
  acc[5] = fmaf(w, v.y, acc[5]);
  acc[6] = fmaf(w, v.z, acc[6]);
  acc[7] = fmaf(w, v.w, acc[7]);
}

__device__ __forceinline__ void spread_store(float2* __restrict__ grid, int C, int G, int c0, int gy, int gx,
                                             const float acc[8]) {
  const float s = ((gx + gy) & 1) ? -1.f : 1.f;  // the k-side sign (-1)^(gx + gy)
#pragma unroll
  for (int j = 0; j < kSpreadCoils; ++j)
    if (c0 + j < C) grid[((size_t)(c0 + j) * G + gy) * G + gx] = make_float2(s * acc[2 * j], s * acc[2 * j + 1]);
}

// Output-driven spreading, sparse cells: thread (gy, gx, coil group) sums the
// samples whose W x W footprint covers its cell, i.e. whose first tap is
// (gy - a, gx - b) (mod G) for 0 <= a, b < W, and stores the cell once; no
// atomics.  A cell whose window holds more than kSpreadDense samples is left
// to k_nufft_spread_dense (its thread would hold the CTA up).
template <int W>
__global__ void __launch_bounds__(256, 4) k_nufft_spread(const float4* __restrict__ ys, int C, int Cp, int G,
                                                         const int32_t* __restrict__ cell_ptr,
                                                         const int32_t* __restrict__ cell_sx,
                                                         const float* __restrict__ cell_w,
                                                         float2* __restrict__ grid) {
  mpi_ptx::pdl_trigger();
  const int gx = blockIdx.x * 32 + threadIdx.x, gy = blockIdx.y * 8 + threadIdx.y;
  const int c0 = blockIdx.z * kSpreadCoils;
  mpi_ptx::pdl_wait();
  if (gx >= G || gy >= G) return;
  int n = 0;
#pragma unroll
  for (int a = 0; a < W; ++a) {
    int sy = gy - a;
    if (sy < 0) sy += G;
    int r[4];
    spread_row_ranges<W>(cell_ptr + sy * G, gx, G, r);
    n += r[1] - r[0] + r[3] - r[2];
  }
  if (n > kSpreadDense) return;
  const int ystride = Cp / 2;
  const float4* yc = ys + c0 / 2;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (n > 0) {
    for (int a = 0; a < W; ++a) {  // the ranges again (L1 hits), rather than W x 4 live registers
      int sy = gy - a;
      if (sy < 0) sy += G;
      int r[4];
      spread_row_ranges<W>(cell_ptr + sy * G, gx, G, r);
      for (int k = r[0]; k < r[1]; ++k) spread_term<W>(cell_w, cell_sx, yc, ystride, k, gx, a, G, acc);
      for (int k = r[2]; k < r[3]; ++k) spread_term<W>(cell_w, cell_sx, yc, ystride, k, gx, a, G, acc);
    }
  }
  spread_store(grid, C, G, c0, gy, gx, acc);
}

// Output-driven spreading, dense cells (the plan's list of cells whose window
// holds more than kSpreadDense samples): warp (cell, coil group), the lanes
// taking every 32nd sample of each row range, then a butterfly sum.
template <int W>
__global__ void __launch_bounds__(256) k_nufft_spread_dense(const float4* __restrict__ ys, int C, int Cp, int G,
                                                            const int32_t* __restrict__ cell_ptr,
                                                            const int32_t* __restrict__ cell_sx,
                                                            const float* __restrict__ cell_w,
                                                            const int32_t* __restrict__ dense, int n_dense,
                                                            float2* __restrict__ grid) {
  mpi_ptx::pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int c0 = blockIdx.y * kSpreadCoils;
  mpi_ptx::pdl_wait();
  if (i >= n_dense) return;
  const int cell = dense[i], gy = cell / G, gx = cell % G;
  const int ystride = Cp / 2;
  const float4* yc = ys + c0 / 2;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < W; ++a) {
    int sy = gy - a;
    if (sy < 0) sy += G;
    int r[4];
    spread_row_ranges<W>(cell_ptr + sy * G, gx, G, r);
    for (int k = r[0] + lane; k < r[1]; k += 32) spread_term<W>(cell_w, cell_sx, yc, ystride, k, gx, a, G, acc);
    for (int k = r[2] + lane; k < r[3]; k += 32) spread_term<W>(cell_w, cell_sx, yc, ystride, k, gx, a, G, acc);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  if (lane == 0) spread_store(grid, C, G, c0, gy, gx, acc);
}

float axis_sign(int n) { return ((n / 2) & 1) ? -1.f : 1.f; }

unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// load_lo, load_hi: the elements of each line read (the rest taken as zero);
// keep_lo, keep_hi: the elements of each transformed line stored back (default: all)
mpi_status launch_fft_rows_inplace(mpi_ctx* ctx, float2* data, long n_rows, int L, bool inverse, int load_lo = 0,
                                   int load_hi = -1, int keep_lo = 0, int keep_hi = -1);

size_t nufft_grid_elems(const mpi_plan* plan, int C) {
  return (size_t)C * plan->G * plan->G + (size_t)spread_coils_padded(C) * plan->M;
}

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
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "nufft plan setup");
  // Spreading CSR, built from the device's own first taps and weights (so it
  // agrees with the interpolation bit for bit): a counting sort of the samples
  // by first-tap cell sy * G + sx, stable in the sample index.
  if (M > 0) {
    std::vector<int32_t> gs((size_t)2 * M);
    std::vector<float> w((size_t)2 * M * W);
    e = cudaMemcpy(gs.data(), plan->gstart, gs.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(w.data(), plan->gw, w.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(ctx, e, "nufft spreading index");
    const size_t GG = (size_t)G * G;
    std::vector<int32_t> ptr(GG + 1, 0), samp(M), rank(M), sx(M), dense;
    std::vector<float> cw((size_t)2 * M * W);
    for (int m = 0; m < M; ++m) ++ptr[(size_t)gs[2 * m + 1] * G + gs[2 * m] + 1];
    for (size_t t = 0; t < GG; ++t) ptr[t + 1] += ptr[t];
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int m = 0; m < M; ++m) {
      const int k = fill[(size_t)gs[2 * m + 1] * G + gs[2 * m]]++;
      samp[k] = m;
      rank[m] = k;
      sx[k] = gs[2 * m];
      std::copy(w.begin() + (size_t)2 * m * W, w.begin() + (size_t)(2 * m + 2) * W, cw.begin() + (size_t)2 * k * W);
    }
    // Cells whose W x W window of first taps holds more than kSpreadDense
    // samples (a radial trajectory's centre), counted the way the kernels do.
    for (int gy = 0; gy < G; ++gy)
      for (int gx = 0; gx < G; ++gx) {
        long cnt = 0;
        for (int a = 0; a < W; ++a) {
          const int sy = (gy - a + G) % G;
          for (int b = 0; b < W; ++b) {
            const size_t t = (size_t)sy * G + (gx - b + G) % G;
            cnt += ptr[t + 1] - ptr[t];
          }
        }
        if (cnt > kSpreadDense) dense.push_back(gy * G + gx);
      }
    plan->n_dense = (int)dense.size();
    e = cudaMalloc(&plan->cell_ptr, ptr.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&plan->cell_rank, (size_t)M * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&plan->cell_sx, (size_t)M * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&plan->cell_w, cw.size() * sizeof(float));
    if (e == cudaSuccess && !dense.empty()) e = cudaMalloc(&plan->cell_dense, dense.size() * sizeof(int32_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(plan->cell_ptr, ptr.data(), ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(plan->cell_rank, rank.data(), (size_t)M * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(plan->cell_sx, sx.data(), (size_t)M * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(plan->cell_w, cw.data(), cw.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !dense.empty())
      e = cudaMemcpy(plan->cell_dense, dense.data(), dense.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    // Interpolation work list: a counting sort of the samples by the 32 x 32
    // tile of their first tap, then one item per chunk of a tile's samples.
    const int tpr = (G + kInterpTile - 1) / kInterpTile, n_tiles = tpr * tpr;
    std::vector<int32_t> tcount(n_tiles + 1, 0), tsorted(M), items;
    for (int m = 0; m < M; ++m)
      ++tcount[(gs[2 * m + 1] / kInterpTile) * tpr + gs[2 * m] / kInterpTile + 1];
    for (int t = 0; t < n_tiles; ++t) tcount[t + 1] += tcount[t];
    std::vector<int32_t> tfill(tcount.begin(), tcount.end() - 1);
    for (int m = 0; m < M; ++m) tsorted[tfill[(gs[2 * m + 1] / kInterpTile) * tpr + gs[2 * m] / kInterpTile]++] = m;
    for (int t = 0; t < n_tiles; ++t)
      for (int s0 = tcount[t]; s0 < tcount[t + 1]; s0 += kInterpChunk) {
        items.push_back(t);
        items.push_back(s0);
        items.push_back(std::min(kInterpChunk, tcount[t + 1] - s0));
      }
    plan->n_tile_items = (int)(items.size() / 3);
    if (e == cudaSuccess) e = cudaMalloc(&plan->tile_items, items.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&plan->tile_samples, (size_t)M * sizeof(int32_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(plan->tile_items, items.data(), items.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(plan->tile_samples, tsorted.data(), (size_t)M * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_check(ctx, e, "nufft spreading index");
  }
  return MPI_OK;
}

mpi_status nufft_forward(mpi_ctx* ctx, const mpi_plan* plan, const float2* v, int C, float2* y, float2* grid) {
  const int n = plan->nx, G = plan->G, M = plan->M;
  // zero-pad with deapodisation and sign, folded into the pass along y
  mpi_status st = launch_fft_cols_window(ctx, grid, C, G, v, nullptr, plan->deap, n, false);
  if (st) return st;
  // the pass along y wrote only the window's columns; the rest are zero
  const int o = G / 2 - n / 2;
  st = launch_fft_rows_inplace(ctx, grid, (long)C * G, G, false, o, o + n);
  if (st) return st;
  if (M == 0) return MPI_OK;
  const float ks = axis_sign(G) * axis_sign(G);
  const dim3 igrid((unsigned)plan->n_tile_items, (unsigned)C);
  MPI_PROF(ctx, KF_NUFFT);
  switch (plan->W) {
#define MPI_W_CASE(w)                                                                                \
  case w:                                                                                            \
    launch_pdl(ctx, k_nufft_interp_tiled<w>, igrid, dim3(kInterpChunk), 0,                                         \
               grid, C, G, M, plan->gstart, plan->gw, ks, plan->tile_items, plan->tile_samples, y);         \
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
  if (M == 0) {
    cudaError_t e = cudaMemsetAsync(grid, 0, total * sizeof(float2), ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "grid clear");
  } else {
    const float ks = axis_sign(G) * axis_sign(G);
    const int Cp = spread_coils_padded(C);
    float2* ys = grid + total;  // nufft_grid_elems reserves the sorted copy after the grid
    MPI_PROF(ctx, KF_NUFFT);
    launch_pdl(ctx, k_nufft_sort_y, dim3(blocks_for((size_t)M * Cp, 256)), dim3(256), 0, y, C, Cp, M,
               plan->cell_rank, ks, ys);
    MPI_LAUNCH_CHECK(ctx, "k_nufft_sort_y");
    const unsigned groups = (unsigned)(Cp / kSpreadCoils);
    const dim3 sgrid((unsigned)((G + 31) / 32), (unsigned)((G + 7) / 8), groups);
    const dim3 dgrid((unsigned)((plan->n_dense + 7) / 8), groups);
    const float4* ys4 = (const float4*)ys;
    switch (plan->W) {
#define MPI_W_CASE(w)                                                                                      \
  case w:                                                                                                  \
    MPI_PROF(ctx, KF_NUFFT);                                                                               \
    launch_pdl(ctx, k_nufft_spread<w>, sgrid, dim3(32, 8), 0, ys4, C, Cp, G, plan->cell_ptr, plan->cell_sx,  \
               plan->cell_w, grid);                                                                        \
    if (plan->n_dense > 0) {                                                                               \
      MPI_LAUNCH_CHECK(ctx, "k_nufft_spread");                                                             \
      MPI_PROF(ctx, KF_NUFFT);                                                                             \
      launch_pdl(ctx, k_nufft_spread_dense<w>, dgrid, dim3(256), 0, ys4, C, Cp, G, plan->cell_ptr,          \
                 plan->cell_sx, plan->cell_w, plan->cell_dense, plan->n_dense, grid);                      \
    }                                                                                                      \
    break;
      MPI_W_CASE(2) MPI_W_CASE(3) MPI_W_CASE(4) MPI_W_CASE(5) MPI_W_CASE(6) MPI_W_CASE(7) MPI_W_CASE(8)
#undef MPI_W_CASE
      default:
        return set_err(ctx, MPI_ERR_ARG, "kernel width");
    }
    MPI_LAUNCH_CHECK(ctx, "k_nufft_spread");
  }
  // only the columns of the centred window reach the cropping pass along y
  const int o = G / 2 - n / 2;
  mpi_status st = launch_fft_rows_inplace(ctx, grid, (long)C * G, G, true, 0, G, o, o + n);
  if (st) return st;
  // the inverse pass along y stores only the centred window, with deapodisation and sign
  return launch_fft_cols_window(ctx, grid, C, G, nullptr, out, plan->deap, n, true);
}
