// Tucker compression of a dense basis on the GPU ("A Compression Scheme for
// Maxwell Basis": Eqs. 19-21).  The basis columns reshaped onto the voxel grid
// form T [q][n1][n2][n3]; the factors U_k are the leading eigenvectors of the
// mode-k Gram matrices G_k = T_(k) T_(k)^H (the left singular vectors of the
// mode-k unfoldings, HOSVD), truncated per mode to the fewest r_k whose
// discarded eigenvalues sum to at most eps^2 ||T||^2 / 3, so that the HOSVD
// bound sqrt(sum_k tail_k) <= eps ||T|| of Eq. 21 holds; the core is
// T x1 U1^H x2 U2^H x3 U3^H.
//
//  - G_k in FP64: the products of the FP32 entries are exact in FP64, and the
//    sums over the q N / n_k fibres run in a fixed order (per-CTA partial tiles
//    of 64 x 64, reduced in order), so eigenvalues down to ~1e-12 of the
//    largest decide the ranks.  Only the tiles on or above the diagonal are
//    formed; the rest is their conjugate transpose.
//  - eigenvectors: one-sided Jacobi on the columns of G_k (for a Hermitian PSD
//    matrix the singular vectors and values are the eigenvectors and values).
//  - the core by the FP32 conjugate mode products of the Tucker adjoint.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "mpi_internal.h"
#include "ptx.cuh"

namespace {

constexpr int kGT = 64;    // Gram tile
constexpr int kGK = 32;    // fibre positions staged per step
constexpr int kGThreads = 256;

// Partial Gram tiles.  T viewed as [Qn][nk][Bk]; K = Qn Bk fibre positions
// kappa = (Qi, bk).  CTA (x, y): tile pair pairs[x] = (ti, tj), ti <= tj, and
// positions [K y / S, K (y + 1) / S).  Thread (tr, tc) accumulates rows
// 4 tr .. 4 tr + 3 of block ti against columns 4 tc .. 4 tc + 3 of block tj.
// A_CONTIG: Bk == 1, so the nk values of a position are contiguous (else the
// positions of one row are).
template <bool A_CONTIG>
__global__ void __launch_bounds__(kGThreads) k_gram(const float2* __restrict__ T, int nk, long Bk, long K, int S,
                                                    const int2* __restrict__ pairs, int npairs,
                                                    double2* __restrict__ part) {
  __shared__ float2 sA[kGT][kGK + 1], sB[kGT][kGK + 1];
  const int2 pr = pairs[blockIdx.x];
  const int split = blockIdx.y;
  const long k0 = K * split / S, k1 = K * (split + 1) / S;
  const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (long kc = k0; kc < k1; kc += kGK) {
    __syncthreads();
    for (int e = tid; e < kGT * kGK; e += kGThreads) {
      int al, kl;
      if (A_CONTIG) {
        al = e % kGT;
        kl = e / kGT;
      } else {
        kl = e % kGK;
        al = e / kGK;
      }
      const long kap = kc + kl;
      const int a = pr.x * kGT + al, b = pr.y * kGT + al;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      if (kap < k1) {
        const long Qi = kap / Bk, bk = kap - Qi * Bk;
        const size_t base = (size_t)Qi * nk * Bk + bk;
        if (a < nk) va = T[base + (size_t)a * Bk];
        if (b < nk) vb = T[base + (size_t)b * Bk];
      }
      sA[al][kl] = va;
      sB[al][kl] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int kl = 0; kl < kGK; ++kl) {
      double2 x[4], y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 u = sA[4 * tr + i][kl], v = sB[4 * tc + i][kl];
        x[i] = make_double2(u.x, u.y);
        y[i] = make_double2(v.x, v.y);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // x_i conj(y_j)
          acc[i][j].x = fma(x[i].x, y[j].x, fma(x[i].y, y[j].y, acc[i][j].x));
          acc[i][j].y = fma(x[i].y, y[j].x, fma(-x[i].x, y[j].y, acc[i][j].y));
        }
    }
  }
  double2* out = part + ((size_t)split * npairs + blockIdx.x) * kGT * kGT;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(4 * tr + i) * kGT + 4 * tc + j] = acc[i][j];
}

// M (column-major, nj columns of length nk; column nk zero when nj > nk) =
// G_k from the partial tiles summed over the splits in order.
__global__ void k_gram_reduce(const double2* __restrict__ part, int S, int npairs, const int* __restrict__ pair_of,
                              int ntile, int nk, int nj, double2* __restrict__ M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= nk) return;
  if (j >= nk) {
    M[(size_t)j * nk + i] = make_double2(0.0, 0.0);
    return;
  }
  const int ti = i / kGT, tj = j / kGT;
  const bool upper = ti <= tj;
  const int p = upper ? pair_of[ti * ntile + tj] : pair_of[tj * ntile + ti];
  const int e = upper ? (i % kGT) * kGT + (j % kGT) : (j % kGT) * kGT + (i % kGT);
  double2 s = make_double2(0.0, 0.0);
  for (int sp = 0; sp < S; ++sp) {
    const double2 v = part[((size_t)sp * npairs + p) * kGT * kGT + e];
    s.x += v.x;
    s.y += v.y;
  }
  M[(size_t)j * nk + i] = upper ? s : make_double2(s.x, -s.y);
}

// F [nk][r] complex64: F[i][c] = V[order[c]][i] (eigenvector column order[c]).
__global__ void k_factor_out(const double2* __restrict__ V, int nj, const int* __restrict__ order, int nk, int r,
                             float2* __restrict__ F) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nk * r) return;
  const int i = e / r, c = e - i * r;
  const double2 v = V[(size_t)order[c] * nj + i];
  F[e] = make_float2((float)v.x, (float)v.y);
}

struct Buf {
  void* p = nullptr;
  ~Buf() {
    if (p) cudaFree(p);
  }
};

// Eigen-decomposition of the mode-k Gram matrix: eigenvalues (descending) and
// their eigenvectors' column order in V.
mpi_status mode_gram_eig(mpi_ctx* ctx, const float2* T, int q, const int n[3], int k, double2* M, double2* V,
                         double* sig_dev, int* flag, double2* part, size_t part_elems, int2* d_pairs, int* d_pair_of,
                         std::vector<double>& lam, std::vector<int>& order) {
  const int nk = n[k];
  const int nj = nk + (nk & 1);
  const long Qn = k == 0 ? q : (k == 1 ? (long)q * n[0] : (long)q * n[0] * n[1]);
  const long Bk = k == 0 ? (long)n[1] * n[2] : (k == 1 ? n[2] : 1);
  const long K = Qn * Bk;
  const int ntile = (nk + kGT - 1) / kGT;
  std::vector<int2> pairs;
  std::vector<int> pair_of(ntile * ntile, -1);
  for (int ti = 0; ti < ntile; ++ti)
    for (int tj = ti; tj < ntile; ++tj) {
      pair_of[ti * ntile + tj] = (int)pairs.size();
      pairs.push_back(make_int2(ti, tj));
    }
  const int npairs = (int)pairs.size();
  const long want = std::max<long>(1, 2L * std::max(ctx->num_sms, 1) / npairs);
  const int S = (int)std::min<long>(want, std::max<long>(1, K / kGK));
  if ((size_t)S * npairs * kGT * kGT > part_elems) return set_err(ctx, MPI_ERR_OOM, "Tucker compression: Gram partials");
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(d_pairs, pairs.data(), npairs * sizeof(int2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_pair_of, pair_of.data(), pair_of.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "Tucker compression: tile list");
  MPI_PROF(ctx, KF_OTHER);
  if (Bk == 1)
    k_gram<true><<<dim3((unsigned)npairs, (unsigned)S), kGThreads, 0, st>>>(T, nk, Bk, K, S, d_pairs, npairs, part);
  else
    k_gram<false><<<dim3((unsigned)npairs, (unsigned)S), kGThreads, 0, st>>>(T, nk, Bk, K, S, d_pairs, npairs, part);
  MPI_LAUNCH_CHECK(ctx, "k_gram");
  MPI_PROF(ctx, KF_OTHER);
  k_gram_reduce<<<dim3((unsigned)((nk + 127) / 128), (unsigned)nj), 128, 0, st>>>(part, S, npairs, d_pair_of, ntile,
                                                                                  nk, nj, M);
  MPI_LAUNCH_CHECK(ctx, "k_gram_reduce");
  std::vector<double> sig;
  mpi_status s2 = jacobi_columns(ctx, M, nk, nj, V, sig_dev, flag, sig, "Tucker compression");
  if (s2) return s2;
  order.resize(nj);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sig[x] > sig[y]; });
  lam.resize(nk);
  for (int i = 0; i < nk; ++i) lam[i] = sig[order[i]];
  return MPI_OK;
}

}  // namespace

extern "C" mpi_status mpi_tucker_compress(mpi_ctx* ctx, const mpi_c32* T, const int n[3], int q, double eps,
                                          mpi_basis** out, int ranks_out[3], double* bound_out) {
  if (!ctx) return MPI_ERR_ARG;
  if (!T || !n || !out || !(eps > 0.0)) return set_err(ctx, MPI_ERR_ARG, "Tucker compression: bad argument");
  *out = nullptr;
  for (int k = 0; k < 3; ++k)
    if (n[k] < 1 || n[k] > 256) return set_err(ctx, MPI_ERR_SHAPE, "Tucker compression: 1 <= n_k <= 256");
  if (q < 1 || q > 256) return set_err(ctx, MPI_ERR_SHAPE, "Tucker compression: 1 <= q <= 256");
  const long N = (long)n[0] * n[1] * n[2];
  if (N % 4) return set_err(ctx, MPI_ERR_SHAPE, "Tucker compression: n1 n2 n3 must be a multiple of 4");
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const int nmax = std::max(n[0], std::max(n[1], n[2]));
  const int njmax = nmax + (nmax & 1);
  const int tmax = (nmax + kGT - 1) / kGT;
  const size_t part_elems = (size_t)(2 * std::max(ctx->num_sms, 1) + tmax * tmax) * kGT * kGT;
  Buf bM, bV, bSig, bFlag, bPart, bPairs, bPairOf, bOrd;
  cudaError_t e = cudaMalloc(&bM.p, (size_t)nmax * njmax * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&bV.p, (size_t)njmax * njmax * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&bSig.p, (size_t)njmax * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&bFlag.p, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&bPart.p, part_elems * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&bPairs.p, (size_t)tmax * tmax * sizeof(int2));
  if (e == cudaSuccess) e = cudaMalloc(&bPairOf.p, (size_t)tmax * tmax * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&bOrd.p, (size_t)njmax * sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_OOM, "Tucker compression workspace");
  }
  // per mode: eigen-decomposition, rank, factor
  Buf bF[3];
  int r[3];
  double tails = 0.0, fro2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    std::vector<double> lam;
    std::vector<int> order;
    mpi_status s2 = mode_gram_eig(ctx, (const float2*)T, q, n, k, (double2*)bM.p, (double2*)bV.p, (double*)bSig.p,
                                  (int*)bFlag.p, (double2*)bPart.p, part_elems, (int2*)bPairs.p, (int*)bPairOf.p,
                                  lam, order);
    if (s2) return s2;
    // eigenvalues of a PSD matrix; rounding can leave the smallest slightly negative in exact
    // arithmetic, but column norms are >= 0.  tail[i] = sum_{j >= i} lam_j
    double total = 0.0;
    for (double v : lam) total += v;
    if (k == 0) fro2 = total;
    const double budget = eps * eps * total / 3.0;
    std::vector<double> tail(n[k] + 1, 0.0);
    for (int i = n[k] - 1; i >= 0; --i) tail[i] = tail[i + 1] + lam[i];
    int rk = 1;
    while (rk < n[k] && tail[rk] > budget) ++rk;
    r[k] = rk;
    if (r[k] > 128) return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker compression: a rank above 128 for this eps");
    // keep the order for the factor write below (after a possible rank increase)
    e = cudaMemcpyAsync(bOrd.p, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, "Tucker compression: order");
    // the Tucker basis needs r1 r2 r3 to be a multiple of 4: the last mode takes
    // the extra eigenvectors (a larger rank only lowers the error)
    if (k == 2) {
      while ((r[0] * r[1] * r[2]) % 4 && r[2] < std::min(n[2], 128)) ++r[2];
      if ((r[0] * r[1] * r[2]) % 4)
        return set_err(ctx, MPI_ERR_UNSUPPORTED, "Tucker compression: ranks cannot be made a multiple of 4");
    }
    tails += tail[r[k]];
    e = cudaMalloc(&bF[k].p, (size_t)n[k] * r[k] * sizeof(float2));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, MPI_ERR_OOM, "Tucker compression: factor");
    }
    MPI_PROF(ctx, KF_OTHER);
    k_factor_out<<<(n[k] * r[k] + 255) / 256, 256, 0, st>>>((const double2*)bV.p, n[k] + (n[k] & 1),
                                                           (const int*)bOrd.p, n[k], r[k], (float2*)bF[k].p);
    MPI_LAUNCH_CHECK(ctx, "k_factor_out");
  }
  // core = T x1 U1^H x2 U2^H x3 U3^H
  Buf bCore, bTmp;
  const size_t core_elems = (size_t)q * r[0] * r[1] * r[2];
  const size_t tmp_elems = (size_t)q * r[0] * ((size_t)n[1] * n[2] + (size_t)r[1] * n[2]);
  e = cudaMalloc(&bCore.p, core_elems * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&bTmp.p, tmp_elems * sizeof(float2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_OOM, "Tucker compression: core");
  }
  mpi_status s3 = tucker_project(ctx, (const float2*)T, q, n, r, (const float2*)bF[0].p, (const float2*)bF[1].p,
                                 (const float2*)bF[2].p, (float2*)bCore.p, (float2*)bTmp.p);
  if (s3) return s3;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "Tucker compression");
  s3 = mpi_basis_load_tucker(ctx, (const mpi_c32*)bCore.p, (const mpi_c32*)bF[0].p, (const mpi_c32*)bF[1].p,
                             (const mpi_c32*)bF[2].p, n, r, q, 1, out);
  if (s3) return s3;
  if (ranks_out)
    for (int k = 0; k < 3; ++k) ranks_out[k] = r[k];
  if (bound_out) *bound_out = fro2 > 0.0 ? std::sqrt(tails / fro2) : 0.0;
  return MPI_OK;
}
