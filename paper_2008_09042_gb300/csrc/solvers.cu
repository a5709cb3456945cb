// The two solvers that drive the encoding operator, on the device:
//   MPI-BL  IRGN with CG on the normal equations of Eq. 6 (mpi_sm_estimate);
//   MPI-L   scaled ADMM for the constrained TV problem of Eq. 8 with the
//           updates of Eq. 11 (mpi_image_solve), FGP TV prox, l2-ball projection;
// and the FP64 Gram / Cholesky projection of maps onto the basis (Fig. 2 caption).
//
// Vectors are FP32 complex; every inner product and norm is accumulated in
// FP64 (block partials summed in a fixed order, so results are deterministic).
// CG and ADMM scalars live in a small device array, so the loops never wait on
// the host; only the residual histories are copied back at the end.
#include <math.h>

#include <string.h>

#include <algorithm>
#include <vector>

#include "mpi_internal.h"

namespace {

constexpr int kVecThreads = 256;
constexpr int kRedBlocks = 304;  // partial sums per reduction

// device scalar slots
enum Slot {
  S_RR = 0, S_DAD, S_A, S_BETA, S_SCALE, S_RHO, S_R2, S_S2, S_UFAC, S_TMP, S_COUNT
};

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partials[b] = sum Re(conj(a) b)  (b == nullptr: sum |a|^2)
__global__ void k_dot_partial(const float2* __restrict__ a, const float2* __restrict__ b, long n,
                              double* __restrict__ partials) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 x = a[i];
    if (b) {
      const float2 y = b[i];
      s += (double)x.x * y.x + (double)x.y * y.y;
    } else {
      s += (double)x.x * x.x + (double)x.y * x.y;
    }
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// partials[b] = sum |a - b|^2
__global__ void k_diffnorm_partial(const float2* __restrict__ a, const float2* __restrict__ b, long n,
                                   double* __restrict__ partials) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 x = a[i], y = b[i];
    const double dx = (double)x.x - y.x, dy = (double)x.y - y.y;
    s += dx * dx + dy * dy;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

enum FinOp {
  FIN_STORE = 0,      // S[slot] = sum
  FIN_ADD,            // S[slot] += sum
  FIN_CG_ALPHA,       // S[S_DAD] = sum; S[S_A] = S[S_RR] / sum (0 if sum <= 0)
  FIN_CG_BETA,        // S[S_BETA] = sum / S[S_RR] (0 if S[S_RR] <= 0); S[S_RR] = sum
  FIN_SCALE,          // S[S_SCALE] = target / sqrt(sum) (1 if sum == 0)
  FIN_SQRT_TO_HIST,   // hist[idx] = sqrt(sum)
};

__global__ void k_finalize(const double* __restrict__ partials, int nblk, double* __restrict__ S, int op, int slot,
                           double target, double* __restrict__ hist, int idx) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += partials[i];
  s = block_sum(s, sh);
  if (threadIdx.x != 0) return;
  switch (op) {
    case FIN_STORE: S[slot] = s; break;
    case FIN_ADD: S[slot] += s; break;
    case FIN_CG_ALPHA:
      S[S_DAD] = s;
      S[S_A] = s > 0.0 ? S[S_RR] / s : 0.0;
      break;
    case FIN_CG_BETA:
      S[S_BETA] = S[S_RR] > 0.0 ? s / S[S_RR] : 0.0;
      S[S_RR] = s;
      break;
    case FIN_SCALE: S[S_SCALE] = s > 0.0 ? target / sqrt(s) : 1.0; break;
    case FIN_SQRT_TO_HIST: hist[idx] = sqrt(s); break;
  }
}

// Ad = h + lam(i) d, lam = lam1 for i < n1 else lam2; partials of Re(conj(d) Ad)
__global__ void k_normal_finish(const float2* __restrict__ h, const float2* __restrict__ d, long n, long n1,
                                float lam1, float lam2, float2* __restrict__ Ad, double* __restrict__ partials) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float lam = i < n1 ? lam1 : lam2;
    const float2 hv = h[i], dv = d[i];
    const float2 a = make_float2(hv.x + lam * dv.x, hv.y + lam * dv.y);
    Ad[i] = a;
    s += (double)dv.x * a.x + (double)dv.y * a.y;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// x += a d; r -= a Ad; partials of |r|^2
__global__ void k_cg_update(float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ d,
                            const float2* __restrict__ Ad, long n, const double* __restrict__ S,
                            double* __restrict__ partials) {
  __shared__ double sh[32];
  const float a = (float)S[S_A];
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 dv = d[i], av = Ad[i];
    float2 xv = x[i], rv = r[i];
    xv.x = fmaf(a, dv.x, xv.x);
    xv.y = fmaf(a, dv.y, xv.y);
    rv.x = fmaf(-a, av.x, rv.x);
    rv.y = fmaf(-a, av.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    s += (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// d = r + beta d
__global__ void k_cg_dir(float2* __restrict__ d, const float2* __restrict__ r, long n, const double* __restrict__ S) {
  const float beta = (float)S[S_BETA];
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 rv = r[i];
    float2 dv = d[i];
    d[i] = make_float2(fmaf(beta, dv.x, rv.x), fmaf(beta, dv.y, rv.y));
  }
}

// out = a1 x + a2 y (host constants; y may be null)
__global__ void k_lincomb(float2* __restrict__ out, const float2* __restrict__ x, float a1,
                          const float2* __restrict__ y, float a2, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 xv = x[i];
    float2 o = make_float2(a1 * xv.x, a1 * xv.y);
    if (y) {
      const float2 yv = y[i];
      o.x = fmaf(a2, yv.x, o.x);
      o.y = fmaf(a2, yv.y, o.y);
    }
    out[i] = o;
  }
}

// out = x * S[slot]^pw  (pw = +1 or -1)
__global__ void k_scale_dev(float2* __restrict__ out, const float2* __restrict__ x, long n, const double* __restrict__ S,
                            int slot, int inverse) {
  const double sd = S[slot];
  const float s = (float)(inverse ? 1.0 / sd : sd);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 v = x[i];
    out[i] = make_float2(v.x * s, v.y * s);
  }
}

__global__ void k_fill(float2* __restrict__ x, float2 v, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] = v;
}

// ---------------------------------------------------------------- TV prox (FGP)

struct Grid3 {
  int nz, ny, nx, nd;  // nd = 2 (y, x) or 3 (z, y, x)
};

// axis d of a component: 0 = x, 1 = y, 2 = z (stride 1, nx, nx*ny)
__device__ __forceinline__ void coords(const Grid3& g, long i, int& x, int& y, int& z) {
  x = (int)(i % g.nx);
  long t = i / g.nx;
  y = (int)(t % g.ny);
  z = (int)(t / g.ny);
}

// x = b - lam D^H R, with (D^H R)_i = sum_d (R_d[i - e_d] if i_d >= 1) - (R_d[i] if i_d <= n_d - 2)
// lam = 1 / S[S_RHO] (rho_slot >= 0) or lam_host.
__global__ void k_tv_primal(const float2* __restrict__ b, const float2* __restrict__ R, Grid3 g, long N,
                            const double* __restrict__ S, int use_rho, float lam_host, float2* __restrict__ x) {
  const float lam = use_rho ? (float)(1.0 / S[S_RHO]) : lam_host;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    coords(g, i, cx, cy, cz);
    float2 dh = make_float2(0.f, 0.f);
    const int pos[3] = {cx, cy, cz};
    const int len[3] = {g.nx, g.ny, g.nz};
    const long stride[3] = {1, g.nx, (long)g.nx * g.ny};
    for (int d = 0; d < g.nd; ++d) {
      const float2* Rd = R + (size_t)d * N;
      if (pos[d] >= 1) {
        const float2 v = Rd[i - stride[d]];
        dh.x += v.x;
        dh.y += v.y;
      }
      if (pos[d] <= len[d] - 2) {
        const float2 v = Rd[i];
        dh.x -= v.x;
        dh.y -= v.y;
      }
    }
    const float2 bv = b[i];
    x[i] = make_float2(bv.x - lam * dh.x, bv.y - lam * dh.y);
  }
}

// Pn = proj(R + D x * rho / L); R = Pn + c (Pn - P); P = Pn
__global__ void k_tv_dual(const float2* __restrict__ x, float2* __restrict__ P, float2* __restrict__ R, Grid3 g,
                          long N, const double* __restrict__ S, int use_rho, float lam_host, float c) {
  const float L = 4.0f * g.nd;
  const float step = use_rho ? (float)(S[S_RHO] / L) : 1.0f / (L * lam_host);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    int cx, cy, cz;
    coords(g, i, cx, cy, cz);
    const int pos[3] = {cx, cy, cz};
    const int len[3] = {g.nx, g.ny, g.nz};
    const long stride[3] = {1, g.nx, (long)g.nx * g.ny};
    const float2 xi = x[i];
    float2 pn[3];
    float mag2 = 0.f;
    for (int d = 0; d < g.nd; ++d) {
      float2 gd = make_float2(0.f, 0.f);
      if (pos[d] <= len[d] - 2) {
        const float2 xn = x[i + stride[d]];
        gd = make_float2(xn.x - xi.x, xn.y - xi.y);
      }
      const float2 rv = R[(size_t)d * N + i];
      pn[d] = make_float2(fmaf(step, gd.x, rv.x), fmaf(step, gd.y, rv.y));
      mag2 += pn[d].x * pn[d].x + pn[d].y * pn[d].y;
    }
    const float inv = 1.0f / fmaxf(1.0f, sqrtf(mag2));
    for (int d = 0; d < g.nd; ++d) {
      const float2 p_old = P[(size_t)d * N + i];
      const float2 pv = make_float2(pn[d].x * inv, pn[d].y * inv);
      P[(size_t)d * N + i] = pv;
      R[(size_t)d * N + i] = make_float2(pv.x + c * (pv.x - p_old.x), pv.y + c * (pv.y - p_old.y));
    }
  }
}

// ------------------------------------------------------------ ball projection

// partials[c * nblk + b] = sum_m |z + u - y|^2 over coil c
__global__ void k_ball_norm_partial(const float2* __restrict__ z, const float2* __restrict__ u,
                                    const float2* __restrict__ y, int M, double* __restrict__ partials) {
  __shared__ double sh[32];
  const int c = blockIdx.y;
  double s = 0.0;
  for (long m = (long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
    const size_t i = (size_t)c * M + m;
    const float2 zv = z[i], uv = u[i], yv = y[i];
    const double dx = (double)zv.x + uv.x - yv.x, dy = (double)zv.y + uv.y - yv.y;
    s += dx * dx + dy * dy;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[(size_t)c * gridDim.x + blockIdx.x] = s;
}

// f_c = eps_c / max(||.||, eps_c) (FP64)
__global__ void k_ball_factor(const double* __restrict__ partials, int nblk, int C, const double* __restrict__ eps,
                              double* __restrict__ f) {
  __shared__ double sh[32];
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += partials[(size_t)c * nblk + i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      const double nrm = sqrt(s);
      f[c] = eps[c] / fmax(nrm, eps[c]);
    }
    __syncthreads();
  }
}

// zk = y + f_c (z + u - y)
__global__ void k_ball_apply(const float2* __restrict__ z, const float2* __restrict__ u, const float2* __restrict__ y,
                             int C, int M, const double* __restrict__ f, float2* __restrict__ out) {
  const long n = (long)C * M;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i / M);
    const float fc = (float)f[c];
    const float2 zv = z[i], uv = u[i], yv = y[i];
    out[i] = make_float2(yv.x + fc * (zv.x + uv.x - yv.x), yv.y + fc * (zv.y + uv.y - yv.y));
  }
}

// u += a - z (elementwise)
__global__ void k_dual_update(float2* __restrict__ u, const float2* __restrict__ a, const float2* __restrict__ z, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float2 av = a[i], zv = z[i];
    float2 uv = u[i];
    u[i] = make_float2(uv.x + av.x - zv.x, uv.y + av.y - zv.y);
  }
}

// residual balancing; S[S_R2], S[S_S2] hold the squared norms
__global__ void k_rho_update(double* __restrict__ S, double mu, double tau, double* __restrict__ hist, int it) {
  const double r = sqrt(S[S_R2]);
  const double s = S[S_RHO] * sqrt(S[S_S2]);
  hist[3 * it] = r;
  hist[3 * it + 1] = s;
  hist[3 * it + 2] = S[S_RHO];
  double f = 1.0;
  if (r > mu * s) {
    S[S_RHO] *= tau;
    f = 1.0 / tau;
  } else if (s > mu * r) {
    S[S_RHO] /= tau;
    f = tau;
  }
  S[S_UFAC] = f;
}

__global__ void k_set_slot(double* S, int slot, double v) { S[slot] = v; }

// ---------------------------------------------------------------- Gram / Cholesky (FP64)

// G[i][j] = sum_n conj(U[i][n]) U[j][n]; block (i, j) tile; chunks of 64 pixels
// accumulate in FP32 and are added to an FP64 sum.
__global__ void k_gram(const float2* __restrict__ U, int N, int q, double2* __restrict__ G) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.y + threadIdx.y;
  double sre = 0.0, sim = 0.0;
  if (j < q) {
    for (int n0 = threadIdx.x * 64; n0 < N; n0 += 32 * 64) {
      float re = 0.f, im = 0.f;
      const int n1 = min(N, n0 + 64);
      for (int n = n0; n < n1; ++n) {
        const float2 a = U[(size_t)i * N + n], b = U[(size_t)j * N + n];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
      }
      sre += re;
      sim += im;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sre += __shfl_down_sync(0xffffffffu, sre, o);
    sim += __shfl_down_sync(0xffffffffu, sim, o);
  }
  if (threadIdx.x == 0 && j < q) G[(size_t)i * q + j] = make_double2(sre, sim);
}

// rhs[c][i] = sum_n conj(U[i][n]) S[c][n]
__global__ void k_uh_s(const float2* __restrict__ U, int N, int q, const float2* __restrict__ Smaps, int C,
                       double2* __restrict__ rhs) {
  const int i = blockIdx.y;
  const int c = blockIdx.x * blockDim.y + threadIdx.y;
  double sre = 0.0, sim = 0.0;
  if (c < C) {
    for (int n0 = threadIdx.x * 64; n0 < N; n0 += 32 * 64) {
      float re = 0.f, im = 0.f;
      const int n1 = min(N, n0 + 64);
      for (int n = n0; n < n1; ++n) {
        const float2 a = U[(size_t)i * N + n], b = Smaps[(size_t)c * N + n];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
      }
      sre += re;
      sim += im;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sre += __shfl_down_sync(0xffffffffu, sre, o);
    sim += __shfl_down_sync(0xffffffffu, sim, o);
  }
  if (threadIdx.x == 0 && c < C) rhs[(size_t)c * q + i] = make_double2(sre, sim);
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zmulc(double2 a, double2 b) {  // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// In-place lower Cholesky factor of the Hermitian positive definite G (one CTA),
// then forward and back substitution for every coil's right-hand side:
//   L w = rhs_c, L^H alpha_c = w.  Writes alpha (FP32) [C][q].
__global__ void k_cholesky_solve(double2* __restrict__ G, int q, double2* __restrict__ rhs, int C,
                                 float2* __restrict__ alpha, int* __restrict__ status) {
  for (int k = 0; k < q; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const double d = G[(size_t)k * q + k].x;
      if (!(d > 0.0)) *status = 1;
      G[(size_t)k * q + k] = make_double2(d > 0.0 ? sqrt(d) : 1.0, 0.0);
    }
    __syncthreads();
    const double dk = G[(size_t)k * q + k].x;
    for (int i = k + 1 + threadIdx.x; i < q; i += blockDim.x) {
      double2 v = G[(size_t)i * q + k];
      G[(size_t)i * q + k] = make_double2(v.x / dk, v.y / dk);
    }
    __syncthreads();
    // trailing update of the lower triangle: G[i][j] -= L[i][k] conj(L[j][k]), k < j <= i
    const int m = q - k - 1;
    const long tri = (long)m * (m + 1) / 2;
    for (long e = threadIdx.x; e < tri; e += blockDim.x) {
      // map e to (i, j) with 0 <= jj <= ii < m
      int ii = (int)((sqrt(8.0 * e + 1.0) - 1.0) / 2.0);
      while ((long)ii * (ii + 1) / 2 > e) --ii;
      while ((long)(ii + 1) * (ii + 2) / 2 <= e) ++ii;
      const int jj = (int)(e - (long)ii * (ii + 1) / 2);
      const int i = k + 1 + ii, j = k + 1 + jj;
      const double2 t = zmulc(G[(size_t)i * q + k], G[(size_t)j * q + k]);
      double2 g = G[(size_t)i * q + j];
      G[(size_t)i * q + j] = make_double2(g.x - t.x, g.y - t.y);
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double2* b = rhs + (size_t)c * q;
    for (int i = 0; i < q; ++i) {  // L w = b
      double2 s = b[i];
      for (int j = 0; j < i; ++j) {
        const double2 t = zmul(G[(size_t)i * q + j], b[j]);
        s.x -= t.x;
        s.y -= t.y;
      }
      const double d = G[(size_t)i * q + i].x;
      b[i] = make_double2(s.x / d, s.y / d);
    }
    for (int i = q - 1; i >= 0; --i) {  // L^H a = w
      double2 s = b[i];
      for (int j = i + 1; j < q; ++j) {
        const double2 l = G[(size_t)j * q + i];
        const double2 t = make_double2(l.x * b[j].x + l.y * b[j].y, l.x * b[j].y - l.y * b[j].x);  // conj(l) b
        s.x -= t.x;
        s.y -= t.y;
      }
      const double d = G[(size_t)i * q + i].x;
      b[i] = make_double2(s.x / d, s.y / d);
    }
    for (int i = 0; i < q; ++i) alpha[(size_t)c * q + i] = make_float2((float)b[i].x, (float)b[i].y);
  }
}

// ----------------------------------------------------------------- host side

unsigned grid_for(long n) {
  const long b = (n + kVecThreads - 1) / kVecThreads;
  return (unsigned)std::max(1L, std::min(b, (long)kRedBlocks));
}

struct Solver {
  mpi_ctx* ctx;
  double* S;         // [S_COUNT]
  double* partials;  // [kRedBlocks * 64]
  void* mem = nullptr;

  mpi_status dot(const float2* a, const float2* b, long n, int op, int slot = 0, double target = 0,
                 double* hist = nullptr, int idx = 0) {
    MPI_PROF(ctx, KF_SOLVER);
    k_dot_partial<<<kRedBlocks, kVecThreads, 0, ctx->stream>>>(a, b, n, partials);
    MPI_LAUNCH_CHECK(ctx, "k_dot_partial");
    return fin(op, slot, target, hist, idx);
  }
  mpi_status fin(int op, int slot = 0, double target = 0, double* hist = nullptr, int idx = 0) {
    MPI_PROF(ctx, KF_SOLVER);
    k_finalize<<<1, kVecThreads, 0, ctx->stream>>>(partials, kRedBlocks, S, op, slot, target, hist, idx);
    MPI_LAUNCH_CHECK(ctx, "k_finalize");
    return MPI_OK;
  }
  mpi_status diffnorm(const float2* a, const float2* b, long n, int op, int slot) {
    MPI_PROF(ctx, KF_SOLVER);
    k_diffnorm_partial<<<kRedBlocks, kVecThreads, 0, ctx->stream>>>(a, b, n, partials);
    MPI_LAUNCH_CHECK(ctx, "k_diffnorm_partial");
    return fin(op, slot);
  }
  mpi_status lincomb(float2* out, const float2* x, float a1, const float2* y, float a2, long n) {
    MPI_PROF(ctx, KF_SOLVER);
    k_lincomb<<<grid_for(n), kVecThreads, 0, ctx->stream>>>(out, x, a1, y, a2, n);
    MPI_LAUNCH_CHECK(ctx, "k_lincomb");
    return MPI_OK;
  }
  mpi_status fill(float2* x, float2 v, long n) {
    MPI_PROF(ctx, KF_SOLVER);
    k_fill<<<grid_for(n), kVecThreads, 0, ctx->stream>>>(x, v, n);
    MPI_LAUNCH_CHECK(ctx, "k_fill");
    return MPI_OK;
  }
  mpi_status scale_dev(float2* out, const float2* x, long n, int slot, int inverse) {
    MPI_PROF(ctx, KF_SOLVER);
    k_scale_dev<<<grid_for(n), kVecThreads, 0, ctx->stream>>>(out, x, n, S, slot, inverse);
    MPI_LAUNCH_CHECK(ctx, "k_scale_dev");
    return MPI_OK;
  }
  mpi_status set(int slot, double v) {
    MPI_PROF(ctx, KF_SOLVER);
    k_set_slot<<<1, 1, 0, ctx->stream>>>(S, slot, v);
    MPI_LAUNCH_CHECK(ctx, "k_set_slot");
    return MPI_OK;
  }
};

#define TRY(x)                  \
  do {                          \
    mpi_status st__ = (x);      \
    if (st__ != MPI_OK) return st__; \
  } while (0)

// Solver buffers live in their own allocation (the operator calls use ctx->work).
struct SolverMem {
  void* p = nullptr;
  ~SolverMem() {
    if (p) cudaFree(p);
  }
};

mpi_status alloc_solver(mpi_ctx* ctx, SolverMem& m, size_t complex_elems, size_t extra_doubles, Solver& sv,
                        float2** base, double** dbase) {
  const size_t bytes = complex_elems * sizeof(float2) + (S_COUNT + (size_t)kRedBlocks * 64 + extra_doubles) * sizeof(double) + 1024;
  cudaError_t e = cudaMalloc(&m.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_OOM, "solver buffers");
  }
  *base = (float2*)m.p;
  double* d = (double*)(((uintptr_t)((float2*)m.p + complex_elems) + 255) & ~(uintptr_t)255);
  sv.ctx = ctx;
  sv.S = d;
  sv.partials = d + S_COUNT;
  *dbase = d + S_COUNT + (size_t)kRedBlocks * 64;
  const size_t nd = S_COUNT + (size_t)kRedBlocks * 64 + extra_doubles;
  return cuda_check(ctx, cudaMemsetAsync(d, 0, nd * sizeof(double), ctx->stream), "memset");
}

Grid3 grid_of(const mpi_plan* plan) {
  Grid3 g;
  g.nz = plan->nz;
  g.ny = plan->ny;
  g.nx = plan->nx;
  g.nd = plan->ndim == 3 ? 3 : 2;
  return g;
}

// z = prox_{lam TV}(b) by n_iter FGP iterations; P, R are [nd][N] scratch, x the output.
mpi_status tv_prox_run(Solver& sv, const Grid3& g, long N, const float2* b, int n_iter, int use_rho, float lam,
                       float2* P, float2* R, float2* x) {
  mpi_ctx* ctx = sv.ctx;
  TRY(sv.fill(P, make_float2(0.f, 0.f), (long)g.nd * N));
  TRY(sv.fill(R, make_float2(0.f, 0.f), (long)g.nd * N));
  double t = 1.0;
  for (int it = 0; it < n_iter; ++it) {
    MPI_PROF(ctx, KF_SOLVER);
    k_tv_primal<<<grid_for(N), kVecThreads, 0, ctx->stream>>>(b, R, g, N, sv.S, use_rho, lam, x);
    MPI_LAUNCH_CHECK(ctx, "k_tv_primal");
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const float c = (float)((t - 1.0) / tn);
    MPI_PROF(ctx, KF_SOLVER);
    k_tv_dual<<<grid_for(N), kVecThreads, 0, ctx->stream>>>(x, P, R, g, N, sv.S, use_rho, lam, c);
    MPI_LAUNCH_CHECK(ctx, "k_tv_dual");
    t = tn;
  }
  MPI_PROF(ctx, KF_SOLVER);
  k_tv_primal<<<grid_for(N), kVecThreads, 0, ctx->stream>>>(b, P, g, N, sv.S, use_rho, lam, x);
  MPI_LAUNCH_CHECK(ctx, "k_tv_primal");
  return MPI_OK;
}

}  // namespace

// ------------------------------------------------------- solver graph cache
//
// A solve enqueues thousands of small kernels; on small grids their launch
// cost dominates.  Each solve is therefore recorded once into a CUDA graph
// over solver buffers that the context keeps (keyed by plan, basis, coils,
// precision and parameters), with its inputs copied into and its outputs
// copied out of those buffers around one graph launch.  Destroying a plan or
// basis drops the graphs that reference it; growing the context workspace
// (which the graphs also reference) drops all of them.

namespace {

struct SolverGraph {
  int kind = 0;  // 0 = MPI-BL, 1 = MPI-L
  const mpi_plan* plan = nullptr;
  const mpi_basis* basis = nullptr;
  int C = 0;
  int prec = 0;
  std::vector<unsigned char> key;
  std::vector<const mpi_plan*> others;  // every plan the graph reads (the frames of a dynamic solve)
  void* work = nullptr;  // ctx->work at capture time
  SolverMem mem;
  Solver sv;
  float2* base = nullptr;  // solver vectors
  double* dbase = nullptr;
  float2* in_y = nullptr;
  float2* in_alpha = nullptr;
  double* in_eps = nullptr;
  float2* out_alpha = nullptr;
  float2* out_p = nullptr;
  double* hist = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  ~SolverGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

struct SolverCache {
  std::vector<SolverGraph*> entries;
};

SolverCache* cache_of(mpi_ctx* ctx) {
  if (!ctx->solver_cache) ctx->solver_cache = new SolverCache();
  return (SolverCache*)ctx->solver_cache;
}

SolverGraph* cache_find(mpi_ctx* ctx, int kind, const mpi_plan* plan, const mpi_basis* basis, int C, int prec,
                        const void* prm, size_t prm_bytes) {
  SolverCache* c = cache_of(ctx);
  for (size_t i = 0; i < c->entries.size(); ++i) {
    SolverGraph* e = c->entries[i];
    if (e->kind == kind && e->plan == plan && e->basis == basis && e->C == C && e->prec == prec &&
        e->key.size() == prm_bytes && memcmp(e->key.data(), prm, prm_bytes) == 0) {
      if (e->work != ctx->work) {  // the workspace moved: the recorded kernels point at the old one
        delete e;
        c->entries.erase(c->entries.begin() + i);
        return nullptr;
      }
      return e;
    }
  }
  return nullptr;
}

void cache_insert(mpi_ctx* ctx, SolverGraph* g) {
  SolverCache* c = cache_of(ctx);
  constexpr size_t kMaxEntries = 8;
  if (c->entries.size() >= kMaxEntries) {
    delete c->entries.front();
    c->entries.erase(c->entries.begin());
  }
  c->entries.push_back(g);
}

// Record `body` (which enqueues on ctx->stream) into a graph on a private stream.
template <class F>
mpi_status capture(mpi_ctx* ctx, SolverGraph* g, F body) {
  cudaStream_t cap = nullptr, user = ctx->stream;
  cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_check(ctx, e, "solver capture stream");
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  ctx->stream = cap;
  const int64_t l0 = ctx->launches;
  mpi_status st = MPI_OK;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = body();
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (st == MPI_OK && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st == MPI_OK && e2 != cudaSuccess) st = cuda_check(ctx, e2, "solver graph");
  } else {
    st = cuda_check(ctx, e, "solver capture begin");
  }
  g->kernels = ctx->launches - l0;
  ctx->launches = l0;
  ctx->stream = user;
  ctx->profiling = prof;
  cudaStreamDestroy(cap);
  return st;
}

mpi_status launch_graph(mpi_ctx* ctx, SolverGraph* g) {
  cudaError_t e = cudaGraphLaunch(g->exec, ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "solver graph launch");
  ctx->launches += g->kernels;
  return MPI_OK;
}

// ------------------------------------------------------------------ MPI-BL

// Start of the extra sets of maps (m >= 1): the first basis coefficient of
// every coil is 0.1 (sets that start proportional to the first stay so).
__global__ void k_first_coef(float2* __restrict__ al, int rows, int q, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows) al[(size_t)i * q] = make_float2(v, 0.f);
}

// Enqueue the IRGN solve with `nm` sets of maps (1: the model of Eq. 5; more:
// the extra bilinear terms of the Forward Model Extensions discussion).  The
// unknowns are x = [p_1 .. p_nm ; alpha_1 .. alpha_nm]; Eq. 6's penalties
// weigh every image by alpha_n and every coefficient set by beta_n.  Inputs:
// y (C x M).  Outputs: alpha_out (nm C q), p_out (nm N), hist.
mpi_status irgn_body(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int nm, int C,
                     const mpi_irgn_params* prm, mpi_precision prec, Solver& sv, float2* base, const float2* yc,
                     float2* alpha_out, float2* p_out, double* hist) {
  const long N = (long)nm * plan->N, Cq = (long)nm * C * basis->q, CM = (long)C * plan->M, X = N + Cq;
  float2 *x = base, *dx = x + X, *res = dx + X, *d = res + X, *Ad = d + X, *h = Ad + X;
  float2 *bn = h + X;  // right-hand side
  float2 *ys = bn + 2 * X, *yt = ys + std::max(CM, 1L), *r = yt + std::max(CM, 1L);
  float2 *p = x, *al = x + N;
  // MIXED: the CG iterations apply BF16 operators; the data residual
  // r = y - G(x) and the right-hand side J^H r - 2 L x of every Gauss-Newton
  // step are FP32, so the outer iteration refines x against FP32 residuals
  // (the inner solve stays the same fixed number of CG iterations).
  const mpi_precision pin = prec == MPI_PREC_MIXED ? MPI_PREC_BF16 : prec;
  const mpi_precision pout = prec == MPI_PREC_MIXED ? MPI_PREC_FP32 : prec;
  // data scale: ys = y * target / ||y||
  if (CM > 0) {
    TRY(sv.dot(yc, nullptr, CM, FIN_SCALE, 0, prm->scale_target));
    TRY(sv.scale_dev(ys, yc, CM, S_SCALE, 0));
  } else {
    TRY(sv.set(S_SCALE, 1.0));
  }
  TRY(sv.fill(p, make_float2(1.f, 0.f), N));
  TRY(sv.fill(al, make_float2(0.f, 0.f), Cq));
  if (nm > 1) {
    const int rows = (nm - 1) * C;
    MPI_PROF(ctx, KF_SOLVER);
    k_first_coef<<<(rows + 255) / 256, 256, 0, ctx->stream>>>(al + (long)C * basis->q, rows, basis->q, 0.1f);
    MPI_LAUNCH_CHECK(ctx, "k_first_coef");
  }
  float l1 = 0.f, l2 = 0.f;
  // (J^H J + 2L) v into Ad, v in `v`, operators at precision pr
  auto normal = [&](const float2* v, mpi_precision pr) -> mpi_status {
    TRY(mpi_jacobian_maps(ctx, plan, basis, nm, (const mpi_c32*)al, C, (const mpi_c32*)p, (const mpi_c32*)v,
                          (const mpi_c32*)(v + N), (mpi_c32*)yt, pr));
    TRY(mpi_jacobian_adjoint_maps(ctx, plan, basis, nm, (const mpi_c32*)al, C, (const mpi_c32*)p,
                                  (const mpi_c32*)yt, (mpi_c32*)h, (mpi_c32*)(h + N), pr));
    MPI_PROF(ctx, KF_SOLVER);
    k_normal_finish<<<kRedBlocks, kVecThreads, 0, ctx->stream>>>(h, v, X, N, l1, l2, Ad, sv.partials);
    MPI_LAUNCH_CHECK(ctx, "k_normal_finish");
    return MPI_OK;
  };
  // `iters` CG iterations for (J^H J + 2L) sol = rhs from sol = 0
  auto cg = [&](float2* sol, const float2* rhs, int iters, mpi_precision pr) -> mpi_status {
    TRY(sv.fill(sol, make_float2(0.f, 0.f), X));
    TRY(sv.lincomb(res, rhs, 1.f, nullptr, 0.f, X));
    TRY(sv.lincomb(d, res, 1.f, nullptr, 0.f, X));
    TRY(sv.dot(res, nullptr, X, FIN_STORE, S_RR));
    for (int it = 0; it < iters; ++it) {
      TRY(normal(d, pr));
      TRY(sv.fin(FIN_CG_ALPHA));
      MPI_PROF(ctx, KF_SOLVER);
      k_cg_update<<<kRedBlocks, kVecThreads, 0, ctx->stream>>>(sol, res, d, Ad, X, sv.S, sv.partials);
      MPI_LAUNCH_CHECK(ctx, "k_cg_update");
      TRY(sv.fin(FIN_CG_BETA));
      MPI_PROF(ctx, KF_SOLVER);
      k_cg_dir<<<grid_for(X), kVecThreads, 0, ctx->stream>>>(d, res, X, sv.S);
      MPI_LAUNCH_CHECK(ctx, "k_cg_dir");
    }
    return MPI_OK;
  };
  for (int n = 0; n <= prm->n_outer; ++n) {
    // r = ys - G(x)
    TRY(mpi_forward_maps(ctx, plan, basis, nm, (const mpi_c32*)al, C, (const mpi_c32*)p, (mpi_c32*)yt, pout));
    if (CM > 0) TRY(sv.lincomb(r, ys, 1.f, yt, -1.f, CM));
    if (CM > 0) TRY(sv.dot(r, nullptr, CM, FIN_SQRT_TO_HIST, 0, 0, hist, n));
    if (n == prm->n_outer) break;
    const double an = std::max(prm->a0 * pow(prm->decay, n), prm->floor_);
    const double bnn = std::max(prm->b0 * pow(prm->decay, n), prm->floor_);
    l1 = (float)(2.0 * an);
    l2 = (float)(2.0 * bnn);
    // b = J^H r - 2 L x
    TRY(mpi_jacobian_adjoint_maps(ctx, plan, basis, nm, (const mpi_c32*)al, C, (const mpi_c32*)p,
                                  (const mpi_c32*)r, (mpi_c32*)h, (mpi_c32*)(h + N), pout));
    TRY(sv.lincomb(bn, h, 1.f, x, -l1, N));
    TRY(sv.lincomb(bn + N, h + N, 1.f, x + N, -l2, Cq));
    TRY(cg(dx, bn, prm->n_cg, pin));
    TRY(sv.lincomb(x, x, 1.f, dx, (float)prm->gamma, X));
  }
  // outputs: alpha, p / scale
  TRY(sv.lincomb(alpha_out, al, 1.f, nullptr, 0.f, Cq));
  TRY(sv.scale_dev(p_out, p, N, S_SCALE, 1));
  return MPI_OK;
}

}  // namespace

namespace {

mpi_status sm_estimate_impl(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int nm, const mpi_c32* y,
                            int C, const mpi_irgn_params* prm, mpi_c32* alpha_out, mpi_c32* p_out,
                            double* resid_out, mpi_precision prec) {
  if (!ctx) return MPI_ERR_ARG;
  if (!plan || !basis || !prm || !alpha_out || !p_out || C < 1 || nm < 1 || (plan->M > 0 && !y))
    return set_err(ctx, MPI_ERR_ARG, "sm_estimate: bad argument");
  if (prm->n_outer < 0 || prm->n_cg < 0) return set_err(ctx, MPI_ERR_ARG, "negative iteration count");
  if (nm > 1 && basis->tucker) return set_err(ctx, MPI_ERR_UNSUPPORTED, "several sets of maps: dense bases only");
  cudaSetDevice(ctx->device);
  TRY(mpi_ctx_reserve(ctx, plan, basis, C));
  const long N = (long)nm * plan->N, Cq = (long)nm * C * basis->q, CM = (long)C * plan->M, X = N + Cq;
  const long CMs = std::max(CM, 1L);
  SolverGraph* g = cache_find(ctx, nm == 1 ? 0 : 100 + nm, plan, basis, C, prec, prm, sizeof(*prm));
  if (!g) {
    g = new SolverGraph();
    g->kind = nm == 1 ? 0 : 100 + nm;
    g->plan = plan;
    g->basis = basis;
    g->C = C;
    g->prec = prec;
    g->key.assign((const unsigned char*)prm, (const unsigned char*)prm + sizeof(*prm));
    // x, dx, res, d, Ad, h, b, spare (X each); ys, yt, r (CM each); in_y, out_alpha, out_p
    mpi_status st = alloc_solver(ctx, g->mem, 8 * X + 4 * CMs + Cq + N, prm->n_outer + 1, g->sv, &g->base, &g->dbase);
    if (st) {
      delete g;
      return st;
    }
    g->in_y = g->base + 8 * X + 3 * CMs;
    g->out_alpha = g->in_y + CMs;
    g->out_p = g->out_alpha + Cq;
    g->hist = g->dbase;
    g->work = ctx->work;
    if ((st = tune_line_passes(ctx, plan, C))) {
      delete g;
      return st;
    }
    st = capture(ctx, g, [&]() {
      return irgn_body(ctx, plan, basis, nm, C, prm, prec, g->sv, g->base, g->in_y, g->out_alpha, g->out_p,
                       g->hist);
    });
    if (st) {
      delete g;
      return st;
    }
    cache_insert(ctx, g);
  }
  if (CM > 0)
    TRY(cuda_check(ctx, cudaMemcpyAsync(g->in_y, y, CM * sizeof(float2), cudaMemcpyDeviceToDevice, ctx->stream),
                   "input copy"));
  TRY(launch_graph(ctx, g));
  TRY(cuda_check(ctx, cudaMemcpyAsync(alpha_out, g->out_alpha, Cq * sizeof(float2), cudaMemcpyDeviceToDevice,
                                      ctx->stream), "output copy"));
  TRY(cuda_check(ctx, cudaMemcpyAsync(p_out, g->out_p, N * sizeof(float2), cudaMemcpyDeviceToDevice, ctx->stream),
                 "output copy"));
  if (resid_out) {
    if (CM > 0)
      TRY(cuda_check(ctx, cudaMemcpyAsync(resid_out, g->hist, (prm->n_outer + 1) * sizeof(double),
                                          cudaMemcpyDeviceToHost, ctx->stream), "history copy"));
    else
      for (int i = 0; i <= prm->n_outer; ++i) resid_out[i] = 0.0;
  }
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sm_estimate");
}

}  // namespace

extern "C" mpi_status mpi_sm_estimate(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, const mpi_c32* y,
                                      int C, const mpi_irgn_params* prm, mpi_c32* alpha_out, mpi_c32* p_out,
                                      double* resid_out, mpi_precision prec) {
  return sm_estimate_impl(ctx, plan, basis, 1, y, C, prm, alpha_out, p_out, resid_out, prec);
}

extern "C" mpi_status mpi_sm_estimate_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                                           const mpi_c32* y, int C, const mpi_irgn_params* prm, mpi_c32* alpha_out,
                                           mpi_c32* p_out, double* resid_out, mpi_precision prec) {
  return sm_estimate_impl(ctx, plan, basis, M, y, C, prm, alpha_out, p_out, resid_out, prec);
}

// ------------------------------------------------------------------- MPI-L

namespace {

// Enqueue the ADMM solve over T frames (T = 1: MPI-L, Eqs. 8-11; T > 1: the
// dynamic problem with a spatiotemporal regulariser, frame t sampled by
// plans[t], the maps shared, TV over the (t, y, x) grid of 2D frames).
// Inputs: alpha (C x q), y (T x C x M), eps_d (T C, device).  Outputs: p_out
// (T x N), hist (n_outer x 3).
mpi_status admm_body(mpi_ctx* ctx, const mpi_plan* const* plans, int T, const mpi_basis* basis, int C,
                     const mpi_admm_params* prm, mpi_precision prec, Solver& sv, float2* base, double* dx,
                     const mpi_c32* A, const float2* yc, const double* eps_d, float2* p_out, double* hist) {
  Grid3 g = grid_of(plans[0]);
  if (T > 1) {
    g.nz = T;
    g.nd = 3;
  }
  const long N1 = plans[0]->N, M = plans[0]->M, CM1 = (long)C * M;
  const long N = (long)T * N1, TC = (long)T * C, CM = TC * M, CMs = std::max(CM, 1L);
  float2 *p = base, *p_prev = p + N, *u0 = p_prev + N, *z0 = u0 + N, *rhs = z0 + N, *t = rhs + N;
  float2 *r = t + N, *d = r + N, *Ad = d + N, *tvx = Ad + N, *P = tvx + N, *R = P + (size_t)g.nd * N;
  float2 *uk = R + (size_t)g.nd * N, *zk = uk + CMs, *Apk = zk + CMs, *Apk_prev = Apk + CMs, *wk = Apk_prev + CMs;
  (void)tvx;
  double* fball = dx;
  double* bpart = fball + TC;
  TRY(sv.fill(p, make_float2(0.f, 0.f), N));
  TRY(sv.fill(u0, make_float2(0.f, 0.f), N));
  if (CM > 0) {
    TRY(sv.fill(uk, make_float2(0.f, 0.f), CM));
    TRY(sv.fill(Apk, make_float2(0.f, 0.f), CM));
  }
  TRY(sv.set(S_RHO, prm->rho0));
  const unsigned ball_blocks = (unsigned)std::max(1L, std::min((M + kVecThreads - 1) / kVecThreads, (long)kRedBlocks));

  // MIXED: BF16 operators in the CG iterations; FP32 for the constraint-side
  // products (A p for the projections and the dual update), the right-hand
  // side and the CG's starting residual (each p-update warm-starts from the
  // previous p, so every outer step refines it against an FP32 residual).
  const mpi_precision pin = prec == MPI_PREC_MIXED ? MPI_PREC_BF16 : prec;
  const mpi_precision pout = prec == MPI_PREC_MIXED ? MPI_PREC_FP32 : prec;
  auto normal = [&](const float2* v, float2* out, mpi_precision pr) -> mpi_status {
    // out = v + S^H F^H F S v, frame by frame
    for (int t = 0; t < T; ++t) {
      TRY(mpi_forward(ctx, plans[t], basis, A, C, (const mpi_c32*)(v + t * N1), (mpi_c32*)(wk + t * CM1), pr));
      TRY(mpi_adjoint(ctx, plans[t], basis, A, C, (const mpi_c32*)(wk + t * CM1), (mpi_c32*)(out + t * N1), pr));
    }
    return sv.lincomb(out, out, 1.f, v, 1.f, N);
  };

  for (int it = 0; it < prm->n_outer; ++it) {
    // z0 = prox_{TV/rho}(p + u0)
    TRY(sv.lincomb(t, p, 1.f, u0, 1.f, N));
    TRY(tv_prox_run(sv, g, N, t, prm->n_tv, 1, 0.f, P, R, z0));
    // zk = Pi(F S p + uk)
    if (CM > 0) {
      MPI_PROF(ctx, KF_SOLVER);
      k_ball_norm_partial<<<dim3(ball_blocks, (unsigned)TC), kVecThreads, 0, ctx->stream>>>(Apk, uk, yc, (int)M,
                                                                                            bpart);
      MPI_LAUNCH_CHECK(ctx, "k_ball_norm_partial");
      MPI_PROF(ctx, KF_SOLVER);
      k_ball_factor<<<1, kVecThreads, 0, ctx->stream>>>(bpart, ball_blocks, (int)TC, eps_d, fball);
      MPI_LAUNCH_CHECK(ctx, "k_ball_factor");
      MPI_PROF(ctx, KF_SOLVER);
      k_ball_apply<<<grid_for(CM), kVecThreads, 0, ctx->stream>>>(Apk, uk, yc, (int)TC, (int)M, fball, zk);
      MPI_LAUNCH_CHECK(ctx, "k_ball_apply");
      TRY(sv.lincomb(wk, zk, 1.f, uk, -1.f, CM));
      for (int t = 0; t < T; ++t)
        TRY(mpi_adjoint(ctx, plans[t], basis, A, C, (const mpi_c32*)(wk + t * CM1), (mpi_c32*)(rhs + t * N1), pout));
      TRY(sv.lincomb(rhs, rhs, 1.f, z0, 1.f, N));
      TRY(sv.lincomb(rhs, rhs, 1.f, u0, -1.f, N));
    } else {
      TRY(sv.lincomb(rhs, z0, 1.f, u0, -1.f, N));
    }
    // p = (I + S^H F^H F S)^{-1} rhs by CG from the previous p
    TRY(sv.lincomb(p_prev, p, 1.f, nullptr, 0.f, N));
    if (CM > 0) TRY(sv.lincomb(Apk_prev, Apk, 1.f, nullptr, 0.f, CM));
    TRY(normal(p, Ad, pout));
    TRY(sv.lincomb(r, rhs, 1.f, Ad, -1.f, N));
    TRY(sv.lincomb(d, r, 1.f, nullptr, 0.f, N));
    TRY(sv.dot(r, nullptr, N, FIN_STORE, S_RR));
    for (int k = 0; k < prm->n_cg; ++k) {
      TRY(normal(d, t, pin));
      MPI_PROF(ctx, KF_SOLVER);
      k_normal_finish<<<kRedBlocks, kVecThreads, 0, ctx->stream>>>(t, d, N, N, 0.f, 0.f, Ad, sv.partials);
      MPI_LAUNCH_CHECK(ctx, "k_normal_finish");
      TRY(sv.fin(FIN_CG_ALPHA));
      MPI_PROF(ctx, KF_SOLVER);
      k_cg_update<<<kRedBlocks, kVecThreads, 0, ctx->stream>>>(p, r, d, Ad, N, sv.S, sv.partials);
      MPI_LAUNCH_CHECK(ctx, "k_cg_update");
      TRY(sv.fin(FIN_CG_BETA));
      MPI_PROF(ctx, KF_SOLVER);
      k_cg_dir<<<grid_for(N), kVecThreads, 0, ctx->stream>>>(d, r, N, sv.S);
      MPI_LAUNCH_CHECK(ctx, "k_cg_dir");
    }
    // dual update u += A p - z
    MPI_PROF(ctx, KF_SOLVER);
    k_dual_update<<<grid_for(N), kVecThreads, 0, ctx->stream>>>(u0, p, z0, N);
    MPI_LAUNCH_CHECK(ctx, "k_dual_update");
    if (CM > 0) {
      for (int t = 0; t < T; ++t)
        TRY(mpi_forward(ctx, plans[t], basis, A, C, (const mpi_c32*)(p + t * N1), (mpi_c32*)(Apk + t * CM1), pout));
      MPI_PROF(ctx, KF_SOLVER);
      k_dual_update<<<grid_for(CM), kVecThreads, 0, ctx->stream>>>(uk, Apk, zk, CM);
      MPI_LAUNCH_CHECK(ctx, "k_dual_update");
    }
    // residuals and rho
    TRY(sv.diffnorm(p, z0, N, FIN_STORE, S_R2));
    if (CM > 0) TRY(sv.diffnorm(Apk, zk, CM, FIN_ADD, S_R2));
    TRY(sv.diffnorm(p, p_prev, N, FIN_STORE, S_S2));
    if (CM > 0) TRY(sv.diffnorm(Apk, Apk_prev, CM, FIN_ADD, S_S2));
    MPI_PROF(ctx, KF_SOLVER);
    k_rho_update<<<1, 1, 0, ctx->stream>>>(sv.S, prm->mu, prm->tau, hist, it);
    MPI_LAUNCH_CHECK(ctx, "k_rho_update");
    TRY(sv.scale_dev(u0, u0, N, S_UFAC, 0));
    if (CM > 0) TRY(sv.scale_dev(uk, uk, CM, S_UFAC, 0));
  }
  return sv.lincomb(p_out, p, 1.f, nullptr, 0.f, N);
}

}  // namespace

namespace {

mpi_status image_solve_impl(mpi_ctx* ctx, const mpi_plan* const* plans, int T, const mpi_basis* basis,
                            const mpi_c32* alpha, int C, const mpi_c32* y, const double* eps,
                            const mpi_admm_params* prm, mpi_c32* p_out, double* hist_out, mpi_precision prec) {
  if (!ctx) return MPI_ERR_ARG;
  if (!plans || T < 1 || !plans[0] || !basis || !alpha || !eps || !prm || !p_out || C < 1 ||
      (plans[0]->M > 0 && !y))
    return set_err(ctx, MPI_ERR_ARG, "image_solve: bad argument");
  for (int t = 1; t < T; ++t) {
    const mpi_plan* a = plans[0];
    const mpi_plan* b = plans[t];
    if (!b) return set_err(ctx, MPI_ERR_ARG, "image_solve: null plan");
    if (b->ndim != 2 || a->ndim != 2 || b->ny != a->ny || b->nx != a->nx || b->M != a->M || b->ctx != a->ctx)
      return set_err(ctx, MPI_ERR_SHAPE, "dynamic image_solve: frames need 2D plans of one grid and sample count");
  }
  if (prm->n_outer < 0 || prm->n_cg < 0 || prm->n_tv < 0 || !(prm->rho0 > 0) || !(prm->tau > 0))
    return set_err(ctx, MPI_ERR_ARG, "image_solve: bad parameters");
  const long TC = (long)T * C;
  for (long c = 0; c < TC; ++c)
    if (!(eps[c] >= 0)) return set_err(ctx, MPI_ERR_ARG, "eps must be >= 0");
  cudaSetDevice(ctx->device);
  for (int t = 0; t < T; ++t) TRY(mpi_ctx_reserve(ctx, plans[t], basis, C));
  Grid3 gr = grid_of(plans[0]);
  if (T > 1) gr.nd = 3;
  const long N = (long)T * plans[0]->N, CM = TC * plans[0]->M, CMs = std::max(CM, 1L), Cq = (long)C * basis->q;
  // the cache key: the parameters, then the frame count and every frame's plan
  std::vector<unsigned char> key((const unsigned char*)prm, (const unsigned char*)prm + sizeof(*prm));
  key.insert(key.end(), (const unsigned char*)&T, (const unsigned char*)&T + sizeof(T));
  key.insert(key.end(), (const unsigned char*)plans, (const unsigned char*)(plans + T));
  SolverGraph* g = cache_find(ctx, 1, plans[0], basis, C, prec, key.data(), key.size());
  if (!g) {
    g = new SolverGraph();
    g->kind = 1;
    g->plan = plans[0];
    g->others.assign(plans, plans + T);
    g->basis = basis;
    g->C = C;
    g->prec = prec;
    g->key = key;
    // image side: 10 N + 2 nd N; k-space: 5 CM; inputs y (CM), alpha (Cq); output p (N)
    const size_t elems = 10 * N + 2 * (size_t)gr.nd * N + 5 * CMs + CMs + Cq + N;
    const size_t extra = 2 * (size_t)TC + (size_t)TC * kRedBlocks + 3 * (size_t)prm->n_outer + TC + 8;
    mpi_status st = alloc_solver(ctx, g->mem, elems, extra, g->sv, &g->base, &g->dbase);
    if (st) {
      delete g;
      return st;
    }
    float2* io = g->base + 10 * N + 2 * (size_t)gr.nd * N + 5 * CMs;
    g->in_y = io;
    g->in_alpha = io + CMs;
    g->out_p = g->in_alpha + Cq;
    double* scratch = g->dbase;                                     // fball, bpart
    g->hist = scratch + 2 * (size_t)TC + (size_t)TC * kRedBlocks;  // [n_outer][3]
    g->in_eps = g->hist + 3 * (size_t)prm->n_outer;
    g->work = ctx->work;
    for (int t = 0; t < T && st == MPI_OK; ++t) st = tune_line_passes(ctx, plans[t], C);
    if (st) {
      delete g;
      return st;
    }
    st = capture(ctx, g, [&]() {
      return admm_body(ctx, plans, T, basis, C, prm, prec, g->sv, g->base, scratch, (const mpi_c32*)g->in_alpha,
                       g->in_y, g->in_eps, g->out_p, g->hist);
    });
    if (st) {
      delete g;
      return st;
    }
    cache_insert(ctx, g);
  }
  TRY(cuda_check(ctx, cudaMemcpyAsync(g->in_alpha, alpha, Cq * sizeof(float2), cudaMemcpyDeviceToDevice, ctx->stream),
                 "input copy"));
  if (CM > 0)
    TRY(cuda_check(ctx, cudaMemcpyAsync(g->in_y, y, CM * sizeof(float2), cudaMemcpyDeviceToDevice, ctx->stream),
                   "input copy"));
  TRY(cuda_check(ctx, cudaMemcpyAsync(g->in_eps, eps, TC * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
                 "eps copy"));
  TRY(launch_graph(ctx, g));
  TRY(cuda_check(ctx, cudaMemcpyAsync(p_out, g->out_p, N * sizeof(float2), cudaMemcpyDeviceToDevice, ctx->stream),
                 "output copy"));
  if (hist_out && prm->n_outer > 0)
    TRY(cuda_check(ctx, cudaMemcpyAsync(hist_out, g->hist, 3 * (size_t)prm->n_outer * sizeof(double),
                                        cudaMemcpyDeviceToHost, ctx->stream), "history copy"));
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "image_solve");
}

}  // namespace

extern "C" mpi_status mpi_image_solve(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                      const mpi_c32* alpha, int C, const mpi_c32* y, const double* eps,
                                      const mpi_admm_params* prm, mpi_c32* p_out, double* hist_out,
                                      mpi_precision prec) {
  return image_solve_impl(ctx, &plan, 1, basis, alpha, C, y, eps, prm, p_out, hist_out, prec);
}

extern "C" mpi_status mpi_image_solve_dynamic(mpi_ctx* ctx, const mpi_plan* const* plans, int T,
                                              const mpi_basis* basis, const mpi_c32* alpha, int C, const mpi_c32* y,
                                              const double* eps, const mpi_admm_params* prm, mpi_c32* p_out,
                                              double* hist_out, mpi_precision prec) {
  return image_solve_impl(ctx, plans, T, basis, alpha, C, y, eps, prm, p_out, hist_out, prec);
}

void solver_cache_forget(mpi_ctx* ctx, const void* object) {
  if (!ctx || !ctx->solver_cache) return;
  SolverCache* c = (SolverCache*)ctx->solver_cache;
  for (size_t i = 0; i < c->entries.size();) {
    const std::vector<const mpi_plan*>& o = c->entries[i]->others;
    if (c->entries[i]->plan == object || c->entries[i]->basis == object ||
        std::find(o.begin(), o.end(), (const mpi_plan*)object) != o.end()) {
      delete c->entries[i];
      c->entries.erase(c->entries.begin() + i);
    } else {
      ++i;
    }
  }
}

void solver_cache_clear(mpi_ctx* ctx) {
  if (!ctx || !ctx->solver_cache) return;
  SolverCache* c = (SolverCache*)ctx->solver_cache;
  for (SolverGraph* e : c->entries) delete e;
  delete c;
  ctx->solver_cache = nullptr;
}

extern "C" mpi_status mpi_tv_prox(mpi_ctx* ctx, const mpi_plan* plan, const mpi_c32* v, double lam, int n_iter,
                                  mpi_c32* x) {
  if (!ctx) return MPI_ERR_ARG;
  if (!plan || !v || !x || n_iter < 0 || !(lam >= 0)) return set_err(ctx, MPI_ERR_ARG, "tv_prox: bad argument");
  cudaSetDevice(ctx->device);
  const Grid3 g = grid_of(plan);
  const long N = plan->N;
  SolverMem mem;
  Solver sv;
  float2* base;
  double* dx;
  TRY(alloc_solver(ctx, mem, 2 * (size_t)g.nd * N, 0, sv, &base, &dx));
  if (lam == 0) {
    TRY(sv.lincomb((float2*)x, (const float2*)v, 1.f, nullptr, 0.f, N));
  } else {
    TRY(tv_prox_run(sv, g, N, (const float2*)v, n_iter, 0, (float)lam, base, base + (size_t)g.nd * N, (float2*)x));
  }
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "tv_prox");
}

// --------------------------------------------------------------- projection

extern "C" mpi_status mpi_basis_project(mpi_ctx* ctx, const mpi_basis* basis, const mpi_c32* maps, int C,
                                        mpi_c32* alpha) {
  if (!ctx) return MPI_ERR_ARG;
  if (!basis || !maps || !alpha || C < 1) return set_err(ctx, MPI_ERR_ARG, "basis_project: bad argument");
  cudaSetDevice(ctx->device);
  const int q = basis->q, N = basis->N;
  double2* buf = nullptr;
  const size_t elems = (size_t)q * q + (size_t)C * q;
  cudaError_t e = cudaMalloc(&buf, elems * sizeof(double2) + sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_OOM, "projection buffers");
  }
  double2* G = buf;
  double2* rhs = buf + (size_t)q * q;
  int* status = (int*)(rhs + (size_t)C * q);
  mpi_status st = MPI_OK;
  e = cudaMemsetAsync(status, 0, sizeof(int), ctx->stream);
  if (e == cudaSuccess) {
    MPI_PROF(ctx, KF_OTHER);
    k_gram<<<dim3((q + 7) / 8, q), dim3(32, 8), 0, ctx->stream>>>(basis->U, N, q, G);
    ctx->launches++;
    prof_end(ctx, "k_gram");
    MPI_PROF(ctx, KF_OTHER);
    k_uh_s<<<dim3((C + 7) / 8, q), dim3(32, 8), 0, ctx->stream>>>(basis->U, N, q, (const float2*)maps, C, rhs);
    ctx->launches++;
    prof_end(ctx, "k_uh_s");
    MPI_PROF(ctx, KF_OTHER);
    k_cholesky_solve<<<1, 1024, 0, ctx->stream>>>(G, q, rhs, C, (float2*)alpha, status);
    ctx->launches++;
    prof_end(ctx, "k_cholesky_solve");
    e = cudaGetLastError();
  }
  int hstat = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) st = cuda_check(ctx, e, "basis_project");
  else if (hstat) st = set_err(ctx, MPI_ERR_NOT_CONVERGED, "Gram matrix not positive definite");
  cudaFree(buf);
  return st;
}
