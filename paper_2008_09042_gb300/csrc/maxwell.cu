// Maxwell basis of a 2D slice on the GPU (Maxwell Regularization section:
// Eqs. 15-18, the randomized range sampling with random boundary excitations
// of Fig. 1).
//
//  1. Field synthesis (FP64).  Every source site s carries three electric and
//     three magnetic point dipoles; column 6 s + t of B is the circularly
//     polarised magnetic field b = (H_x - i H_y) / sqrt(2) of dipole t at the
//     pixel centroids, through the free-space dyadic Green's functions with
//     g = exp(-j k R) / (4 pi R):
//        electric current element along e:  H = grad g x e
//        magnetic current element m:        H = (grad grad g + k^2 g) m / (j k)
//     (the magnetic block scaled by the free-space impedance; k = 2 pi f / c0).
//     Identically zero fields (three per site for sites in the slice plane)
//     are dropped, with their rows of Omega, before step 2.
//  2. Y = B Omega with the caller's random excitations Omega (6 D x L).  Its
//     q leading left singular vectors are the basis (Eq. 16: the truncation
//     error is sigma_{q+1}).  They are computed without forming Y:
//       a. B = Q R, Householder QR of the N x 6D field matrix on the GPU
//          (unblocked, FP64, backward stable, so singular values down to
//          ~1e-16 sigma_1 keep their subspaces where the gaps allow);
//       b. X = R Omega (6D x L) on the GPU; Y = Q X, so sigma(Y) = sigma(X)
//          and the left singular vectors of Y are Q times those of X;
//       c. one-sided Jacobi on the columns of X^H (round-robin pairs, one
//          CTA per pair, FP64): X^H V = U' Sigma, so X = V Sigma U'^H and the
//          columns of V are the left singular vectors of X;
//       d. U = Q [V_q; 0], applying the reflectors to the q leading columns of
//          V (ordered by singular value), then rounded to complex64.
// All FP64 reductions run in a fixed order, so the result is reproducible.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "mpi_internal.h"
#include "ptx.cuh"

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kRowsW = 512;     // rows per CTA of the reflector dot products
constexpr int kThreadsW = 256;  // 8 warps
constexpr int kNormBlocks = 256;
constexpr int kColsW = 32;      // target columns per CTA of the reflector dot products

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zcmul(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
// z / (j k) = -j z / k
__device__ __forceinline__ double2 zdiv_jk(double2 z, double k) { return make_double2(z.y / k, -z.x / k); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Field of dipole t (0-5) of site s at pixel n.  With B: written to packed
// column pos[6 s + t] (skipped where pos = -1), column-major with ld = N.
// Without B: |b|^2 summed per dipole into norm2 (per-CTA sums, then one
// atomic add per CTA and dipole; only used to find the identically zero fields).
__global__ void k_dipole_fields(double2* __restrict__ B, const int* __restrict__ pos, double* __restrict__ norm2,
                                int N, int nz, int ny, int nx, double dz, double dy, double dx,
                                const double* __restrict__ src, double k) {
  __shared__ double s_n2[6][8];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  double2 b[6];
  if (n < N) {
    const int ix = n % nx, t = n / nx, iy = t % ny, iz = t / ny;  // raster order, x fastest, z slowest
    const double px = (ix - 0.5 * nx + 0.5) * dx, py = (iy - 0.5 * ny + 0.5) * dy, pz = (iz - 0.5 * nz + 0.5) * dz;
    const double rx = px - src[3 * s + 0], ry = py - src[3 * s + 1], rz = pz - src[3 * s + 2];
    const double R = sqrt(rx * rx + ry * ry + rz * rz);
    const double ux = rx / R, uy = ry / R, uz = rz / R;
    double sn, cs;
    sincos(k * R, &sn, &cs);
    const double inv4piR = 1.0 / (4.0 * kPi * R);
    const double2 g = make_double2(cs * inv4piR, -sn * inv4piR);  // exp(-j k R) / (4 pi R)
    const double2 jk1 = make_double2(1.0 / R, k);                   // j k + 1 / R
    const double2 g1 = zscale(zmul(jk1, g), -1.0);                  // dg/dR
    const double2 jk1sq = zmul(jk1, jk1);
    const double2 g2 = zmul(make_double2(jk1sq.x + 1.0 / (R * R), jk1sq.y), g);  // d2g/dR2
    const double is2 = 0.70710678118654752440;
    // electric elements: H = g1 (u x e); b = g1 (c_x - i c_y) / sqrt 2 with c = u x e
    b[0] = zscale(zmul(g1, make_double2(0.0, -uz)), is2);   // e = x: c = (0, uz, -uy)
    b[1] = zscale(g1, -uz * is2);                            // e = y: c = (-uz, 0, ux)
    b[2] = zscale(zmul(g1, make_double2(uy, ux)), is2);     // e = z: c = (uy, -ux, 0)
    // magnetic elements: H = a (u . m) u + c m, a = (g2 - g1 / R) / (j k), c = (g1 / R + k^2 g) / (j k)
    const double2 a = zdiv_jk(zsub(g2, zscale(g1, 1.0 / R)), k);
    const double2 c = zdiv_jk(zadd(zscale(g1, 1.0 / R), zscale(g, k * k)), k);
    const double2 uxy = make_double2(ux, -uy);  // u_x - i u_y
    b[3] = zscale(zadd(zscale(zmul(a, uxy), ux), c), is2);
    b[4] = zscale(zadd(zscale(zmul(a, uxy), uy), zmul(c, make_double2(0.0, -1.0))), is2);
    b[5] = zscale(zscale(zmul(a, uxy), uz), is2);
  } else {
#pragma unroll
    for (int t = 0; t < 6; ++t) b[t] = make_double2(0.0, 0.0);
  }
  if (B) {
    if (n < N) {
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const int c = pos[6 * s + t];
        if (c >= 0) B[(size_t)c * N + n] = b[t];
      }
    }
    return;
  }
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const double v = warp_sum(b[t].x * b[t].x + b[t].y * b[t].y);
    if ((threadIdx.x & 31) == 0) s_n2[t][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) v += s_n2[threadIdx.x][w2];
    atomicAdd(&norm2[6 * s + threadIdx.x], v);
  }
}

// Partial sums of |A[j][i]|^2 over rows i > j (grid-stride, fixed order).
__global__ void k_hh_norm(const double2* __restrict__ A, int N, int j, double* __restrict__ part) {
  __shared__ double s_w[8];
  const double2* col = A + (size_t)j * N;
  double acc = 0.0;
  for (long i = (long)j + 1 + (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
    const double2 v = col[i];
    acc += v.x * v.x + v.y * v.y;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
    part[blockIdx.x] = t;
  }
}

// The reflector of column j (the convention of LAPACK's zlarfg): beta real,
// H = I - tau v v^H with v_j = 1 and H^H [alpha; x] = [beta; 0].  Writes
// tau[j], beta into A[j][j] and the scale 1 / (alpha - beta) of x into *scal.
__global__ void k_hh_make(double2* __restrict__ A, int N, int j, const double* __restrict__ part, int nb,
                          double2* __restrict__ tau, double2* __restrict__ scal) {
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) t += part[b];
  t = warp_sum(t);
  if (threadIdx.x != 0) return;
  const double2 alpha = A[(size_t)j * N + j];
  if (t == 0.0 && alpha.y == 0.0) {  // nothing to annihilate: H = I
    tau[j] = make_double2(0.0, 0.0);
    *scal = make_double2(0.0, 0.0);
    return;
  }
  const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + t);
  const double beta = -copysign(nrm, alpha.x);
  tau[j] = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
  const double2 d = make_double2(alpha.x - beta, alpha.y);
  const double dd = d.x * d.x + d.y * d.y;
  *scal = make_double2(d.x / dd, -d.y / dd);
  A[(size_t)j * N + j] = make_double2(beta, 0.0);
}

// x -> v = x / (alpha - beta) for rows i > j of column j (after k_hh_make).
__global__ void k_hh_scale(double2* __restrict__ A, int N, int j, const double2* __restrict__ tau,
                           const double2* __restrict__ scal) {
  const double2 t = tau[j];
  if (t.x == 0.0 && t.y == 0.0) return;  // H_j = I: x is already zero
  const long i = (long)j + 1 + (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double2* p = A + (size_t)j * N + i;
  *p = zmul(*p, *scal);
}

// w_k = sum_{i >= j} conj(v_i) T[k][i] for target columns k in [c0, c0 + nc):
// per-CTA partials over rows [j + 512 bx, + 512) and columns [c0 + 32 by, + 32)
// (four per warp); nothing to do when tau_j = 0 (H_j = I).
__global__ void __launch_bounds__(kThreadsW) k_refl_w(const double2* __restrict__ A, const double2* __restrict__ T,
                                                     int N, int j, int c0, int nc, const double2* __restrict__ tau,
                                                     double2* __restrict__ part) {
  const double2 t = tau[j];
  if (t.x == 0.0 && t.y == 0.0) return;
  __shared__ double2 s_v[kRowsW];
  const long r0 = (long)j + (long)blockIdx.x * kRowsW;
  const int rows = (int)(((long)N - r0) < kRowsW ? ((long)N - r0) : kRowsW);
  const double2* vcol = A + (size_t)j * N;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const long i = r0 + r;
    s_v[r] = (i == j) ? make_double2(1.0, 0.0) : vcol[i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kend = min(nc, (int)(blockIdx.y + 1) * kColsW);
  for (int kk = blockIdx.y * kColsW + warp; kk < kend; kk += kThreadsW / 32) {
    const double2* tc = T + (size_t)(c0 + kk) * N + r0;
    double ax = 0.0, ay = 0.0;
    for (int r = lane; r < rows; r += 32) {
      const double2 p = zcmul(s_v[r], tc[r]);
      ax += p.x;
      ay += p.y;
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    if (lane == 0) part[(size_t)blockIdx.x * nc + kk] = make_double2(ax, ay);
  }
}

__global__ void k_refl_wsum(const double2* __restrict__ part, int nb, int nc, int j, const double2* __restrict__ tau,
                            double2* __restrict__ w) {
  const double2 t = tau[j];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nc || (t.x == 0.0 && t.y == 0.0)) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nb; ++b) s = zadd(s, part[(size_t)b * nc + k]);
  w[k] = s;
}

// T[k][i] -= t v_i w_k for rows i >= j, t = conj(tau_j) (the QR's H^H) or
// tau_j (applying Q); eight target columns per thread.
__global__ void k_refl_update(const double2* __restrict__ A, double2* __restrict__ T, int N, int j, int c0, int nc,
                              const double2* __restrict__ w, const double2* __restrict__ tau, int conj_tau) {
  const long i = (long)j + (long)blockIdx.x * blockDim.x + threadIdx.x;
  double2 t = tau[j];
  if (i >= N || (t.x == 0.0 && t.y == 0.0)) return;
  const double2 v = (i == j) ? make_double2(1.0, 0.0) : A[(size_t)j * N + i];
  if (conj_tau) t.y = -t.y;
  const double2 tv = zmul(t, v);
  const int k0 = blockIdx.y * 8, k1 = min(nc, k0 + 8);
  for (int kk = k0; kk < k1; ++kk) {
    double2* p = T + (size_t)(c0 + kk) * N + i;
    *p = zsub(*p, zmul(tv, w[kk]));
  }
}

// M = X^H with X = R Omega: column a of M (length L) holds conj(X[a][:]),
// X[a][l] = sum_{i >= a} R[a][i] Omega[i][l], R[a][i] = A[i][a].
__global__ void k_small_x(const double2* __restrict__ A, int N, int n, const double2* __restrict__ Om, int L,
                          double2* __restrict__ M) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (l >= L) return;
  double2 s = make_double2(0.0, 0.0);
  for (int i = a; i < n; ++i) s = zadd(s, zmul(A[(size_t)i * N + a], Om[(size_t)i * L + l]));
  M[(size_t)a * L + l] = make_double2(s.x, -s.y);
}

// One round-robin step of one-sided Jacobi (Hestenes) on the n columns of M (length L),
// accumulating the same rotations into V (n x n, column-major): pair p of step
// `step` is (step, n - 1) for p = 0 and ((step + p) mod (n - 1), (step - p)
// mod (n - 1)) otherwise, so every column meets every other once per n - 1 steps.
__global__ void __launch_bounds__(128) k_jacobi_step(double2* __restrict__ M, int L, double2* __restrict__ V, int n,
                                                     int step, double tol, double floor2, int* __restrict__ rotated) {
  __shared__ double s_red[4][4];
  __shared__ double s_rot[5];
  const int m = n - 1, p = blockIdx.x;
  int a, b;
  if (p == 0) {
    a = step % m;
    b = n - 1;
  } else {
    a = (step + p) % m;
    b = (step - p + m) % m;
  }
  double2* ma = M + (size_t)a * L;
  double2* mb = M + (size_t)b * L;
  double al = 0.0, be = 0.0, gx = 0.0, gy = 0.0;
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const double2 x = ma[l], y = mb[l];
    al += x.x * x.x + x.y * x.y;
    be += y.x * y.x + y.y * y.y;
    const double2 g = zcmul(x, y);
    gx += g.x;
    gy += g.y;
  }
  al = warp_sum(al);
  be = warp_sum(be);
  gx = warp_sum(gx);
  gy = warp_sum(gy);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_red[warp][0] = al;
    s_red[warp][1] = be;
    s_red[warp][2] = gx;
    s_red[warp][3] = gy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A2 = 0.0, B2 = 0.0, Gx = 0.0, Gy = 0.0;
    for (int w = 0; w < 4; ++w) {
      A2 += s_red[w][0];
      B2 += s_red[w][1];
      Gx += s_red[w][2];
      Gy += s_red[w][3];
    }
    const double ag = hypot(Gx, Gy);
    s_rot[0] = 0.0;
    // a pair with a column at the rounding floor of M (|m|^2 <= floor2) counts
    // as converged: such a column is noise, and rotating it moves the other by
    // less than the rounding of M
    if (fmin(A2, B2) > floor2 && ag > tol * sqrt(A2) * sqrt(B2)) {
      const double zeta = (B2 - A2) / (2.0 * ag);
      const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
      const double c = 1.0 / sqrt(1.0 + t * t);
      s_rot[0] = 1.0;
      s_rot[1] = c;
      s_rot[2] = c * t;
      s_rot[3] = Gx / ag;  // conj(gamma) / |gamma|, the phase taken off column b
      s_rot[4] = -Gy / ag;
      *rotated = 1;
    }
  }
  __syncthreads();
  if (s_rot[0] == 0.0) return;
  const double c = s_rot[1], s = s_rot[2];
  const double2 e = make_double2(s_rot[3], s_rot[4]);
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    const double2 x = ma[l], y = zmul(e, mb[l]);
    ma[l] = zsub(zscale(x, c), zscale(y, s));
    mb[l] = zadd(zscale(x, s), zscale(y, c));
  }
  double2* va = V + (size_t)a * n;
  double2* vb = V + (size_t)b * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 x = va[i], y = zmul(e, vb[i]);
    va[i] = zsub(zscale(x, c), zscale(y, s));
    vb[i] = zadd(zscale(x, s), zscale(y, c));
  }
}

__global__ void k_identity(double2* __restrict__ V, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * n) V[e] = make_double2((e % n) == (e / n) ? 1.0 : 0.0, 0.0);
}

__global__ void k_col_norms(const double2* __restrict__ M, int L, double* __restrict__ sig) {
  __shared__ double s_w[4];
  const double2* col = M + (size_t)blockIdx.x * L;
  double acc = 0.0;
  for (int l = threadIdx.x; l < L; l += blockDim.x) acc += col[l].x * col[l].x + col[l].y * col[l].y;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) sig[blockIdx.x] = sqrt(s_w[0] + s_w[1] + s_w[2] + s_w[3]);
}

// Z[k][i] = V[order[k]][i] for i < n, 0 below (the N x q start of U = Q [V_q; 0]).
__global__ void k_init_z(const double2* __restrict__ V, int n, const int* __restrict__ order, int N,
                         double2* __restrict__ Z) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= N) return;
  Z[(size_t)k * N + i] = i < n ? V[(size_t)order[k] * n + i] : make_double2(0.0, 0.0);
}

__global__ void k_z_to_c64(const double2* __restrict__ Z, size_t total, float2* __restrict__ U) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) U[e] = make_float2((float)Z[e].x, (float)Z[e].y);
}

struct SweepGraph {
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~SweepGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
  }
};

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// H_j applied to target columns [c0, c0 + nc) of T, rows >= j: the dot
// products, their fixed-order sums and the update (each a no-op when tau_j = 0).
mpi_status apply_reflector(mpi_ctx* ctx, const double2* A, double2* T, int N, int j, int c0, int nc,
                           const double2* tau, int conj_tau, double2* part, double2* w) {
  if (nc == 0) return MPI_OK;
  cudaStream_t st = ctx->stream;
  const int nb = (int)(((long)N - j + kRowsW - 1) / kRowsW);
  MPI_PROF(ctx, KF_OTHER);
  k_refl_w<<<dim3((unsigned)nb, (unsigned)((nc + kColsW - 1) / kColsW)), kThreadsW, 0, st>>>(A, T, N, j, c0, nc, tau,
                                                                                           part);
  MPI_LAUNCH_CHECK(ctx, "k_refl_w");
  MPI_PROF(ctx, KF_OTHER);
  k_refl_wsum<<<(nc + 127) / 128, 128, 0, st>>>(part, nb, nc, j, tau, w);
  MPI_LAUNCH_CHECK(ctx, "k_refl_wsum");
  const dim3 g((unsigned)(((long)N - j + 255) / 256), (unsigned)((nc + 7) / 8));
  MPI_PROF(ctx, KF_OTHER);
  k_refl_update<<<g, 256, 0, st>>>(A, T, N, j, c0, nc, w, tau, conj_tau);
  MPI_LAUNCH_CHECK(ctx, "k_refl_update");
  return MPI_OK;
}

}  // namespace

// One-sided Jacobi on the nj (even) columns of M (L x nj, column-major, FP64),
// accumulating the rotations into V (nj x nj, set to I here), until no pair
// rotates (at most 60 sweeps).  A pair counts as orthogonal once
// |m_a^H m_b| <= L eps |m_a| |m_b| (the rounding bound of the L-term dot
// product itself: a tighter test keeps rotating on rounding noise); columns with
// |m|^2 below eps^2 ||M||_F^2 (invariant under the rotations) are at M's
// rounding floor.  One sweep is a CUDA graph of nj - 1 steps.  On return
// sig_host holds the final column norms (the singular values of M, in column
// order).  sig_dev: nj doubles; flag: one int (device scratch).
mpi_status jacobi_columns(mpi_ctx* ctx, double2* M, int L, int nj, double2* V, double* sig_dev, int* flag,
                          std::vector<double>& sig_host, const char* what) {
  cudaStream_t st = ctx->stream;
  MPI_PROF(ctx, KF_OTHER);
  k_identity<<<(nj * nj + 255) / 256, 256, 0, st>>>(V, nj);
  MPI_LAUNCH_CHECK(ctx, "k_identity");
  constexpr double kEps = 2.220446049250313e-16;
  const double tol = (double)L * kEps;
  MPI_PROF(ctx, KF_OTHER);
  k_col_norms<<<nj, 128, 0, st>>>(M, L, sig_dev);
  MPI_LAUNCH_CHECK(ctx, "k_col_norms");
  sig_host.assign(nj, 0.0);
  cudaError_t e = cudaMemcpyAsync(sig_host.data(), sig_dev, nj * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(ctx, e, what);
  double fro2 = 0.0;
  for (double v : sig_host) fro2 += v * v;
  const double floor2 = kEps * kEps * fro2;
  SweepGraph sg;
  e = cudaStreamCreateWithFlags(&sg.cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(sg.cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int s = 0; s < nj - 1; ++s) k_jacobi_step<<<nj / 2, 128, 0, sg.cap>>>(M, L, V, nj, s, tol, floor2, flag);
    cudaError_t e2 = cudaStreamEndCapture(sg.cap, &sg.graph);
    e = e2 != cudaSuccess ? e2 : cudaGraphInstantiate(&sg.exec, sg.graph, 0);
  }
  if (e != cudaSuccess) return cuda_check(ctx, e, what);
  int rot = 1;
  for (int sweeps = 0; sweeps < 60 && rot; ++sweeps) {
    e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_check(ctx, e, what);
    MPI_PROF(ctx, KF_OTHER);
    e = cudaGraphLaunch(sg.exec, st);
    if (e != cudaSuccess) return cuda_check(ctx, e, what);
    ctx->launches += nj - 2;  // the sweep's kernels (MPI_LAUNCH_CHECK counts one)
    MPI_LAUNCH_CHECK(ctx, "k_jacobi_step (sweep)");
    e = cudaMemcpyAsync(&rot, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(ctx, e, what);
  }
  if (rot) return set_err(ctx, MPI_ERR_CUDA, std::string(what) + ": Jacobi SVD did not converge");
  MPI_PROF(ctx, KF_OTHER);
  k_col_norms<<<nj, 128, 0, st>>>(M, L, sig_dev);
  MPI_LAUNCH_CHECK(ctx, "k_col_norms");
  e = cudaMemcpyAsync(sig_host.data(), sig_dev, nj * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? MPI_OK : cuda_check(ctx, e, what);
}

namespace {

mpi_status maxwell_basis(mpi_ctx* ctx, int nz, int ny, int nx, double fov_z, double fov_y, double fov_x,
                         double f_hz, const double* sources, int n_sites, const mpi_c64* omega, int L, int q,
                         mpi_c32* U_out, double* sv_out) {
  if (!ctx) return MPI_ERR_ARG;
  if (!sources || !omega || !U_out || !sv_out) return set_err(ctx, MPI_ERR_ARG, "null argument");
  if (nz < 1 || !(fov_z > 0)) return set_err(ctx, MPI_ERR_SHAPE, "Maxwell basis: bad sizes");
  const long Nl = (long)nz * ny * nx;
  const int n = 6 * n_sites;
  if (ny < 1 || nx < 1 || n_sites < 1 || L < 1 || q < 1 || n_sites > 4096 || L > 65536)
    return set_err(ctx, MPI_ERR_SHAPE, "Maxwell basis: bad sizes");
  if (Nl < n || Nl > (1L << 28)) return set_err(ctx, MPI_ERR_SHAPE, "Maxwell basis: need 6 n_sites <= N <= 2^28");
  if (q > std::min(n, L)) return set_err(ctx, MPI_ERR_SHAPE, "Maxwell basis: q > min(6 n_sites, L)");
  if (!(fov_y > 0 && fov_x > 0 && f_hz > 0)) return set_err(ctx, MPI_ERR_ARG, "Maxwell basis: fov and f must be > 0");
  const int N = (int)Nl;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const double k = 2.0 * kPi * f_hz / kC0;
  const dim3 fgrid((unsigned)((N + 255) / 256), (unsigned)n_sites);
  // 1. fields.  Identically zero fields (e.g. the three that vanish in the
  // plane of in-plane sources) add nothing to Y = B Omega: they are dropped
  // with their rows of Omega before the factorisation.
  DevBuf bSrc, bPos, bN2;
  cudaError_t e = cudaMalloc(&bSrc.p, (size_t)n_sites * 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&bPos.p, (size_t)n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&bN2.p, (size_t)n * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bSrc.p, sources, (size_t)n_sites * 3 * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bN2.p, 0, (size_t)n * sizeof(double), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_OOM, "Maxwell basis sources");
  }
  MPI_PROF(ctx, KF_OTHER);
  k_dipole_fields<<<fgrid, 256, 0, st>>>(nullptr, nullptr, (double*)bN2.p, N, nz, ny, nx, fov_z / nz, fov_y / ny,
                                         fov_x / nx, (const double*)bSrc.p, k);
  MPI_LAUNCH_CHECK(ctx, "k_dipole_fields (norms)");
  std::vector<double> n2(n);
  e = cudaMemcpyAsync(n2.data(), bN2.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "Maxwell basis field norms");
  std::vector<int> pos(n, -1), keep;
  for (int j = 0; j < n; ++j)
    if (n2[j] > 0.0) {
      pos[j] = (int)keep.size();
      keep.push_back(j);
    }
  const int ne = (int)keep.size();     // columns of B that are not identically zero
  const int nj = ne + (ne & 1);        // Jacobi columns (round-robin pairs need an even count)
  if (ne == 0) return set_err(ctx, MPI_ERR_SHAPE, "Maxwell basis: every field is zero");
  if (q > std::min(ne, L)) return set_err(ctx, MPI_ERR_SHAPE, "Maxwell basis: q exceeds the rank bound of B omega");
  std::vector<double2> om_nz((size_t)ne * L);
  for (int c = 0; c < ne; ++c)
    for (int l = 0; l < L; ++l) {
      const mpi_c64 v = omega[(size_t)keep[c] * L + l];
      om_nz[(size_t)c * L + l] = make_double2(v.x, v.y);
    }
  const int nbw = (N + kRowsW - 1) / kRowsW;
  const int wmax = std::max(ne, q);
  DevBuf bA, bZ, bM, bV, bOm, bPart, bW, bTau, bScal, bNorm, bSig, bOrd, bFlag;
  auto alloc = [&](DevBuf& b, size_t bytes) { return cudaMalloc(&b.p, std::max<size_t>(bytes, 16)); };
  e = alloc(bA, (size_t)N * ne * sizeof(double2));
  if (e == cudaSuccess) e = alloc(bZ, (size_t)N * q * sizeof(double2));
  if (e == cudaSuccess) e = alloc(bM, (size_t)L * nj * sizeof(double2));
  if (e == cudaSuccess) e = alloc(bV, (size_t)nj * nj * sizeof(double2));
  if (e == cudaSuccess) e = alloc(bOm, (size_t)ne * L * sizeof(double2));
  if (e == cudaSuccess) e = alloc(bPart, (size_t)nbw * wmax * sizeof(double2));
  if (e == cudaSuccess) e = alloc(bW, (size_t)wmax * sizeof(double2));
  if (e == cudaSuccess) e = alloc(bTau, (size_t)ne * sizeof(double2));
  if (e == cudaSuccess) e = alloc(bScal, sizeof(double2));
  if (e == cudaSuccess) e = alloc(bNorm, kNormBlocks * sizeof(double));
  if (e == cudaSuccess) e = alloc(bSig, (size_t)nj * sizeof(double));
  if (e == cudaSuccess) e = alloc(bOrd, (size_t)q * sizeof(int));
  if (e == cudaSuccess) e = alloc(bFlag, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_OOM, "Maxwell basis workspace");
  }
  double2* A = (double2*)bA.p;
  double2* Z = (double2*)bZ.p;
  double2* M = (double2*)bM.p;
  double2* V = (double2*)bV.p;
  double2* Om = (double2*)bOm.p;
  double2* part = (double2*)bPart.p;
  double2* w = (double2*)bW.p;
  double2* tau = (double2*)bTau.p;
  double2* scal = (double2*)bScal.p;
  int* flag = (int*)bFlag.p;
  e = cudaMemcpyAsync(bPos.p, pos.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Om, om_nz.data(), (size_t)ne * L * sizeof(double2), cudaMemcpyHostToDevice, st);
  // the padded Jacobi column (odd ne) stays zero
  if (e == cudaSuccess) e = cudaMemsetAsync(M, 0, (size_t)L * nj * sizeof(double2), st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "Maxwell basis inputs");
  MPI_PROF(ctx, KF_OTHER);
  k_dipole_fields<<<fgrid, 256, 0, st>>>(A, (const int*)bPos.p, nullptr, N, nz, ny, nx, fov_z / nz, fov_y / ny,
                                         fov_x / nx, (const double*)bSrc.p, k);
  MPI_LAUNCH_CHECK(ctx, "k_dipole_fields");
  // 2a. Householder QR
  for (int j = 0; j < ne; ++j) {
    MPI_PROF(ctx, KF_OTHER);
    k_hh_norm<<<kNormBlocks, 256, 0, st>>>(A, N, j, (double*)bNorm.p);
    MPI_LAUNCH_CHECK(ctx, "k_hh_norm");
    MPI_PROF(ctx, KF_OTHER);
    k_hh_make<<<1, 32, 0, st>>>(A, N, j, (const double*)bNorm.p, kNormBlocks, tau, scal);
    MPI_LAUNCH_CHECK(ctx, "k_hh_make");
    MPI_PROF(ctx, KF_OTHER);
    k_hh_scale<<<(unsigned)(((long)N - j + 255) / 256), 256, 0, st>>>(A, N, j, tau, scal);
    MPI_LAUNCH_CHECK(ctx, "k_hh_scale");
    mpi_status s2 = apply_reflector(ctx, A, A, N, j, j + 1, ne - j - 1, tau, 1, part, w);
    if (s2) return s2;
  }
  // 2b. M = (R Omega)^H
  MPI_PROF(ctx, KF_OTHER);
  k_small_x<<<dim3((unsigned)((L + 127) / 128), (unsigned)ne), 128, 0, st>>>(A, N, ne, Om, L, M);
  MPI_LAUNCH_CHECK(ctx, "k_small_x");
  // 2c. one-sided Jacobi on the columns of M = X^H
  std::vector<double> sig;
  {
    mpi_status s2 = jacobi_columns(ctx, M, L, nj, V, (double*)bSig.p, flag, sig, "Maxwell basis");
    if (s2) return s2;
  }
  std::vector<int> order(nj);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return sig[x] > sig[y]; });
  const int nsv = std::min(n, L);  // the dropped zero fields add zero singular values
  for (int i = 0; i < nsv; ++i) sv_out[i] = i < nj ? sig[order[i]] : 0.0;
  e = cudaMemcpyAsync(bOrd.p, order.data(), q * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_check(ctx, e, "Maxwell basis order");
  // 2d. U = Q [V_q; 0]: reflectors ne - 1 .. 0 (V's padded row, if any, is zero
  // in every column but its own)
  MPI_PROF(ctx, KF_OTHER);
  k_init_z<<<dim3((unsigned)((N + 255) / 256), (unsigned)q), 256, 0, st>>>(V, nj, (const int*)bOrd.p, N, Z);
  MPI_LAUNCH_CHECK(ctx, "k_init_z");
  for (int j = ne - 1; j >= 0; --j) {
    mpi_status s2 = apply_reflector(ctx, A, Z, N, j, 0, q, tau, 0, part, w);
    if (s2) return s2;
  }
  const size_t total = (size_t)N * q;
  MPI_PROF(ctx, KF_OTHER);
  k_z_to_c64<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Z, total, (float2*)U_out);
  MPI_LAUNCH_CHECK(ctx, "k_z_to_c64");
  e = cudaStreamSynchronize(st);  // the workspace is freed on return
  return e == cudaSuccess ? MPI_OK : cuda_check(ctx, e, "Maxwell basis");
}

}  // namespace

extern "C" mpi_status mpi_maxwell_basis_2d(mpi_ctx* ctx, int ny, int nx, double fov_y, double fov_x, double f_hz,
                                           const double* sources, int n_sites, const mpi_c64* omega, int L, int q,
                                           mpi_c32* U_out, double* sv_out) {
  return maxwell_basis(ctx, 1, ny, nx, 1.0, fov_y, fov_x, f_hz, sources, n_sites, omega, L, q, U_out, sv_out);
}

extern "C" mpi_status mpi_maxwell_basis_3d(mpi_ctx* ctx, int nz, int ny, int nx, double fov_z, double fov_y,
                                           double fov_x, double f_hz, const double* sources, int n_sites,
                                           const mpi_c64* omega, int L, int q, mpi_c32* U_out, double* sv_out) {
  return maxwell_basis(ctx, nz, ny, nx, fov_z, fov_y, fov_x, f_hz, sources, n_sites, omega, L, q, U_out, sv_out);
}
