// Cartesian F_s (Eq. 1): centred unitary DFT per coil followed by selection of
// the sampled points, as shared-memory FFT passes.
//
// The centred DFT along an axis of even length n is
//   F_c = (-1)^(n/2) D F D / sqrt(n),  D = diag((-1)^j),
// with F the plain DFT.  The image-side sign D and the 1/sqrt(N) scale are
// applied by the expansion kernels; these passes do the plain FFTs, the
// k-side sign and the gather / zero-fill of the sampled points.
//
// Every line (one row, or one column of a tile) is transformed by one warp in
// shared memory (padded by one element per 8, see pad8) with a mixed-radix
// (2, 3, 4, 5, 8) Stockham auto-sort FFT: for
// a stage of radix R after Ns points have been combined, butterfly j reads
// x[j + r N/R], r < R, multiplies input r by w^(r (j mod Ns)) with w =
// exp(-+2 pi i / (Ns R)), takes an R-point DFT and writes output r to
// (j div Ns) Ns R + (j mod Ns) + r Ns.  Each lane keeps its butterflies in
// registers across a __syncwarp, so the stage runs in place.
#include <stdio.h>

#include <cuda.h>

#include <algorithm>

#include "dft_reg.cuh"
#include "mpi_internal.h"
#include "ptx.cuh"

namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// R-point DFT in registers, y[a] = sum_r x[r] exp(-+2 pi i a r / R).
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  static __device__ __forceinline__ void go(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct Dft<4, INV> {
  static __device__ __forceinline__ void go(float2* v) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

template <bool INV>
struct Dft<8, INV> {
  static __device__ __forceinline__ void go(float2* v) {
    // two 4-point DFTs on the even and odd inputs, then the radix-2 combine
    // with twiddles exp(-+2 pi i m / 8), m = 0..3.
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4, INV>::go(e);
    Dft<4, INV>::go(o);
    const float h = 0.70710678118654752f;  // 1/sqrt(2)
    // o[1] *= exp(-+i pi/4), o[2] *= -+i, o[3] *= exp(-+3 i pi/4)
    const float2 o1 = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                          : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    const float2 o2 = rot90<INV>(o[2]);
    const float2 o3 = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                          : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

template <bool INV>
struct Dft<3, INV> {
  static __device__ __forceinline__ void go(float2* v) {
    // c = cos(2 pi / 3) = -1/2, s = sin(2 pi / 3) = sqrt(3)/2
    const float s = INV ? -0.86602540378443865f : 0.86602540378443865f;
    const float2 t = cadd(v[1], v[2]);
    const float2 d = csub(v[1], v[2]);
    const float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    // -+ i s d
    const float2 isd = make_float2(s * d.y, -s * d.x);
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, isd);
    v[2] = csub(m, isd);
  }
};

template <bool INV>
struct Dft<5, INV> {
  static __device__ __forceinline__ void go(float2* v) {
    // c1 = cos(2 pi/5) = (sqrt 5 - 1)/4, c2 = cos(4 pi/5) = -(sqrt 5 + 1)/4,
    // s1 = sin(2 pi/5), s2 = sin(4 pi/5)
    const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;
    const float s1 = INV ? -0.95105651629515357f : 0.95105651629515357f;
    const float s2 = INV ? -0.58778525229247313f : 0.58778525229247313f;
    const float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    const float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    const float2 x0 = v[0];
    const float2 r1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
    const float2 r2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
    // forward: y1 = r1 - i (s1 b1 + s2 b2), y2 = r2 - i (s2 b1 - s1 b2)
    const float2 i1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
    const float2 i2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
    v[0] = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
    v[1] = make_float2(r1.x + i1.y, r1.y - i1.x);
    v[4] = make_float2(r1.x - i1.y, r1.y + i1.x);
    v[2] = make_float2(r2.x + i2.y, r2.y - i2.x);
    v[3] = make_float2(r2.x - i2.y, r2.y + i2.x);
  }
};

// Shared-memory index of element i of a line: one float2 of padding per 8,
// which leaves every Stockham stage's strided loads and stores at most
// two-way bank conflicted for the supported lengths.
__host__ __device__ __forceinline__ constexpr int pad8(int i) { return i + (i >> 3); }
__host__ __device__ constexpr int padded_len(int n) { return n + n / 8; }

// One radix-R Stockham stage of an N-point line held in shared memory, its
// N / R butterflies spread over LANES lanes (a warp, or half a warp for short
// lines, two lines per warp).
template <int N, int R, int NS, bool INV, int LANES>
__device__ __forceinline__ void fft_stage(float2* buf, const float2* tw, int lane) {
  constexpr int NB = N / R;
  constexpr int PER = (NB + LANES - 1) / LANES;
  float2 v[PER][R];
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = lane + LANES * b;
    if (j < NB) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = buf[pad8(j + r * NB)];
    }
  }
  __syncwarp();
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = lane + LANES * b;
    if (j < NB) {
      const int k = j % NS;
      if (NS > 1) {
        // w^r for r = 1 .. R-1 from one table read: w^r = w^(r/2) w^(r - r/2),
        // so each power is at most three products deep (a few ulp)
        float2 w[R];
        w[1] = tw[k * (N / (NS * R))];
        if (INV) w[1].y = -w[1].y;
#pragma unroll
        for (int r = 2; r < R; ++r) w[r] = cmul(w[r / 2], w[r - r / 2]);
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
      }
      Dft<R, INV>::go(v[b]);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pad8(base + r * NS)] = v[b][r];
    }
  }
  __syncwarp();
}

template <int N, bool INV, int LANES, int NS, int R, int... Rest>
struct Run {
  static __device__ __forceinline__ void go(float2* b, const float2* tw, int lane) {
    fft_stage<N, R, NS, INV, LANES>(b, tw, lane);
    Run<N, INV, LANES, NS * R, Rest...>::go(b, tw, lane);
  }
};
template <int N, bool INV, int LANES, int NS, int R>
struct Run<N, INV, LANES, NS, R> {
  static __device__ __forceinline__ void go(float2* b, const float2* tw, int lane) {
    fft_stage<N, R, NS, INV, LANES>(b, tw, lane);
  }
};

template <int N, bool INV>
struct Fft;
#define MPI_FFT_PLAN(n, ...)                                                    \
  template <bool INV>                                                           \
  struct Fft<n, INV> {                                                          \
    template <int LANES = 32>                                                   \
    static __device__ __forceinline__ void go(float2* b, const float2* tw, int lane) { \
      Run<n, INV, LANES, 1, __VA_ARGS__>::go(b, tw, lane);                      \
    }                                                                           \
  };
MPI_FFT_PLAN(16, 4, 4)
MPI_FFT_PLAN(32, 8, 4)
MPI_FFT_PLAN(48, 4, 4, 3)
MPI_FFT_PLAN(64, 8, 8)
MPI_FFT_PLAN(96, 8, 4, 3)
MPI_FFT_PLAN(128, 8, 4, 4)
MPI_FFT_PLAN(192, 8, 8, 3)
MPI_FFT_PLAN(256, 8, 8, 4)
MPI_FFT_PLAN(320, 8, 8, 5)
MPI_FFT_PLAN(512, 8, 8, 8)
#undef MPI_FFT_PLAN

constexpr int kRowWarps = 4;

// One warp per (coil, k-space row), the warps striding over all rows (the grid
// is capped at a few CTAs per SM: volumes have hundreds of thousands of rows,
// most of them without samples, and one CTA each would make the pass bound by
// CTA launches).  Forward: FFT along x, k-side centring sign, gather the row's
// samples (contiguous in the sorted list); rows without samples are skipped.
template <int NX>
__global__ void __launch_bounds__(kRowWarps * 32) k_rows_fwd_gather(
    const float2* __restrict__ data, int C, int n_rows, int ny, const int32_t* __restrict__ idx,
    const int32_t* __restrict__ row_ptr, float2* __restrict__ y, int M, float ksign,
    const float2* __restrict__ tw_g) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  __shared__ float2 tw[NX];
  __shared__ float2 buf[kRowWarps][padded_len(NX)];
  for (int i = threadIdx.x; i < NX; i += blockDim.x) tw[i] = tw_g[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* b = buf[warp];
  const int total = C * n_rows;
  for (int gr = blockIdx.x * kRowWarps + warp; gr < total; gr += gridDim.x * kRowWarps) {
    const int c = gr / n_rows, row = gr - c * n_rows;
    const int m0 = row_ptr[row], m1 = row_ptr[row + 1];
    if (m1 <= m0) continue;  // warp-uniform
    const float2* src = data + ((size_t)c * n_rows + row) * NX;
    constexpr int PL = (NX + 31) / 32;
    float2 v[PL];
#pragma unroll
    for (int u = 0; u < PL; ++u)
      if (lane + 32 * u < NX) v[u] = src[lane + 32 * u];
#pragma unroll
    for (int u = 0; u < PL; ++u)
      if (lane + 32 * u < NX) b[pad8(lane + 32 * u)] = v[u];
    __syncwarp();
    Fft<NX, false>::go(b, tw, lane);
    const int rpar = (row / ny + row % ny) & 1;  // (kz + ky) parity
    const size_t rbase = (size_t)row * NX;
    for (int m = m0 + lane; m < m1; m += 32) {
      const int kx = (int)(idx[m] - rbase);
      const float sg = ((kx + rpar) & 1) ? -ksign : ksign;
      const float2 t = b[pad8(kx)];
      y[(size_t)c * M + m] = make_float2(t.x * sg, t.y * sg);
    }
    __syncwarp();  // the buffer is refilled for the next row
  }
}

// Adjoint: zero-fill the row from its samples (with the k-side sign), inverse
// FFT.  Rows without samples are not written: the pass along y that follows
// reads them as zeros.  Same row striding.
template <int NX>
__global__ void __launch_bounds__(kRowWarps * 32) k_rows_scatter_inv(
    const float2* __restrict__ y, int C, int n_rows, int ny, const int32_t* __restrict__ idx,
    const int32_t* __restrict__ row_ptr, float2* __restrict__ data, int M, float ksign,
    const float2* __restrict__ tw_g) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  __shared__ float2 tw[NX];
  __shared__ float2 buf[kRowWarps][padded_len(NX)];
  for (int i = threadIdx.x; i < NX; i += blockDim.x) tw[i] = tw_g[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* b = buf[warp];
  const int total = C * n_rows;
  for (int gr = blockIdx.x * kRowWarps + warp; gr < total; gr += gridDim.x * kRowWarps) {
    const int c = gr / n_rows, row = gr - c * n_rows;
    const int m0 = row_ptr[row], m1 = row_ptr[row + 1];
    float2* dst = data + ((size_t)c * n_rows + row) * NX;
    if (m1 <= m0) continue;  // warp-uniform
    for (int i = lane; i < padded_len(NX); i += 32) b[i] = make_float2(0.f, 0.f);
    __syncwarp();
    const int rpar = (row / ny + row % ny) & 1;
    const size_t rbase = (size_t)row * NX;
    for (int m = m0 + lane; m < m1; m += 32) {
      const int kx = (int)(idx[m] - rbase);
      const float sg = ((kx + rpar) & 1) ? -ksign : ksign;
      const float2 t = y[(size_t)c * M + m];
      b[pad8(kx)] = make_float2(t.x * sg, t.y * sg);
    }
    __syncwarp();
    Fft<NX, true>::go(b, tw, lane);
    for (int i = lane; i < NX; i += 32) dst[i] = b[pad8(i)];
    __syncwarp();
  }
}

constexpr int kLineWarps = 8;  // warps per CTA of the line pass

// The FFTs of a line pass's TILE lines, in shared memory at buf + line * S.
// Lines of up to 128 points take half a warp each (no stage of theirs has more
// than 16 butterflies), two lines per warp; every line of the tile is
// transformed, whether or not it is stored, so both halves of a warp run the
// same stages.
template <int L, bool INV, int TILE, int S>
__device__ __forceinline__ void fft_tile_lines(float2* buf, const float2* tw, int warp, int lane) {
  if constexpr (L <= 128) {
    for (int line = 2 * warp + (lane >> 4); line < TILE; line += 2 * kLineWarps)
      Fft<L, INV>::template go<16>(buf + line * S, tw, lane & 15);
  } else {
    for (int line = warp; line < TILE; line += kLineWarps) Fft<L, INV>::go(buf + line * S, tw, lane);
  }
}

// In-place FFT of lines of length L with element stride `stride`.  A CTA takes
// TILE lines that are adjacent in memory (consecutive x): it loads them as
// TILE-element row segments (64, 128 or 256 bytes), transposes into shared
// memory (one contiguous padded line each), transforms them (TILE / 8 lines
// per warp) and writes back.  Wide tiles make long DRAM bursts for passes over
// volumes that do not fit in L2; narrow ones give more CTAs for small grids.
// Tiles are enumerated as (slab, x-tile) with slab base offset
// (slab / inner) * outer_stride + (slab % inner) * inner_stride.
// Column stride of the transposed tile: the padded line length rounded to
// 2 mod 16 float2 for TILE <= 16 (a warp's transposing accesses then cover 8
// or 16 lines x 4 or 2 rows) and to 1 mod 16 for TILE = 32 (32 lines of one
// row); either way they take the minimum two shared-memory wavefronts.
__host__ __device__ constexpr int col_stride(int L, int TILE) {
  return padded_len(L) + (((TILE == 32 ? 1 : 2) - padded_len(L)) % 16 + 16) % 16;
}

template <int L, bool INV, int TILE>
__global__ void __launch_bounds__(kLineWarps * 32, (L * TILE <= 2048) ? 4 : (L * TILE >= 4096 ? 2 : 3)) k_fft_lines(float2* __restrict__ data, int nx,
                                                              long stride, int n_slabs, int inner,
                                                              long outer_stride, long inner_stride,
                                                              const float2* __restrict__ tw_g,
                                                              const uint8_t* __restrict__ rmask, int mask_nz) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  constexpr int S = col_stride(L, TILE);
  constexpr int T = kLineWarps * 32;         // threads
  constexpr int RSTEP = T / TILE;            // rows covered per pass of the CTA
  constexpr int PER = (L + RSTEP - 1) / RSTEP;  // elements per thread
  __shared__ float2 tw[L];
  __shared__ float2 buf[TILE * S];
  const int tid = threadIdx.x;
  for (int i = tid; i < L; i += T) tw[i] = tw_g[i];
  const int x_tiles = (nx + TILE - 1) / TILE;
  const int tile = (int)blockIdx.x;
  const int slab = tile / x_tiles;
  const int x0 = (tile - slab * x_tiles) * TILE;
  if (slab >= n_slabs) return;
  const size_t base = (size_t)(slab / inner) * outer_stride + (size_t)(slab % inner) * inner_stride + x0;
  // thread -> (column cx, rows r0 + RSTEP u): all PER loads are issued before any is used
  const int cx = tid % TILE, r0 = tid / TILE;
  const bool ok = x0 + cx < nx;
  const float2* src = data + base + cx;
  // With a row mask (rmask[z * L + r], z = slab % mask_nz: 1 where k-space row r
  // of this slab has samples): inverse, the rows without samples are taken as
  // zeros without being read, whatever the buffer holds there (the adjoint's
  // row pass does not write them); forward, only the rows with samples are
  // stored (the row pass that follows reads no other row).
  const uint8_t* rm = rmask ? rmask + (size_t)(slab % mask_nz) * L : nullptr;
  float2 v[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int r = r0 + RSTEP * u;
    if (ok && r < L) v[u] = (INV && rm && !rm[r]) ? make_float2(0.f, 0.f) : src[(size_t)r * stride];
  }
#pragma unroll
  for (int u = 0; u < PER; ++u)
    if (ok && r0 + RSTEP * u < L) buf[cx * S + pad8(r0 + RSTEP * u)] = v[u];
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  fft_tile_lines<L, INV, TILE, S>(buf, tw, warp, lane);
  __syncthreads();
  float2* dst = data + base + cx;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int r = r0 + RSTEP * u;
    if (ok && r < L && (INV || !rm || rm[r])) dst[(size_t)r * stride] = buf[cx * S + pad8(r)];
  }
}

template <int L, bool INV, int TILE>
void lines_launch(mpi_ctx* ctx, long blocks, float2* data, int nx, long stride, int n_slabs, int inner,
                  long outer_stride, long inner_stride, const float2* tw, const uint8_t* rmask, int mask_nz) {
  launch_pdl(ctx, k_fft_lines<L, INV, TILE>, dim3((unsigned)blocks), dim3(kLineWarps * 32), 0, data, nx, stride,
             n_slabs, inner, outer_stride, inner_stride, tw, rmask, mask_nz);
}

// Tile width: the widest (longest row segments) that keeps at most 16 elements
// per thread in the copy phases and still gives every SM four or more CTAs.
int lines_tile(const mpi_ctx* ctx, int L, int nx, int n_slabs) {
  const long want = 4L * std::max(ctx->num_sms, 1);
  const int tiles[3] = {32, 16, 8};
  for (int t : tiles) {
    if (L * t / (kLineWarps * 32) > 16) continue;
    if (t == 8 || (long)n_slabs * ((nx + t - 1) / t) >= want) return t;
  }
  return 8;
}

// The pass along y as a two-step FFT in registers: L = R1 R2 points per
// column, y = r + R2 m.  A CTA takes 32 adjacent columns (one per lane) of one
// (coil, z) plane.  Step 1: for each r, the R1 values y = r + R2 m are loaded
// (rows of 32 columns: coalesced), transformed (R1-point DFT in registers) and
// twiddled by w_L^(r k1) into shared memory [k1][r][column].  Step 2: for each
// k1, the R2 values are read back, transformed (R2-point DFT) and stored to
// rows k = k1 + R1 k2.  One shared-memory write and read per element (the
// Stockham passes take one per radix stage plus two transposes).  The inverse
// is the forward of the conjugated data, conjugated back.  Row mask as in
// k_fft_lines: inverse, rows without samples are read as zeros; forward, only
// rows with samples are stored.
template <int R1, int R2, bool INV>
__global__ void __launch_bounds__(256, 2) k_fft_cols_reg(float2* __restrict__ data, int nx, int n_slabs, long plane,
                                                      const float2* __restrict__ tw_g,
                                                      const uint8_t* __restrict__ rmask, int mask_nz) {
  constexpr int L = R1 * R2;
  __shared__ float2 sY[L * 32];  // [k1][r][column]
  __shared__ float2 tw[L];
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < L; i += 256) tw[i] = tw_g[i];
  const int x_tiles = (nx + 31) / 32;
  const int slab = (int)blockIdx.x / x_tiles, x0 = ((int)blockIdx.x - slab * x_tiles) * 32;
  const bool ok = x0 + lane < nx;
  float2* col = data + (size_t)slab * plane + x0 + lane;
  const uint8_t* rm = rmask ? rmask + (size_t)(slab % mask_nz) * L : nullptr;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < (R2 + 7) / 8; ++it) {
    const int r = w + 8 * it;
    if (r >= R2) break;
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const int y = r + R2 * m;
      float2 t = make_float2(0.f, 0.f);
      if (ok && !(INV && rm && !rm[y])) t = col[(size_t)y * nx];
      v[m] = INV ? make_float2(t.x, -t.y) : t;
    }
    mpi_dft::dft_r<R1>(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) v[k1] = mpi_dft::cmulf(v[k1], tw[r * k1]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) sY[(k1 * R2 + r) * 32 + lane] = v[k1];
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < (R1 + 7) / 8; ++it) {
    const int k1 = w + 8 * it;
    if (k1 >= R1) break;
    float2 u[R2];
#pragma unroll
    for (int r = 0; r < R2; ++r) u[r] = sY[(k1 * R2 + r) * 32 + lane];
    mpi_dft::dft_r<R2>(u);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      const int k = k1 + R1 * k2;
      if (ok && (INV || !rm || rm[k])) col[(size_t)k * nx] = INV ? make_float2(u[k2].x, -u[k2].y) : u[k2];
    }
  }
}

// Launch of the register pass along y for length L; false where L has no
// (R1, R2) split or the geometry is not a y pass (lines of stride nx in
// planes of `outer_stride`).
template <bool INV>
bool cols_reg_launch(mpi_ctx* ctx, int L, float2* data, int nx, long stride, int n_slabs, int inner,
                     long outer_stride, const float2* tw, const uint8_t* rmask, int mask_nz) {
  if (stride != nx || inner != 1) return false;
  const long blocks = (long)n_slabs * ((nx + 31) / 32);
  if (blocks == 0 || blocks > 0x7fffffffL) return false;
#define MPI_CREG(n, r1, r2)                                                                                   \
  case n:                                                                                                    \
    launch_pdl(ctx, k_fft_cols_reg<r1, r2, INV>, dim3((unsigned)blocks), dim3(256), 0, data, nx, n_slabs,       \
               outer_stride, tw, rmask, mask_nz);                                                            \
    return true;
  switch (L) {
    MPI_CREG(64, 8, 8)
    MPI_CREG(96, 8, 12)
    MPI_CREG(128, 8, 16)
    MPI_CREG(192, 16, 12)
    MPI_CREG(256, 16, 16)
    default:
      return false;
  }
#undef MPI_CREG
}

// Launch of one line pass with tile width `tile` (8, 16 or 32 lines, or -1
// for the register pass along y); false when the length / tile pair is not
// compiled.
template <bool INV>
bool lines_launch_tile(mpi_ctx* ctx, int tile, int L, long blocks, float2* data, int nx, long stride, int n_slabs,
                       int inner, long outer_stride, long inner_stride, const float2* tw, const uint8_t* rmask,
                       int mask_nz) {
  if (tile == -1) return cols_reg_launch<INV>(ctx, L, data, nx, stride, n_slabs, inner, outer_stride, tw, rmask, mask_nz);
#define MPI_LINES_CASE(n)                                                                                     \
  case n:                                                                                                     \
    if (tile == 32 && n <= 128)                                                                               \
      lines_launch<n, INV, (n <= 128 ? 32 : 8)>(ctx, blocks, data, nx, stride, n_slabs, inner, outer_stride,   \
                                                inner_stride, tw, rmask, mask_nz);                           \
    else if (tile == 16 && n <= 256)                                                                          \
      lines_launch<n, INV, (n <= 256 ? 16 : 8)>(ctx, blocks, data, nx, stride, n_slabs, inner, outer_stride,   \
                                                inner_stride, tw, rmask, mask_nz);                           \
    else if (tile == 8)                                                                                       \
      lines_launch<n, INV, 8>(ctx, blocks, data, nx, stride, n_slabs, inner, outer_stride, inner_stride, tw,    \
                              rmask, mask_nz);                                                               \
    else                                                                                                      \
      return false;                                                                                           \
    return true;
  switch (L) {
    MPI_LINES_CASE(16)
    MPI_LINES_CASE(32)
    MPI_LINES_CASE(48)
    MPI_LINES_CASE(64)
    MPI_LINES_CASE(96)
    MPI_LINES_CASE(128)
    MPI_LINES_CASE(192)
    MPI_LINES_CASE(256)
    MPI_LINES_CASE(320)
    MPI_LINES_CASE(512)
    default:
      return false;
  }
#undef MPI_LINES_CASE
}

// Autotuner of the line passes' tile width.  A pass shape is tuned once per
// context: each candidate width (at most 16 elements per thread in the copy
// phases) is launched once to warm up and then three times between two CUDA
// events on the context's stream, on the tuning scratch buffer (the pass's
// timing does not depend on the values it transforms); the fastest is kept.
// Returns 0 when this call cannot tune (no scratch, capture in progress,
// tuning off).
template <bool INV>
int lines_autotune(mpi_ctx* ctx, const long (&key)[10], int L, float2* data, int nx, long stride, int n_slabs,
                   int inner, long outer_stride, long inner_stride, const float2* tw, const uint8_t* rmask,
                   int mask_nz) {
  if (!ctx->autotune || !ctx->tune_scratch) return 0;
  // the elements the pass touches, from `data`: every slab base plus a full line set
  const long last_slab = n_slabs - 1;
  const size_t extent = (size_t)(last_slab / inner) * outer_stride + (size_t)(last_slab % inner) * inner_stride +
                        (size_t)(L - 1) * stride + nx;
  if (extent * sizeof(float2) > ctx->tune_scratch_bytes) return 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cap != cudaStreamCaptureStatusNone) return 0;
  float2* scratch = (float2*)ctx->tune_scratch;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(e0);
    return 0;
  }
  mpi_ctx::TuneRecord rec;
  for (int i = 0; i < 10; ++i) rec.key[i] = key[i];
  rec.n = 0;
  rec.choice = 0;
  float best = 1e30f;
  const int cands[4] = {8, 16, 32, -1};
  for (int tile : cands) {
    if (tile > 0 && (long)L * tile / (kLineWarps * 32) > 16) continue;
    const int cols = tile < 0 ? 32 : tile;  // columns per CTA
    const long blocks = (long)n_slabs * ((nx + cols - 1) / cols);
    if (blocks > 0x7fffffffL) continue;
    if (!lines_launch_tile<INV>(ctx, tile, L, blocks, scratch, nx, stride, n_slabs, inner, outer_stride,
                                inner_stride, tw, rmask, mask_nz))
      continue;
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 3; ++r)
      lines_launch_tile<INV>(ctx, tile, L, blocks, scratch, nx, stride, n_slabs, inner, outer_stride, inner_stride,
                             tw, rmask, mask_nz);
    cudaEventRecord(e1, ctx->stream);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const float us = 1e3f * ms / 3.f;
    rec.cand[rec.n] = tile;
    rec.us[rec.n] = us;
    rec.n++;
    if (us < best) {
      best = us;
      rec.choice = tile;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rec.choice || cudaGetLastError() != cudaSuccess) return 0;
  char buf[256];
  auto tname = [](int t, char* b, size_t n) {
    if (t < 0) snprintf(b, n, "register two-step");
    else snprintf(b, n, "%d lines", t);
  };
  char tn[32];
  tname(rec.choice, tn, sizeof tn);
  int len = snprintf(buf, sizeof buf, "FFT line pass L=%d %s stride=%ld lines=%ld%s: %s (", L, INV ? "inverse" : "forward",
                     stride, (long)n_slabs * nx, rmask ? " row-masked" : "", tn);
  for (int i = 0; i < rec.n && len < (int)sizeof buf; ++i) {
    tname(rec.cand[i], tn, sizeof tn);
    len += snprintf(buf + len, sizeof buf - len, "%s%s: %.1f us", i ? ", " : "", tn, rec.us[i]);
  }
  if (len < (int)sizeof buf) snprintf(buf + len, sizeof buf - len, ")");
  rec.what = buf;
  ctx->tuned.push_back(rec);
  return rec.choice;
}

// The tile width of a line pass: the caller's fixed choice where it applies,
// else the tuned one (tuning it now if this call can), else 0.
template <bool INV>
int lines_choose(mpi_ctx* ctx, float2* data, int L, int nx, long stride, int n_slabs, int inner, long outer_stride,
                 long inner_stride, const float2* tw, const uint8_t* rmask, int mask_nz) {
  const long key[10] = {L, INV ? 1 : 0, nx, stride, n_slabs, inner, outer_stride, inner_stride, rmask ? 1 : 0,
                        mask_nz};
  int tile = 0;
  // a caller's fixed choice (mpi_ctx_set_line_kernel), where this pass has it
  if (ctx->line_kernel) {
    const int t = ctx->line_kernel;
    const bool ok = t == -1 ? (L == 64 || L == 96 || L == 128 || L == 192 || L == 256) && stride == nx && inner == 1
                            : (t == 8 || (t == 16 && L <= 256) || (t == 32 && L <= 128));
    if (ok) tile = t;
  }
  for (const auto& r : ctx->tuned) {
    if (tile) break;
    if (std::equal(r.key, r.key + 10, key)) tile = r.choice;
  }
  if (!tile)
    tile = lines_autotune<INV>(ctx, key, L, data, nx, stride, n_slabs, inner, outer_stride, inner_stride, tw, rmask,
                               mask_nz);
  return tile;
}

template <bool INV>
mpi_status lines_dispatch(mpi_ctx* ctx, const char* name, float2* data, int L, int nx, long stride, int n_slabs,
                          int inner, long outer_stride, long inner_stride, const uint8_t* rmask = nullptr,
                          int mask_nz = 1) {
  const float2* tw = twiddle_table(ctx, L);
  if (!tw) return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
  if ((long)n_slabs * nx == 0) return MPI_OK;
  int tile = lines_choose<INV>(ctx, data, L, nx, stride, n_slabs, inner, outer_stride, inner_stride, tw, rmask,
                               mask_nz);
  if (!tile) tile = lines_tile(ctx, L, nx, n_slabs);
  const int tw_cols = tile < 0 ? 32 : tile;
  const int x_tiles = (nx + tw_cols - 1) / tw_cols;
  const long blocks = (long)n_slabs * x_tiles;
  if (blocks > 0x7fffffffL) return set_err(ctx, MPI_ERR_SHAPE, "too many FFT tiles");
  MPI_PROF(ctx, KF_FFT_LINES);
  if (!lines_launch_tile<INV>(ctx, tile, L, blocks, data, nx, stride, n_slabs, inner, outer_stride, inner_stride, tw,
                              rmask, mask_nz))
    return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
  MPI_LAUNCH_CHECK(ctx, name);
  return MPI_OK;
}

// Line pass along y over the oversampled radial grid [C][G][G] (L = G) with the
// centred n x n window folded in, in place of separate zero-pad and crop
// passes.  Each grid cell of the window (gy, gx) = (o + y, o + x) carries the
// factor deap[y] deap[x] / n (-1)^(gx + gy).  Forward (src set): the column is
// formed on the fly from the image [C][n][n] (zero outside the window) and its
// transform written to the grid.  Inverse (dst set): the grid column's
// transform is stored only inside the window, scaled, into the image
// [C][n][n]; the grid is not written back.  Tiles of 8 columns; a tile wholly
// outside the window does nothing: forward, those grid columns are zero and
// the row pass that follows reads them as zeros without loading them.
struct LineWin {
  const float2* src;
  float2* dst;
  const float* deap;
  int n, o;
};

template <int L, bool INV>
__global__ void __launch_bounds__(kLineWarps * 32, (L * 8 <= 2048) ? 4 : (L * 8 >= 4096 ? 2 : 3))
    k_fft_lines_win(float2* __restrict__ grid, int C, LineWin win, const float2* __restrict__ tw_g) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  constexpr int TILE = 8;
  constexpr int S = col_stride(L, TILE);
  constexpr int T = kLineWarps * 32;
  constexpr int RSTEP = T / TILE;
  constexpr int PER = (L + RSTEP - 1) / RSTEP;
  __shared__ float2 tw[L];
  __shared__ float2 buf[TILE * S];
  constexpr int x_tiles = L / TILE;
  const int c = (int)blockIdx.x / x_tiles, x0 = ((int)blockIdx.x % x_tiles) * TILE;
  if (c >= C) return;
  const bool tile_in = x0 < win.o + win.n && x0 + TILE > win.o;  // CTA-uniform
  const int tid = threadIdx.x, cx = tid % TILE, r0 = tid / TILE;
  const int gx = x0 + cx, xi = gx - win.o;
  const bool colin = xi >= 0 && xi < win.n;
  float2* gcol = grid + (size_t)c * L * L + gx;
  if (!tile_in) return;  // forward: those columns are zero, and the row pass reads them as such
  for (int i = tid; i < L; i += T) tw[i] = tw_g[i];
  float2 v[PER];
  if (!INV) {
    const float2* src = win.src + (size_t)c * win.n * win.n + xi;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int r = r0 + RSTEP * u, yi = r - win.o;
      v[u] = make_float2(0.f, 0.f);
      if (r < L && colin && yi >= 0 && yi < win.n) {
        const float2 val = src[(size_t)yi * win.n];
        float f = win.deap[yi] * win.deap[xi] / (float)win.n;
        if ((gx + r) & 1) f = -f;
        v[u] = make_float2(val.x * f, val.y * f);
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (r0 + RSTEP * u < L) v[u] = gcol[(size_t)(r0 + RSTEP * u) * L];
  }
#pragma unroll
  for (int u = 0; u < PER; ++u)
    if (r0 + RSTEP * u < L) buf[cx * S + pad8(r0 + RSTEP * u)] = v[u];
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  fft_tile_lines<L, INV, TILE, S>(buf, tw, warp, lane);
  __syncthreads();
  if (!INV) {
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (r0 + RSTEP * u < L) gcol[(size_t)(r0 + RSTEP * u) * L] = buf[cx * S + pad8(r0 + RSTEP * u)];
  } else {
    float2* dst = win.dst + (size_t)c * win.n * win.n + xi;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int r = r0 + RSTEP * u, yi = r - win.o;
      if (r < L && colin && yi >= 0 && yi < win.n) {
        const float2 t = buf[cx * S + pad8(r)];
        float f = win.deap[yi] * win.deap[xi] / (float)win.n;
        if ((gx + r) & 1) f = -f;
        dst[(size_t)yi * win.n] = make_float2(t.x * f, t.y * f);
      }
    }
  }
}

float axis_sign(int n) { return ((n / 2) & 1) ? -1.f : 1.f; }

// The passes along y and x of one (coil, kz) plane of a 3D volume in one CTA,
// the plane held in shared memory S [NY][NX] (NY x NX x 8 bytes, at most 128 KB).
// NX / 8 warps: four per 32-column group.
//  forward: the DFT along y as a register two-step (NY = 8 R2; y = r + R2 m):
//    DFT8 over m straight from the coalesced rows of global memory, twiddle
//    w_NY^(r k1), into S rows r + R2 k1; then for each k1 the R2 rows R2 k1 + r
//    are read back, transformed (R2-point DFT) and written in place, so that
//    row R2 (ky % 8) + ky / 8 holds k-space row ky.  Then each k-space row with
//    samples takes its DFT along x (Stockham, one warp per row) and the gather
//    of its samples with the k-side centring sign.
//  inverse: the rows with samples are zero-filled from theirs, signed and
//    transformed along x into S row ky (the others zeroed), then the inverse
//    two-step along y (the forward one on conjugated data) writes the plane's
//    rows y straight to global memory.
// Rows along x: one per sample row of the plan (row_ptr over (kz, ky)).
template <int NY, int NX, bool INV>
__global__ void __launch_bounds__(NX * 4, 1) k_plane_yx(float2* __restrict__ data, float2* __restrict__ y, int nz,
                                                        const int32_t* __restrict__ idx,
                                                        const int32_t* __restrict__ row_ptr, int M, float ksign,
                                                        const float2* __restrict__ twy_g,
                                                        const float2* __restrict__ twx_g) {
  constexpr int R2 = NY / 8;
  constexpr int NW = NX / 8;
  constexpr int NT = NW * 32;
  constexpr int GROUPS = NX / 32;
  extern __shared__ float2 sh[];
  float2* S = sh;                               // [NY][NX]
  float2* rbuf = S + NY * NX;                   // [NW][padded_len(NX)]
  float2* twy = rbuf + NW * padded_len(NX);     // [NY]
  float2* twx = twy + NY;                       // [NX]
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cg = warp % GROUPS, sub = warp / GROUPS;  // sub < 4
  const int col = cg * 32 + lane;
  const int plane = (int)blockIdx.x;
  const int c = plane / nz, kz = plane - c * nz;
  float2* P = data + (size_t)plane * NY * NX;
  for (int i = tid; i < NY; i += NT) twy[i] = twy_g[i];
  for (int i = tid; i < NX; i += NT) twx[i] = twx_g[i];
  float2* b = rbuf + warp * padded_len(NX);
  const int rbase = kz * NY;  // k-space row (kz, ky) = kz NY + ky
  if (!INV) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < R2 / 4; ++i) {
      const int r = sub + 4 * i;
      float2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = P[(size_t)(r + R2 * m) * NX + col];
      mpi_dft::dft8(v);
#pragma unroll
      for (int k1 = 1; k1 < 8; ++k1) v[k1] = mpi_dft::cmulf(v[k1], twy[r * k1]);
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) S[(r + R2 * k1) * NX + col] = v[k1];
    }
    __syncthreads();
#pragma unroll
    for (int k1 = sub; k1 < 8; k1 += 4) {
      float2 u[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) u[r] = S[(R2 * k1 + r) * NX + col];
      mpi_dft::dft_r<R2>(u);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) S[(R2 * k1 + k2) * NX + col] = u[k2];
    }
    __syncthreads();
    for (int ky = warp; ky < NY; ky += NW) {
      const int row = rbase + ky;
      const int m0 = row_ptr[row], m1 = row_ptr[row + 1];
      if (m1 <= m0) continue;  // warp-uniform
      const float2* src = S + (R2 * (ky % 8) + ky / 8) * NX;
      for (int i = lane; i < NX; i += 32) b[pad8(i)] = src[i];
      __syncwarp();
      Fft<NX, false>::go(b, twx, lane);
      const int rpar = (kz + ky) & 1;
      const size_t rb = (size_t)row * NX;
      for (int m = m0 + lane; m < m1; m += 32) {
        const int kx = (int)(idx[m] - rb);
        const float sg = ((kx + rpar) & 1) ? -ksign : ksign;
        const float2 t = b[pad8(kx)];
        y[(size_t)c * M + m] = make_float2(t.x * sg, t.y * sg);
      }
      __syncwarp();
    }
  } else {
    __syncthreads();
    for (int ky = warp; ky < NY; ky += NW) {
      const int row = rbase + ky;
      const int m0 = row_ptr[row], m1 = row_ptr[row + 1];
      float2* dst = S + ky * NX;
      if (m1 <= m0) {  // warp-uniform
        for (int i = lane; i < NX; i += 32) dst[i] = make_float2(0.f, 0.f);
        continue;
      }
      for (int i = lane; i < padded_len(NX); i += 32) b[i] = make_float2(0.f, 0.f);
      __syncwarp();
      const int rpar = (kz + ky) & 1;
      const size_t rb = (size_t)row * NX;
      for (int m = m0 + lane; m < m1; m += 32) {
        const int kx = (int)(idx[m] - rb);
        const float sg = ((kx + rpar) & 1) ? -ksign : ksign;
        const float2 t = y[(size_t)c * M + m];
        b[pad8(kx)] = make_float2(t.x * sg, t.y * sg);
      }
      __syncwarp();
      Fft<NX, true>::go(b, twx, lane);
      for (int i = lane; i < NX; i += 32) dst[i] = b[pad8(i)];
      __syncwarp();
    }
    __syncthreads();
    // inverse along y: the forward two-step on conjugated values, conjugated back
#pragma unroll
    for (int i = 0; i < R2 / 4; ++i) {
      const int r = sub + 4 * i;
      float2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float2 t = S[(r + R2 * m) * NX + col];
        v[m] = make_float2(t.x, -t.y);
      }
      mpi_dft::dft8(v);
#pragma unroll
      for (int k1 = 1; k1 < 8; ++k1) v[k1] = mpi_dft::cmulf(v[k1], twy[r * k1]);
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) S[(r + R2 * k1) * NX + col] = v[k1];
    }
    __syncthreads();
#pragma unroll
    for (int k1 = sub; k1 < 8; k1 += 4) {
      float2 u[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) u[r] = S[(R2 * k1 + r) * NX + col];
      mpi_dft::dft_r<R2>(u);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) P[(size_t)(k1 + 8 * k2) * NX + col] = make_float2(u[k2].x, -u[k2].y);
    }
  }
}

template <int NY, int NX>
size_t plane_smem() {
  return ((size_t)NY * NX + (size_t)(NX / 8) * padded_len(NX) + NY + NX) * sizeof(float2);
}

// ---------------------------------------------------------------------------
// Pipelined plane passes.  k_plane_yx holds a whole plane per CTA, so at one
// CTA per SM each plane's global traffic waits for its passes.  Here one
// persistent CTA per SM (more where shared memory allows) walks its (coil, kz)
// planes in tiles of TC columns [NY][TC] (pipe_cols):
//  forward: TMA loads the tiles into a ring of buffers, ahead of
//    use; each tile takes the two-step DFT along y in place (as k_plane_yx),
//    and the outputs of the k-space rows with samples go straight to a compact
//    row store R [plane_kmax][padded NX].  When a plane's tiles are done, each
//    warp takes rows of R through the DFT along x and the gather, under the
//    loads of the next plane's tiles.
//  inverse: the rows with samples are scattered into R and transformed along
//    x; each tile then takes the inverse two-step along y with its first step
//    reading R (rows without samples are zero), and the result leaves by TMA
//    stores (8 strided boxes, one per output class ky mod 8), which run under
//    the next tile's work.
// Per plane the CTA keeps its row list (ky, sample range) and each row's slot
// in R in a double-buffered table, the next plane's loaded into registers
// while the current one runs.
constexpr int kPipeThreads = 512;

// Tile width and ring depth: 64 columns in 2 buffers where NX allows (the
// second step along y then has one item per thread), else 32 in 4.
__host__ __device__ constexpr int pipe_cols(int nx) { return nx % 64 == 0 ? 64 : 32; }
__host__ __device__ constexpr int pipe_bufs(int nx) { return pipe_cols(nx) == 64 ? 2 : 4; }

struct PlaneMeta {
  int4 row;  // thread t < kmax: the plane's t-th row with samples
  int slot;  // thread t < NY: position of row ky = t in the list, -1 without samples
  int n;     // number of rows with samples
};

template <int NY>
__device__ __forceinline__ PlaneMeta load_plane_meta(int kz, int kmax, const int4* __restrict__ prow,
                                                     const int32_t* __restrict__ pn,
                                                     const int16_t* __restrict__ pslot) {
  PlaneMeta m;
  const int t = threadIdx.x;
  m.row = t < kmax ? prow[(size_t)kz * kmax + t] : make_int4(-1, 0, 0, 0);
  m.slot = t < NY ? (int)pslot[(size_t)kz * NY + t] : -1;
  m.n = t == 0 ? pn[kz] : 0;
  return m;
}

template <int NY>
__device__ __forceinline__ void store_plane_meta(const PlaneMeta& m, int kmax, int4* rows, int* slot, int* n) {
  const int t = threadIdx.x;
  if (t < kmax) rows[t] = m.row;
  if (t < NY) slot[t] = m.slot;
  if (t == 0) *n = m.n;
}

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory carve-up of k_plane_pipe (byte offsets from a 1024-aligned base).
template <int NY, int NX>
struct PipeLayout {
  static constexpr int TC = pipe_cols(NX), NB = pipe_bufs(NX);
  static constexpr size_t kTile = (size_t)NY * TC * sizeof(float2);
  static __host__ __device__ size_t R(int) { return NB * kTile; }
  static __host__ __device__ size_t tw(int kmax) { return R(kmax) + (size_t)kmax * padded_len(NX) * sizeof(float2); }
  static __host__ __device__ size_t rows(int kmax) { return align_up(tw(kmax) + (NY + NX) * sizeof(float2), 16); }
  static __host__ __device__ size_t slot(int kmax) { return rows(kmax) + 2 * (size_t)kmax * sizeof(int4); }
  static __host__ __device__ size_t n(int kmax) { return slot(kmax) + 2 * (size_t)NY * sizeof(int); }
  static __host__ __device__ size_t bars(int kmax) { return align_up(n(kmax) + 2 * sizeof(int), 8); }
  static __host__ __device__ size_t total(int kmax) { return bars(kmax) + NB * sizeof(uint64_t) + 1024; }
};

template <int NY, int NX, bool INV>
__global__ void __launch_bounds__(kPipeThreads, 1)
    k_plane_pipe(const __grid_constant__ CUtensorMap tmap, float2* __restrict__ y, int nz, int planes, int kmax,
                 const int32_t* __restrict__ idx, const int4* __restrict__ prow, const int32_t* __restrict__ pn,
                 const int16_t* __restrict__ pslot, int M, float ksign, const float2* __restrict__ twy_g,
                 const float2* __restrict__ twx_g, int* err, long long wait_cycles) {
  constexpr int R2 = NY / 8;
  constexpr int TC = pipe_cols(NX), NB = pipe_bufs(NX);
  constexpr int TP = NX / TC;
  constexpr int PL = padded_len(NX);
  constexpr int NT = kPipeThreads;
  constexpr int NW = NT / 32;
  using L = PipeLayout<NY, NX>;
  extern __shared__ unsigned char smraw[];
  // offset from the shared array itself (not a cast integer), so that every
  // access below compiles to shared-memory loads and stores
  unsigned char* base = smraw + ((1024u - (mpi_ptx::smem_addr(smraw) & 1023u)) & 1023u);
  float2* bufs = (float2*)base;
  float2* R = (float2*)(base + L::R(kmax));
  float2* twy = (float2*)(base + L::tw(kmax));
  float2* twx = twy + NY;
  int4* mrows = (int4*)(base + L::rows(kmax));
  int* mslot = (int*)(base + L::slot(kmax));
  int* mn = (int*)(base + L::n(kmax));
  uint64_t* full = (uint64_t*)(base + L::bars(kmax));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  const int first = (int)blockIdx.x, stride = (int)gridDim.x;
  const int nmine = planes > first ? (planes - 1 - first) / stride + 1 : 0;
  if (nmine == 0) return;  // CTA-uniform
  const int total = nmine * TP;
  for (int i = tid; i < NY; i += NT) twy[i] = twy_g[i];
  for (int i = tid; i < NX; i += NT) twx[i] = twx_g[i];
  if (!INV && tid == 0) {
    for (int b = 0; b < NB; ++b) mpi_ptx::mbar_init(&full[b], 1);
    mpi_ptx::fence_mbar_init();
  }
  {
    const PlaneMeta m0 = load_plane_meta<NY>(first % nz, kmax, prow, pn, pslot);
    store_plane_meta<NY>(m0, kmax, mrows, mslot, mn);
  }
  __syncthreads();
  // tile g of this CTA: plane first + (g / TP) stride, columns (g % TP) TC +
  // [0, TC), ring buffer g % NB
  auto issue_load = [&](int g) {
    const int b = g % NB;
    mpi_ptx::mbar_arrive_expect_tx(&full[b], (uint32_t)L::kTile);
    mpi_ptx::tma_load_3d(bufs + (size_t)b * NY * TC, &tmap, (g % TP) * 2 * TC, 0,
                         first + (g / TP) * stride, &full[b]);
  };
  if (!INV && tid == 0)
    for (int g = 0; g < NB && g < total; ++g) issue_load(g);
  int g = 0;
  for (int j = 0; j < nmine; ++j) {
    const int pl = first + j * stride, c = pl / nz, kz = pl - c * nz;
    const int cur = j & 1;
    PlaneMeta nxt;
    if (j + 1 < nmine) nxt = load_plane_meta<NY>((pl + stride) % nz, kmax, prow, pn, pslot);
    const int4* rows = mrows + cur * kmax;
    const int* slot = mslot + cur * NY;
    const int nS = mn[cur];
    if (!INV) {
      for (int t = 0; t < TP; ++t, ++g) {
        const int b = g % NB;
        float2* B = bufs + (size_t)b * NY * TC;
        const bool ok = mpi_ptx::mbar_wait(&full[b], (uint32_t)((g / NB) & 1), err, wait_cycles);
        // first step along y, in place: DFT8 over m of rows r + R2 m, twiddle
        for (int it = tid; it < TC * R2; it += NT) {
          const int col = it % TC, r = it / TC;
          float2 v[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) v[m] = B[(r + R2 * m) * TC + col];
          mpi_dft::dft8(v);
#pragma unroll
          for (int k1 = 1; k1 < 8; ++k1) v[k1] = mpi_dft::cmulf(v[k1], twy[r * k1]);
#pragma unroll
          for (int k1 = 0; k1 < 8; ++k1) B[(r + R2 * k1) * TC + col] = v[k1];
        }
        if (__syncthreads_or(!ok)) return;  // a load timed out (recorded in err)
        // second step: R2-point DFT over r; output ky = k1 + 8 k2 kept where it has samples
        for (int it = tid; it < TC * 8; it += NT) {
          const int col = it % TC, k1 = it / TC;
          float2 u[R2];
#pragma unroll
          for (int r = 0; r < R2; ++r) u[r] = B[(R2 * k1 + r) * TC + col];
          mpi_dft::dft_r<R2>(u);
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const int s = slot[k1 + 8 * k2];
            if (s >= 0) R[s * PL + pad8(t * TC + col)] = u[k2];
          }
        }
        mpi_ptx::fence_proxy_async();  // the buffer's generic accesses before the next TMA load into it
        __syncthreads();
        if (tid == 0 && g + NB < total) issue_load(g + NB);
      }
      // rows along x and the gather (the next plane's tiles load meanwhile)
      for (int k = warp; k < nS; k += NW) {
        float2* rr = R + k * PL;
        Fft<NX, false>::go(rr, twx, lane);
        const int4 rw = rows[k];  // ky, first sample, end
        const int rpar = (kz + rw.x) & 1;
        const size_t rb = ((size_t)kz * NY + rw.x) * NX;
        const bool whole = rw.z - rw.y == NX;
        for (int m = rw.y + lane; m < rw.z; m += 32) {
          const int kx = whole ? m - rw.y : (int)(idx[m] - rb);
          const float sg = ((kx + rpar) & 1) ? -ksign : ksign;
          const float2 v = rr[pad8(kx)];
          y[(size_t)c * M + m] = make_float2(v.x * sg, v.y * sg);
        }
      }
      if (j + 1 < nmine) store_plane_meta<NY>(nxt, kmax, mrows + (cur ^ 1) * kmax, mslot + (cur ^ 1) * NY, mn + (cur ^ 1));
      __syncthreads();
    } else {
      // rows with samples: zero-fill (partial rows), scatter with the k-side sign, inverse DFT along x
      for (int k = warp; k < nS; k += NW) {
        float2* rr = R + k * PL;
        const int4 rw = rows[k];
        const bool whole = rw.z - rw.y == NX;
        if (!whole) {
          for (int i = lane; i < PL; i += 32) rr[i] = make_float2(0.f, 0.f);
          __syncwarp();
        }
        const int rpar = (kz + rw.x) & 1;
        if (whole) {  // a whole readout: all loads first
          float2 v[NX / 32];
#pragma unroll
          for (int u = 0; u < NX / 32; ++u) v[u] = y[(size_t)c * M + rw.y + lane + 32 * u];
#pragma unroll
          for (int u = 0; u < NX / 32; ++u) {
            const int kx = lane + 32 * u;
            const float sg = ((kx + rpar) & 1) ? -ksign : ksign;
            rr[pad8(kx)] = make_float2(v[u].x * sg, v[u].y * sg);
          }
        } else {
          const size_t rb = ((size_t)kz * NY + rw.x) * NX;
          for (int m = rw.y + lane; m < rw.z; m += 32) {
            const int kx = (int)(idx[m] - rb);
            const float sg = ((kx + rpar) & 1) ? -ksign : ksign;
            const float2 v = y[(size_t)c * M + m];
            rr[pad8(kx)] = make_float2(v.x * sg, v.y * sg);
          }
        }
        __syncwarp();
        Fft<NX, true>::go(rr, twx, lane);
      }
      __syncthreads();
      for (int t = 0; t < TP; ++t, ++g) {
        const int b = g % NB;
        float2* B = bufs + (size_t)b * NY * TC;
        // inverse along y: the forward two-step on conjugated values, conjugated back
        for (int it = tid; it < TC * R2; it += NT) {
          const int col = it % TC, r = it / TC;
          float2 v[8];
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int s = slot[r + R2 * m];
            const float2 u = s >= 0 ? R[s * PL + pad8(t * TC + col)] : make_float2(0.f, 0.f);
            v[m] = make_float2(u.x, -u.y);
          }
          mpi_dft::dft8(v);
#pragma unroll
          for (int k1 = 1; k1 < 8; ++k1) v[k1] = mpi_dft::cmulf(v[k1], twy[r * k1]);
#pragma unroll
          for (int k1 = 0; k1 < 8; ++k1) B[(r + R2 * k1) * TC + col] = v[k1];
        }
        if (t == TP - 1 && j + 1 < nmine)
          store_plane_meta<NY>(nxt, kmax, mrows + (cur ^ 1) * kmax, mslot + (cur ^ 1) * NY, mn + (cur ^ 1));
        __syncthreads();
        // rows R2 k1 + k2 of the buffer take output row y = k1 + 8 k2
        for (int it = tid; it < TC * 8; it += NT) {
          const int col = it % TC, k1 = it / TC;
          float2 u[R2];
#pragma unroll
          for (int r = 0; r < R2; ++r) u[r] = B[(R2 * k1 + r) * TC + col];
          mpi_dft::dft_r<R2>(u);
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) B[(R2 * k1 + k2) * TC + col] = make_float2(u[k2].x, -u[k2].y);
        }
        mpi_ptx::fence_proxy_async();  // the buffer's writes before the TMA store reads them
        // the buffer the next tile writes was last stored NB tiles ago
        if (tid == 0) mpi_ptx::bulk_wait_read<NB - 2>();
        __syncthreads();
        if (tid == 0) {
#pragma unroll
          for (int k1 = 0; k1 < 8; ++k1)
            mpi_ptx::tma_store_4d(&tmap, B + (size_t)R2 * k1 * TC, t * 2 * TC, k1, 0, pl);
          mpi_ptx::bulk_commit();
        }
      }
    }
  }
  if (INV && tid == 0) mpi_ptx::bulk_wait_all();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map over FP32 data (no swizzle, no out-of-range fill needed: every
// box lies inside the volume).  strides: bytes, one per dimension above the first.
bool encode_f32_map(CUtensorMap* map, void* ptr, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                    const cuuint32_t* box) {
  static void* fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult qr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
    if (e != cudaSuccess || qr != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      fn = nullptr;
      return false;
    }
  }
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return ((EncodeTiledFn)fn)(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, ptr, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

mpi_status launch_fft_cols(mpi_ctx* ctx, float2* data, int C, int nz, int ny, int nx, bool inverse,
                           const uint8_t* row_has) {
  // lines along y: stride nx; slabs = (c, z); base = slab * ny * nx; row mask [z][y]
  const long plane = (long)ny * nx;
  if (inverse) return lines_dispatch<true>(ctx, "k_fft_lines<y,inv>", data, ny, nx, nx, C * nz, 1, plane, 0, row_has, nz);
  return lines_dispatch<false>(ctx, "k_fft_lines<y,fwd>", data, ny, nx, nx, C * nz, 1, plane, 0, row_has, nz);
}

mpi_status launch_fft_cols_window(mpi_ctx* ctx, float2* grid, int C, int G, const float2* src, float2* dst,
                                  const float* deap, int n, bool inverse) {
  if (C == 0) return MPI_OK;
  const long blocks = (long)C * (G / 8);
  if (blocks > 0x7fffffffL) return set_err(ctx, MPI_ERR_SHAPE, "too many FFT tiles");
  const float2* tw = twiddle_table(ctx, G);
  if (!tw) return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
  const LineWin win{src, dst, deap, n, G / 2 - n / 2};
#define MPI_WIN_CASE(L)                                                                                    \
  case L:                                                                                                  \
    if (inverse)                                                                                           \
      launch_pdl(ctx, k_fft_lines_win<L, true>, dim3((unsigned)blocks), dim3(kLineWarps * 32), 0, grid, C, win, tw); \
    else                                                                                                   \
      launch_pdl(ctx, k_fft_lines_win<L, false>, dim3((unsigned)blocks), dim3(kLineWarps * 32), 0, grid, C, win, tw); \
    break;
  MPI_PROF(ctx, KF_FFT_LINES);
  switch (G) {
    MPI_WIN_CASE(16)
    MPI_WIN_CASE(32)
    MPI_WIN_CASE(48)
    MPI_WIN_CASE(64)
    MPI_WIN_CASE(96)
    MPI_WIN_CASE(128)
    MPI_WIN_CASE(192)
    MPI_WIN_CASE(256)
    MPI_WIN_CASE(320)
    MPI_WIN_CASE(512)
    default:
      return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
  }
#undef MPI_WIN_CASE
  MPI_LAUNCH_CHECK(ctx, "k_fft_lines_win");
  return MPI_OK;
}

mpi_status launch_fft_z(mpi_ctx* ctx, float2* data, int C, int nz, int ny, int nx, bool inverse) {
  // lines along z: stride ny * nx; slabs = (c, y); base = c * vol + y * nx
  const long plane = (long)ny * nx;
  const long vol = plane * nz;
  if (inverse) return lines_dispatch<true>(ctx, "k_fft_lines<z,inv>", data, nz, nx, plane, C * ny, ny, vol, nx);
  return lines_dispatch<false>(ctx, "k_fft_lines<z,fwd>", data, nz, nx, plane, C * ny, ny, vol, nx);
}

mpi_status tune_line_passes(mpi_ctx* ctx, const mpi_plan* plan, int C) {
  if (!ctx->autotune || plan->kind != MPI_TRAJ_CARTESIAN || C < 1) return MPI_OK;
  const size_t cn = (size_t)C * plan->N;
  if (!ctx->work || ctx->work_bytes < 2 * cn * sizeof(float2)) return MPI_OK;
  // the workspace's second [C][N] buffer, as in the operator calls
  void* saved = ctx->tune_scratch;
  const size_t saved_bytes = ctx->tune_scratch_bytes;
  float2* base = (float2*)ctx->work;
  ctx->tune_scratch = base + cn;
  ctx->tune_scratch_bytes = cn * sizeof(float2);
  const int nz = plan->nz, ny = plan->ny, nx = plan->nx;
  const long plane = (long)ny * nx, vol = plane * nz;
  const float2* twy = twiddle_table(ctx, ny);
  if (twy) {
    lines_choose<false>(ctx, base, ny, nx, nx, C * nz, 1, plane, 0, twy, plan->row_has, nz);
    lines_choose<true>(ctx, base, ny, nx, nx, C * nz, 1, plane, 0, twy, plan->row_has, nz);
  }
  const float2* twz = plan->ndim == 3 ? twiddle_table(ctx, nz) : nullptr;
  if (twz) {
    lines_choose<false>(ctx, base, nz, nx, plane, C * ny, ny, vol, nx, twz, nullptr, 1);
    lines_choose<true>(ctx, base, nz, nx, plane, C * ny, ny, vol, nx, twz, nullptr, 1);
  }
  ctx->tune_scratch = saved;
  ctx->tune_scratch_bytes = saved_bytes;
  return cuda_check(ctx, cudaGetLastError(), "line-pass tuning");
}

bool plane_pass_supported(const mpi_plan* plan) {
  if (plan->kind != MPI_TRAJ_CARTESIAN || plan->ndim != 3) return false;
  const int ny = plan->ny, nx = plan->nx;
  return (ny == 64 || ny == 96 || ny == 128) && (nx == 64 || nx == 96 || nx == 128);
}

namespace {

// The pipelined plane passes: false (nothing launched) where they do not
// apply (shared memory for the plane's rows with samples, alignment).
template <int NY, int NX>
bool try_plane_pipe(mpi_ctx* ctx, const mpi_plan* plan, float2* data, int C, float2* y, bool inverse,
                    const float2* twy, const float2* twx, float ks, mpi_status* st) {
  const int kmax = plan->plane_kmax;
  const size_t smem = PipeLayout<NY, NX>::total(kmax);
  if (!plan->plane_rows || smem > 227 * 1024 || ((uintptr_t)data & 15)) return false;
  const long planes = (long)C * plan->nz;
  CUtensorMap map;
  bool ok;
  if (!inverse) {
    const cuuint64_t dims[3] = {(cuuint64_t)2 * NX, (cuuint64_t)NY, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)NX * sizeof(float2), (cuuint64_t)NY * NX * sizeof(float2)};
    const cuuint32_t box[3] = {2 * pipe_cols(NX), NY, 1};
    ok = encode_f32_map(&map, data, 3, dims, strides, box);
  } else {
    // rows y = k1 + 8 k2 as dimensions (k1, k2): one box per k1 holds rows k2 = 0 .. NY/8 - 1
    const cuuint64_t dims[4] = {(cuuint64_t)2 * NX, 8, (cuuint64_t)NY / 8, (cuuint64_t)planes};
    const cuuint64_t strides[3] = {(cuuint64_t)NX * sizeof(float2), (cuuint64_t)8 * NX * sizeof(float2),
                                   (cuuint64_t)NY * NX * sizeof(float2)};
    const cuuint32_t box[4] = {2 * pipe_cols(NX), 1, NY / 8, 1};
    ok = encode_f32_map(&map, data, 4, dims, strides, box);
  }
  if (!ok) return false;
  auto kern = inverse ? k_plane_pipe<NY, NX, true> : k_plane_pipe<NY, NX, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPipeThreads, smem);
  if (e != cudaSuccess) {
    *st = cuda_check(ctx, e, "plane pipe attributes");
    return true;
  }
  const long grid = std::min(planes, (long)ctx->num_sms * std::max(per_sm, 1));
  MPI_PROF(ctx, KF_FFT_ROWS);
  e = launch_pdl(ctx, kern, dim3((unsigned)grid), dim3(kPipeThreads), smem, map, y, plan->nz, (int)planes, kmax,
                 (const int32_t*)plan->idx, (const int4*)plan->plane_rows, (const int32_t*)plan->plane_nrows,
                 (const int16_t*)plan->plane_slot, plan->M, ks, twy, twx, ctx->dev_err, ctx->wait_cycles);
  const char* name = inverse ? "k_plane_pipe<inv>" : "k_plane_pipe<fwd>";
  ctx->launches++;
  prof_end(ctx, name);
  if (e == cudaSuccess) e = cudaGetLastError();
  *st = e == cudaSuccess ? MPI_OK : cuda_check(ctx, e, name);
  return true;
}

}  // namespace

mpi_status launch_plane_yx(mpi_ctx* ctx, const mpi_plan* plan, float2* data, int C, float2* y, bool inverse) {
  if (!plane_pass_supported(plan)) return set_err(ctx, MPI_ERR_UNSUPPORTED, "plane pass: shape");
  const long planes = (long)C * plan->nz;
  if (planes == 0) return MPI_OK;
  if (planes > 0x7fffffffL) return set_err(ctx, MPI_ERR_SHAPE, "plane pass: too many planes");
  const float ks = axis_sign(plan->nx) * axis_sign(plan->ny) * axis_sign(plan->nz);
  const float2* twy = twiddle_table(ctx, plan->ny);
  const float2* twx = twiddle_table(ctx, plan->nx);
  if (!twy || !twx) return set_err(ctx, MPI_ERR_SHAPE, "plane pass: no twiddle table");
  cudaError_t e = cudaSuccess;
  if (ctx->plane_pipe) {
    mpi_status st = MPI_OK;
#define MPI_PIPE(NY_, NX_) \
  if (plan->ny == NY_ && plan->nx == NX_ && try_plane_pipe<NY_, NX_>(ctx, plan, data, C, y, inverse, twy, twx, ks, &st)) \
    return st;
    MPI_PIPE(64, 64) MPI_PIPE(64, 96) MPI_PIPE(64, 128)
    MPI_PIPE(96, 64) MPI_PIPE(96, 96) MPI_PIPE(96, 128)
    MPI_PIPE(128, 64) MPI_PIPE(128, 96) MPI_PIPE(128, 128)
#undef MPI_PIPE
  }
#define MPI_PLANE(NY_, NX_)                                                                                    \
  if (plan->ny == NY_ && plan->nx == NX_) {                                                                    \
    const size_t smem = plane_smem<NY_, NX_>();                                                                \
    auto kern = inverse ? k_plane_yx<NY_, NX_, true> : k_plane_yx<NY_, NX_, false>;                            \
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                    \
    if (e != cudaSuccess) return cuda_check(ctx, e, "plane pass smem attribute");                              \
    MPI_PROF(ctx, KF_FFT_ROWS);                                                                                \
    launch_pdl(ctx, kern, dim3((unsigned)planes), dim3(NX_ * 4), smem, data, y, plan->nz, plan->idx,           \
               plan->row_ptr, plan->M, ks, twy, twx);                                                          \
    MPI_LAUNCH_CHECK(ctx, inverse ? "k_plane_yx<inv>" : "k_plane_yx<fwd>");                                    \
    return MPI_OK;                                                                                             \
  }
  MPI_PLANE(64, 64) MPI_PLANE(64, 96) MPI_PLANE(64, 128)
  MPI_PLANE(96, 64) MPI_PLANE(96, 96) MPI_PLANE(96, 128)
  MPI_PLANE(128, 64) MPI_PLANE(128, 96) MPI_PLANE(128, 128)
#undef MPI_PLANE
  return set_err(ctx, MPI_ERR_UNSUPPORTED, "plane pass: shape");
}

mpi_status launch_rows_fwd_gather(mpi_ctx* ctx, const mpi_plan* plan, const float2* data, int C,
                                  float2* y) {
  if (plan->M == 0 || C == 0) return MPI_OK;
  const int n_rows = plan->n_rows;
  if ((long)C * n_rows > 0x7fffffffL) return set_err(ctx, MPI_ERR_SHAPE, "too many k-space rows");
  const long blocks = std::min(((long)C * n_rows + kRowWarps - 1) / kRowWarps, 16L * std::max(ctx->num_sms, 1));
  const float ks = axis_sign(plan->nx) * axis_sign(plan->ny) * (plan->ndim == 3 ? axis_sign(plan->nz) : 1.f);
  const float2* tw = twiddle_table(ctx, plan->nx);
  if (!tw) return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
#define MPI_ROWS_CASE(n)                                                                          \
  case n:                                                                                         \
    launch_pdl(ctx, k_rows_fwd_gather<n>, dim3((unsigned)blocks), dim3(kRowWarps * 32), 0, data, C, n_rows, \
               plan->ny, plan->idx, plan->row_ptr, y, plan->M, ks, tw);                           \
    break;
  MPI_PROF(ctx, KF_FFT_ROWS);
  switch (plan->nx) {
    MPI_ROWS_CASE(16)
    MPI_ROWS_CASE(32)
    MPI_ROWS_CASE(48)
    MPI_ROWS_CASE(64)
    MPI_ROWS_CASE(96)
    MPI_ROWS_CASE(128)
    MPI_ROWS_CASE(192)
    MPI_ROWS_CASE(256)
    MPI_ROWS_CASE(320)
    MPI_ROWS_CASE(512)
    default:
      return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
  }
#undef MPI_ROWS_CASE
  MPI_LAUNCH_CHECK(ctx, "k_rows_fwd_gather");
  return MPI_OK;
}

mpi_status launch_rows_scatter_inv(mpi_ctx* ctx, const mpi_plan* plan, const float2* y, int C,
                                   float2* data) {
  if (C == 0) return MPI_OK;
  const int n_rows = plan->n_rows;
  if ((long)C * n_rows > 0x7fffffffL) return set_err(ctx, MPI_ERR_SHAPE, "too many k-space rows");
  const long blocks = std::min(((long)C * n_rows + kRowWarps - 1) / kRowWarps, 16L * std::max(ctx->num_sms, 1));
  const float ks = axis_sign(plan->nx) * axis_sign(plan->ny) * (plan->ndim == 3 ? axis_sign(plan->nz) : 1.f);
  const float2* tw = twiddle_table(ctx, plan->nx);
  if (!tw) return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
#define MPI_ROWS_CASE(n)                                                                          \
  case n:                                                                                         \
    launch_pdl(ctx, k_rows_scatter_inv<n>, dim3((unsigned)blocks), dim3(kRowWarps * 32), 0, y, C, n_rows, \
               plan->ny, plan->idx, plan->row_ptr, data, plan->M, ks, tw);                        \
    break;
  MPI_PROF(ctx, KF_FFT_ROWS);
  switch (plan->nx) {
    MPI_ROWS_CASE(16)
    MPI_ROWS_CASE(32)
    MPI_ROWS_CASE(48)
    MPI_ROWS_CASE(64)
    MPI_ROWS_CASE(96)
    MPI_ROWS_CASE(128)
    MPI_ROWS_CASE(192)
    MPI_ROWS_CASE(256)
    MPI_ROWS_CASE(320)
    MPI_ROWS_CASE(512)
    default:
      return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
  }
#undef MPI_ROWS_CASE
  MPI_LAUNCH_CHECK(ctx, "k_rows_scatter_inv");
  return MPI_OK;
}

namespace {

// In-place FFT of contiguous lines of length L, one warp per line.  Elements
// outside [load_lo, load_hi) are taken as zero without being read (the radial
// forward's padded columns), and only [keep_lo, keep_hi) of each transformed
// line is stored back (the radial adjoint keeps the columns that its cropping
// pass along y reads).
template <int L, bool INV>
__global__ void __launch_bounds__(kRowWarps * 32) k_fft_rows_inplace(float2* __restrict__ data, long n_rows,
                                                                    const float2* __restrict__ tw_g, int load_lo,
                                                                    int load_hi, int keep_lo, int keep_hi) {
  mpi_ptx::pdl_trigger();
  mpi_ptx::pdl_wait();
  __shared__ float2 tw[L];
  __shared__ float2 buf[kRowWarps][padded_len(L)];
  for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = tw_g[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long row = (long)blockIdx.x * kRowWarps + warp;
  float2* src = data + (size_t)(row < n_rows ? row : 0) * L;
  float2* b = buf[warp];
  if (row < n_rows) {
#pragma unroll
    for (int i = lane; i < L; i += 32)
      b[pad8(i)] = (i >= load_lo && i < load_hi) ? src[i] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (row >= n_rows) return;
  Fft<L, INV>::go(b, tw, lane);
#pragma unroll
  for (int i = lane; i < L; i += 32)
    if (i >= keep_lo && i < keep_hi) src[i] = b[pad8(i)];
}

template <bool INV>
mpi_status rows_inplace_dispatch(mpi_ctx* ctx, float2* data, long n_rows, int L, int load_lo, int load_hi,
                                 int keep_lo, int keep_hi) {
  const long blocks = (n_rows + kRowWarps - 1) / kRowWarps;
  if (blocks == 0) return MPI_OK;
  const float2* tw = twiddle_table(ctx, L);
  if (!tw) return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
#define MPI_RI_CASE(n)                                                                           \
  case n:                                                                                        \
    launch_pdl(ctx, k_fft_rows_inplace<n, INV>, dim3((unsigned)blocks), dim3(kRowWarps * 32), 0, data, n_rows, \
               tw, load_lo, load_hi, keep_lo, keep_hi);                                           \
    break;
  MPI_PROF(ctx, KF_FFT_ROWS);
  switch (L) {
    MPI_RI_CASE(16)
    MPI_RI_CASE(32)
    MPI_RI_CASE(48)
    MPI_RI_CASE(64)
    MPI_RI_CASE(96)
    MPI_RI_CASE(128)
    MPI_RI_CASE(192)
    MPI_RI_CASE(256)
    MPI_RI_CASE(320)
    MPI_RI_CASE(512)
    default:
      return set_err(ctx, MPI_ERR_SHAPE, "unsupported FFT length");
  }
#undef MPI_RI_CASE
  MPI_LAUNCH_CHECK(ctx, "k_fft_rows_inplace");
  return MPI_OK;
}

}  // namespace

mpi_status launch_fft_rows_inplace(mpi_ctx* ctx, float2* data, long n_rows, int L, bool inverse, int load_lo,
                                   int load_hi, int keep_lo, int keep_hi) {
  if (load_hi < 0) load_hi = L;
  if (keep_hi < 0) keep_hi = L;
  if (inverse) return rows_inplace_dispatch<true>(ctx, data, n_rows, L, load_lo, load_hi, keep_lo, keep_hi);
  return rows_inplace_dispatch<false>(ctx, data, n_rows, L, load_lo, load_hi, keep_lo, keep_hi);
}
