// Small DFTs held in registers (one thread, complex float2 values):
// X[k] = sum_n x[n] exp(-2 pi i n k / R) for R = 3, 4, 8, 12, 16, with the
// constants of the roots of unity written out (cos and sin of multiples of
// pi / 8 and pi / 6).  Shared by the fused Tucker kernels and the register
// column FFT.
#pragma once

#include <cuda_runtime.h>

namespace mpi_dft {

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // -i a
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Forward DFTs in registers, X[k] = sum_n x[n] exp(-2 pi i n k / R).
__host__ __device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

__host__ __device__ __forceinline__ void dft3(float2& x0, float2& x1, float2& x2) {
  // exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
  const float s = 0.86602540378443865f;
  const float2 t = cadd(x1, x2), d = csub(x1, x2);
  const float2 m = make_float2(x0.x - 0.5f * t.x, x0.y - 0.5f * t.y);
  const float2 isd = make_float2(s * d.y, -s * d.x);  // -i s d
  x0 = cadd(x0, t);
  x1 = cadd(m, isd);
  x2 = csub(m, isd);
}

__host__ __device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 s02 = cadd(x0, x2), d02 = csub(x0, x2);
  const float2 s13 = cadd(x1, x3), d13 = mul_mi(csub(x1, x3));
  x0 = cadd(s02, s13);
  x2 = csub(s02, s13);
  x1 = cadd(d02, d13);
  x3 = csub(d02, d13);
}

__host__ __device__ __forceinline__ void dft8(float2 (&v)[8]) {
  // radix-2 split: 4-point DFTs of the even and odd samples, then the combine
  // with exp(-2 pi i m / 8), m < 4
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  const float h = 0.70710678118654752f;
  o1 = make_float2(h * (o1.x + o1.y), h * (o1.y - o1.x));   // x exp(-i pi/4)
  o2 = mul_mi(o2);                                           // x -i
  o3 = make_float2(h * (o3.y - o3.x), -h * (o3.x + o3.y));  // x exp(-3 i pi/4)
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

// 12 = 3 x 4: n = 3 n2 + n1, k = k1 + 4 k2; 4-point DFTs over n2, twiddles
// exp(-2 pi i n1 k1 / 12), 3-point DFTs over n1.
__host__ __device__ __forceinline__ void dft12(float2 (&v)[12]) {
  float2 y[3][4];
#pragma unroll
  for (int n1 = 0; n1 < 3; ++n1) {
    y[n1][0] = v[n1];
    y[n1][1] = v[3 + n1];
    y[n1][2] = v[6 + n1];
    y[n1][3] = v[9 + n1];
    dft4(y[n1][0], y[n1][1], y[n1][2], y[n1][3]);
  }
  const float c30 = 0.86602540378443865f;  // cos(pi/6)
  // n1 = 1: m = k1 (0..3); n1 = 2: m = 2 k1 (0, 2, 4, 6)
  y[1][1] = cmulf(y[1][1], make_float2(c30, -0.5f));
  y[1][2] = cmulf(y[1][2], make_float2(0.5f, -c30));
  y[1][3] = mul_mi(y[1][3]);
  y[2][1] = cmulf(y[2][1], make_float2(0.5f, -c30));
  y[2][2] = cmulf(y[2][2], make_float2(-0.5f, -c30));
  y[2][3] = make_float2(-y[2][3].x, -y[2][3].y);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    dft3(y[0][k1], y[1][k1], y[2][k1]);
    v[k1] = y[0][k1];
    v[k1 + 4] = y[1][k1];
    v[k1 + 8] = y[2][k1];
  }
}

// 16 = 4 x 4: n = 4 n2 + n1, k = k1 + 4 k2; twiddles exp(-2 pi i n1 k1 / 16).
__host__ __device__ __forceinline__ void dft16(float2 (&v)[16]) {
  float2 y[4][4];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    y[n1][0] = v[n1];
    y[n1][1] = v[4 + n1];
    y[n1][2] = v[8 + n1];
    y[n1][3] = v[12 + n1];
    dft4(y[n1][0], y[n1][1], y[n1][2], y[n1][3]);
  }
  const float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  const float2 w1 = make_float2(c1, -s1), w2 = make_float2(h, -h), w3 = make_float2(s1, -c1);
  const float2 w6 = make_float2(-h, -h), w9 = make_float2(-c1, s1);
  y[1][1] = cmulf(y[1][1], w1);
  y[1][2] = cmulf(y[1][2], w2);
  y[1][3] = cmulf(y[1][3], w3);
  y[2][1] = cmulf(y[2][1], w2);
  y[2][2] = mul_mi(y[2][2]);
  y[2][3] = cmulf(y[2][3], w6);
  y[3][1] = cmulf(y[3][1], w3);
  y[3][2] = cmulf(y[3][2], w6);
  y[3][3] = cmulf(y[3][3], w9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    dft4(y[0][k1], y[1][k1], y[2][k1], y[3][k1]);
    v[k1] = y[0][k1];
    v[k1 + 4] = y[1][k1];
    v[k1 + 8] = y[2][k1];
    v[k1 + 12] = y[3][k1];
  }
}

template <int R>
__host__ __device__ __forceinline__ void dft_r(float2 (&v)[R]) {
  if constexpr (R == 8) dft8(v);
  else if constexpr (R == 12) dft12(v);
  else dft16(v);
}


}  // namespace mpi_dft
