// Device helpers of the sliced block storage shared by the Krylov solves and
// the multigrid preconditioner: 16-byte vector loads and stores, one row of
// K times x, and the 3x3 inverse-block product.
#pragma once
#include <cuda_fp16.h>

#include "mpm_internal.cuh"

namespace mpm {

// 4-wide loads and stores (16-byte aligned; two 16-byte halves for double)
__device__ inline void ld4(const float* p, float* v) {
  float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ inline void ld4(const double* p, double* v) {
  double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ inline void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ inline void st4(double* p, const double* v) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// y = storage row r of K (dof row S.row[r]) times x, sliced storage (one
// thread per storage row; a warp is one slice).  XS = 4: x padded to 4
// components per dof; XS = 3: plain 3-vectors.
template <class T, class V, class A, int XS>
__device__ inline void sliced_row(int r, Sliced S, const T* __restrict__ K,
                                  const V* __restrict__ x, A* y) {
  int s = r >> 5, ln = r & 31;
  int W = S.w[s];
  long long b0 = S.base[s];
  const T* Kb = K + 9 * b0;
  const int* cb = S.scol + b0;
  size_t plane = (size_t)32 * W;
  y[0] = y[1] = y[2] = (A)0;
  for (int k4 = 0; k4 < (W >> 2); ++k4) {
    size_t off = ((size_t)k4 * 32 + ln) * 4;
    int4 c = *reinterpret_cast<const int4*>(cb + off);
    int cc[4] = {c.x, c.y, c.z, c.w};
    T v[9][4];
#pragma unroll
    for (int e = 0; e < 9; ++e) ld4(Kb + e * plane + off, v[e]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      A x0, x1, x2;
      if (XS == 4) {
        V xv[4];
        ld4(x + 4 * (size_t)cc[j], xv);
        x0 = (A)xv[0]; x1 = (A)xv[1]; x2 = (A)xv[2];
      } else {
        x0 = (A)x[3 * (size_t)cc[j]]; x1 = (A)x[3 * (size_t)cc[j] + 1]; x2 = (A)x[3 * (size_t)cc[j] + 2];
      }
      y[0] += (A)v[0][j] * x0 + (A)v[1][j] * x1 + (A)v[2][j] * x2;
      y[1] += (A)v[3][j] * x0 + (A)v[4][j] * x1 + (A)v[5][j] * x2;
      y[2] += (A)v[6][j] * x0 + (A)v[7][j] * x1 + (A)v[8][j] * x2;
    }
  }
}

template <class V>
__device__ inline void apply_dinv(const V* __restrict__ Dinv, size_t i, const V* rv, V* zv) {
  V d0[4], d1[4], d2[4];
  ld4(Dinv + 12 * i, d0);
  ld4(Dinv + 12 * i + 4, d1);
  ld4(Dinv + 12 * i + 8, d2);
  zv[0] = d0[0] * rv[0] + d0[1] * rv[1] + d0[2] * rv[2];
  zv[1] = d1[0] * rv[0] + d1[1] * rv[1] + d1[2] * rv[2];
  zv[2] = d2[0] * rv[0] + d2[1] * rv[1] + d2[2] * rv[2];
  zv[3] = (V)0;
}

// y = storage row r of K times x with FP32 values and FP64 x, accumulated in
// double-float arithmetic: each product k * x is split exactly as
// k * x_hi = p + e (Dekker's two-product through one fused multiply-add),
// k * x_lo is added to the error term, and p enters a (hi, lo) pair of floats
// by Knuth's two-sum.  The sum carries about 48 significant bits, enough for
// the FP64 refinement residual, while every operation runs on the FP32 pipe
// (GB300 issues FP64 at 1/64 of the FP32 rate).
__device__ inline void df_acc(float& hi, float& lo, float k, float xh, float xl) {
  float p = k * xh;
  float e = fmaf(k, xh, -p);
  e = fmaf(k, xl, e);
  float s = hi + p;
  float bv = s - hi;
  float err = (hi - (s - bv)) + (p - bv);
  hi = s;
  lo += err + e;
}

__device__ inline void sliced_row_df(int r, Sliced S, const float* __restrict__ K,
                                     const float4* __restrict__ xs, double* y) {
  int s = r >> 5, ln = r & 31;
  int W = S.w[s];
  long long b0 = S.base[s];
  const float* Kb = K + 9 * b0;
  const int* cb = S.scol + b0;
  size_t plane = (size_t)32 * W;
  float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
  for (int k4 = 0; k4 < (W >> 2); ++k4) {
    size_t off = ((size_t)k4 * 32 + ln) * 4;
    int4 c = *reinterpret_cast<const int4*>(cb + off);
    int cc[4] = {c.x, c.y, c.z, c.w};
    float v[9][4];
#pragma unroll
    for (int e = 0; e < 9; ++e) ld4(Kb + e * plane + off, v[e]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // x split into hi and lo floats, two 16-byte loads per column
      float4 p0 = xs[2 * (size_t)cc[j]], p1 = xs[2 * (size_t)cc[j] + 1];
      float xh[3] = {p0.x, p0.z, p1.x}, xl[3] = {p0.y, p0.w, p1.y};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) df_acc(h[a], l[a], v[3 * a + d][j], xh[d], xl[d]);
    }
  }
  for (int a = 0; a < 3; ++a) y[a] = (double)h[a] + (double)l[a];
}

// x (FP64, 3 per dof) -> (hi, lo) float pairs, 8 floats per dof (padding zero)
__global__ inline void k_split_df(int npad, int nd, const double* __restrict__ x, float4* xs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  float hl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (i < nd)
    for (int d = 0; d < 3; ++d) {
      double v = x[3 * (size_t)i + d];
      float hi = (float)v;
      hl[2 * d] = hi;
      hl[2 * d + 1] = (float)(v - (double)hi);
    }
  xs[2 * (size_t)i] = make_float4(hl[0], hl[1], hl[2], hl[3]);
  xs[2 * (size_t)i + 1] = make_float4(hl[4], hl[5], 0.f, 0.f);
}

// The FP16 copy of K keeps the sliced block order but stores the entry
// planes of a slice in pairs: for planes 2q and 2q + 1 (q < 4), the 4 blocks
// of a lane's group of one plane, then the same 4 blocks of the other, in one
// 16-byte word per lane at Kh[9 base + 2q (32 W) + 2 off]; plane 8 as in the
// FP32 layout, 8 bytes per lane at Kh[9 base + 8 (32 W) + off]
// (off = (group 32 + lane) 4).  A group of four blocks is then five loads
// instead of nine.

// one group of four FP16 blocks (the four 16-byte plane pairs and plane 8)
// times x
__device__ inline void acc_h4(const uint4* u, uint2 u8, int4 c, const float* __restrict__ x, float* y) {
  int cc[4] = {c.x, c.y, c.z, c.w};
  float v[9][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float2 a0 = __half22float2(*reinterpret_cast<const __half2*>(&u[q].x));
    float2 a1 = __half22float2(*reinterpret_cast<const __half2*>(&u[q].y));
    float2 b0 = __half22float2(*reinterpret_cast<const __half2*>(&u[q].z));
    float2 b1 = __half22float2(*reinterpret_cast<const __half2*>(&u[q].w));
    v[2 * q][0] = a0.x;
    v[2 * q][1] = a0.y;
    v[2 * q][2] = a1.x;
    v[2 * q][3] = a1.y;
    v[2 * q + 1][0] = b0.x;
    v[2 * q + 1][1] = b0.y;
    v[2 * q + 1][2] = b1.x;
    v[2 * q + 1][3] = b1.y;
  }
  {
    float2 a0 = __half22float2(*reinterpret_cast<const __half2*>(&u8.x));
    float2 a1 = __half22float2(*reinterpret_cast<const __half2*>(&u8.y));
    v[8][0] = a0.x;
    v[8][1] = a0.y;
    v[8][2] = a1.x;
    v[8][3] = a1.y;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float xv[4];
    ld4(x + 4 * (size_t)cc[j], xv);
    y[0] += v[0][j] * xv[0] + v[1][j] * xv[1] + v[2][j] * xv[2];
    y[1] += v[3][j] * xv[0] + v[4][j] * xv[1] + v[5][j] * xv[2];
    y[2] += v[6][j] * xv[0] + v[7][j] * xv[1] + v[8][j] * xv[2];
  }
}

__device__ inline void load_h4(const __half* Kb, size_t plane, size_t off, uint4* u, uint2& u8) {
#pragma unroll
  for (int q = 0; q < 4; ++q) u[q] = *reinterpret_cast<const uint4*>(Kb + 2 * q * plane + 2 * off);
  u8 = *reinterpret_cast<const uint2*>(Kb + 8 * plane + off);
}

// y = storage row r of the FP16 copy of K (values scaled by a power of two) times x;
// FP32 arithmetic, the caller undoes the scale.  Two groups of four blocks
// per trip, all of their loads issued before the arithmetic: FP16 blocks are
// half the bytes of FP32 ones, so a trip over one group would keep half as
// many bytes in flight as the FP32 row product.
__device__ inline void sliced_row_h(int r, Sliced S, const __half* __restrict__ K,
                                    const float* __restrict__ x, float* y) {
  int s = r >> 5, ln = r & 31;
  int W = S.w[s];
  long long b0 = S.base[s];
  const __half* Kb = K + 9 * b0;
  const int* cb = S.scol + b0;
  size_t plane = (size_t)32 * W;
  y[0] = y[1] = y[2] = 0.f;
  int n4 = W >> 2, k4 = 0;
  for (; k4 + 2 <= n4; k4 += 2) {
    size_t off0 = ((size_t)k4 * 32 + ln) * 4, off1 = off0 + 128;
    int4 c0 = *reinterpret_cast<const int4*>(cb + off0);
    int4 c1 = *reinterpret_cast<const int4*>(cb + off1);
    uint4 u0[4], u1[4];
    uint2 v0, v1;
    load_h4(Kb, plane, off0, u0, v0);
    load_h4(Kb, plane, off1, u1, v1);
    acc_h4(u0, v0, c0, x, y);
    acc_h4(u1, v1, c1, x, y);
  }
  if (k4 < n4) {
    size_t off = ((size_t)k4 * 32 + ln) * 4;
    int4 c0 = *reinterpret_cast<const int4*>(cb + off);
    uint4 u0[4];
    uint2 v0;
    load_h4(Kb, plane, off, u0, v0);
    acc_h4(u0, v0, c0, x, y);
  }
}

}  // namespace mpm
