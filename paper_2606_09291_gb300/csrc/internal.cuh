// internal.cuh - device helpers shared by the kernels of libmlsgd (sm_103a).
//
// Discretisation (Sec. 5: -div(exp(a~) grad y) = u on the unit cube, V = H^1_0):
// Q1 hexahedra, N cells per side, mesh width h = 1/N, coefficient a constant per
// cell.  Node (i,j,k) has flat index i + (N+1)(j + (N+1)k); cell (i,j,k) has
// i + N(j + Nk).  Boundary nodes are stored and always hold 0.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "mlsgd.h"

namespace mlsgd {

constexpr int kBlock = 256;

// ---------------------------------------------------------------- precision glue
template <typename T> __device__ __forceinline__ T from_coef(double v) { return (T)v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <typename T> __device__ __forceinline__ T load_coef(const double* p) { return (T)__ldg(p); }
template <typename T> __device__ __forceinline__ T load_coef(const float* p) { return (T)__ldg(p); }
template <typename T> __device__ __forceinline__ T load_coef(const __nv_bfloat16* p) {
  return (T)__bfloat162float(*p);
}

// value already in registers / shared memory, converted to the arithmetic type
template <typename T> __device__ __forceinline__ T smem_coef(double v) { return (T)v; }
template <typename T> __device__ __forceinline__ T smem_coef(float v) { return (T)v; }
template <typename T> __device__ __forceinline__ T smem_coef(__nv_bfloat16 v) { return (T)__bfloat162float(v); }

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): 10 rounds; a round multiplies counter words 0 and 2 by the two
// published multipliers and mixes the high halves with the other words and the
// key; the key is bumped by the two Weyl constants between rounds.
struct U4 { uint32_t x, y, z, w; };
__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * c.x;
    const uint64_t p1 = (uint64_t)M1 * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}
// 53-bit uniform in (0, 1]
__host__ __device__ inline double uniform53(uint32_t hi, uint32_t lo) {
  const uint64_t m = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
  return (double)(m + 1) * 0x1p-53;
}

// ---------------------------------------------------------------- Q1 operator
// For a node with the eight surrounding cells c[p][q][r] (cell (i-1+p, j-1+q,
// k-1+r)), the assembled Q1 stiffness row is h/12 times
//   4 (sum of the 8 cells) x_0
//   - sum over the 12 face-diagonal neighbours (u,v,0), (u,0,w), (0,v,w) of
//     (sum of the two cells sharing that face diagonal) x_nb
//   - sum over the 8 body-diagonal neighbours of (the one shared cell) x_nb;
// edge neighbours have coefficient 0 (element matrix h K_ref, K_ref with
// diagonal 1/3, edge 0, face and body diagonals -1/12).
template <typename T, typename TA>
struct Cells8 {
  T c[2][2][2];
  T sum;
  __device__ __forceinline__ void load(const TA* __restrict__ a, int i, int j, int k, int N) {
    sum = T(0);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const T v = load_coef<T>(a + (i - 1 + p) + (long long)N * ((j - 1 + q) + (long long)N * (k - 1 + r)));
          c[p][q][r] = v;
          sum += v;
        }
  }
};

// (A x)_node / (h/12) for an interior node
template <typename T, typename TA>
__device__ __forceinline__ T q1_row(const Cells8<T, TA>& C, const T* __restrict__ x, int i, int j, int k, int n1) {
  const long long s1 = n1, s2 = (long long)n1 * n1;
  const T* xc = x + i + s1 * j + s2 * k;
  T acc = T(4) * C.sum * xc[0];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const long long du = 2 * p - 1, dv = 2 * q - 1;
      // xy face diagonal (u, v, 0): cells (p, q, 0) and (p, q, 1)
      acc -= (C.c[p][q][0] + C.c[p][q][1]) * xc[du + s1 * dv];
      // xz face diagonal (u, 0, w): cells (p, 0, r) and (p, 1, r), w = 2q-1 here
      acc -= (C.c[p][0][q] + C.c[p][1][q]) * xc[du + s2 * dv];
      // yz face diagonal (0, v, w): cells (0, p, q) and (1, p, q)
      acc -= (C.c[0][p][q] + C.c[1][p][q]) * xc[s1 * du + s2 * dv];
    }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int p = 0; p < 2; ++p)
        acc -= C.c[p][q][r] * xc[(2 * p - 1) + s1 * (2 * q - 1) + s2 * (2 * r - 1)];
  return acc;
}

__device__ __forceinline__ void node_ijk(int n, int n1, int& i, int& j, int& k) {
  const unsigned t = (unsigned)n / (unsigned)n1;
  i = n - (int)t * n1;
  k = (int)(t / (unsigned)n1);
  j = (int)t - k * n1;
}
__device__ __forceinline__ bool interior(int i, int j, int k, int N) {
  return i > 0 && j > 0 && k > 0 && i < N && j < N && k < N;
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// block of kBlock threads (1-, 2- or 3-D); returns the sum in linear thread 0
template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T red[kBlock / 32];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  v = warp_sum(v);
  const int w = tid >> 5, l = tid & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = T(0);
  if (tid < 32) {
    s = (l < kBlock / 32) ? red[l] : T(0);
    s = warp_sum(s);
  }
  return s;
}

// ---------------------------------------------------------------- FP32 pair arithmetic
// A value is the unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h)/2
// (about 48 significant bits).  Sums use Knuth's two-sum, products the FMA to
// recover the rounding error of h*h'; both renormalise.  No FP64 instruction.
// The additions and products are the round-to-nearest intrinsics, which the
// compiler never contracts into an FMA: a contracted "s + a*b" would round once
// where the error-free transformations count on two roundings.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_make(float2 v) { return DF{v.x, v.y}; }
__device__ __forceinline__ float2 df_f2(DF a) { return make_float2(a.h, a.l); }
__device__ __forceinline__ DF df_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return DF{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return df_norm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p)));
  return df_norm(p, e);
}
// product with an FP32 number
__device__ __forceinline__ DF df_mulf(DF a, float w) {
  const float p = __fmul_rn(a.h, w);
  const float e = __fmaf_rn(a.l, w, __fmaf_rn(a.h, w, -p));
  return df_norm(p, e);
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.h + (double)a.l; }
__host__ __device__ inline float2 df_split(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

}  // namespace mlsgd
