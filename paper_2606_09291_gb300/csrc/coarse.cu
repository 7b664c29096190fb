// coarse.cu - the coarse end of the V-cycle (rows a4, a6) in one launch: the levels
// 16^3, 8^3, 4^3 and 2^3 of a sample's hierarchy in the shared memory of one block.
//
// Below the fused fine-grid passes the V-cycle's levels are small (17^3 nodes and
// less): run level by level, each of the dozen steps (pre-smoothing and residual,
// restriction, the 2^3 solve, prolongation, post-smoothing, per level) is a launch
// whose grid is a few blocks per sample and whose time is mostly launch latency and
// tail.  Here one block per launched sample loads the restricted residual r and the
// four coefficient levels once, runs the whole V(1,1)-cycle below the 32^3 level with
// a block barrier between steps, and writes the correction z of the 16^3 level.
//
// The arithmetic is the V-cycle's (Sec. 5, the preconditioner of the PCG): at every
// level damped Jacobi with x0 = 0 (x = omega D^-1 r), the residual t = r - A x,
// restriction P^T t, recursion, x += P e, post-smoothing z = x + omega D^-1 (r - A x);
// on 2^3 the single interior unknown is solved exactly.  D = (h/3) sum_8 a: on the
// 16^3 level D^-1 is formed as the solver's D^-1 pass forms it (the four-cell sums of
// the planes below and above, then the reciprocal), on 8^3 and 4^3 the smoother
// divides by D as the level-by-level kernels do, and pre- and post-smoothing take
// the same D, so the preconditioner stays symmetric.  Boundary nodes hold 0 in every
// array.  The operator rows are those of the assembled Q1 stiffness (q1_row).
#include <cstdio>
#include <type_traits>

#include "internal.cuh"
#include "kernels.h"
#include "launch.h"

namespace mlsgd {

namespace {

constexpr int kCT = 768;  // threads per block (24 warps: two blocks per SM hide the shared-memory latency)

template <int N>
struct Lv {
  static constexpr int n1 = N + 1, nodes = n1 * n1 * n1, cells = N * N * N;
};

// shared-memory layout (elements of T)
template <typename T>
struct CoarseSmem {
  using L16 = Lv<16>;
  using L8 = Lv<8>;
  using L4 = Lv<4>;
  using L2 = Lv<2>;
  static constexpr int r16 = 0, x16 = r16 + L16::nodes, t16 = x16 + L16::nodes, d16 = t16 + L16::nodes,
                       a16 = d16 + L16::nodes;
  static constexpr int r8 = a16 + L16::cells, x8 = r8 + L8::nodes, t8 = x8 + L8::nodes, a8 = t8 + L8::nodes;
  static constexpr int r4 = a8 + L8::cells, x4 = r4 + L4::nodes, t4 = x4 + L4::nodes, a4 = t4 + L4::nodes;
  static constexpr int r2 = a4 + L4::cells, x2 = r2 + L2::nodes, a2 = x2 + L2::nodes;
  static constexpr int total = a2 + L2::cells;
  static constexpr size_t bytes = sizeof(T) * (size_t)total;
};

// the eight cells around interior node (i, j, k) of an N^3 level held in shared memory
template <typename T>
__device__ __forceinline__ void cells8(Cells8<T, T>& C, const T* a, int i, int j, int k, int N) {
  C.sum = T(0);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const T v = a[(i - 1 + p) + N * ((j - 1 + q) + N * (k - 1 + r))];
        C.c[p][q][r] = v;
        C.sum += v;
      }
}

__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }

// D^-1 of the 16^3 level at every node (0 on the boundary)
template <typename T>
__device__ void dinv_level(const T* a, T* d) {
  constexpr int N = 16, n1 = N + 1;
  const T h3 = T(1.0 / (3.0 * N));
  for (int n = threadIdx.x; n < Lv<N>::nodes; n += kCT) {
    int i, j, k;
    node_ijk(n, n1, i, j, k);
    T v = T(0);
    if (interior(i, j, k, N)) {
      auto sum4 = [&](int c) {
        const T* p = a + (i - 1) + N * (j - 1) + N * N * c;
        return (p[0] + p[1]) + (p[N] + p[N + 1]);
      };
      v = rcp(h3 * (sum4(k - 1) + sum4(k)));
    }
    d[n] = v;
  }
}

// pre-smoothing from 0 and the residual: x = omega D^-1 r (from d, or dividing by D),
// t = r - A x
template <int N, bool DTAB, typename T>
__device__ void pre_level(const T* r, const T* a, const T* d, T* x, T* t, T omega) {
  constexpr int n1 = N + 1;
  const T h3 = T(1.0 / (3.0 * N)), sc = T(1.0 / (12.0 * N));
  for (int n = threadIdx.x; n < Lv<N>::nodes; n += kCT) {
    int i, j, k;
    node_ijk(n, n1, i, j, k);
    T v = T(0);
    if (interior(i, j, k, N)) {
      if (DTAB) {
        v = omega * r[n] * d[n];
      } else {
        Cells8<T, T> C;
        cells8(C, a, i, j, k, N);
        v = omega * r[n] / (h3 * C.sum);
      }
    }
    x[n] = v;
  }
  __syncthreads();
  for (int n = threadIdx.x; n < Lv<N>::nodes; n += kCT) {
    int i, j, k;
    node_ijk(n, n1, i, j, k);
    T v = T(0);
    if (interior(i, j, k, N)) {
      Cells8<T, T> C;
      cells8(C, a, i, j, k, N);
      v = r[n] - sc * q1_row(C, x, i, j, k, n1);
    }
    t[n] = v;
  }
}

// rc = P^T tf (coarse level Nc, weights 1 and 1/2 per axis around the even fine node)
template <int NC, typename T>
__device__ void restrict_level(const T* tf, T* rc) {
  constexpr int n1c = NC + 1, n1f = 2 * NC + 1;
  for (int n = threadIdx.x; n < Lv<NC>::nodes; n += kCT) {
    int I, J, K;
    node_ijk(n, n1c, I, J, K);
    T v = T(0);
    if (interior(I, J, K, NC)) {
      const T* f = tf + 2 * I + n1f * (2 * J) + n1f * n1f * (2 * K);
#pragma unroll
      for (int w = -1; w <= 1; ++w)
#pragma unroll
        for (int u = -1; u <= 1; ++u)
#pragma unroll
          for (int q = -1; q <= 1; ++q) {
            const T wt = T((q == 0 ? 1.0 : 0.5) * (u == 0 ? 1.0 : 0.5) * (w == 0 ? 1.0 : 0.5));
            v += wt * f[q + n1f * u + n1f * n1f * w];
          }
    }
    rc[n] = v;
  }
}

// xf += P ec (trilinear; ec holds 0 on its boundary)
template <int NF, typename T>
__device__ void prolong_level(T* xf, const T* ec) {
  constexpr int n1f = NF + 1, n1c = NF / 2 + 1;
  for (int n = threadIdx.x; n < Lv<NF>::nodes; n += kCT) {
    int i, j, k;
    node_ijk(n, n1f, i, j, k);
    if (!interior(i, j, k, NF)) continue;
    const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    const int i1 = i0 + (i & 1), j1 = j0 + (j & 1), k1 = k0 + (k & 1);
    const T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1), wk = (k & 1) ? T(0.5) : T(1);
    auto at = [&](int a, int b, int c) { return ec[a + n1c * b + n1c * n1c * c]; };
    T v;
    if ((i & 1) == 0 && (j & 1) == 0 && (k & 1) == 0) {
      v = at(i0, j0, k0);
    } else {
      v = wi * wj * wk *
          (at(i0, j0, k0) + ((i & 1) ? at(i1, j0, k0) : T(0)) + ((j & 1) ? at(i0, j1, k0) : T(0)) +
           ((k & 1) ? at(i0, j0, k1) : T(0)) + (((i & 1) && (j & 1)) ? at(i1, j1, k0) : T(0)) +
           (((i & 1) && (k & 1)) ? at(i1, j0, k1) : T(0)) + (((j & 1) && (k & 1)) ? at(i0, j1, k1) : T(0)) +
           (((i & 1) && (j & 1) && (k & 1)) ? at(i1, j1, k1) : T(0)));
    }
    xf[n] += v;
  }
}

// post-smoothing z = x + omega D^-1 (r - A x), written to z (shared or global)
template <int N, bool DTAB, typename T>
__device__ void post_level(const T* r, const T* a, const T* d, const T* x, T* z, T omega) {
  constexpr int n1 = N + 1;
  const T h3 = T(1.0 / (3.0 * N)), sc = T(1.0 / (12.0 * N));
  for (int n = threadIdx.x; n < Lv<N>::nodes; n += kCT) {
    int i, j, k;
    node_ijk(n, n1, i, j, k);
    T v = T(0);
    if (interior(i, j, k, N)) {
      Cells8<T, T> C;
      cells8(C, a, i, j, k, N);
      const T res = r[n] - sc * q1_row(C, x, i, j, k, n1);
      v = DTAB ? x[n] + omega * res * d[n] : x[n] + omega * res / (h3 * C.sum);
    }
    z[n] = v;
  }
}

// asynchronous element copy into shared memory (4 or 8 bytes; the thread waits for its
// own copies, a block barrier then publishes them)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(sizeof(T))
               : "memory");
}

struct CoarseArgs {
  const void* r;      // restricted residual on the 16^3 level, [S][17^3]
  const void* a[4];   // cell coefficient of the levels 16^3, 8^3, 4^3, 2^3, [S][cells]
  void* z;            // the V-cycle's correction on the 16^3 level, [S][17^3]
  const SolveScalars* sc;
  const int* act;
  double omega;
};

template <typename T>
__global__ void __launch_bounds__(kCT, sizeof(T) == 4 ? 2 : 1) k_coarse_vcycle(CoarseArgs A) {
  using M = CoarseSmem<T>;
  const int s = A.act != nullptr ? A.act[blockIdx.x] : (int)blockIdx.x;
  if (A.sc != nullptr && !A.sc[s].active) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = (T*)smraw;
  const T omega = (T)A.omega;
  // r and the four coefficient levels, all copies in flight at once
  const T* rg = (const T*)A.r + (long long)s * Lv<16>::nodes;
  for (int n = threadIdx.x; n < Lv<16>::nodes; n += kCT) cp_async_elem(sm + M::r16 + n, rg + n);
  const int aoff[4] = {M::a16, M::a8, M::a4, M::a2};
  const int acnt[4] = {Lv<16>::cells, Lv<8>::cells, Lv<4>::cells, Lv<2>::cells};
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const T* ag = (const T*)A.a[l] + (long long)s * acnt[l];
    for (int n = threadIdx.x; n < acnt[l]; n += kCT) cp_async_elem(sm + aoff[l] + n, ag + n);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  dinv_level<T>(sm + M::a16, sm + M::d16);
  __syncthreads();
  // down: 16^3, 8^3, 4^3
  pre_level<16, true, T>(sm + M::r16, sm + M::a16, sm + M::d16, sm + M::x16, sm + M::t16, omega);
  __syncthreads();
  restrict_level<8, T>(sm + M::t16, sm + M::r8);
  __syncthreads();
  pre_level<8, false, T>(sm + M::r8, sm + M::a8, nullptr, sm + M::x8, sm + M::t8, omega);
  __syncthreads();
  restrict_level<4, T>(sm + M::t8, sm + M::r4);
  __syncthreads();
  pre_level<4, false, T>(sm + M::r4, sm + M::a4, nullptr, sm + M::x4, sm + M::t4, omega);
  __syncthreads();
  restrict_level<2, T>(sm + M::t4, sm + M::r2);
  __syncthreads();
  // 2^3: the single interior unknown (node 13), x = r / D
  for (int n = threadIdx.x; n < Lv<2>::nodes; n += kCT) {
    T v = T(0);
    if (n == 13) {
      Cells8<T, T> C;
      cells8(C, sm + M::a2, 1, 1, 1, 2);
      v = sm[M::r2 + 13] / (T(1.0 / 6.0) * C.sum);
    }
    sm[M::x2 + n] = v;
  }
  __syncthreads();
  // up: 4^3, 8^3 (the smoothed corrections overwrite the dead residuals t), then 16^3
  prolong_level<4, T>(sm + M::x4, sm + M::x2);
  __syncthreads();
  post_level<4, false, T>(sm + M::r4, sm + M::a4, nullptr, sm + M::x4, sm + M::t4, omega);
  __syncthreads();
  prolong_level<8, T>(sm + M::x8, sm + M::t4);
  __syncthreads();
  post_level<8, false, T>(sm + M::r8, sm + M::a8, nullptr, sm + M::x8, sm + M::t8, omega);
  __syncthreads();
  prolong_level<16, T>(sm + M::x16, sm + M::t8);
  __syncthreads();
  post_level<16, true, T>(sm + M::r16, sm + M::a16, sm + M::d16, sm + M::x16,
                          (T*)A.z + (long long)s * Lv<16>::nodes, omega);
}

}  // namespace

bool coarse_vcycle_applies(int N, int j) { return j >= 1 && (N >> j) == 16; }

template <typename T>
void coarse_vcycle(const T* r16, const T* const a[4], T* z16, const SolveScalars* sc, const Batch& bt, double omega,
                   cudaStream_t st) {
  using M = CoarseSmem<T>;
  static bool smem_set = false;  // once per instantiation (capture-friendly)
  if (!smem_set) {
    cudaFuncSetAttribute(k_coarse_vcycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::bytes);
    smem_set = true;
  }
  CoarseArgs A{};
  A.r = r16;
  for (int l = 0; l < 4; ++l) A.a[l] = a[l];
  A.z = z16;
  A.sc = sc;
  A.act = bt.act;
  A.omega = omega;
  // per sample: r and z on 17^3 nodes, the four coefficient levels
  const double bytes = (double)bt.n * sizeof(T) *
                       (2.0 * Lv<16>::nodes + Lv<16>::cells + Lv<8>::cells + Lv<4>::cells + Lv<2>::cells);
  launch(sizeof(T) == 4 ? "coarse_f32" : "coarse_f64", bytes, k_coarse_vcycle<T>, dim3((unsigned)bt.n), dim3(kCT),
         M::bytes, st, A);
}

template void coarse_vcycle<float>(const float*, const float* const[4], float*, const SolveScalars*, const Batch&,
                                   double, cudaStream_t);
template void coarse_vcycle<double>(const double*, const double* const[4], double*, const SolveScalars*,
                                    const Batch&, double, cudaStream_t);

}  // namespace mlsgd
