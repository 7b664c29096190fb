// solver.cu - batched, matrix-free, geometric-multigrid-preconditioned CG for
// the discrete state and adjoint problems (rows a4, a6).
//
// The paper solves its FE systems with a multigrid-preconditioned CG (Sec. 5);
// this is a GPU design of that solver, not a port: S independent samples are
// advanced in lock step, each with its own scalars and an `active` flag that
// freezes it the iteration it converges, so a sample's iterates do not depend
// on the batch it is in.  Preconditioner: one V(1,1)-cycle with damped Jacobi
// on rediscretised Q1 operators (coarse coefficient = mean of the 8 child
// cells), trilinear prolongation P and restriction P^T, down to 2^3 cells
// (one unknown, solved exactly).  Stop rule: ||r||_2 <= rtol ||b||_2.
//
// Mixed precision: iterative refinement in FP64 (residual b - A x with x in
// FP64 and the accurate FP32-stored coefficient) around a fixed number of FP32
// PCG iterations whose V-cycle reads the BF16 coefficient.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "internal.cuh"
#include "kernels.h"
#include "launch.h"

namespace mlsgd {

enum ScalarMode { SM_INIT = 0, SM_RZ0, SM_ALPHA, SM_CONV, SM_BETA, SM_OUTER_CONV, SM_INNER_BEGIN, SM_OUTER_STEP };

// ---------------------------------------------------------------- vector kernels
// blockIdx.y indexes the launched samples: act[blockIdx.y] when the active samples
// have been compacted into a list, else blockIdx.y itself
#define SAMPLE_GUARD(sc)                                                     \
  const int s = act != nullptr ? act[blockIdx.y] : (int)blockIdx.y;          \
  if ((sc) != nullptr && !(sc)[s].active) return;

template <typename T, typename TA>
__global__ void k_apply_dot(const T* __restrict__ x, const TA* __restrict__ a, T* __restrict__ y,
                            double* __restrict__ partial, const SolveScalars* __restrict__ sc, int N,
                            const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n1 = N + 1;
  const long long nodes = (long long)n1 * n1 * n1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const T* xs = x + s * nodes;
  T contrib = T(0);
  if (n < nodes) {
    int i, j, k;
    node_ijk(n, n1, i, j, k);
    T v = T(0);
    if (interior(i, j, k, N)) {
      Cells8<T, TA> C;
      C.load(a + s * (long long)N * N * N, i, j, k, N);
      v = T(1.0 / (12.0 * N)) * q1_row(C, xs, i, j, k, n1);
    }
    y[s * nodes + n] = v;
    contrib = xs[n] * v;
  }
  const T b = block_sum(contrib);
  if (threadIdx.x == 0) partial[(long long)s * gridDim.x + blockIdx.x] = (double)b;
}

template <typename T>
__global__ void k_dot(const T* __restrict__ u, const T* __restrict__ v, double* __restrict__ partial,
                      const SolveScalars* __restrict__ sc, long long nodes, const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  T contrib = T(0);
  if (n < nodes) contrib = u[s * nodes + n] * v[s * nodes + n];
  const T b = block_sum(contrib);
  if (threadIdx.x == 0) partial[(long long)s * gridDim.x + blockIdx.x] = (double)b;
}

// x += alpha p; r -= alpha q; partial = r.r
template <typename T, bool REDUCE>
__global__ void k_update_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ q,
                            double* __restrict__ partial, const SolveScalars* __restrict__ sc, long long nodes,
                            const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const T al = (T)sc[s].alpha;
  T contrib = T(0);
  if (n < nodes) {
    const long long o = s * nodes + n;
    x[o] += al * p[o];
    const T rn = r[o] - al * q[o];
    r[o] = rn;
    contrib = rn * rn;
  }
  if (REDUCE) {
    const T b = block_sum(contrib);
    if (threadIdx.x == 0) partial[(long long)s * gridDim.x + blockIdx.x] = (double)b;
  }
}

template <typename T>
__global__ void k_p_update(T* __restrict__ p, const T* __restrict__ z, const SolveScalars* __restrict__ sc,
                           long long nodes, int first, const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nodes) {
    const long long o = s * nodes + n;
    p[o] = first ? z[o] : z[o] + (T)sc[s].beta * p[o];
  }
}

// r = b (shared or per sample), x = 0, partial = b.b  (not masked)
template <typename T>
__global__ void k_init(const double* __restrict__ b, long long bstride, T* __restrict__ r, T* __restrict__ x,
                       double* __restrict__ partial, long long nodes) {
  const int s = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (n < nodes) {
    const double bv = b[s * bstride + n];
    r[s * nodes + n] = (T)bv;
    x[s * nodes + n] = T(0);
    contrib = bv * bv;
  }
  const double bs = block_sum(contrib);
  if (threadIdx.x == 0) partial[(long long)s * gridDim.x + blockIdx.x] = bs;
}

// one warp per launched sample: sum the block partials in a fixed order, then the
// scalar update
__global__ void k_scalar(const double* __restrict__ partial, int nblk, SolveScalars* __restrict__ sc, int n,
                         const int* __restrict__ act, int mode, double tol2, int max_iter, int inner_iters,
                         const SolveScalars* __restrict__ outer) {
  const int t = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const int s = act != nullptr ? act[t] : t;
  SolveScalars& c = sc[s];
  if (mode == SM_INNER_BEGIN) {
    if (lane == 0) c.active = outer[s].active;
    return;
  }
  if (mode == SM_OUTER_STEP) {
    if (lane == 0 && c.active) { c.iters += 1; c.pad += inner_iters; }
    return;
  }
  if (mode != SM_INIT && !c.active) return;
  double v = 0.0;
  for (int t = lane; t < nblk; t += 32) v += partial[(long long)s * nblk + t];
  v = warp_sum(v);
  if (lane != 0) return;
  switch (mode) {
    case SM_INIT:
      c.bb = v; c.rr = v; c.active = (v > 0.0) ? 1 : 0; c.iters = 0; c.status = 0; c.pad = 0;
      c.rz = 0.0; c.alpha = 0.0; c.beta = 0.0;
      if (!(v < INFINITY)) { c.active = 0; c.status = 2; }
      break;
    case SM_RZ0: c.rz = v; break;
    case SM_ALPHA: c.alpha = (v > 0.0 && c.rz != 0.0) ? c.rz / v : 0.0; break;
    case SM_CONV:
      c.rr = v; c.iters += 1;
      if (v <= tol2 * c.bb) c.active = 0;
      else if (!(v < INFINITY)) { c.active = 0; c.status = 2; }
      else if (c.iters >= max_iter) { c.active = 0; c.status = 1; }
      break;
    case SM_BETA: c.beta = (c.rz != 0.0) ? v / c.rz : 0.0; c.rz = v; break;
    case SM_OUTER_CONV:
      c.rr = v;
      if (v <= tol2 * c.bb) c.active = 0;
      else if (!(v < INFINITY)) { c.active = 0; c.status = 2; }
      else if (c.iters >= max_iter) { c.active = 0; c.status = 1; }
      break;
  }
}

// Ordered compaction of the active samples: act[0..count) = the indices s with
// sc[s].active, ascending.  One block of kBlock threads walks the batch in chunks;
// each chunk's offsets come from warp ballots and a scan of the warp counts.
__global__ void __launch_bounds__(kBlock) k_compact(const SolveScalars* __restrict__ sc, int S, int* __restrict__ act,
                                                    int* __restrict__ count) {
  __shared__ int wcount[kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int base = 0;
  for (int s0 = 0; s0 < S; s0 += kBlock) {
    const int s = s0 + threadIdx.x;
    const bool a = s < S && sc[s].active;
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (lane == 0) wcount[w] = __popc(m);
    __syncthreads();
    int off = base;
    for (int v = 0; v < w; ++v) off += wcount[v];
    if (a) act[off + __popc(m & ((1u << lane) - 1u))] = s;
    for (int v = 0; v < kBlock / 32; ++v) base += wcount[v];
    __syncthreads();  // wcount is rewritten by the next chunk
  }
  if (threadIdx.x == 0) *count = base;
}

// ---------------------------------------------------------------- multigrid kernels
// x = omega D^{-1} r  (pre-smoothing from a zero initial guess), D = (h/3) sum_8 a
template <typename T, typename TA>
__global__ void k_jacobi0(const T* __restrict__ r, const TA* __restrict__ a, T* __restrict__ x,
                          const SolveScalars* __restrict__ sc, int N, T omega, const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n1 = N + 1;
  const long long nodes = (long long)n1 * n1 * n1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nodes) return;
  int i, j, k;
  node_ijk(n, n1, i, j, k);
  T v = T(0);
  if (interior(i, j, k, N)) {
    Cells8<T, TA> C;
    C.load(a + s * (long long)N * N * N, i, j, k, N);
    v = omega * r[s * nodes + n] / (T(1.0 / (3.0 * N)) * C.sum);
  }
  x[s * nodes + n] = v;
}

// t = r - A x   (mode 0)   or   t = x + omega D^{-1} (r - A x)   (mode 1, smoothing)
template <typename T, typename TA, int MODE>
__global__ void k_resid_smooth(const T* __restrict__ r, const T* __restrict__ x, const TA* __restrict__ a,
                               T* __restrict__ t, const SolveScalars* __restrict__ sc, int N, T omega,
                               const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n1 = N + 1;
  const long long nodes = (long long)n1 * n1 * n1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nodes) return;
  int i, j, k;
  node_ijk(n, n1, i, j, k);
  T v = T(0);
  if (interior(i, j, k, N)) {
    Cells8<T, TA> C;
    C.load(a + s * (long long)N * N * N, i, j, k, N);
    const T* xs = x + s * nodes;
    const T res = r[s * nodes + n] - T(1.0 / (12.0 * N)) * q1_row(C, xs, i, j, k, n1);
    v = (MODE == 0) ? res : xs[n] + omega * res / (T(1.0 / (3.0 * N)) * C.sum);
  }
  t[s * nodes + n] = v;
}

// coarse = P^T fine: weights 1, 1/2 per axis around (2I, 2J, 2K)
template <typename T, int NCC = 0>
__global__ void k_restrict(const T* __restrict__ tf, T* __restrict__ rc, const SolveScalars* __restrict__ sc,
                           int Nc_, const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int Nc = NCC ? NCC : Nc_;  // a compile-time grid makes the index divisions multiplications
  const int n1c = Nc + 1, Nf = 2 * Nc, n1f = Nf + 1;
  const long long nc = (long long)n1c * n1c * n1c, nf = (long long)n1f * n1f * n1f;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nc) return;
  int I, J, K;
  node_ijk(n, n1c, I, J, K);
  T v = T(0);
  if (interior(I, J, K, Nc)) {
    const T* f = tf + s * nf + (2 * I) + (long long)n1f * (2 * J) + (long long)n1f * n1f * (2 * K);
#pragma unroll
    for (int w = -1; w <= 1; ++w)
#pragma unroll
      for (int u = -1; u <= 1; ++u)
#pragma unroll
        for (int q = -1; q <= 1; ++q) {
          const T wt = T((q == 0 ? 1.0 : 0.5) * (u == 0 ? 1.0 : 0.5) * (w == 0 ? 1.0 : 0.5));
          v += wt * f[q + (long long)n1f * u + (long long)n1f * n1f * w];
        }
  }
  rc[s * nc + n] = v;
}

// The same restriction marching in z: one thread per coarse node column (I, J) and
// chunk of kRestrictPlanes coarse planes (blockIdx.z); the xy-weighted sum of fine
// plane 2K+1 serves coarse planes K and K+1, so a coarse node reads 18 fine values
// instead of 27.  rc holds 0 on the coarse boundary.
constexpr int kRestrictPlanes = 8;
template <typename T, int NCC>
__global__ void k_restrict_zm(const T* __restrict__ tf, T* __restrict__ rc, const SolveScalars* __restrict__ sc,
                              const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  constexpr int Nc = NCC, n1c = Nc + 1, n1f = 2 * Nc + 1;
  constexpr long long nc = (long long)n1c * n1c * n1c, nf = (long long)n1f * n1f * n1f;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n1c * n1c) return;
  const int I = col % n1c, J = col / n1c;
  const int K0 = kRestrictPlanes * (int)blockIdx.z, K1 = min(Nc, K0 + kRestrictPlanes - 1);
  T* out = rc + s * nc + col;
  if (I == 0 || J == 0 || I == Nc || J == Nc) {
    for (int K = K0; K <= K1; ++K) out[K * (n1c * n1c)] = T(0);
    return;
  }
  const T* f = tf + s * nf + 2 * I + (long long)n1f * (2 * J);
  auto rxy = [&](int k) {  // sum over the 3 x 3 fine nodes around (2I, 2J) of fine plane k
    const T* p = f + (long long)n1f * n1f * k;
    T v = T(0);
#pragma unroll
    for (int u = -1; u <= 1; ++u)
#pragma unroll
      for (int q = -1; q <= 1; ++q) v += T((q == 0 ? 1.0 : 0.5) * (u == 0 ? 1.0 : 0.5)) * p[q + n1f * u];
    return v;
  };
  if (K0 == 0) out[0] = T(0);
  if (K1 == Nc) out[Nc * (n1c * n1c)] = T(0);
  const int Ka = K0 > 1 ? K0 : 1, Kb = K1 < Nc - 1 ? K1 : Nc - 1;  // interior coarse planes
  T prev = rxy(2 * Ka - 1);
#pragma unroll 2
  for (int K = Ka; K <= Kb; ++K) {
    const T mid = rxy(2 * K), up = rxy(2 * K + 1);
    out[K * (n1c * n1c)] = T(0.5) * prev + mid + T(0.5) * up;
    prev = up;
  }
}

// fine += P coarse (trilinear)
template <typename T>
__global__ void k_prolong_add(T* __restrict__ xf, const T* __restrict__ ec, const SolveScalars* __restrict__ sc,
                              int Nf, const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n1f = Nf + 1, Nc = Nf / 2, n1c = Nc + 1;
  const long long nf = (long long)n1f * n1f * n1f, nc = (long long)n1c * n1c * n1c;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nf) return;
  int i, j, k;
  node_ijk(n, n1f, i, j, k);
  if (!interior(i, j, k, Nf)) return;
  const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
  const int i1 = i0 + (i & 1), j1 = j0 + (j & 1), k1 = k0 + (k & 1);
  const T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1), wk = (k & 1) ? T(0.5) : T(1);
  const T* e = ec + s * nc;
  auto at = [&](int a, int b, int c) { return e[a + (long long)n1c * b + (long long)n1c * n1c * c]; };
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
  xf[s * nf + n] += v;
}

// 2^3 cells: the single interior unknown, x = r / D; all other nodes 0
template <typename T, typename TA>
__global__ void k_coarsest(const T* __restrict__ r, const TA* __restrict__ a, T* __restrict__ x,
                           const SolveScalars* __restrict__ sc, int n, const int* __restrict__ act) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int s = act != nullptr ? act[t] : t;
  if (sc != nullptr && !sc[s].active) return;
  T* xs = x + (long long)s * 27;
  for (int n = 0; n < 27; ++n) xs[n] = T(0);
  Cells8<T, TA> C;
  C.load(a + (long long)s * 8, 1, 1, 1, 2);
  xs[13] = r[(long long)s * 27 + 13] / (T(1.0 / 6.0) * C.sum);
}

// coarse cell coefficient = mean of the 8 children
template <typename TI, typename TO>
// (one thread per coarse cell of a sample, blockIdx.y the sample).  The mixed path's
// FP32 levels sum in FP32: the eight BF16 children of the first coarsening sum exactly
// (8-bit significands, the coefficient's range spans well under 16 binary orders), and
// the coarse coefficients only shape the preconditioner; the FP64 path sums in FP64.
__global__ void k_coarsen_coef(const TI* __restrict__ af, TO* __restrict__ ac, int Nc) {
  using Acc = typename std::conditional<std::is_same<TO, double>::value, double, float>::type;
  const int cc = Nc * Nc * Nc;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cc) return;
  const int s = blockIdx.y;
  const unsigned t = (unsigned)c / (unsigned)Nc;
  const int I = c - (int)t * Nc, K = (int)(t / (unsigned)Nc), J = (int)t - K * Nc;
  const int Nf = 2 * Nc;
  const TI* f = af + (long long)s * Nf * Nf * Nf + 2 * I + Nf * (2 * J + Nf * 2 * K);
  Acc acc = Acc(0);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int p = 0; p < 2; ++p) acc += smem_coef<Acc>(f[p + Nf * (q + Nf * r)]);
  ac[(long long)s * cc + c] = (TO)(Acc(0.125) * acc);
}

// ---------------------------------------------------------------- mixed-precision kernels
// r64 = b - A(a) x64 in FP64, partial = r.r
template <typename TA>
__global__ void k_residual64(const double* __restrict__ b, long long bstride, const double* __restrict__ x,
                             const TA* __restrict__ a, double* __restrict__ r, double* __restrict__ partial,
                             const SolveScalars* __restrict__ sc, int N, const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n1 = N + 1;
  const long long nodes = (long long)n1 * n1 * n1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (n < nodes) {
    int i, j, k;
    node_ijk(n, n1, i, j, k);
    double v = 0.0;
    if (interior(i, j, k, N)) {
      Cells8<double, TA> C;
      C.load(a + s * (long long)N * N * N, i, j, k, N);
      v = b[s * bstride + n] - (1.0 / (12.0 * N)) * q1_row(C, x + s * nodes, i, j, k, n1);
    }
    r[s * nodes + n] = v;
    contrib = v * v;
  }
  const double bs = block_sum(contrib);
  if (threadIdx.x == 0) partial[(long long)s * gridDim.x + blockIdx.x] = bs;
}

// r32 = (float) r64, d = 0
__global__ void k_demote(const double* __restrict__ r64, float* __restrict__ r32, float* __restrict__ d,
                         const SolveScalars* __restrict__ sc, long long nodes, const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nodes) {
    r32[s * nodes + n] = (float)r64[s * nodes + n];
    d[s * nodes + n] = 0.0f;
  }
}

// r32 = (float) b (shared or per sample), bdf = b as an FP32 (hi, lo) pair (written
// once when b is shared), partial = b.b  (not masked).  Each thread takes kInitPer
// nodes so that the FP64 block reduction is amortised.
constexpr int kInitPer = 8;
static inline int init_blocks(int N) { return (int)((nodes_of(N) + kBlock * kInitPer - 1) / (kBlock * kInitPer)); }
// PAIR_B: b is already given as FP32 pairs (bp; nothing to split, b.b from the heads).
// Boundary rows of b are taken as 0 whatever the buffer holds there.
template <bool PAIR_B, int NN = 0>
__global__ void k_init32(const double* __restrict__ b, const float2* __restrict__ bp, long long bstride,
                         float* __restrict__ r32, float2* __restrict__ bdf, double* __restrict__ partial,
                         long long nodes, int N_) {
  const int N = NN ? NN : N_;
  const int s = blockIdx.y;
  const long long n0 = (long long)blockIdx.x * blockDim.x * kInitPer + threadIdx.x;
  const bool write_pair = bstride != 0 || s == 0;
  double contrib = 0.0;
  float contrib32 = 0.0f;
#pragma unroll
  for (int i = 0; i < kInitPer; ++i) {
    const long long n = n0 + (long long)i * blockDim.x;
    if (n < nodes) {
      int ii, jj, kk;
      node_ijk((int)n, N + 1, ii, jj, kk);
      if (!interior(ii, jj, kk, N)) {
        r32[s * nodes + n] = 0.0f;
        if (!PAIR_B && write_pair) bdf[s * bstride + n] = make_float2(0.0f, 0.0f);
        continue;
      }
      if constexpr (PAIR_B) {
        const float hi = bp[s * bstride + n].x;
        r32[s * nodes + n] = hi;
        contrib32 = __fmaf_rn(hi, hi, contrib32);
      } else {
        const double bv = b[s * bstride + n];
        const float hi = (float)bv;
        r32[s * nodes + n] = hi;
        if (write_pair) bdf[s * bstride + n] = make_float2(hi, (float)(bv - (double)hi));
        contrib = fma(bv, bv, contrib);
      }
    }
  }
  if (PAIR_B) contrib = (double)contrib32;
  const double bs = block_sum(contrib);
  if (threadIdx.x == 0) partial[(long long)s * gridDim.x + blockIdx.x] = bs;
}

// the inner solve's last update fused with the refinement step: the solution is
// kept as an FP32 (hi, lo) pair x, x (+)= d + alpha p (pair addition: two-sum and
// renormalisation, about 48 significant bits), d taken as 0 when never written.
// The first step (assign) launches every sample and writes x = 0 for the samples that
// take no step (b = 0, or a non-finite b), so every sample's solution is defined.
template <int NN = 0>
__global__ void k_finish_step(float2* __restrict__ x, const float* __restrict__ d, const float* __restrict__ p,
                              const SolveScalars* __restrict__ sci, const SolveScalars* __restrict__ sco,
                              long long nodes, int N_, int assign, int d_zero, const int* __restrict__ act) {
  const int N = NN ? NN : N_;
  const int s = act != nullptr ? act[blockIdx.y] : (int)blockIdx.y;
  const bool on = sco[s].active != 0;
  if (!on && !assign) return;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nodes) return;
  const long long o = s * nodes + n;
  int i, j, k;
  node_ijk(n, N + 1, i, j, k);
  if (!on || !interior(i, j, k, N)) {  // d and p are never written on the boundary
    x[o] = make_float2(0.0f, 0.0f);
    return;
  }
  const float dv = d_zero ? 0.0f : d[o];
  const float inc = dv + (float)sci[s].alpha * p[o];
  if (assign) {
    x[o] = make_float2(inc, 0.0f);
    return;
  }
  const float2 xv = x[o];
  const float sh = xv.x + inc;  // two-sum of hi and inc
  const float bb = sh - xv.x;
  const float se = (xv.x - (sh - bb)) + (inc - bb);
  const float lo = xv.y + se;
  const float h = sh + lo;      // renormalise
  x[o] = make_float2(h, lo - (h - sh));
}

// x64 = hi + lo of the FP32 pair solution (every sample, after the refinement)
__global__ void k_store_pair(double* __restrict__ x, const float2* __restrict__ xp, long long nodes) {
  const int s = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nodes) return;
  const float2 v = xp[s * nodes + n];
  x[s * nodes + n] = (double)v.x + (double)v.y;
}

// x64 += d
__global__ void k_accumulate(double* __restrict__ x, const float* __restrict__ d, const SolveScalars* __restrict__ sc,
                             long long nodes, const int* __restrict__ act) {
  SAMPLE_GUARD(sc);
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nodes) x[s * nodes + n] += (double)d[s * nodes + n];
}

// ---------------------------------------------------------------- host side
static inline dim3 grid_nodes(int N, int S) { return dim3((unsigned)node_blocks(N), (unsigned)S); }

// f(std::integral_constant<int, N>) for the grids of the hierarchies (N a power of two,
// 16 .. 256), f(std::integral_constant<int, 0>) (N at run time) otherwise
template <typename F>
static void with_grid(int N, F&& f) {
  switch (N) {
    case 16: f(std::integral_constant<int, 16>()); break;
    case 32: f(std::integral_constant<int, 32>()); break;
    case 64: f(std::integral_constant<int, 64>()); break;
    case 128: f(std::integral_constant<int, 128>()); break;
    case 256: f(std::integral_constant<int, 256>()); break;
    default: f(std::integral_constant<int, 0>()); break;
  }
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }
// bytes after every node vector: the slab passes copy 16-byte aligned spans that may
// reach up to 12 bytes past a vector's last node
constexpr size_t kVecSlack = 64;

static int mg_levels(int N) {
  int J = 0;
  while ((N >> J) > 2) ++J;
  return J;
}

// the whole-row slab passes run the FP32 fused passes of grid N
static bool uses_slab(const SolverBufs& B, int N, int elem) { return elem == 4 && B.stencil == 0 && slab_supported(N); }

// levels whose smoothing runs in the tiled passes (they read a precomputed D^{-1})
static bool tiled_level(int N, int j) { return N >= kTiledMinN && mg_levels(N) >= 1 && (N >> j) >= kTiledMinN; }

size_t solver_bytes(int N, int S, int elem) {
  size_t b = 0;
  const int J = mg_levels(N);
  b += 7 * align_up((size_t)S * nodes_of(N) * elem + kVecSlack);
  for (int j = 1; j <= J; ++j) {
    const int Nj = N >> j;
    b += 3 * align_up((size_t)S * nodes_of(Nj) * elem + kVecSlack) + align_up((size_t)S * cells_of(Nj) * elem);
  }
  for (int j = 0; j <= J; ++j)
    if (tiled_level(N, j)) b += align_up((size_t)S * nodes_of(N >> j) * elem + kVecSlack);
  if (elem == 4 && tiled_level(N, 0)) b += align_up((size_t)S * nodes_of(N) * sizeof(float2)) +
                                           align_up((size_t)nodes_of(N) * sizeof(float2));
  b += align_up((size_t)S * node_blocks(N) * sizeof(double));
  b += 2 * align_up((size_t)S * sizeof(SolveScalars));
  b += align_up(sizeof(int)) + align_up((size_t)S * sizeof(int));
  return b;
}

void carve_solver(SolverBufs& B, int N, int S, int elem, char*& ptr) {
  auto take = [&](size_t n) { void* p = ptr; ptr += align_up(n); return p; };
  B.N = N;
  B.S = S;
  B.J = mg_levels(N);
  const size_t v0 = (size_t)S * nodes_of(N) * elem + kVecSlack;
  B.x = take(v0); B.r = take(v0); B.r2 = take(v0); B.p = take(v0); B.q = take(v0);
  B.vx[0] = take(v0); B.vt[0] = take(v0); B.vr[0] = nullptr; B.acoef[0] = nullptr;
  for (int j = 1; j <= B.J; ++j) {
    const int Nj = N >> j;
    const size_t vj = (size_t)S * nodes_of(Nj) * elem + kVecSlack;
    B.vx[j] = take(vj); B.vt[j] = take(vj); B.vr[j] = take(vj);
    B.acoef[j] = take((size_t)S * cells_of(Nj) * elem);
  }
  for (int j = 0; j < 8; ++j) B.dinv[j] = nullptr;
  for (int j = 0; j <= B.J; ++j)
    if (tiled_level(N, j)) B.dinv[j] = take((size_t)S * nodes_of(N >> j) * elem + kVecSlack);
  B.bdf = (elem == 4 && tiled_level(N, 0)) ? (float2*)take((size_t)S * nodes_of(N) * sizeof(float2)) : nullptr;
  B.bsh = (elem == 4 && tiled_level(N, 0)) ? (float2*)take((size_t)nodes_of(N) * sizeof(float2)) : nullptr;
  B.partial = (double*)take((size_t)S * node_blocks(N) * sizeof(double));
  B.sc = (SolveScalars*)take((size_t)2 * S * sizeof(SolveScalars));
  B.count = (int*)take(sizeof(int));
  B.act = (int*)take((size_t)S * sizeof(int));
  B.n_act = S;
  B.actp = nullptr;
}

// algorithmic bytes of a node kernel: `vec` vectors of T over S samples of grid N
// plus `coef` reads of the cell coefficient TA
template <typename T, typename TA>
static double nbytes(int N, int S, double vec, double coef) {
  return (double)S * (vec * (double)nodes_of(N) * sizeof(T) + coef * (double)cells_of(N) * sizeof(TA));
}
template <typename T> struct Tag;
template <> struct Tag<double> { static constexpr const char* s = "f64"; };
template <> struct Tag<float> { static constexpr const char* s = "f32"; };
template <typename T>
static const char* cls(const char* base, bool fine) {
  static thread_local char buf[64];
  snprintf(buf, sizeof(buf), "%s_%s%s", base, Tag<T>::s, fine ? "" : "_coarse");
  return buf;
}

// D^{-1} = 1 / ((h/3) sum_8 a) at interior nodes, 0 on the boundary (computed once per
// coefficient hierarchy; the tiled smoothing passes stage it like a vector).  FP32:
// the fast approximate reciprocal (the diagonal only scales the smoother; pre- and
// post-smoothing read the same values, so the V-cycle stays symmetric).
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
// One thread per node column (i, j) and chunk of kDinvPlanes planes (blockIdx.z),
// marching in z: the four cells of the column below a node are summed once and
// reused by the node above (the chunk's first node sums both).
constexpr int kDinvPlanes = 8;
template <typename T, typename TA>
__global__ void k_dinv(const TA* __restrict__ a, T* __restrict__ dinv, int N, T omega) {
  const int s = blockIdx.y;
  const int n1 = N + 1;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n1 * n1) return;
  const int i = col % n1, j = col / n1;
  const long long plane = (long long)n1 * n1;
  const int k0 = 1 + kDinvPlanes * (int)blockIdx.z, k1 = min(N - 1, k0 + kDinvPlanes - 1);
  T* out = dinv + s * plane * n1 + col;
  if (blockIdx.z == 0) out[0] = T(0);
  if (k1 == N - 1) out[N * plane] = T(0);
  if (i == 0 || j == 0 || i == N || j == N) {
    T* o = out + (long long)k0 * plane;
    for (int k = k0; k <= k1; ++k, o += plane) *o = T(0);
    return;
  }
  const int cpl = N * N;
  // pointers advanced by addition (64-bit multiplies issue on the FP64 pipe here)
  const TA* ac = a + (long long)s * cpl * N + (i - 1) + N * (j - 1) + (long long)(k0 - 1) * cpl;
  auto sum4 = [&](const TA* p) {
    return (load_coef<T>(p) + load_coef<T>(p + 1)) + (load_coef<T>(p + N) + load_coef<T>(p + N + 1));
  };
  const T h3 = T(1.0 / (3.0 * N));
  T below = sum4(ac);
  T* o = out + (long long)k0 * plane;
  for (int k = k0; k <= k1; ++k, o += plane) {
    ac += cpl;
    const T above = sum4(ac);
    *o = omega * recip(h3 * (below + above));
    below = above;
  }
}

template <typename T, typename TA0>
static void build_dinv(SolverBufs& B, const TA0* a0, double omega, cudaStream_t st) {
  for (int j = 0; j <= B.J; ++j) {
    if (!B.dinv[j]) continue;
    const int Nj = B.N >> j;
    const dim3 g((unsigned)(((Nj + 1) * (Nj + 1) + kBlock - 1) / kBlock), (unsigned)B.S,
                 (unsigned)((Nj - 1 + kDinvPlanes - 1) / kDinvPlanes));
    if (j == 0)
      launch("dinv", nbytes<T, TA0>(Nj, B.S, 1, 1), k_dinv<T, TA0>, g, kBlock, 0, st, a0, (T*)B.dinv[0], Nj,
             (T)omega);
    else
      launch("dinv", nbytes<T, T>(Nj, B.S, 1, 1), k_dinv<T, T>, g, kBlock, 0, st, (const T*)B.acoef[j],
             (T*)B.dinv[j], Nj, (T)omega);
  }
}

template <typename TI, typename TO>
static void coarsen_all(SolverBufs& B, const TI* a0, cudaStream_t st) {
  for (int j = 1; j <= B.J; ++j) {
    const int Nc = B.N >> j;
    const long long n = cells_of(Nc) * B.S;
    const dim3 g((unsigned)((cells_of(Nc) + 255) / 256), (unsigned)B.S);
    if (j == 1)
      launch("coarsen", (double)n * (8 * sizeof(TI) + sizeof(TO)), k_coarsen_coef<TI, TO>, g, 256, 0, st, a0,
             (TO*)B.acoef[1], Nc);
    else
      launch("coarsen", (double)n * 9 * sizeof(TO), k_coarsen_coef<TO, TO>, g, 256, 0, st, (const TO*)B.acoef[j - 1],
             (TO*)B.acoef[j], Nc);
  }
}
void build_hierarchy_fp64(SolverBufs& B, const double* a64, double omega, cudaStream_t st) {
  coarsen_all<double, double>(B, a64, st);
  build_dinv<double, double>(B, a64, omega, st);
}
void build_hierarchy_mixed(SolverBufs& B, const __nv_bfloat16* abf, double omega, cudaStream_t st) {
  coarsen_all<__nv_bfloat16, float>(B, abf, st);
  build_dinv<float, __nv_bfloat16>(B, abf, omega, st);
}

// One V(1,1)-cycle on r0 (level-0 coefficient a0); the result is left in vt[0].
// Grids with N >= kTiledMinN run the fine level with the tiled passes (PRE
// fuses the pre-smoothing into the residual, POST fuses prolongation,
// post-smoothing and the r.z partial sums, which land in B.partial);
// returns the partial-sum blocks per sample of r.z, or 0 if not computed.
// With fuse_q the fine-level PRE first applies the CG residual update
// r_new = r0 - alpha fuse_q (written to r_new) and the V-cycle runs on r_new.
template <typename T, typename TA0>
static int vcycle(SolverBufs& B, const T* r0, const TA0* a0, const SolveScalars* sc, T omega, cudaStream_t st,
                  const T* fuse_q = nullptr, T* r_new = nullptr, T* z0 = nullptr) {
  const int S = B.S, J = B.J;
  const int n = B.n_act;            // samples launched (the active ones when compacted)
  const int* act = B.actp;
  const Batch bt = B.batch();
  const bool tiled = B.N >= kTiledMinN && J >= 1;
  const T* rfine = fuse_q ? r_new : r0;  // residual the V-cycle works on after the fused update
  auto rin = [&](int j) { return j == 0 ? rfine : (const T*)B.vr[j]; };
  // the levels from a coarse 16^3 level down to 2^3 run as one fused launch; jc is
  // the first of them (J: none)
  int jc = J;
  if (tiled)
    for (int j = 1; j < J; ++j)
      if (coarse_vcycle_applies(B.N, j) && J - j == 3) jc = j;
  for (int j = 0; j < jc; ++j) {
    const int Nj = B.N >> j;
    const bool fine = j == 0;
    T* rc = (T*)B.vr[j + 1];
    bool restricted = false;  // the pre-smoothing pass restricted its residual itself
    if (fine && tiled && fuse_q) {
      if constexpr (std::is_same<T, float>::value && std::is_same<TA0, __nv_bfloat16>::value)
        restricted = tiled_pre_update(r0, fuse_q, a0, (const T*)B.dinv[0], (T*)B.vt[0], r_new, rc, sc, Nj, bt, st);
    } else if (fine && tiled) {
      restricted = tiled_pre<T, TA0>(r0, a0, (const T*)B.dinv[0], (T*)B.vt[0], rc, sc, Nj, bt, st);
    } else if (!fine && tiled && Nj >= kTiledMinN) {
      restricted = tiled_pre<T, T>(rin(j), (const T*)B.acoef[j], (const T*)B.dinv[j], (T*)B.vt[j], rc, sc, Nj, bt, st);
    } else if (fine) {
      launch(cls<T>("jacobi0", true), nbytes<T, TA0>(Nj, n, 2, 1), k_jacobi0<T, TA0>, grid_nodes(Nj, n), kBlock, 0,
             st, rin(0), a0, (T*)B.vx[0], sc, Nj, omega, act);
      launch(cls<T>("resid", true), nbytes<T, TA0>(Nj, n, 3, 1), k_resid_smooth<T, TA0, 0>, grid_nodes(Nj, n), kBlock,
             0, st, rin(0), (const T*)B.vx[0], a0, (T*)B.vt[0], sc, Nj, omega, act);
    } else {
      const T* aj = (const T*)B.acoef[j];
      launch(cls<T>("jacobi0", false), nbytes<T, T>(Nj, n, 2, 1), k_jacobi0<T, T>, grid_nodes(Nj, n), kBlock, 0, st,
             rin(j), aj, (T*)B.vx[j], sc, Nj, omega, act);
      launch(cls<T>("resid", false), nbytes<T, T>(Nj, n, 3, 1), k_resid_smooth<T, T, 0>, grid_nodes(Nj, n), kBlock, 0,
             st, rin(j), (const T*)B.vx[j], aj, (T*)B.vt[j], sc, Nj, omega, act);
    }
    if (restricted) continue;
    with_grid(Nj / 2, [&](auto c) {
      constexpr int NCC = decltype(c)::value;
      const double rb = nbytes<T, T>(Nj, n, 1, 0) + nbytes<T, T>(Nj / 2, n, 1, 0);
      if constexpr (NCC >= 32) {  // on smaller grids the per-node kernel has more threads in flight
        const int n1c = Nj / 2 + 1;
        const dim3 gr((unsigned)((n1c * n1c + kBlock - 1) / kBlock), (unsigned)n,
                      (unsigned)((Nj / 2 + kRestrictPlanes) / kRestrictPlanes));
        launch(cls<T>("restrict", fine), rb, k_restrict_zm<T, NCC>, gr, kBlock, 0, st, (const T*)B.vt[j],
               (T*)B.vr[j + 1], sc, act);
      } else {
        launch(cls<T>("restrict", fine), rb, k_restrict<T, NCC>, grid_nodes(Nj / 2, n), kBlock, 0, st,
               (const T*)B.vt[j], (T*)B.vr[j + 1], sc, Nj / 2, act);
      }
    });
  }
  if (jc < J) {
    const T* const al[4] = {(const T*)B.acoef[jc], (const T*)B.acoef[jc + 1], (const T*)B.acoef[jc + 2],
                            (const T*)B.acoef[jc + 3]};
    coarse_vcycle<T>(rin(jc), al, (T*)B.vt[jc], sc, bt, (double)omega, st);
  } else if (J == 0) {
    launch("coarsest", 0.0, k_coarsest<T, TA0>, dim3((n + 127) / 128), 128, 0, st, rin(0), a0, (T*)B.vt[0], sc, n,
           act);
  } else {
    launch("coarsest", 0.0, k_coarsest<T, T>, dim3((n + 127) / 128), 128, 0, st, rin(J), (const T*)B.acoef[J],
           (T*)B.vt[J], sc, n, act);
  }
  for (int j = jc - 1; j >= 0; --j) {
    const int Nj = B.N >> j;
    const bool fine = j == 0;
    if (fine && tiled) {
      tiled_post<T, TA0>(rfine, a0, (const T*)B.dinv[0], (const T*)B.vt[1], z0 ? z0 : (T*)B.vt[0], B.partial, sc, Nj,
                         bt, st);
      return tiled_blocks_per_sample(Nj, S, (int)sizeof(T), uses_slab(B, Nj, (int)sizeof(T)));
    }
    if (!fine && tiled && Nj >= kTiledMinN) {
      // the r.z partial sums of a coarse level are overwritten by the fine level's POST
      tiled_post<T, T>(rin(j), (const T*)B.acoef[j], (const T*)B.dinv[j], (const T*)B.vt[j + 1], (T*)B.vt[j],
                       B.partial, sc, Nj, bt, st);
      continue;
    }
    launch(cls<T>("prolong", fine), nbytes<T, T>(Nj, n, 2, 0) + nbytes<T, T>(Nj / 2, n, 1, 0), k_prolong_add<T>,
           grid_nodes(Nj, n), kBlock, 0, st, (T*)B.vx[j], (const T*)B.vt[j + 1], sc, Nj, act);
    if (fine)
      launch(cls<T>("smooth", true), nbytes<T, TA0>(Nj, n, 3, 1), k_resid_smooth<T, TA0, 1>, grid_nodes(Nj, n), kBlock,
             0, st, rin(0), (const T*)B.vx[0], a0, (T*)B.vt[0], sc, Nj, omega, act);
    else
      launch(cls<T>("smooth", false), nbytes<T, T>(Nj, n, 3, 1), k_resid_smooth<T, T, 1>, grid_nodes(Nj, n), kBlock, 0,
             st, rin(j), (const T*)B.vx[j], (const T*)B.acoef[j], (T*)B.vt[j], sc, Nj, omega, act);
  }
  return 0;
}

static void scalar(SolverBufs& B, SolveScalars* sc, int mode, double tol2, int max_iter, cudaStream_t st, int nblk,
                   int inner_iters = 0, const SolveScalars* outer = nullptr) {
  const int warps = 8;
  launch("scalar", 0.0, k_scalar, dim3((B.n_act + warps - 1) / warps), 32 * warps, 0, st, (const double*)B.partial,
         nblk, sc, B.n_act, B.actp, mode, tol2, max_iter, inner_iters, outer);
}

// All samples launched again (the start of a solve).
static void launch_all(SolverBufs& B) {
  B.n_act = B.S;
  B.actp = nullptr;
}

// Host-checked modes: compact the active samples of `sc` into B.act, read their
// count back (one synchronisation) and launch only them from now on, so retired
// samples start no blocks and are credited with no bytes.
static cudaError_t compact_active(SolverBufs& B, const SolveScalars* sc, cudaStream_t st, int& n) {
  launch("compact", (double)B.S * (sizeof(SolveScalars) + sizeof(int)), k_compact, dim3(1), kBlock, 0, st, sc, B.S,
         B.act, B.count);
  cudaError_t e = cudaMemcpyAsync(B.count_host, B.count, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  n = *B.count_host;
  if (n < 0 || n > B.S) return cudaErrorInvalidValue;
  B.n_act = n;
  B.actp = n < B.S ? B.act : nullptr;
  return cudaSuccess;
}

// Krylov loop shared by the FP64 solve and the FP32 inner solve.
// fixed_iters > 0: run exactly that many iterations without a stop test (over the
// samples the caller's compaction left active).  Otherwise the stop test runs every
// iteration on the device and every prm.check_every iterations on the host, which
// then compacts the still-active samples.
template <typename T, typename TAop, typename TA0>
static cudaError_t pcg_loop(SolverBufs& B, const TAop* aop, const TA0* a0, T* x, T* r, SolveScalars* sc,
                            const PcgParams& prm, int fixed_iters, cudaStream_t st) {
  const int S = B.S, N = B.N;
  const long long nodes = nodes_of(N);
  const int nb = node_blocks(N);
  const T omega = (T)prm.omega;
  const bool tiled = N >= kTiledMinN && B.J >= 1;
  T* pbuf[2] = {(T*)B.p, (T*)B.vx[0]};  // tiled: ping-pong p (vx[0] is unused there)
  int cur = 0;
  T* q = (T*)B.q;
  const T* z = (const T*)B.vt[0];
  auto g = [&]() { return grid_nodes(N, B.n_act); };
  auto precondition = [&](int mode) {
    const int nrz = vcycle<T, TA0>(B, r, a0, sc, omega, st);
    if (nrz == 0) {
      launch(cls<T>("dot", true), nbytes<T, T>(N, B.n_act, 2, 0), k_dot<T>, g(), kBlock, 0, st, (const T*)r, z,
             B.partial, (const SolveScalars*)sc, nodes, B.actp);
      scalar(B, sc, mode, 0, 0, st, nb);
    } else {
      scalar(B, sc, mode, 0, 0, st, nrz);
    }
  };
  precondition(SM_RZ0);
  if (!tiled)
    launch(cls<T>("pupdate", true), nbytes<T, T>(N, B.n_act, 2, 0), k_p_update<T>, g(), kBlock, 0, st, pbuf[0], z,
           (const SolveScalars*)sc, nodes, 1, B.actp);
  const double tol2 = prm.rtol * prm.rtol;
  const int nit = fixed_iters > 0 ? fixed_iters : prm.max_iter;
  const int napply = tiled ? tiled_blocks_per_sample(N, S, (int)sizeof(T), uses_slab(B, N, (int)sizeof(T))) : nb;
  for (int it = 0; it < nit; ++it) {
    T* p;
    if (tiled) {
      p = pbuf[cur ^ 1];
      tiled_apply<T, TAop>(z, pbuf[cur], p, aop, q, B.partial, sc, N, B.batch(), it == 0, st);
      cur ^= 1;
    } else {
      p = pbuf[0];
      launch(cls<T>("apply", true), nbytes<T, TAop>(N, B.n_act, 2, 1), k_apply_dot<T, TAop>, g(), kBlock, 0, st,
             (const T*)p, aop, q, B.partial, (const SolveScalars*)sc, N, B.actp);
    }
    scalar(B, sc, SM_ALPHA, 0, 0, st, napply);
    if (fixed_iters > 0) {
      launch(cls<T>("update", true), nbytes<T, T>(N, B.n_act, 6, 0), k_update_xr<T, false>, g(), kBlock, 0, st, x, r,
             (const T*)p, (const T*)q, B.partial, (const SolveScalars*)sc, nodes, B.actp);
      if (it == nit - 1) break;
    } else {
      launch(cls<T>("update", true), nbytes<T, T>(N, B.n_act, 6, 0), k_update_xr<T, true>, g(), kBlock, 0, st, x, r,
             (const T*)p, (const T*)q, B.partial, (const SolveScalars*)sc, nodes, B.actp);
      scalar(B, sc, SM_CONV, tol2, prm.max_iter, st, nb);
      if ((it + 1) % prm.check_every == 0 || it + 1 == nit) {
        int n = 0;
        cudaError_t e = compact_active(B, sc, st, n);
        if (e != cudaSuccess) return e;
        if (n == 0) break;
      }
    }
    precondition(SM_BETA);
    if (!tiled)
      launch(cls<T>("pupdate", true), nbytes<T, T>(N, B.n_act, 3, 0), k_p_update<T>, g(), kBlock, 0, st, pbuf[0], z,
             (const SolveScalars*)sc, nodes, 0, B.actp);
  }
  return cudaGetLastError();
}

// Mixed inner solve on a tiled grid, `iters` PCG iterations with the vector
// updates fused into the stencil passes: x += alpha_prev p_old happens inside the
// next A p pass, r -= alpha q inside the next fine pre-smoothing pass; r and p are
// double-buffered (neighbouring tiles read the old values in their halos).
// x need not be initialised: the first iteration that updates it assigns.  Instead
// of the last x += alpha p, the final update is fused with the refinement step into
// x_out (+)= x + alpha p (k_finish_step; assign on the first refinement step), or,
// with p_last, left to the next refinement step's pass (its p is returned there).
// Runs over the samples the refinement left active (B.n_act, B.actp).
static cudaError_t pcg_inner_fused(SolverBufs& B, const float* a32, const __nv_bfloat16* abf, float* x, float* r,
                                   SolveScalars* sc, const PcgParams& prm, int iters, cudaStream_t st,
                                   float2* x_out, const SolveScalars* sco, bool assign_out,
                                   const float** p_last = nullptr) {
  const int S = B.S, N = B.N, n = B.n_act;
  const Batch bt = B.batch();
  const long long nodes = nodes_of(N);
  const float omega = (float)prm.omega;
  float* rb[2] = {r, (float*)B.r2};
  float* q = (float*)B.q;
  // z and p rotate through three vectors: a new p never overwrites the z or the old p
  // it is formed from, and the V-cycle's z never overwrites the p the next pass reads.
  // With the slab passes the first p equals z and is not stored (p aliases z).
  float* const vb[3] = {(float*)B.vt[0], (float*)B.p, (float*)B.vx[0]};
  const bool alias_first = uses_slab(B, N, 4);
  auto other = [&](const float* a, const float* b) {
    for (float* v : vb)
      if (v != a && v != b) return v;
    return vb[0];
  };
  float* z = vb[0];
  float* pold = vb[1];  // not read by the first pass
  const int napply = tiled_blocks_per_sample(N, S, 4, uses_slab(B, N, 4));
  int nrz = vcycle<float, __nv_bfloat16>(B, rb[0], abf, sc, omega, st, nullptr, nullptr, z);
  scalar(B, sc, SM_RZ0, 0, 0, st, nrz);
  int rc = 0;
  for (int it = 0; it < iters; ++it) {
    float* pnew;
    if (it == 0) {
      pnew = alias_first ? z : other(z, pold);
      tiled_apply<float, float>(z, pold, alias_first ? nullptr : pnew, a32, q, B.partial, sc, N, bt, 1, st);
    } else {
      pnew = other(z, pold);
      // the last pass needs only p.q (for alpha): with the slab passes q is not stored
      tiled_apply_x(z, pold, pnew, a32, (alias_first && it == iters - 1) ? nullptr : q, x, B.partial, sc, N, bt, st,
                    it == 1);
    }
    float* znext = z != pnew ? z : other(pnew, pnew);  // z is dead unless it is the new p
    pold = pnew;
    z = znext;
    scalar(B, sc, SM_ALPHA, 0, 0, st, napply);
    if (it == iters - 1) {
      if (p_last) {  // the refinement step applies x (+)= x + alpha p itself
        *p_last = pnew;
        break;
      }
      with_grid(N, [&](auto c) {
        launch("finish_step", (double)n * nodes * ((iters > 1 ? 4 : 0) + 4 + (assign_out ? 8 : 16)),
               k_finish_step<decltype(c)::value>, grid_nodes(N, n), kBlock, 0, st, x_out, (const float*)x,
               (const float*)pnew, (const SolveScalars*)sc, sco, nodes, N, assign_out ? 1 : 0, iters > 1 ? 0 : 1,
               B.actp);
      });
      break;
    }
    nrz = vcycle<float, __nv_bfloat16>(B, rb[rc], abf, sc, omega, st, q, rb[rc ^ 1], z);
    rc ^= 1;
    scalar(B, sc, SM_BETA, 0, 0, st, nrz);
  }
  return cudaGetLastError();
}

// Buffers the tiled passes write only on interior nodes must hold zero
// boundary nodes: clear them once per solve.
// zero the boundary nodes (2 (N+1)^2 + 4 N (N-1) per sample) of up to 6 vectors
struct ZeroList { void* v[6]; };
template <typename T>
__global__ void k_zero_boundary(ZeroList zl, int nv, int N) {
  const int s = blockIdx.y;
  const int n1 = N + 1;
  const long long plane = (long long)n1 * n1;
  const long long nb = 2 * plane + 4LL * N * (N - 1);
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb) return;
  long long o;
  if (idx < 2 * plane) {
    o = (idx < plane ? 0 : (long long)N * plane) + idx % plane;  // planes z = 0 and z = N
  } else {
    const long long r = idx - 2 * plane;
    const int k = 1 + (int)(r / (4 * N));
    const int p = (int)(r % (4 * N));
    int i, j;
    if (p < n1) { i = p; j = 0; }                       // row y = 0
    else if (p < 2 * n1) { i = p - n1; j = N; }         // row y = N
    else if (p < 2 * n1 + N - 1) { i = 0; j = p - 2 * n1 + 1; }  // column x = 0
    else { i = N; j = p - (2 * n1 + N - 1) + 1; }       // column x = N
    o = i + (long long)n1 * j + plane * k;
  }
  const long long so = (long long)s * plane * n1 + o;
  for (int t = 0; t < nv; ++t) ((T*)zl.v[t])[so] = T(0);
}

template <typename T>
static void zero_boundary(void* const* bufs, int nv, int N, int S, cudaStream_t st) {
  ZeroList zl{};
  for (int t = 0; t < nv; ++t) zl.v[t] = bufs[t];
  const long long nb = 2LL * (N + 1) * (N + 1) + 4LL * N * (N - 1);
  launch("zero_boundary", (double)S * nb * nv * sizeof(T), k_zero_boundary<T>,
         dim3((unsigned)((nb + kBlock - 1) / kBlock), (unsigned)S), kBlock, 0, st, zl, nv, N);
}

// The FP64 tiled passes write interior nodes only: the vectors they produce (and the
// inner solve's correction, which is first assigned by a tiled pass) get zero
// boundary nodes once per solve.
// The mixed path needs none of this: its z-marching passes zero-fill boundary nodes
// when staging, its slab passes take them as 0 when deriving the operand plane and
// interpolating the coarse correction, and the kernels that read whole vectors (the
// refinement's init and accumulation) take the boundary as 0 themselves.
static cudaError_t clear_tiled(SolverBufs& B, int elem, cudaStream_t st) {
  if (!(B.N >= kTiledMinN && B.J >= 1) || elem == 4) return cudaSuccess;
  void* bufs[5] = {B.p, B.vx[0], B.q, B.vt[0], B.r2};
  zero_boundary<double>(bufs, 5, B.N, B.S, st);
  for (int j = 1; j < B.J; ++j)  // coarse levels run by the tiled passes
    if ((B.N >> j) >= kTiledMinN) zero_boundary<double>(&B.vt[j], 1, B.N >> j, B.S, st);
  return cudaGetLastError();
}

cudaError_t pcg_fp64(SolverBufs& B, const double* a64, const double* b, long long bstride, double* x_out,
                     const PcgParams& prm, cudaStream_t st) {
  launch_all(B);
  const dim3 g = grid_nodes(B.N, B.S);
  double* r = (double*)B.r;
  cudaError_t e = clear_tiled(B, 8, st);
  if (e != cudaSuccess) return e;
  const double bb = (double)(bstride ? B.S : 1) * nodes_of(B.N) * 8;
  launch("init_f64", bb + nbytes<double, double>(B.N, B.S, 2, 0), k_init<double>, g, kBlock, 0, st, b, bstride, r,
         x_out, B.partial, nodes_of(B.N));
  scalar(B, B.sc, SM_INIT, 0, 0, st, node_blocks(B.N));
  return pcg_loop<double, double, double>(B, a64, a64, x_out, r, B.sc, prm, 0, st);
}

cudaError_t ir_mixed(SolverBufs& B, const float* a32, const __nv_bfloat16* abf, const double* b, long long bstride,
                     double* x_out, double* r64, const PcgParams& prm, int inner_iters, cudaStream_t st,
                     int fixed_steps, const float2* b_pair, bool pair_out, int inner_next) {
  const int N = B.N, S = B.S;
  const long long nodes = nodes_of(N);
  const int nb = node_blocks(N);
  const bool tiled = N >= kTiledMinN && B.J >= 1;
  SolveScalars* sco = B.sc;
  SolveScalars* sci = B.sc + S;
  float* d = (float*)B.x;
  float* r32 = (float*)B.r;
  const double tol2 = prm.rtol * prm.rtol;
  const double bb = (double)(bstride ? S : 1) * nodes * 8;
  launch_all(B);
  auto g = [&]() { return grid_nodes(N, B.n_act); };
  cudaError_t e = clear_tiled(B, 4, st);
  if (e != cudaSuccess) return e;
  // tiled grids: the FP32 residual is written directly (first from b, then by the
  // refinement residual pass), b and the solution are kept as FP32 (hi, lo) pairs
  // (the solution in r64's storage, assigned by the first step and stored to x_out
  // in FP64 at the end), so the refinement loop executes no FP64 arithmetic.
  if (!tiled && (b_pair || pair_out)) return cudaErrorInvalidValue;  // pairs only on tiled grids
  float2* xdf = pair_out ? (float2*)x_out : (float2*)r64;
  // b as pairs: given, or split by the init pass (per sample, or once when shared)
  float2* bsplit = bstride ? B.bdf : B.bsh;
  const float2* bdf = b_pair ? b_pair : bsplit;
  // 32^3 and 64^3 grids: one slab pass per refinement step applies the inner solve's
  // last update to x and updates the residual pairs rr (B.bdf; b on the first step) by
  // rr -= A inc, so x is only written at nodes its block owns; the first step also
  // writes x's boundary nodes (0), each by the block that owns its rows and planes
  const bool sres = tiled && uses_slab(B, N, 4);
  const float* p_last = nullptr;
  if (inner_next <= 0) inner_next = inner_iters;
  int last_inner = inner_iters;  // inner iterations of the step the next refinement pass completes
  if (tiled) {
    const dim3 gi((unsigned)init_blocks(N), (unsigned)S);
    with_grid(N, [&](auto c) {
      constexpr int NN = decltype(c)::value;
      if (b_pair) {
        launch("init_f32", bb + nbytes<float, float>(N, S, 1, 0), k_init32<true, NN>, gi, kBlock, 0, st, b, b_pair,
               bstride, r32, bsplit, B.partial, nodes, N);
      } else if (bstride) {
        launch("init_f32", bb + nbytes<float, float>(N, S, 1, 0) + (double)S * nodes * 8, k_init32<false, NN>, gi,
               kBlock, 0, st, b, b_pair, bstride, r32, bsplit, B.partial, nodes, N);
      } else {
        // a b shared by every sample is split into pairs once (sample 0's launch), and
        // every sample's FP32 residual and b.b then come from the pairs in FP32
        const dim3 g1((unsigned)init_blocks(N), 1u);
        launch("init_f32", (double)nodes * 20, k_init32<false, NN>, g1, kBlock, 0, st, b, b_pair, bstride, r32, bsplit,
               B.partial, nodes, N);
        launch("init_f32", (double)nodes * 8 + nbytes<float, float>(N, S, 1, 0), k_init32<true, NN>, gi, kBlock, 0, st,
               b, (const float2*)bsplit, bstride, r32, bsplit, B.partial, nodes, N);
      }
    });
    scalar(B, sco, SM_INIT, 0, 0, st, init_blocks(N));
  } else {
    launch("init_f64", bb + nbytes<double, double>(N, S, 2, 0), k_init<double>, g(), kBlock, 0, st, b, bstride, r64,
           x_out, B.partial, nodes);
    scalar(B, sco, SM_INIT, 0, 0, st, nb);
  }
  for (int step = 0;; ++step) {
    if (step > 0) {
      const int cap = fixed_steps > 0 ? fixed_steps : prm.max_iter;
      if (sres) {
        slab_res(d, p_last, last_inner <= 1, sci, step == 1 ? bdf : B.bdf, step == 1 ? bstride : nodes, B.bdf, xdf,
                 step == 1, a32, r32, B.partial, sco, N, B.batch(), st);
        scalar(B, sco, SM_OUTER_CONV, tol2, cap, st, tiled_blocks_per_sample(N, S, 4, true));
      } else if (tiled) {
        tiled_res64(bdf, bstride, xdf, a32, r32, B.partial, sco, N, B.batch(), st);
        scalar(B, sco, SM_OUTER_CONV, tol2, cap, st, tiled_blocks_per_sample(N, S, 8, false));
      } else {
        launch("resid64", (double)(bstride ? B.n_act : 1) * nodes * 8 + nbytes<double, float>(N, B.n_act, 2, 1),
               k_residual64<float>, g(), kBlock, 0, st, b, bstride, (const double*)x_out, a32, r64, B.partial,
               (const SolveScalars*)sco, N, B.actp);
        scalar(B, sco, SM_OUTER_CONV, tol2, cap, st, nb);
      }
    }
    if (fixed_steps > 0) {
      if (step == fixed_steps) break;  // masked steps: no host round trip
    } else if (step > 0) {
      // host-checked: only the samples still above rtol take the next step (the first
      // step launches every sample: it also defines x of those that take no step)
      int n = 0;
      e = compact_active(B, sco, st, n);
      if (e != cudaSuccess) return e;
      if (n == 0) break;
    }
    if (!tiled)
      launch("demote", (double)B.n_act * nodes * 16, k_demote, g(), kBlock, 0, st, (const double*)r64, r32, d,
             (const SolveScalars*)sco, nodes, B.actp);
    scalar(B, sci, SM_INNER_BEGIN, 0, 0, st, nb, 0, sco);
    const int inner = step == 0 ? inner_iters : inner_next;
    last_inner = inner;
    if (tiled) {
      e = pcg_inner_fused(B, a32, abf, d, r32, sci, prm, inner, st, xdf, sco, step == 0, sres ? &p_last : nullptr);
      if (e != cudaSuccess) return e;
    } else {
      e = pcg_loop<float, float, __nv_bfloat16>(B, a32, abf, d, r32, sci, prm, inner, st);
      if (e != cudaSuccess) return e;
      launch("accum", (double)B.n_act * nodes * 20, k_accumulate, g(), kBlock, 0, st, x_out, (const float*)d,
             (const SolveScalars*)sco, nodes, B.actp);
    }
    scalar(B, sco, SM_OUTER_STEP, 0, 0, st, nb, inner);
  }
  launch_all(B);
  if (tiled && !pair_out)
    launch("store_x", (double)S * nodes * 16, k_store_pair, grid_nodes(N, S), kBlock, 0, st, x_out,
           (const float2*)xdf, nodes);
  return cudaGetLastError();
}

}  // namespace mlsgd
