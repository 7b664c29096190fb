// estimator.cu - right-hand sides, Phi, B*q, entropic weights, level
// differences, Chan statistics and the multilevel step (rows a3, a5, a7-a10).
#include <math.h>

#include <algorithm>

#include <type_traits>

#include "internal.cuh"
#include "kernels.h"
#include "launch.h"

namespace mlsgd {

// (B z)_n = int z phi_n (<B u, v> = int u v, Sec. 5) for a cellwise-constant control
// z on the control grid Nc.
//
// Control coarser than the grid (N = r Nc): each of the 8 cells around node n lies in
// one control cell (its parent) and int_e phi_n = h^3 / 8.
__global__ void k_rhs_state(const double* __restrict__ z, int Nc, int N, double* __restrict__ b) {
  const int n1 = N + 1;
  const long long nodes = (long long)n1 * n1 * n1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nodes) return;
  int i, j, k;
  node_ijk(n, n1, i, j, k);
  double acc = 0.0;
  if (interior(i, j, k, N)) {
    const int r = N / Nc;
    for (int dz = -1; dz <= 0; ++dz)
      for (int dy = -1; dy <= 0; ++dy)
        for (int dx = -1; dx <= 0; ++dx)
          acc += z[(i + dx) / r + (long long)Nc * ((j + dy) / r + (long long)Nc * ((k + dz) / r))];
    const double h = 1.0 / N;
    acc *= 0.125 * h * h * h;
  }
  b[n] = acc;
}

// Control grid at least as fine as the grid (Nc = r N): the midpoint rule on each
// control cell c is exact for the multilinear phi_n, so (B z)_n = h_c^3 sum_c z_c
// phi_n(x_c) over the (2r)^3 control cells of the support.  phi_n(x_c) is a product of
// one hat weight per axis, w(m) = 1 - |(m + 1/2) / r - 1| for the m-th of the 2r control
// cells along that axis.  One block per node row (j, k): threads along cx contract
// the (2r)^2 control rows (cy, cz) of the row's support with w(y) w(z) into a column
// sum per cx, then each node i of the row contracts its 2r columns with w(x).
__global__ void __launch_bounds__(kBlock) k_rhs_rows(const double* __restrict__ z, int Nc, int N,
                                                     double* __restrict__ b) {
  extern __shared__ double sm[];  // w[2r], col[Nc]
  const int n1 = N + 1, r = Nc / N, w2 = 2 * r;
  const int j = blockIdx.x, k = blockIdx.y;
  double* brow = b + (long long)n1 * (j + (long long)n1 * k);
  if (j == 0 || j == N || k == 0 || k == N) {
    for (int i = threadIdx.x; i < n1; i += blockDim.x) brow[i] = 0.0;
    return;
  }
  double* w = sm;
  double* col = sm + w2;
  const double inv_r = 1.0 / r;
  for (int m = threadIdx.x; m < w2; m += blockDim.x) w[m] = 1.0 - fabs((m + 0.5) * inv_r - 1.0);
  __syncthreads();
  const long long y0 = (long long)r * (j - 1), z0 = (long long)r * (k - 1);
  for (int cx = threadIdx.x; cx < Nc; cx += blockDim.x) {
    double acc = 0.0;
    for (int mz = 0; mz < w2; ++mz) {
      const double* zp = z + cx + (long long)Nc * (y0 + (long long)Nc * (z0 + mz));
      double accz = 0.0;
      for (int my = 0; my < w2; ++my) accz = fma(w[my], zp[(long long)Nc * my], accz);
      acc = fma(w[mz], accz, acc);
    }
    col[cx] = acc;
  }
  __syncthreads();
  const double hc = 1.0 / Nc;
  const double hc3 = hc * hc * hc;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) {
    double v = 0.0;
    if (i > 0 && i < N) {
      const double* cp = col + r * (i - 1);
      for (int m = 0; m < w2; ++m) v = fma(w[m], cp[m], v);
      v *= hc3;
    }
    brow[i] = v;
  }
}

void launch_rhs_state(const double* z, int Nc, int N, double* b, cudaStream_t st) {
  const double bytes = (double)cells_of(Nc) * 8 + (double)nodes_of(N) * 8;
  if (N > Nc) {
    launch("rhs", bytes, k_rhs_state, dim3(node_blocks(N)), kBlock, 0, st, z, Nc, N, b);
  } else {
    const size_t smem = (size_t)(2 * (Nc / N) + Nc) * sizeof(double);
    launch("rhs", bytes, k_rhs_rows, dim3((unsigned)(N + 1), (unsigned)(N + 1)), kBlock, smem, st, z, Nc, N, b);
  }
}

// e = y - g_h with g_h the nodal interpolant of sin(pi x) sin(pi y) sin(pi z);
// (M e)_n with the consistent Q1 mass M = (h/6)^3 [1 4 1]^(x3); badj = M e on
// interior rows (adjoint right-hand side <y - g, v>_H, Sec. 2.2) and
// Phi = 1/2 e^T M e (eq:cost), reduced per sample in FP64.
__global__ void k_phi_adjrhs(const double* __restrict__ y, int N, double* __restrict__ badj,
                             double* __restrict__ partial, int freq) {
  const int s = blockIdx.y;
  const int n1 = N + 1;
  const long long nodes = (long long)n1 * n1 * n1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const double* ys = y + s * nodes;
  double contrib = 0.0;
  if (n < nodes) {
    int i, j, k;
    node_ijk(n, n1, i, j, k);
    double me = 0.0;
    if (interior(i, j, k, N)) {
      const double invN = (double)freq / N;  // g = prod sin(freq pi x)
      double gx[3], gy[3], gz[3];
      for (int d = -1; d <= 1; ++d) {
        gx[d + 1] = sinpi((i + d) * invN);
        gy[d + 1] = sinpi((j + d) * invN);
        gz[d + 1] = sinpi((k + d) * invN);
      }
      for (int w = -1; w <= 1; ++w) {
        const int kk = k + w;
        const double mz = (w == 0) ? 4.0 : 1.0;
        const double gzv = (kk == 0 || kk == N) ? 0.0 : gz[w + 1];
        for (int v = -1; v <= 1; ++v) {
          const int jj = j + v;
          const double my = (v == 0) ? 4.0 : 1.0;
          const double gyv = (jj == 0 || jj == N) ? 0.0 : gy[v + 1];
          for (int u = -1; u <= 1; ++u) {
            const int ii = i + u;
            const double mx = (u == 0) ? 4.0 : 1.0;
            const double gxv = (ii == 0 || ii == N) ? 0.0 : gx[u + 1];
            const double e = ys[ii + (long long)n1 * (jj + (long long)n1 * kk)] - gxv * gyv * gzv;
            me += mx * my * mz * e;
          }
        }
      }
      const double h6 = 1.0 / (6.0 * N);
      me *= h6 * h6 * h6;
      contrib = (ys[n] - gx[1] * gy[1] * gz[1]) * me;
    }
    badj[s * nodes + n] = me;
  }
  const double bs = block_sum(contrib);
  if (threadIdx.x == 0) partial[(long long)s * gridDim.x + blockIdx.x] = bs;
}

__global__ void k_phi_finish(const double* __restrict__ partial, int nblk, int S, double* __restrict__ phi) {
  const int s = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= S) return;
  double v = 0.0;
  for (int t = lane; t < nblk; t += 32) v += partial[(long long)s * nblk + t];
  v = warp_sum(v);
  if (lane == 0) phi[s] = 0.5 * v;
}

// the state as FP32 pairs on a tiled grid: M e written as pairs (tables as pairs)
void launch_phi_adjrhs_df(const float2* y, int N, int S, float2* badj, double* phi, double* partial,
                          const float2* gtab, const float2* mgtab, cudaStream_t st) {
  if (S == 0) return;
  const int nb = tiled_phi_df(y, N, S, gtab, mgtab, badj, partial, st);
  launch("phi_finish", 0.0, k_phi_finish, dim3((S + 7) / 8), 256, 0, st, (const double*)partial, nb, S, phi);
}

void launch_phi_adjrhs(const double* y, int N, int S, double* badj, double* phi, double* partial, const double* gtab,
                       const double* mgtab, cudaStream_t st, int freq) {
  if (S == 0) return;
  if (N >= kTiledMinN && gtab != nullptr) {
    const int nb = tiled_phi(y, N, S, gtab, mgtab, badj, partial, st);
    launch("phi_finish", 0.0, k_phi_finish, dim3((S + 7) / 8), 256, 0, st, (const double*)partial, nb, S, phi);
    return;
  }
  const int nb = node_blocks(N);
  launch("phi_adjrhs", (double)S * nodes_of(N) * 16, k_phi_adjrhs, dim3(nb, S), kBlock, 0, st, y, N, badj, partial,
         freq);
  launch("phi_finish", 0.0, k_phi_finish, dim3((S + 7) / 8), 256, 0, st, (const double*)partial, nb, S, phi);
}

// ---------------------------------------------------------------- level statistics
// work layout: [0] shift_new, [1] scale_old = exp(theta (shift_old - shift_new)),
// [2] n_old, [3] n_batch, [4..4+S) w_fine, [4+S..4+2S) w_coarse, then the same
// weights as FP32 (hi, lo) pairs (8 bytes each): [4+2S..4+3S) fine, [4+3S..4+4S) coarse.
//
// Single block: shift, per-sample weights Y~ = exp(theta (Phi - shift)), and
// the scalar statistics of dY~ = Y~_l - Y~_{l-1} (Welford over the batch,
// then the Chan merge with the rescaled old sums; Algorithm 1, PairwiseUpdate).
__global__ void k_level_scalars(const double* __restrict__ phif, const double* __restrict__ phic, int S,
                                double theta, double* __restrict__ sc, double* __restrict__ work,
                                const int* __restrict__ iters, const int* __restrict__ status) {
  __shared__ double smax[kBlock / 32];
  double m = -INFINITY;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    m = fmax(m, phif[s]);
    if (phic) m = fmax(m, phic[s]);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bm = smax[0];
    for (int w = 1; w < kBlock / 32; ++w) bm = fmax(bm, smax[w]);
    const double n_old = sc[MLSGD_S_COUNT];
    const double shift_old = sc[MLSGD_S_SHIFT];
    const double shift = (n_old > 0.0) ? fmax(shift_old, bm) : bm;
    work[0] = shift;
    work[1] = (n_old > 0.0) ? exp(theta * (shift_old - shift)) : 0.0;
    work[2] = n_old;
    work[3] = (double)S;
  }
  __syncthreads();
  const double shift = work[0];
  // a sample whose solve went non-finite (status bit 1) gets NaN weights, so the
  // record, and the step that reads it, report the failure instead of using it
  float2* wpair = (float2*)(work + 4 + 2 * S);
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const bool bad = status != nullptr && ((status[s] | (phic ? status[S + s] : 0)) & 2);
    const double wf = bad ? NAN : exp(theta * (phif[s] - shift));
    const double wc = bad ? NAN : (phic ? exp(theta * (phic[s] - shift)) : 0.0);
    work[4 + s] = wf;
    work[4 + S + s] = wc;
    wpair[s] = df_split(wf);
    wpair[S + s] = df_split(wc);
  }
  __syncthreads();
  // batch mean and M2 of dY~ by shifted sums over the block (deviations from the
  // first sample), and the sample-wise maxima / counts, all in parallel
  const double ref = work[4] - work[4 + S];
  double sd = 0.0, sd2 = 0.0, pm = -INFINITY, itp = 0.0, ncp = 0.0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const double d = (work[4 + s] - work[4 + S + s]) - ref;
    sd += d;
    sd2 = fma(d, d, sd2);
    pm = fmax(pm, fmax(phif[s], phic ? phic[s] : -INFINITY));
  }
  if (iters) {
    const int nsolve = phic ? 2 * S : S;
    for (int t = threadIdx.x; t < nsolve; t += blockDim.x) {
      itp += iters[t];
      ncp += (status[t] != 0) ? 1.0 : 0.0;
    }
  }
  sd = block_sum(sd);
  __syncthreads();
  sd2 = block_sum(sd2);
  __syncthreads();
  itp = block_sum(itp);
  __syncthreads();
  ncp = block_sum(ncp);
  for (int o = 16; o > 0; o >>= 1) pm = fmax(pm, __shfl_xor_sync(0xffffffffu, pm, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = pm;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kBlock / 32; ++w) pm = fmax(pm, smax[w]);
    const double mean = ref + sd / S;
    const double s2 = fmax(sd2 - sd * (sd / S), 0.0);
    const double n_old = work[2], scale = work[1];
    const double n = n_old + S;
    const double mo = sc[MLSGD_S_MEAN_DY] * scale;
    const double so = sc[MLSGD_S_S2_DY] * scale * scale;
    const double delta = mo - mean;
    sc[MLSGD_S_MEAN_DY] = mean + (n_old / n) * delta;
    sc[MLSGD_S_S2_DY] = so + s2 + delta * delta * n_old * S / n;
    sc[MLSGD_S_COUNT] = n;
    sc[MLSGD_S_SHIFT] = shift;
    sc[MLSGD_S_PHI_MAX] = fmax(sc[MLSGD_S_PHI_MAX], pm);
    sc[MLSGD_S_ITERS] += itp;
    sc[MLSGD_S_NOCONV] += ncp;
  }
}

// Average of the nodal function q (grid N) over control cell (cx, cy, cz) of the
// Nc grid.  N <= Nc (r = Nc / N): q is trilinear on the control cell, so the
// average is its value at the cell centre.  N > Nc (r = N / Nc): trapezoid
// weights per axis over the r + 1 grid nodes of the cell, 1/r inside and
// 1/(2r) at the two ends.
__device__ __forceinline__ double eval_at_ctrl(const double* __restrict__ q, int N, int Nc, int cx, int cy, int cz) {
  const int n1 = N + 1;
  if (N > Nc) {
    const int r = N / Nc;
    const double wi = 1.0 / r, we = 0.5 / r;
    double acc = 0.0;
    for (int c = 0; c <= r; ++c) {
      const double wz = (c == 0 || c == r) ? we : wi;
      for (int b = 0; b <= r; ++b) {
        const double wy = (b == 0 || b == r) ? we : wi;
        const double* row = q + (long long)r * cx + (long long)n1 * ((long long)r * cy + b + (long long)n1 * ((long long)r * cz + c));
        double rs = 0.5 * (row[0] + row[r]);
        for (int a = 1; a < r; ++a) rs += row[a];
        acc += wz * wy * rs * wi;
      }
    }
    return acc;
  }
  const int r = Nc / N;
  const int ex = cx / r, ey = cy / r, ez = cz / r;
  const double tx = ((cx % r) + 0.5) / r, ty = ((cy % r) + 0.5) / r, tz = ((cz % r) + 0.5) / r;
  const double* b = q + ex + (long long)n1 * (ey + (long long)n1 * ez);
  const long long sy = n1, sz = (long long)n1 * n1;
  const double c00 = b[0] * (1 - tx) + b[1] * tx;
  const double c10 = b[sy] * (1 - tx) + b[sy + 1] * tx;
  const double c01 = b[sz] * (1 - tx) + b[sz + 1] * tx;
  const double c11 = b[sy + sz] * (1 - tx) + b[sy + sz + 1] * tx;
  return (c00 * (1 - ty) + c10 * ty) * (1 - tz) + (c01 * (1 - ty) + c11 * ty) * tz;
}

// The eight trilinear weights of a control-cell centre inside a level cell
// (level no finer than the control grid), set up once per control cell.
struct CellInterp {
  long long base;  // node (ex, ey, ez) of the level cell holding the control cell
  long long sy, sz;
  double w[8];     // weight of node (ex + a, ey + b, ez + c) at index a + 2b + 4c
  float w32[8];    // the same weights (exact in FP32: r is a power of two)
  __device__ void setup(int N, int Nc, int cx, int cy, int cz) {
    const int n1 = N + 1, r = Nc / N;
    const double tx = ((cx % r) + 0.5) / r, ty = ((cy % r) + 0.5) / r, tz = ((cz % r) + 0.5) / r;
    base = (cx / r) + (long long)n1 * ((cy / r) + (long long)n1 * (cz / r));
    sy = n1;
    sz = (long long)n1 * n1;
#pragma unroll
    for (int e = 0; e < 8; ++e)
      w[e] = ((e & 1) ? tx : 1.0 - tx) * ((e & 2) ? ty : 1.0 - ty) * ((e & 4) ? tz : 1.0 - tz);
#pragma unroll
    for (int e = 0; e < 8; ++e) w32[e] = (float)w[e];
  }
  // the same average of an FP32 pair field, in pair arithmetic
  __device__ __forceinline__ DF eval(const float2* __restrict__ q) const {
    const float2* b = q + base;
    const float2 v[8] = {b[0], b[1], b[sy], b[sy + 1], b[sz], b[sz + 1], b[sz + sy], b[sz + sy + 1]};
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float p = __fmul_rn(w32[e], v[e].x);
      const float pe = __fmaf_rn(w32[e], v[e].y, __fmaf_rn(w32[e], v[e].x, -p));
      const float t = __fadd_rn(s, p);  // two-sum (intrinsics: never contracted)
      const float bb = __fsub_rn(t, s);
      c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb)), pe));
      s = t;
    }
    return df_norm(s, c);
  }
  __device__ __forceinline__ double eval(const double* __restrict__ q) const {
    const double* b = q + base;
    double v = w[0] * b[0];
    v = fma(w[1], b[1], v);
    v = fma(w[2], b[sy], v);
    v = fma(w[3], b[sy + 1], v);
    v = fma(w[4], b[sz], v);
    v = fma(w[5], b[sz + 1], v);
    v = fma(w[6], b[sz + sy], v);
    return fma(w[7], b[sz + sy + 1], v);
  }
};

// The same trilinear average for FP32 pair fields with the weights kept as three
// per-axis pairs (exact dyadic values, so each product equals CellInterp's w32) and a
// 32-bit node index: fewer registers per thread, so more threads in flight.
struct PairInterp {
  int base, sy, sz;
  float wx[2], wy[2], wz[2];
  __device__ void setup(int N, int Nc, int cx, int cy, int cz) {
    const int n1 = N + 1, r = Nc / N;
    const float ir = 1.0f / (float)r;  // r a power of two: exact
    const float tx = ((cx % r) + 0.5f) * ir, ty = ((cy % r) + 0.5f) * ir, tz = ((cz % r) + 0.5f) * ir;
    wx[0] = 1.0f - tx; wx[1] = tx;
    wy[0] = 1.0f - ty; wy[1] = ty;
    wz[0] = 1.0f - tz; wz[1] = tz;
    base = (cx / r) + n1 * ((cy / r) + n1 * (cz / r));
    sy = n1;
    sz = n1 * n1;
  }
  __device__ __forceinline__ DF eval(const float2* __restrict__ q) const {
    const float2* b = q + base;
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float w = (wx[e & 1] * wy[(e >> 1) & 1]) * wz[e >> 2];  // exact
      const float2 v = b[(e & 1) + ((e >> 1) & 1) * sy + (e >> 2) * sz];
      const float p = __fmul_rn(w, v.x);
      const float pe = __fmaf_rn(w, v.y, __fmaf_rn(w, v.x, -p));
      const float t = __fadd_rn(s, p);  // two-sum (intrinsics: never contracted)
      const float bb = __fsub_rn(t, s);
      c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb)), pe));
      s = t;
    }
    return df_norm(s, c);
  }
};

// eval_at_ctrl for an FP32 pair field, in pair arithmetic (trapezoid weights are
// exact in FP32 since r is a power of two)
__device__ DF eval_at_ctrl(const float2* __restrict__ q, int N, int Nc, int cx, int cy, int cz) {
  const int n1 = N + 1;
  const int r = N / Nc;
  const float wi = 1.0f / r, we = 0.5f / r;
  DF acc{0.f, 0.f};
  for (int c = 0; c <= r; ++c) {
    const float wz = (c == 0 || c == r) ? we : wi;
    for (int b = 0; b <= r; ++b) {
      const float wy = (b == 0 || b == r) ? we : wi;
      const float2* row = q + (long long)r * cx + (long long)n1 * ((long long)r * cy + b + (long long)n1 * ((long long)r * cz + c));
      DF rs = df_mulf(df_add(df_make(row[0]), df_make(row[r])), 0.5f);
      for (int a = 1; a < r; ++a) rs = df_add(rs, df_make(row[a]));
      acc = df_add(acc, df_mulf(rs, wz * wy * wi));
    }
  }
  return acc;
}

// One thread per control cell: B*q as the cell average for both grids,
// dX~_s = w_f[s] B*q_f[s] - w_c[s] B*q_c[s]; batch mean and M2 by the
// shifted-data sums (deviations from the first sample: no division per
// sample, stable when the first sample is typical), then the Chan merge with
// the rescaled old mean; block partials of h_c^3 (M2_batch + delta^2 n_old S / n).
// PF / PC: the fine / coarse adjoint solutions are FP32 (hi, lo) pairs (the mixed
// path on tiled grids); their control-cell averages are then formed in pair
// arithmetic (exact weights, about 48 significant bits), and with both grids in
// pairs so is the weighted difference w_f X_f - w_c X_c (weights rounded to pairs
// from their FP64 values; error below 6 u^2 (|w_f X_f| + |w_c X_c|), u = 2^-24), a
// function of the sample alone.  The sums of the cancelling differences, the
// deviations from the first sample and the merge are FP64 in every case
// (eq:delta-notation, eq:sec-order-sum), so a record does not depend on how the
// samples were split into calls beyond FP64 rounding.  (This part has about 2 FP64
// operations per FP32 one; GB300 issues FP64 at 1/58 of the FP32 rate, so the FP64
// count sets the kernel's time.)
__device__ __forceinline__ double ctrl_avg(const CellInterp& I, bool fast, const double* q, int N, int Nc, int cx,
                                           int cy, int cz) {
  return fast ? I.eval(q) : eval_at_ctrl(q, N, Nc, cx, cy, cz);
}
// FP32 -> FP64 by moving the fields (IEEE 754 binary32 and binary64 layouts), in
// integer instructions instead of the FP64 conversion: exponent rebiased by
// 1023 - 127, mantissa shifted into the top of the 52-bit field; 0 and subnormals
// give a signed 0, Inf and NaN keep their class (a NaN stays a NaN).
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const uint32_t e11 = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);
  const uint32_t mh = e == 0u ? 0u : ((m >> 3) | ((e == 0xffu && m != 0u) ? 0x80000u : 0u));
  const uint32_t hi = (u & 0x80000000u) | (e11 << 20) | mh;
  const uint32_t lo = e == 0u ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ DF ctrl_avg_df(const CellInterp& I, bool fast, const float2* q, int N, int Nc, int cx,
                                          int cy, int cz) {
  return fast ? I.eval(q) : eval_at_ctrl(q, N, Nc, cx, cy, cz);
}
__device__ __forceinline__ double ctrl_avg(const CellInterp& I, bool fast, const float2* q, int N, int Nc, int cx,
                                           int cy, int cz) {
  return df_to_double(ctrl_avg_df(I, fast, q, N, Nc, cx, cy, cz));
}
template <bool PF, bool PC, bool FAST = false>
__global__ void k_level_field(const void* __restrict__ qf_, int Nf, const void* __restrict__ qc_, int Ncs, int S,
                              int Nc, const double* __restrict__ work, double* __restrict__ field,
                              double* __restrict__ partial) {
  using QF = typename std::conditional<PF, float2, double>::type;
  using QC = typename std::conditional<PC, float2, double>::type;
  const QF* qf = (const QF*)qf_;
  const QC* qc = (const QC*)qc_;
  const long long ncell = (long long)Nc * Nc * Nc;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (c < ncell) {
    const int cx = (int)(c % Nc), cy = (int)((c / Nc) % Nc), cz = (int)(c / ((long long)Nc * Nc));
    const long long nf = nodes_of(Nf), ncn = qc ? nodes_of(Ncs) : 0;
    const double* wf = work + 4;
    const double* wc = work + 4 + S;
    const float2* wfp = (const float2*)(work + 4 + 2 * S);
    const float2* wcp = wfp + S;
    // level grids no finer than the control grid: weights hoisted out of the sample loop
    const bool fast_f = Nf <= Nc, fast_c = !qc || Ncs <= Nc;
    double ref = 0.0, sd = 0.0, sd2 = 0.0;
    if constexpr (PF && PC && FAST) {  // both grids no finer than the control grid
      PairInterp Pf{}, Pc{};
      Pf.setup(Nf, Nc, cx, cy, cz);
      Pc.setup(Ncs, Nc, cx, cy, cz);
      // sample pointers advanced by addition: a 64-bit multiply per sample would issue
      // on the FP64 pipe of this part, the kernel's bottleneck
      const QF* qfs = qf;
      const QC* qcs = qc;
      for (int s = 0; s < S; ++s, qfs += nf, qcs += ncn) {
        const DF vf = df_mul(df_make(wfp[s]), Pf.eval(qfs));
        const DF vc = df_mul(df_make(wcp[s]), Pc.eval(qcs));
        const DF vd = df_add(vf, df_neg(vc));
        const double v = f2d(vd.h) + f2d(vd.l);
        if (s == 0) ref = v;
        const double d = v - ref;
        sd += d;
        sd2 = fma(d, d, sd2);
      }
    } else {
    CellInterp If{}, Ic{};
    if (fast_f) If.setup(Nf, Nc, cx, cy, cz);
    if (qc && fast_c) Ic.setup(Ncs, Nc, cx, cy, cz);
    for (int s = 0; s < S; ++s) {
      double v;
      if constexpr (PF && PC) {
        const DF vf = df_mul(df_make(wfp[s]), ctrl_avg_df(If, fast_f, qf + s * nf, Nf, Nc, cx, cy, cz));
        const DF vc = df_mul(df_make(wcp[s]), ctrl_avg_df(Ic, fast_c, qc + s * ncn, Ncs, Nc, cx, cy, cz));
        const DF vd = df_add(vf, df_neg(vc));
        v = f2d(vd.h) + f2d(vd.l);
      } else {
        v = wf[s] * ctrl_avg(If, fast_f, qf + s * nf, Nf, Nc, cx, cy, cz);
        if (qc) v = fma(-wc[s], ctrl_avg(Ic, fast_c, qc + s * ncn, Ncs, Nc, cx, cy, cz), v);
      }
      if (s == 0) ref = v;
      const double d = v - ref;
      sd += d;
      sd2 = fma(d, d, sd2);
    }
    }
    const double mean = ref + sd / S;
    const double m2 = fmax(sd2 - sd * (sd / S), 0.0);
    const double n_old = work[2], scale = work[1];
    const double n = n_old + S;
    const double mo = (n_old > 0.0) ? field[c] * scale : 0.0;
    const double delta = mo - mean;
    field[c] = mean + (n_old / n) * delta;
    const double hc = 1.0 / Nc;
    contrib = hc * hc * hc * (m2 + delta * delta * n_old * S / n);
  }
  const double bs = block_sum(contrib);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs;
}

// ---- statistics of a level whose grids are coarser than the control grid (Nc = r Nf,
// r >= 2).  Interpolation to the control grid is linear, so with the nodal values
// x_s = w_f[s] q_f[s] - w_c[s] P q_c[s] on the level's fine grid (P q_c: the coarse
// trilinear function at the fine nodes, which interpolation to the control cells
// reproduces exactly) the batch mean field is the interpolation of the nodal mean,
// and ||I x||_U^2 = sum over level cells e of x_e^T G x_e with the fixed 8 x 8 Gram
// matrix G = h_f^3 (g x g x g), g = (1/r) sum_m w(t_m) w(t_m)^T, w(t) = (1 - t, t),
// t_m = (m + 1/2)/r (the midpoint rule over the r^3 control cells of a level cell is
// exact for the integrand of these trilinear weights).  M2 of the batch is then
// sum_s ||d_s||_G^2 - S ||mean d||_G^2 with d_s = x_s - x_0 (deviations from the
// first sample, as in k_level_field).  Work per sample: the level's nodes and cells,
// not the control cells.
__device__ __forceinline__ double ldq(const double* p, long long i) { return p[i]; }
__device__ __forceinline__ double ldq(const float2* p, long long i) {
  const float2 v = p[i];
  return (double)v.x + (double)v.y;
}
template <typename QF, typename QC>
__device__ __forceinline__ double lvl_x(const QF* qfs, const QC* qcs, int Nf, int i, int j, int k, double wf,
                                        double wc) {
  const int n1 = Nf + 1;
  double v = wf * ldq(qfs, i + (long long)n1 * (j + (long long)n1 * k));
  if (qcs) {
    const int c1 = Nf / 2 + 1;
    const int di = i & 1, dj = j & 1, dk = k & 1;
    const long long b = (i >> 1) + (long long)c1 * ((j >> 1) + (long long)c1 * (k >> 1));
    double acc = 0.0;
    for (int c = 0; c <= dk; ++c)
      for (int bb = 0; bb <= dj; ++bb)
        for (int a = 0; a <= di; ++a) acc += ldq(qcs, b + a + (long long)c1 * (bb + (long long)c1 * c));
    v -= wc * acc * (1.0 / (double)(1 << (di + dj + dk)));
  }
  return v;
}
// x_s at every node of the level grid, written over q_f (same 8-byte slots; q_f is
// not needed after the statistics)
template <typename QF, typename QC>
__global__ void k_lvl_x(QF* __restrict__ qf, int Nf, const QC* __restrict__ qc, int S,
                        const double* __restrict__ work) {
  const int s = blockIdx.y;
  const int n1 = Nf + 1;
  const long long nodes = (long long)n1 * n1 * n1;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nodes) return;
  const int i = (int)(n % n1), j = (int)((n / n1) % n1), k = (int)(n / ((long long)n1 * n1));
  const long long ncn = qc ? nodes_of(Nf / 2) : 0;
  const double x = lvl_x(qf + s * nodes, qc ? qc + s * ncn : (const QC*)nullptr, Nf, i, j, k, work[4 + s],
                         work[4 + S + s]);
  reinterpret_cast<double*>(qf)[s * nodes + n] = x;
}
// nodal x_0 and sum_s (x_s - x_0)
__global__ void k_lvl_nodes(const double* __restrict__ x, long long nodes, int S, double* __restrict__ x0,
                            double* __restrict__ dsum) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nodes) return;
  const double xr = x[n];
  double ds = 0.0;
  for (int s = 1; s < S; ++s) ds += x[s * nodes + n] - xr;
  x0[n] = xr;
  dsum[n] = ds;
}
// d^T G d for the 8 nodal values of a level cell (index a + 2b + 4c)
__device__ __forceinline__ double gram8(const double* d, double A, double B) {
  double t[8], u[8];
#pragma unroll
  for (int e = 0; e < 8; e += 2) { t[e] = A * d[e] + B * d[e + 1]; t[e + 1] = B * d[e] + A * d[e + 1]; }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    if (e & 2) continue;
    u[e] = A * t[e] + B * t[e + 2];
    u[e + 2] = B * t[e] + A * t[e + 2];
  }
  double q = 0.0;
#pragma unroll
  for (int e = 0; e < 4; ++e) q += d[e] * (A * u[e] + B * u[e + 4]) + d[e + 4] * (B * u[e] + A * u[e + 4]);
  return q;
}
// per level cell: sum_s ||d_s||^2 - S ||mean d||^2 over the cell, block partials;
// blockIdx.y takes samples y, y + gridDim.y, ... (the mean term goes with y = 0)
__global__ void k_lvl_cells(const double* __restrict__ x, int Nf, int S, const double* __restrict__ x0,
                            const double* __restrict__ dsum, double A, double B, double hf3,
                            double* __restrict__ partial) {
  const long long cells = (long long)Nf * Nf * Nf;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double contrib = 0.0;
  if (e < cells) {
    const int ci = (int)(e % Nf), cj = (int)((e / Nf) % Nf), ck = (int)(e / ((long long)Nf * Nf));
    const int n1 = Nf + 1;
    const long long nodes = (long long)n1 * n1 * n1;
    long long nv[8];
    double xr[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      nv[v] = (ci + (v & 1)) + (long long)n1 * ((cj + ((v >> 1) & 1)) + (long long)n1 * (ck + (v >> 2)));
      xr[v] = x0[nv[v]];
    }
    double acc = 0.0;
    for (int s = blockIdx.y; s < S; s += gridDim.y) {
      const double* xs = x + s * nodes;
      double d[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) d[v] = xs[nv[v]] - xr[v];
      acc += gram8(d, A, B);
    }
    if (blockIdx.y == 0) {
      double db[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) db[v] = dsum[nv[v]] / S;
      acc -= S * gram8(db, A, B);
    }
    contrib = hf3 * acc;
  }
  const double bs = block_sum(contrib);
  if (threadIdx.x == 0) partial[blockIdx.x + (long long)gridDim.x * blockIdx.y] = bs;
}
// per control cell: batch mean = interpolated nodal mean; Chan merge with the old
// field; block partials of h_c^3 delta^2 n_old S / n.  A block takes kLvlRows rows
// (cy, cz) of control cells, 256 cells of a row per block in x; per row the
// level-node columns are first interpolated in (y, z) into shared memory, then each
// cell interpolates linearly in x between the two columns of its level cell.
constexpr int kLvlRows = 16;
__global__ void __launch_bounds__(kBlock) k_lvl_field(const double* __restrict__ x0, const double* __restrict__ dsum,
                                                      int Nf, int Nc, int S, const double* __restrict__ work,
                                                      double* __restrict__ field, double* __restrict__ partial) {
  extern __shared__ double col[];  // [2][Nf + 1]: x0 and dsum interpolated in (y, z)
  const int n1 = Nf + 1, r = Nc / Nf;
  const long long sz = (long long)n1 * n1;
  const double inv_r = 1.0 / r;
  const double n_old = work[2], scale = work[1];
  const double n = n_old + S;
  const double inv_s = 1.0 / S, a = n_old / n;
  const int cx = blockIdx.x * blockDim.x + threadIdx.x;
  const int ex = cx / r;
  const double tx = (cx - ex * r + 0.5) * inv_r;
  const long long rows = (long long)Nc * Nc;
  double contrib = 0.0;
  for (long long row = (long long)blockIdx.y * kLvlRows; row < rows && row < (long long)(blockIdx.y + 1) * kLvlRows;
       ++row) {
    const int cy = (int)(row % Nc), cz = (int)(row / Nc);
    const int ey = cy / r, ez = cz / r;
    const double ty = (cy - ey * r + 0.5) * inv_r, tz = (cz - ez * r + 0.5) * inv_r;
    __syncthreads();  // the previous row's columns are no longer read
    for (int c = threadIdx.x; c < n1; c += blockDim.x) {
      const long long b = c + (long long)n1 * ey + sz * ez;
      const double w00 = (1.0 - ty) * (1.0 - tz), w10 = ty * (1.0 - tz), w01 = (1.0 - ty) * tz, w11 = ty * tz;
      col[c] = w00 * x0[b] + w10 * x0[b + n1] + w01 * x0[b + sz] + w11 * x0[b + sz + n1];
      col[n1 + c] = w00 * dsum[b] + w10 * dsum[b + n1] + w01 * dsum[b + sz] + w11 * dsum[b + sz + n1];
    }
    __syncthreads();
    if (cx < Nc) {
      const double xv = fma(tx, col[ex + 1] - col[ex], col[ex]);
      const double dv = fma(tx, col[n1 + ex + 1] - col[n1 + ex], col[n1 + ex]);
      const double mean = fma(dv, inv_s, xv);
      const long long c = cx + row * Nc;
      const double mo = (n_old > 0.0) ? field[c] * scale : 0.0;
      const double delta = mo - mean;
      field[c] = fma(a, delta, mean);
      contrib = fma(delta, delta, contrib);
    }
  }
  const double hc = 1.0 / Nc;
  contrib *= hc * hc * hc * n_old * S / n;
  const double bs = block_sum(contrib);
  if (threadIdx.x == 0) partial[blockIdx.x + (long long)gridDim.x * blockIdx.y] = bs;
}

// returns the number of block partials written (at most level_partial_cap(Nc, Nf))
template <typename QF, typename QC>
static int launch_lvl(const void* qf, int Nf, const void* qc, int S, int Nc, const double* work, double* field,
                      double* partial, double* nodebuf, cudaStream_t st) {
  const long long nodes = nodes_of(Nf), cells = cells_of(Nf), ncell = cells_of(Nc);
  double* x0 = nodebuf;
  double* dsum = nodebuf + nodes;
  const int r = Nc / Nf;
  double A = 0.0, B = 0.0;
  for (int m = 0; m < r; ++m) {
    const double t = (m + 0.5) / r;
    A += (1.0 - t) * (1.0 - t) / r;
    B += t * (1.0 - t) / r;
  }
  const double hf = 1.0 / Nf;
  const double qb = (double)S * sizeof(QF) * (nodes + (qc ? nodes_of(Nf / 2) : 0));
  const unsigned nbn = (unsigned)((nodes + kBlock - 1) / kBlock);
  launch("level_x", qb + (double)S * nodes * 8, k_lvl_x<QF, QC>, dim3(nbn, (unsigned)S), kBlock, 0, st,
         (QF*)const_cast<void*>(qf), Nf, (const QC*)qc, S, work);
  const double* x = (const double*)qf;
  launch("level_nodes", (double)S * nodes * 8 + (double)nodes * 16, k_lvl_nodes, dim3(nbn), kBlock, 0, st, x, nodes,
         S, x0, dsum);
  const unsigned fx = (unsigned)((Nc + kBlock - 1) / kBlock);
  const unsigned fy = (unsigned)(((long long)Nc * Nc + kLvlRows - 1) / kLvlRows);
  const long long nf = (long long)fx * fy;
  launch("level_field", (double)nodes * 16 + (double)ncell * 16, k_lvl_field, dim3(fx, fy), kBlock,
         (size_t)2 * (Nf + 1) * sizeof(double), st, (const double*)x0, (const double*)dsum, Nf, Nc, S, work, field,
         partial);
  // samples spread over blockIdx.y: about 4 blocks per SM, within the partial buffer
  const long long cb = (cells + kBlock - 1) / kBlock;
  long long g = std::min<long long>((level_partial_cap(Nc, Nf) - nf) / cb, (4LL * 152 + cb - 1) / cb);
  g = std::max<long long>(1, std::min<long long>(g, S));
  launch("level_cells", (double)S * nodes * 8 + (double)nodes * 16, k_lvl_cells, dim3((unsigned)cb, (unsigned)g),
         kBlock, 0, st, x, Nf, S, (const double*)x0, (const double*)dsum, A, B, hf * hf * hf, partial + nf);
  return (int)(nf + cb * g);
}

// s2_dx = old * scale^2 + sum of partials (fixed order, one warp)
__global__ void k_level_finish(const double* __restrict__ partial, int nblk, const double* __restrict__ work,
                               double* __restrict__ sc) {
  const int lane = threadIdx.x;
  double v = 0.0;
  for (int t = lane; t < nblk; t += 32) v += partial[t];
  v = warp_sum(v);
  if (lane == 0) {
    const double scale = work[1];
    sc[MLSGD_S_S2_DX] = (work[2] > 0.0 ? sc[MLSGD_S_S2_DX] * scale * scale : 0.0) + v;
  }
}

void launch_level_stats(const double* qf, const double* phif, int Nf, const double* qc, const double* phic,
                        int Ncoarse, int S, int Nc, double theta, double* field, double* scalars, double* work,
                        double* partial, const int* iters, const int* status, cudaStream_t st, bool qf_pairs,
                        bool qc_pairs, double* nodebuf) {
  if (S == 0) return;
  launch("level_scalars", 0.0, k_level_scalars, dim3(1), kBlock, 0, st, phif, phic, S, theta, scalars, work, iters,
         status);
  // levels at least 4x coarser than the control grid (per axis): statistics on the level
  // grid (cost ~ level nodes and cells per sample instead of control cells per sample;
  // at 2x the control-cell path in pair arithmetic is cheaper).  q_f is overwritten.
  if (nodebuf && 4 * Nf <= Nc) {
    const int nb = (qf_pairs && qc_pairs) ? launch_lvl<float2, float2>(qf, Nf, qc, S, Nc, work, field, partial, nodebuf, st)
                   : qf_pairs             ? launch_lvl<float2, double>(qf, Nf, qc, S, Nc, work, field, partial, nodebuf, st)
                                          : launch_lvl<double, double>(qf, Nf, qc, S, Nc, work, field, partial, nodebuf, st);
    launch("level_finish", 0.0, k_level_finish, dim3(1), 32, 0, st, (const double*)partial, nb, (const double*)work,
           scalars);
    return;
  }
  const long long ncell = (long long)Nc * Nc * Nc;
  const int nblk = (int)((ncell + kBlock - 1) / kBlock);
  const double qbytes = (double)S * 8 * (nodes_of(Nf) + (qc ? nodes_of(Ncoarse) : 0));
  // pairs on the coarse grid only come with pairs on the fine grid (it is at least as large)
  const bool fast = Nf <= Nc && (!qc || Ncoarse <= Nc);
  auto lf = qf_pairs ? (qc_pairs ? (fast ? k_level_field<true, true, true> : k_level_field<true, true>)
                                 : k_level_field<true, false>)
                     : k_level_field<false, false>;
  // FP64 operations per control cell and sample: both grids in pairs, the pair value
  // to FP64 (2 conversions, 1 add), its deviation and the two sums; otherwise also the
  // FP64 weighting and, for FP64 fields, the 8-node averages
  const double f64ops = qf_pairs && qc_pairs ? (fast ? 4.0 : 6.0) : (qf_pairs ? 16.0 : 21.0);
  launch_flops("level_field", qbytes + (double)ncell * 16, (double)S * ncell * f64ops, lf, dim3(nblk), kBlock, 0, st,
               (const void*)qf, Nf, (const void*)qc, Ncoarse, S, Nc, (const double*)work, field, partial);
  launch("level_finish", 0.0, k_level_finish, dim3(1), 32, 0, st, (const double*)partial, nblk, (const double*)work,
         scalars);
}

__global__ void k_stats_reset(double* __restrict__ field, double* __restrict__ sc, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) field[i] = 0.0;
  if (i < MLSGD_NSCALARS) sc[i] = (i == MLSGD_S_SHIFT || i == MLSGD_S_PHI_MAX) ? -INFINITY : 0.0;
}

void launch_stats_reset(double* field, double* scalars, long long ncells, cudaStream_t st) {
  const long long n = ncells > MLSGD_NSCALARS ? ncells : MLSGD_NSCALARS;
  launch("stats_reset", (double)ncells * 8, k_stats_reset, dim3((unsigned)((n + kBlock - 1) / kBlock)), kBlock, 0, st,
         field, scalars, ncells);
}

// Chan merge of two statistics records: src into dst, both rescaled to the larger shift.
__global__ void k_merge_field(double* __restrict__ df, const double* __restrict__ dsc, const double* __restrict__ sf,
                              const double* __restrict__ ssc, long long n, double theta, double hc3,
                              double* __restrict__ partial) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double na = dsc[MLSGD_S_COUNT], nb = ssc[MLSGD_S_COUNT];
  const double shift = fmax(dsc[MLSGD_S_SHIFT], ssc[MLSGD_S_SHIFT]);
  const double fa = na > 0.0 ? exp(theta * (dsc[MLSGD_S_SHIFT] - shift)) : 0.0;
  const double fb = nb > 0.0 ? exp(theta * (ssc[MLSGD_S_SHIFT] - shift)) : 0.0;
  const double nt = na + nb;
  double contrib = 0.0;
  if (i < n && nt > 0.0) {
    const double a = df[i] * fa, b = sf[i] * fb;
    const double d = a - b;
    df[i] = b + (na / nt) * d;
    contrib = hc3 * d * d * na * nb / nt;
  }
  const double bs = block_sum(contrib);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs;
}

__global__ void k_merge_scalars(const double* __restrict__ partial, int nblk, double* __restrict__ dsc,
                                const double* __restrict__ ssc, double theta) {
  const int lane = threadIdx.x;
  double v = 0.0;
  for (int t = lane; t < nblk; t += 32) v += partial[t];
  v = warp_sum(v);
  if (lane != 0) return;
  const double na = dsc[MLSGD_S_COUNT], nb = ssc[MLSGD_S_COUNT];
  const double nt = na + nb;
  if (nt <= 0.0) return;
  const double shift = fmax(dsc[MLSGD_S_SHIFT], ssc[MLSGD_S_SHIFT]);
  const double fa = na > 0.0 ? exp(theta * (dsc[MLSGD_S_SHIFT] - shift)) : 0.0;
  const double fb = nb > 0.0 ? exp(theta * (ssc[MLSGD_S_SHIFT] - shift)) : 0.0;
  const double ya = dsc[MLSGD_S_MEAN_DY] * fa, yb = ssc[MLSGD_S_MEAN_DY] * fb;
  const double d = ya - yb;
  dsc[MLSGD_S_MEAN_DY] = yb + (na / nt) * d;
  dsc[MLSGD_S_S2_DY] = dsc[MLSGD_S_S2_DY] * fa * fa + ssc[MLSGD_S_S2_DY] * fb * fb + d * d * na * nb / nt;
  dsc[MLSGD_S_S2_DX] = dsc[MLSGD_S_S2_DX] * fa * fa + ssc[MLSGD_S_S2_DX] * fb * fb + v;
  dsc[MLSGD_S_COUNT] = nt;
  dsc[MLSGD_S_SHIFT] = shift;
  dsc[MLSGD_S_PHI_MAX] = fmax(dsc[MLSGD_S_PHI_MAX], ssc[MLSGD_S_PHI_MAX]);
  dsc[MLSGD_S_ITERS] += ssc[MLSGD_S_ITERS];
  dsc[MLSGD_S_NOCONV] += ssc[MLSGD_S_NOCONV];
}

void launch_stats_merge(double* dfield, double* dsc, const double* sfield, const double* ssc, long long ncells,
                        double hc3, double theta, double* partial, cudaStream_t st) {
  const int nblk = (int)((ncells + kBlock - 1) / kBlock);
  launch("merge", (double)ncells * 24, k_merge_field, dim3(nblk), kBlock, 0, st, dfield, (const double*)dsc, sfield,
         ssc, ncells, theta, hc3, partial);
  launch("merge_scalars", 0.0, k_merge_scalars, dim3(1), 32, 0, st, (const double*)partial, nblk, dsc, ssc, theta);
}

// ---------------------------------------------------------------- combine and step
// EX = sum_l f_l mean_l (f_l = exp(theta (c_l - c*))), grad = EX / denom + alpha z,
// z <- z - tau grad when `update`.  partial rows: 0 = ||grad||^2, 1 = ||EX||^2,
// 2 = ||grad - gprev||^2, 3 = ||gprev||^2 (0 without gprev), 4 = ||z||^2 (before the
// step), 5+l = ||mean_l||^2
// (unscaled, counted without h_c^3).
struct FieldList { const double* f[16]; };

__global__ void k_combine_step(FieldList fl, const double* __restrict__ factors, int L, long long n, double denom,
                               double alpha, double tau, int update, double* __restrict__ z,
                               double* __restrict__ grad, const double* __restrict__ gprev,
                               double* __restrict__ partial, int nblk) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double ex = 0.0, g = 0.0, d = 0.0, gp = 0.0, zz = 0.0;
  double ml[16];
  for (int l = 0; l < L; ++l) ml[l] = 0.0;
  if (i < n) {
    for (int l = 0; l < L; ++l) {
      const double m = fl.f[l][i];
      ml[l] = m * m;
      ex += factors[l] * m;
    }
    const double zi = z[i];
    zz = zi * zi;
    g = ex / denom + alpha * zi;
    if (gprev) {
      gp = gprev[i];
      d = g - gp;
    }
    if (grad) grad[i] = g;
    if (update) z[i] = zi - tau * g;
  }
  const double rowv[5] = {g * g, ex * ex, d * d, gp * gp, zz};
  for (int r = 0; r < 5; ++r) {
    if (r) __syncthreads();
    const double v = block_sum(rowv[r]);
    if (threadIdx.x == 0) partial[(long long)r * nblk + blockIdx.x] = v;
  }
  for (int l = 0; l < L; ++l) {
    __syncthreads();
    const double v = block_sum(ml[l]);
    if (threadIdx.x == 0) partial[(long long)(5 + l) * nblk + blockIdx.x] = v;
  }
}

// z <- z - tau g, and gout <- g (the gradient kept for the next step size)
__global__ void k_step_apply(long long n, double tau, const double* __restrict__ g, double* __restrict__ z,
                             double* __restrict__ gout) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gi = g[i];
  z[i] -= tau * gi;
  gout[i] = gi;
}

__global__ void k_rows_finish(const double* __restrict__ partial, int nblk, int rows, double* __restrict__ out) {
  const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  double v = 0.0;
  for (int t = lane; t < nblk; t += 32) v += partial[(long long)r * nblk + t];
  v = warp_sum(v);
  if (lane == 0) out[r] = v;
}

void launch_combine_step(const double* const* fields, const double* factors, int L, long long ncells, double denom,
                         double alpha, double tau, bool update, double* z, double* grad, const double* gprev,
                         double* partial, int nblk, cudaStream_t st) {
  FieldList fl;
  for (int l = 0; l < L && l < 16; ++l) fl.f[l] = fields[l];
  const double bytes = (double)ncells * 8 * (L + 1 + (update ? 1 : 0) + (grad ? 1 : 0) + (gprev ? 1 : 0));
  launch("combine", bytes, k_combine_step, dim3(nblk), kBlock, 0, st, fl, factors, L, ncells, denom, alpha, tau,
         update ? 1 : 0, z, grad, gprev, partial, nblk);
  const int rows = L + 5;
  launch("combine_finish", 0.0, k_rows_finish, dim3((rows + 7) / 8), 256, 0, st, (const double*)partial, nblk, rows,
         partial + (long long)rows * nblk);
}

void launch_step_apply(long long ncells, double tau, const double* g, double* z, double* gout, cudaStream_t st) {
  const int nblk = (int)((ncells + kBlock - 1) / kBlock);
  launch("step_apply", (double)ncells * 32, k_step_apply, dim3(nblk), kBlock, 0, st, ncells, tau, g, z, gout);
}

}  // namespace mlsgd
