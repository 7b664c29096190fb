// api.cu - the C ABI of libmlsgd (declared in include/mlsgd.h).
//
// Orchestrates one level's batch of samples: draw xi (row a1), fields on the
// level and its coarse partner (a2), B z (a3), state solve (a4), Phi and the
// adjoint right-hand side (a5), adjoint solve (a6), B*q, weights, level
// differences and the Chan merge (a7-a9); the multilevel combine, projected
// step (a10) and the adaptive plan (a11, host).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "launch.h"
#include "kl_table.h"
#include "mlsgd.h"

using namespace mlsgd;

struct mlsgd_ctx {
  mlsgd_config cfg;
  std::string err;
  KLTable kl;
  int n1x = 0;
  int* d_ix = nullptr;
  int* d_iy = nullptr;
  int* d_iz = nullptr;
  double* d_scale = nullptr;
  int* d_order = nullptr;
  int* d_offs = nullptr;
  std::vector<double*> d_phi;  // per level: [n1d][N] at cell centres
  std::vector<double*> d_gtab;   // per level: [N+1] sin(pi i / N), 0 at i = 0, N (nodal interpolant of g)
  std::vector<double*> d_mgtab;  // per level: [N+1] (h/6)(g[i-1] + 4 g[i] + g[i+1]) (1D mass times g)
  std::vector<float2*> d_gtab2, d_mgtab2;  // the same tables as FP32 (hi, lo) pairs
  char* ws = nullptr;
  size_t ws_size = 0;
  bool ws_external = false;  // ws belongs to the caller (mlsgd_set_workspace): never grown or freed
  std::vector<__nv_bfloat16*> d_phiT;  // per level: tensor-core B operand [N^3][K] (built on first use)
  int* d_err = nullptr;                // device error flag of the tensor-core kernel
  int* count_host = nullptr;
  double* host_buf = nullptr;  // pinned, for small read-backs
  ModeTable mt() const {
    ModeTable m;
    m.iy = d_iy; m.iz = d_iz; m.scale = d_scale; m.order = d_order; m.offs = d_offs;
    m.n1x = n1x; m.n1d = kl.n1d;
    return m;
  }
  int N(int l) const { return cfg.n0 << l; }
  int freq() const { return cfg.target_freq > 0 ? cfg.target_freq : 1; }
  double xi_half_width() const { return cfg.field_model == 1 ? 4.0 : 0.0; }
  int Nc() const { return cfg.n0 << cfg.ctrl_level; }
  bool mixed() const { return cfg.precision == MLSGD_MIXED; }
  bool tc_ok(int level) const {
    const long long cells = cells_of(N(level));
    return cfg.n_modes % 64 == 0 && cells % 128 == 0 && kl_gemm_b_bytes(N(level), cfg.n_modes) <= ((size_t)1 << 30);
  }
  bool use_tc(int level) const { return mixed() && cfg.field_tc && tc_ok(level); }
};

namespace {

mlsgd_status fail(mlsgd_ctx* c, mlsgd_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, MLSGD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

struct Bump {
  char* p;
  template <typename T>
  T* take(size_t n) { T* r = (T*)p; p += al(n * sizeof(T)); return r; }
};

// scratch of one grid solve (solver buffers, y, badj, b, r64)
size_t solve_scratch_bytes(const mlsgd_ctx* ctx, int N, int S) {
  const size_t nodes = (size_t)nodes_of(N);
  size_t b = solver_bytes(N, S, ctx->mixed() ? 4 : 8);
  b += 2 * al(S * nodes * 8) + al(nodes * 8);
  if (ctx->mixed()) b += al(S * nodes * 8);
  return b + 4096;
}
size_t field_bytes(const mlsgd_ctx* ctx, int N, int S) {
  const size_t cells = (size_t)cells_of(N);
  return ctx->mixed() ? al(S * cells * 4) + al(S * cells * 2) : al(S * cells * 8);
}
// persistent per-grid results kept until the statistics kernel
size_t grid_keep_bytes(const mlsgd_ctx* ctx, int N, int S) {
  return field_bytes(ctx, N, S) + al((size_t)S * nodes_of(N) * 8) + al(S * 8);
}
size_t level_bytes(const mlsgd_ctx* ctx, int level, int S) {
  const int N = ctx->N(level);
  size_t b = al((size_t)S * ctx->cfg.n_modes * 8);
  b += grid_keep_bytes(ctx, N, S);
  if (level > 0) b += grid_keep_bytes(ctx, N / 2, S);
  b += 2 * al((size_t)2 * S * 4);
  b += al(kl_gemm_a_bytes(S, ctx->cfg.n_modes));
  b += solve_scratch_bytes(ctx, N, S);
  b += al((4 + 4 * (size_t)S) * 8) + al((size_t)level_partial_cap(ctx->Nc(), N) * 8);
  b += al(2 * (size_t)nodes_of(N) * 8);
  return b;
}

mlsgd_status ensure_ws(mlsgd_ctx* ctx, size_t bytes, cudaStream_t st) {
  if (bytes <= ctx->ws_size) return MLSGD_OK;
  if (ctx->ws_external)
    return fail(ctx, MLSGD_ENOMEM, "the caller's workspace holds " + std::to_string(ctx->ws_size) + " bytes, " +
                                       std::to_string(bytes) + " needed");
  CK(cudaStreamSynchronize(st));
  if (ctx->ws) CK(cudaFree(ctx->ws));
  ctx->ws = nullptr;
  ctx->ws_size = 0;
  if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return fail(ctx, MLSGD_ENOMEM, "cannot allocate " + std::to_string(bytes) + " bytes of scratch");
  }
  ctx->ws_size = bytes;
  return MLSGD_OK;
}

struct GridFields {
  double* a64 = nullptr;
  float* a32 = nullptr;
  __nv_bfloat16* abf = nullptr;
};

GridFields carve_fields(const mlsgd_ctx* ctx, int N, int S, Bump& bp) {
  GridFields f;
  const size_t cells = (size_t)cells_of(N);
  if (ctx->mixed()) { f.a32 = bp.take<float>(S * cells); f.abf = bp.take<__nv_bfloat16>(S * cells); }
  else f.a64 = bp.take<double>(S * cells);
  return f;
}

// Per-sample status flags: 1 = a solve hit its iteration cap, 2 = a solve went
// non-finite (NaN/Inf right-hand side or iterate); the state and adjoint flags of a
// sample are OR-ed.
__global__ void k_record(const SolveScalars* __restrict__ sc, int S, int mixed, int* __restrict__ iters,
                         int* __restrict__ status, int accumulate) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int it = mixed ? sc[s].pad : sc[s].iters;
  const int stv = sc[s].status;
  iters[s] = accumulate ? iters[s] + it : it;
  status[s] = accumulate ? (status[s] | stv) : stv;
}

// OR of the S per-sample status flags into *out (one block of kAnyBlock threads)
constexpr int kAnyBlock = 256;
__global__ void k_status_any(const int* __restrict__ status, int S, int* __restrict__ out) {
  int v = 0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) v |= status[s];
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  __shared__ int w[kAnyBlock / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kAnyBlock / 32; ++i) v |= w[i];
    *out = v;
  }
}

// status of a solve call from the OR of its per-sample flags
mlsgd_status solve_verdict(mlsgd_ctx* ctx, int flags, const char* who) {
  if (flags & 2) return fail(ctx, MLSGD_ENONFINITE, std::string(who) + ": a solve went non-finite (NaN/Inf input?)");
  if (flags & 1) return fail(ctx, MLSGD_ENOCONV, std::string(who) + ": a solve hit max_iter");
  return MLSGD_OK;
}

// state + Phi + adjoint for S samples on grid N; scratch carved from bp (not kept).
// want_pairs (internal callers): on tiled grids of the mixed path, y stays and q is
// returned as FP32 (hi, lo) pairs in the FP64 buffers' storage (*pairs_out = true),
// and Phi / the adjoint right-hand side are formed in pair arithmetic.
mlsgd_status solve_grid(mlsgd_ctx* ctx, int N, int S, const GridFields& f, const double* z, double* y, double* q,
                        double* phi, int* iters, int* status, char* scratch, cudaStream_t st,
                        bool want_pairs = false, bool* pairs_out = nullptr) {
  const size_t nodes = (size_t)nodes_of(N);
  char* p = scratch;
  SolverBufs B;
  carve_solver(B, N, S, ctx->mixed() ? 4 : 8, p);
  B.count_host = ctx->count_host;
  B.err = ctx->d_err;
  B.stencil = ctx->cfg.stencil;
  B.zchunks = ctx->cfg.z_chunks;
  Bump bp{p};
  double* badj = bp.take<double>(S * nodes);
  double* b = bp.take<double>(nodes);
  double* r64 = ctx->mixed() ? bp.take<double>(S * nodes) : nullptr;
  double* ytmp = y ? y : bp.take<double>(S * nodes);
  PcgParams prm{ctx->cfg.rtol, ctx->cfg.max_iter, ctx->cfg.omega > 0 ? ctx->cfg.omega : 0.6, 4};
  const int inner = ctx->cfg.inner_iters > 0 ? ctx->cfg.inner_iters : 6;
  const int inner2 = ctx->cfg.inner_iters_next > 0 ? ctx->cfg.inner_iters_next : inner;
  if (ctx->mixed()) build_hierarchy_mixed(B, f.abf, prm.omega, st);
  else build_hierarchy_fp64(B, f.a64, prm.omega, st);
  launch_rhs_state(z, ctx->Nc(), N, b, st);
  const int fixed = ctx->cfg.ir_steps > 0 ? ctx->cfg.ir_steps : 0;
  const bool pairs = want_pairs && ctx->mixed() && N >= kTiledMinN && B.J >= 1;
  if (pairs_out) *pairs_out = pairs;
  cudaError_t e = ctx->mixed() ? ir_mixed(B, f.a32, f.abf, b, 0, ytmp, r64, prm, inner, st, fixed, nullptr, pairs, inner2)
                               : pcg_fp64(B, f.a64, b, 0, ytmp, prm, st);
  CK(e);
  launch("record", 0.0, k_record, dim3((S + 127) / 128), 128, 0, st, (const SolveScalars*)B.sc, S, (int)ctx->mixed(),
         iters, status, 0);
  int lev = 0;
  while ((ctx->cfg.n0 << lev) < N) ++lev;
  if (!pairs) CK(cudaMemsetAsync(badj, 0, S * nodes * sizeof(double), st));  // boundary rows stay 0
  if (pairs) {
    launch_phi_adjrhs_df((const float2*)ytmp, N, S, (float2*)badj, phi, B.partial, ctx->d_gtab2[lev],
                         ctx->d_mgtab2[lev], st);
    e = ir_mixed(B, f.a32, f.abf, nullptr, (long long)nodes, q, r64, prm, inner, st, fixed, (const float2*)badj, true,
                 inner2);
  } else {
    launch_phi_adjrhs(ytmp, N, S, badj, phi, B.partial, ctx->d_gtab[lev], ctx->d_mgtab[lev], st, ctx->freq());
    e = ctx->mixed() ? ir_mixed(B, f.a32, f.abf, badj, (long long)nodes, q, r64, prm, inner, st, fixed, nullptr, false, inner2)
                     : pcg_fp64(B, f.a64, badj, (long long)nodes, q, prm, st);
  }
  CK(e);
  launch("record", 0.0, k_record, dim3((S + 127) / 128), 128, 0, st, (const SolveScalars*)B.sc, S, (int)ctx->mixed(),
         iters, status, 1);
  CK(cudaGetLastError());
  return MLSGD_OK;
}

mlsgd_status ensure_phiT(mlsgd_ctx* ctx, int grid, cudaStream_t st) {
  if (ctx->d_phiT[grid]) return MLSGD_OK;
  __nv_bfloat16* b = nullptr;
  if (cudaMalloc(&b, kl_gemm_b_bytes(ctx->N(grid), ctx->cfg.n_modes)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, MLSGD_ENOMEM, "cannot allocate the tensor-core mode table");
  }
  kl_gemm_build_b(ctx->d_phi[grid], ctx->d_ix, ctx->d_iy, ctx->d_iz, ctx->N(grid), ctx->cfg.n_modes, b, st);
  ctx->d_phiT[grid] = b;
  return MLSGD_OK;
}

// fields of one grid; with the tensor-core option the BF16 coefficient comes from the GEMM
mlsgd_status make_field(mlsgd_ctx* ctx, const double* xi, int grid, int S, const GridFields& f, double* log_a,
                        cudaStream_t st, __nv_bfloat16* gemm_a = nullptr) {
  const bool tc = gemm_a != nullptr && f.abf != nullptr && ctx->use_tc(grid);
  FieldOut o{log_a, f.a64, f.a32, tc ? nullptr : f.abf};
  CK(launch_field(xi, ctx->cfg.n_modes, ctx->mt(), ctx->d_phi[grid], ctx->N(grid), S, o, st));
  if (tc) {
    mlsgd_status s = ensure_phiT(ctx, grid, st);
    if (s != MLSGD_OK) return s;
    CK(kl_gemm(xi, ctx->d_scale, S, ctx->cfg.n_modes, ctx->d_phiT[grid], ctx->N(grid), gemm_a, f.abf, nullptr,
               ctx->d_err, st));
  }
  return MLSGD_OK;
}

// ---------------------------------------------------------------- adaptive plan (host)
// Sec. 4.1 with the readings stated in the header of mlsgd.h's mlsgd_step:
// Giles-form batch sizes, Giles bias extrapolation, least-squares rates.
double cost_model(int n0, int l) {
  const double N = (double)(n0 << l);
  return (N - 1) * (N - 1) * (N - 1) * (1.0 + (l >= 1 ? 0.125 : 0.0));
}
double ls_slope(const std::vector<double>& x, const std::vector<double>& y) {
  double xm = 0, ym = 0;
  for (size_t i = 0; i < x.size(); ++i) { xm += x[i]; ym += y[i]; }
  xm /= x.size(); ym /= y.size();
  double num = 0, den = 0;
  for (size_t i = 0; i < x.size(); ++i) { num += (x[i] - xm) * (y[i] - ym); den += (x[i] - xm) * (x[i] - xm); }
  return num / den;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

const char* mlsgd_status_string(mlsgd_status s) {
  switch (s) {
    case MLSGD_OK: return "ok";
    case MLSGD_EINVAL: return "invalid argument";
    case MLSGD_ENOMEM: return "out of device memory";
    case MLSGD_ENOCONV: return "solver did not converge within max_iter";
    case MLSGD_ENONFINITE: return "non-finite value";
    case MLSGD_ECUDA: return "CUDA error";
    case MLSGD_ENOTIMPL: return "not implemented";
  }
  return "unknown status";
}

const char* mlsgd_last_error(const mlsgd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mlsgd_status mlsgd_create(const mlsgd_config* cfg, mlsgd_ctx** out) {
  if (!cfg || !out) return MLSGD_EINVAL;
  *out = nullptr;
  const mlsgd_config& c = *cfg;
  if (c.n_levels < 1 || c.n_levels > 16 || c.n0 < 2 || (c.n0 & (c.n0 - 1)) != 0 || c.ctrl_level < 0 ||
      c.ctrl_level >= c.n_levels || c.n_modes < 2 || (c.field_model == 0 && (c.n_modes % 2) != 0) || c.n_modes > 4096 ||
      !(c.corr_len > 0) || !(c.rtol > 0) || c.max_iter < 1 || (c.precision != MLSGD_FP64 && c.precision != MLSGD_MIXED) ||
      (c.n0 << (c.n_levels - 1)) > 1024 || c.field_model < 0 || c.field_model > 1 || c.target_freq < 0 ||
      c.stencil < 0 || c.stencil > 1 || c.z_chunks < 0 || !(c.omega >= 0.0 && c.omega < 1.0) ||
      c.inner_iters_next < 0)
    return MLSGD_EINVAL;
  int mcube = 0;
  if (c.field_model == 1) {
    while ((mcube + 1) * (mcube + 1) * (mcube + 1) <= c.n_modes) ++mcube;
    if (mcube * mcube * mcube != c.n_modes) return MLSGD_EINVAL;
  }
  mlsgd_ctx* ctx = new mlsgd_ctx();
  ctx->cfg = c;
  if (ctx->cfg.max_batch <= 0) ctx->cfg.max_batch = 256;
  ctx->kl = c.field_model == 1 ? build_paper_table(c.corr_len, mcube) : build_kl_table(c.corr_len, c.n_modes);
  const int K = c.n_modes;
  std::vector<int> iy(K), iz(K), order(K);
  std::vector<double> scale(K);
  int n1x = 0;
  for (int k = 0; k < K; ++k) {
    iy[k] = ctx->kl.iy[k];
    iz[k] = ctx->kl.iz[k];
    scale[k] = c.sigma * std::sqrt(ctx->kl.lam3[k]);
    n1x = std::max(n1x, ctx->kl.ix[k] + 1);
  }
  std::vector<int> offs(n1x + 1, 0);
  for (int k = 0; k < K; ++k) offs[ctx->kl.ix[k] + 1]++;
  for (int i = 0; i < n1x; ++i) offs[i + 1] += offs[i];
  std::vector<int> fill(offs.begin(), offs.end() - 1);
  for (int k = 0; k < K; ++k) order[fill[ctx->kl.ix[k]]++] = k;
  ctx->n1x = n1x;
  auto up = [&](void** d, const void* h, size_t n) -> bool {
    return cudaMalloc(d, n) == cudaSuccess && cudaMemcpy(*d, h, n, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  std::vector<int> ixv(ctx->kl.ix.begin(), ctx->kl.ix.end());
  const int zero = 0;
  bool ok = up((void**)&ctx->d_ix, ixv.data(), K * sizeof(int)) && up((void**)&ctx->d_err, &zero, sizeof(int)) &&
            up((void**)&ctx->d_iy, iy.data(), K * sizeof(int)) && up((void**)&ctx->d_iz, iz.data(), K * sizeof(int)) &&
            up((void**)&ctx->d_scale, scale.data(), K * sizeof(double)) &&
            up((void**)&ctx->d_order, order.data(), K * sizeof(int)) &&
            up((void**)&ctx->d_offs, offs.data(), (n1x + 1) * sizeof(int));
  ctx->d_phiT.assign(c.n_levels, nullptr);
  for (int l = 0; ok && l < c.n_levels; ++l) {
    std::vector<double> phi = kl_cell_table(ctx->kl, ctx->N(l));
    double* d = nullptr;
    ok = up((void**)&d, phi.data(), phi.size() * sizeof(double));
    ctx->d_phi.push_back(d);
    const int N = ctx->N(l);
    std::vector<double> g(N + 1, 0.0), mg(N + 1, 0.0);
    for (int i = 1; i < N; ++i) g[i] = std::sin(M_PI * (double)(ctx->freq() * i) / N);
    for (int i = 1; i < N; ++i) mg[i] = (g[i - 1] + 4.0 * g[i] + g[i + 1]) / (6.0 * N);
    double *dg = nullptr, *dmg = nullptr;
    ok = ok && up((void**)&dg, g.data(), g.size() * sizeof(double)) && up((void**)&dmg, mg.data(), mg.size() * sizeof(double));
    ctx->d_gtab.push_back(dg);
    ctx->d_mgtab.push_back(dmg);
    std::vector<float2> g2(N + 1), mg2(N + 1);
    auto split = [](double v) { const float h = (float)v; return make_float2(h, (float)(v - (double)h)); };
    for (int i = 0; i <= N; ++i) { g2[i] = split(g[i]); mg2[i] = split(mg[i]); }
    float2 *dg2 = nullptr, *dmg2 = nullptr;
    ok = ok && up((void**)&dg2, g2.data(), g2.size() * sizeof(float2)) &&
         up((void**)&dmg2, mg2.data(), mg2.size() * sizeof(float2));
    ctx->d_gtab2.push_back(dg2);
    ctx->d_mgtab2.push_back(dmg2);
  }
  ok = ok && cudaHostAlloc((void**)&ctx->count_host, sizeof(int), cudaHostAllocDefault) == cudaSuccess;
  ok = ok && cudaHostAlloc((void**)&ctx->host_buf, 4096 * sizeof(double), cudaHostAllocDefault) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mlsgd_destroy(ctx);
    return MLSGD_ECUDA;
  }
  *out = ctx;
  return MLSGD_OK;
}

void mlsgd_destroy(mlsgd_ctx* ctx) {
  if (!ctx) return;
  cudaFree(ctx->d_ix); cudaFree(ctx->d_err);
  for (__nv_bfloat16* b : ctx->d_phiT) cudaFree(b);
  cudaFree(ctx->d_iy); cudaFree(ctx->d_iz); cudaFree(ctx->d_scale); cudaFree(ctx->d_order); cudaFree(ctx->d_offs);
  for (double* d : ctx->d_phi) cudaFree(d);
  for (double* d : ctx->d_gtab) cudaFree(d);
  for (double* d : ctx->d_mgtab) cudaFree(d);
  for (float2* d : ctx->d_gtab2) cudaFree(d);
  for (float2* d : ctx->d_mgtab2) cudaFree(d);
  if (ctx->ws && !ctx->ws_external) cudaFree(ctx->ws);
  if (ctx->count_host) cudaFreeHost(ctx->count_host);
  if (ctx->host_buf) cudaFreeHost(ctx->host_buf);
  delete ctx;
}

int64_t mlsgd_n_ctrl_cells(const mlsgd_ctx* ctx) { return ctx ? cells_of(ctx->Nc()) : 0; }

mlsgd_status mlsgd_set_workspace(mlsgd_ctx* ctx, void* ws_dev, size_t bytes) {
  if (!ctx || (ws_dev == nullptr) != (bytes == 0) || ((uintptr_t)ws_dev & 255) != 0)
    return fail(ctx, MLSGD_EINVAL, "mlsgd_set_workspace: a 256-byte aligned device range, or NULL and 0");
  if (ctx->ws && !ctx->ws_external) {
    cudaDeviceSynchronize();  // the context's own scratch may still be in use
    cudaFree(ctx->ws);
  }
  ctx->ws = (char*)ws_dev;
  ctx->ws_size = bytes;
  ctx->ws_external = ws_dev != nullptr;
  return MLSGD_OK;
}

size_t mlsgd_workspace_bytes(const mlsgd_ctx* ctx, int level, int n_samples) {
  if (!ctx || level < 0 || level >= ctx->cfg.n_levels || n_samples < 0) return 0;
  const int S = std::min(n_samples, ctx->cfg.max_batch);
  return level_bytes(ctx, level, S);
}

int mlsgd_mode_table(const mlsgd_ctx* ctx, int* idx, double* lam) {
  if (!ctx) return 0;
  for (int k = 0; k < ctx->cfg.n_modes; ++k) {
    if (idx) { idx[3 * k] = ctx->kl.ix[k]; idx[3 * k + 1] = ctx->kl.iy[k]; idx[3 * k + 2] = ctx->kl.iz[k]; }
    if (lam) lam[k] = ctx->kl.lam3[k];
  }
  return ctx->kl.n1d;
}

mlsgd_status mlsgd_sample_field(mlsgd_ctx* ctx, int iter, int level, int grid, int64_t first_sample, int n_samples,
                                double* xi_dev, double* log_a_dev, void* stream) {
  if (!ctx) return MLSGD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (level < 0 || level >= ctx->cfg.n_levels || (grid != level && grid != level - 1) || grid < 0 || n_samples < 0 ||
      first_sample < 0 || iter < 0 || (!log_a_dev && !xi_dev) || (n_samples > 0 && !log_a_dev && !xi_dev))
    return fail(ctx, MLSGD_EINVAL, "mlsgd_sample_field: bad level/grid/sizes");
  if (n_samples == 0) return MLSGD_OK;
  const int K = ctx->cfg.n_modes;
  double* xi = xi_dev;
  if (!xi) {
    mlsgd_status s = ensure_ws(ctx, al((size_t)n_samples * K * 8), st);
    if (s != MLSGD_OK) return s;
    xi = (double*)ctx->ws;
  }
  launch_draw_xi(ctx->cfg.seed, iter, level, first_sample, n_samples, K, xi, st, ctx->xi_half_width());
  if (log_a_dev) {
    GridFields none;
    mlsgd_status s = make_field(ctx, xi, grid, n_samples, none, log_a_dev, st);
    if (s != MLSGD_OK) return s;
  }
  CK(cudaGetLastError());
  return MLSGD_OK;
}

mlsgd_status mlsgd_sample_field_tc(mlsgd_ctx* ctx, int iter, int level, int grid, int64_t first_sample,
                                   int n_samples, float* log_a_f32_dev, void* a_bf16_dev, void* stream) {
  if (!ctx) return MLSGD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (level < 0 || level >= ctx->cfg.n_levels || (grid != level && grid != level - 1) || grid < 0 || n_samples < 0 ||
      first_sample < 0 || iter < 0)
    return fail(ctx, MLSGD_EINVAL, "mlsgd_sample_field_tc: bad level/grid/sizes");
  if (!ctx->tc_ok(grid)) return fail(ctx, MLSGD_ENOTIMPL, "mlsgd_sample_field_tc: needs n_modes % 64 == 0 and N^3 % 128 == 0");
  if (n_samples == 0) return MLSGD_OK;
  const int K = ctx->cfg.n_modes, S = n_samples;
  mlsgd_status s = ensure_ws(ctx, al((size_t)S * K * 8) + al(kl_gemm_a_bytes(S, K)), st);
  if (s != MLSGD_OK) return s;
  Bump bp{ctx->ws};
  double* xi = bp.take<double>((size_t)S * K);
  __nv_bfloat16* A = bp.take<__nv_bfloat16>((size_t)S * K);
  launch_draw_xi(ctx->cfg.seed, iter, level, first_sample, S, K, xi, st, ctx->xi_half_width());
  s = ensure_phiT(ctx, grid, st);
  if (s != MLSGD_OK) return s;
  CK(kl_gemm(xi, ctx->d_scale, S, K, ctx->d_phiT[grid], ctx->N(grid), A, (__nv_bfloat16*)a_bf16_dev, log_a_f32_dev,
             ctx->d_err, st));
  CK(cudaMemcpyAsync(ctx->count_host, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*ctx->count_host != 0) return fail(ctx, MLSGD_ECUDA, "tensor-core KL synthesis timed out on a barrier");
  return MLSGD_OK;
}

mlsgd_status mlsgd_solve_state_adjoint(mlsgd_ctx* ctx, int grid, int n_samples, const double* log_a_dev,
                                       const double* z_dev, double* y_dev, double* q_dev, double* phi_dev,
                                       int* iters_dev, int* status_dev, void* stream) {
  if (!ctx) return MLSGD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (grid < 0 || grid >= ctx->cfg.n_levels || n_samples < 0)
    return fail(ctx, MLSGD_EINVAL, "mlsgd_solve_state_adjoint: bad grid or sample count");
  if (n_samples == 0) return MLSGD_OK;
  if (!log_a_dev || !z_dev || !y_dev || !q_dev || !phi_dev || !iters_dev || !status_dev)
    return fail(ctx, MLSGD_EINVAL, "mlsgd_solve_state_adjoint: null pointer");
  const int N = ctx->N(grid);
  const int S = n_samples;
  const size_t need = field_bytes(ctx, N, S) + solve_scratch_bytes(ctx, N, S);
  mlsgd_status s = ensure_ws(ctx, need, st);
  if (s != MLSGD_OK) return s;
  Bump bp{ctx->ws};
  GridFields f = carve_fields(ctx, N, S, bp);
  FieldOut o{nullptr, f.a64, f.a32, f.abf};
  launch_exp_field(log_a_dev, o, (long long)S * cells_of(N), st);
  s = solve_grid(ctx, N, S, f, z_dev, y_dev, q_dev, phi_dev, iters_dev, status_dev, bp.p, st);
  if (s != MLSGD_OK) return s;
  // report non-convergence / non-finite solves (synchronous check of the status flags)
  std::vector<int> h(S);
  CK(cudaMemcpyAsync(h.data(), status_dev, S * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->count_host, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*ctx->count_host != 0) return fail(ctx, MLSGD_ECUDA, "mlsgd_solve_state_adjoint: a kernel timed out on a barrier");
  int flags = 0;
  for (int v : h) flags |= v;
  return solve_verdict(ctx, flags, "mlsgd_solve_state_adjoint");
}

// ---------------------------------------------------------------- allocation-free solve
// Some callers cannot allocate device memory at the time they need a solve: a
// latency-critical loop where cudaMalloc's implicit device-wide synchronisation is
// not acceptable, or a host application whose own allocator has reserved the
// device memory and forbids libraries to call the CUDA allocator.  For them the
// solve below takes its scratch from a fixed array compiled into the library
// instead of the context's growable workspace.  The array is
// MLSGD_NOALLOC_SCRATCH_BYTES large and every GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) char g_noalloc_scratch[MLSGD_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
char* g_noalloc_addr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of the static array on the current device, looked up once per
// device with that device current (host code only sees a host-side stand-in under
// the array's name, never a device address).
mlsgd_status noalloc_scratch(mlsgd_ctx* ctx, char** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ctx, MLSGD_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(ctx, MLSGD_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = (char*)p;
  }
  *out = g_noalloc_addr[dev];
  return MLSGD_OK;
}
}  // namespace

mlsgd_status mlsgd_solve_state_adjoint_noalloc(mlsgd_ctx* ctx, int grid, int n_samples, const double* log_a_dev,
                                               const double* z_dev, double* y_dev, double* q_dev, double* phi_dev,
                                               int* iters_dev, int* status_dev, void* stream) {
  if (!ctx) return MLSGD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (grid < 0 || grid >= ctx->cfg.n_levels || n_samples < 0)
    return fail(ctx, MLSGD_EINVAL, "mlsgd_solve_state_adjoint_noalloc: bad grid or sample count");
  if (n_samples == 0) return MLSGD_OK;
  if (!log_a_dev || !z_dev || !y_dev || !q_dev || !phi_dev || !iters_dev || !status_dev)
    return fail(ctx, MLSGD_EINVAL, "mlsgd_solve_state_adjoint_noalloc: null pointer");
  const int N = ctx->N(grid);
  const int S = n_samples;
  const size_t need = al(sizeof(int)) + field_bytes(ctx, N, S) + solve_scratch_bytes(ctx, N, S);
  if (need > (size_t)MLSGD_NOALLOC_SCRATCH_BYTES)
    return fail(ctx, MLSGD_EINVAL,
                "mlsgd_solve_state_adjoint_noalloc: " + std::to_string(S) + " samples on a " + std::to_string(N) +
                    "^3 grid need " + std::to_string(need) + " bytes of scratch; the static array holds " +
                    std::to_string((size_t)MLSGD_NOALLOC_SCRATCH_BYTES) + " (use fewer samples per call)");
  char* scratch = nullptr;
  mlsgd_status s = noalloc_scratch(ctx, &scratch);
  if (s != MLSGD_OK) return s;
  // Nothing in the scratch has to start at zero: every kernel of the solve writes
  // a buffer (all nodes, boundary included) before any kernel reads it.
  Bump bp{scratch};
  int* flags_dev = bp.take<int>(1);
  GridFields f = carve_fields(ctx, N, S, bp);
  FieldOut o{nullptr, f.a64, f.a32, f.abf};
  launch_exp_field(log_a_dev, o, (long long)S * cells_of(N), st);
  s = solve_grid(ctx, N, S, f, z_dev, y_dev, q_dev, phi_dev, iters_dev, status_dev, bp.p, st);
  if (s != MLSGD_OK) return s;
  // the OR of the per-sample flags is formed on the device and one int read back
  // through the context's pinned word (no allocation, any batch size)
  launch("status_any", (double)S * sizeof(int), k_status_any, dim3(1), kAnyBlock, 0, st, (const int*)status_dev, S,
         flags_dev);
  CK(cudaMemcpyAsync(ctx->count_host, flags_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->host_buf, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*(const int*)ctx->host_buf != 0)
    return fail(ctx, MLSGD_ECUDA, "mlsgd_solve_state_adjoint_noalloc: a kernel timed out on a barrier");
  return solve_verdict(ctx, *ctx->count_host, "mlsgd_solve_state_adjoint_noalloc");
}

mlsgd_status mlsgd_stats_reset(mlsgd_ctx* ctx, mlsgd_level_stats* stats, void* stream) {
  if (!ctx || !stats || !stats->field_dev || !stats->scalars_dev) return MLSGD_EINVAL;
  launch_stats_reset(stats->field_dev, stats->scalars_dev, cells_of(ctx->Nc()), (cudaStream_t)stream);
  CK(cudaGetLastError());
  return MLSGD_OK;
}

mlsgd_status mlsgd_stats_merge(mlsgd_ctx* ctx, mlsgd_level_stats* dst, const mlsgd_level_stats* src, void* stream) {
  if (!ctx || !dst || !src || dst->level != src->level) return MLSGD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const long long nc = cells_of(ctx->Nc());
  mlsgd_status s = ensure_ws(ctx, al(((nc + 255) / 256 + 64) * 8), st);
  if (s != MLSGD_OK) return s;
  const double hc = 1.0 / ctx->Nc();
  launch_stats_merge(dst->field_dev, dst->scalars_dev, src->field_dev, src->scalars_dev, nc, hc * hc * hc,
                     ctx->cfg.theta, (double*)ctx->ws, st);
  CK(cudaGetLastError());
  return MLSGD_OK;
}

mlsgd_status mlsgd_level_gradient(mlsgd_ctx* ctx, int iter, int level, int64_t first_sample, int n_samples,
                                  const double* z_dev, mlsgd_level_stats* stats, void* stream) {
  if (!ctx) return MLSGD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (level < 0 || level >= ctx->cfg.n_levels || n_samples < 0 || first_sample < 0 ||
      iter < 0 || !z_dev || !stats || !stats->field_dev || !stats->scalars_dev || stats->level != level)
    return fail(ctx, MLSGD_EINVAL, "mlsgd_level_gradient: bad arguments");
  if (n_samples == 0) return MLSGD_OK;
  const int chunk = std::min(n_samples, ctx->cfg.max_batch);
  mlsgd_status s = ensure_ws(ctx, level_bytes(ctx, level, chunk), st);
  if (s != MLSGD_OK) return s;
  const int N = ctx->N(level), K = ctx->cfg.n_modes;
  for (int64_t done = 0; done < n_samples; done += chunk) {
    const int S = (int)std::min<int64_t>(chunk, n_samples - done);
    Bump bp{ctx->ws};
    double* xi = bp.take<double>((size_t)S * K);
    GridFields ff = carve_fields(ctx, N, S, bp);
    double* qf = bp.take<double>((size_t)S * nodes_of(N));
    double* phif = bp.take<double>(S);
    GridFields fc;
    double *qc = nullptr, *phic = nullptr;
    if (level > 0) {
      fc = carve_fields(ctx, N / 2, S, bp);
      qc = bp.take<double>((size_t)S * nodes_of(N / 2));
      phic = bp.take<double>(S);
    }
    int* iters = bp.take<int>(2 * (size_t)S);
    int* status = bp.take<int>(2 * (size_t)S);
    __nv_bfloat16* gemm_a = bp.take<__nv_bfloat16>((size_t)S * K);
    double* work = bp.take<double>(4 + 4 * (size_t)S);
    double* spartial = bp.take<double>((size_t)level_partial_cap(ctx->Nc(), N));
    double* lvl_nodes = bp.take<double>(2 * (size_t)nodes_of(N));
    char* scratch = bp.p;
    launch_draw_xi(ctx->cfg.seed, iter, level, first_sample + done, S, K, xi, st, ctx->xi_half_width());
    s = make_field(ctx, xi, level, S, ff, nullptr, st, gemm_a);
    if (s != MLSGD_OK) return s;
    bool pf = false, pc = false;
    s = solve_grid(ctx, N, S, ff, z_dev, nullptr, qf, phif, iters, status, scratch, st, true, &pf);
    if (s != MLSGD_OK) return s;
    if (level > 0) {
      s = make_field(ctx, xi, level - 1, S, fc, nullptr, st, gemm_a);
      if (s != MLSGD_OK) return s;
      s = solve_grid(ctx, N / 2, S, fc, z_dev, nullptr, qc, phic, iters + S, status + S, scratch, st, true, &pc);
      if (s != MLSGD_OK) return s;
    }
    launch_level_stats(qf, phif, N, qc, phic, N / 2, S, ctx->Nc(), ctx->cfg.theta, stats->field_dev,
                       stats->scalars_dev, work, spartial, iters, status, st, pf, pc, lvl_nodes);
    CK(cudaGetLastError());
  }
  return MLSGD_OK;
}

namespace {
// slope of a least-squares line through (l, y_l), l = 1..L-1; NaN with fewer than two points
double diff_level_slope(const std::vector<double>& y) {
  if (y.size() < 3) return NAN;
  std::vector<double> x, v;
  for (size_t l = 1; l < y.size(); ++l) { x.push_back((double)l); v.push_back(y[l]); }
  return ls_slope(x, v);
}
}  // namespace

// Shared body of mlsgd_step and mlsgd_step_adaptive.  Fixed: one pass computes the
// gradient and takes the step with `tau`.  Adaptive: the first pass computes the
// gradient into scratch together with ||grad - grad_prev|| (read only when
// tau_prev > 0), the host evaluates eq:adaptive-step-size, and a second pass takes
// the step and stores the gradient into grad_prev.
static mlsgd_status step_core(mlsgd_ctx* ctx, const mlsgd_level_stats* stats, int n_levels, double eta,
                              int max_levels, double* z_dev, double* grad_dev, bool adaptive, double tau,
                              double tau_prev, double* grad_prev_dev, mlsgd_step_report* rep, cudaStream_t st) {
  if (!stats || n_levels < 1 || n_levels > 16 || !z_dev || !rep || n_levels > ctx->cfg.n_levels)
    return fail(ctx, MLSGD_EINVAL, "mlsgd_step: bad arguments");
  if (adaptive && (!grad_prev_dev || !(tau > 0) || !std::isfinite(tau_prev)))
    return fail(ctx, MLSGD_EINVAL, "mlsgd_step_adaptive: needs grad_prev_dev, tau0 > 0 and a finite tau_prev");
  for (int l = 0; l < n_levels; ++l)
    if (stats[l].level != l || !stats[l].field_dev || !stats[l].scalars_dev)
      return fail(ctx, MLSGD_EINVAL, "mlsgd_step: stats[l] must hold level l");
  const double theta = ctx->cfg.theta;
  double* hb = ctx->host_buf;
  for (int l = 0; l < n_levels; ++l)
    CK(cudaMemcpyAsync(hb + l * MLSGD_NSCALARS, stats[l].scalars_dev, MLSGD_NSCALARS * sizeof(double),
                       cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ctx->count_host, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (*ctx->count_host != 0) return fail(ctx, MLSGD_ECUDA, "a kernel timed out on a barrier");
  std::vector<double> sc(hb, hb + n_levels * MLSGD_NSCALARS);
  double cstar = -INFINITY;
  for (int l = 0; l < n_levels; ++l) {
    if (!(sc[l * MLSGD_NSCALARS + MLSGD_S_COUNT] >= 2))
      return fail(ctx, MLSGD_EINVAL, "mlsgd_step: every level needs at least 2 samples");
    cstar = std::max(cstar, sc[l * MLSGD_NSCALARS + MLSGD_S_SHIFT]);
  }
  std::vector<double> fac(n_levels);
  double ey = 0.0;
  for (int l = 0; l < n_levels; ++l) {
    fac[l] = std::exp(theta * (sc[l * MLSGD_NSCALARS + MLSGD_S_SHIFT] - cstar));
    ey += fac[l] * sc[l * MLSGD_NSCALARS + MLSGD_S_MEAN_DY];
  }
  const double floor_y = std::exp(-theta * cstar);
  const double denom = std::max(floor_y, ey);
  if (!std::isfinite(denom) || !std::isfinite(cstar)) return fail(ctx, MLSGD_ENONFINITE, "mlsgd_step: non-finite shift");
  const long long nc = cells_of(ctx->Nc());
  const int nblk = (int)((nc + 255) / 256);
  const int rows = n_levels + 5;
  const size_t part_bytes = al((size_t)(rows + 1) * nblk * 8 + 64 * 8);
  mlsgd_status s = ensure_ws(ctx, part_bytes + al(16 * 8) + (adaptive ? al((size_t)nc * 8) : 0), st);
  if (s != MLSGD_OK) return s;
  double* partial = (double*)ctx->ws;
  double* dfac = (double*)(ctx->ws + part_bytes);
  double* gnew = adaptive ? (double*)(ctx->ws + part_bytes + al(16 * 8)) : nullptr;
  const double* gprev = (adaptive && tau_prev > 0) ? grad_prev_dev : nullptr;
  CK(cudaMemcpyAsync(dfac, fac.data(), n_levels * sizeof(double), cudaMemcpyHostToDevice, st));
  std::vector<const double*> fields(n_levels);
  for (int l = 0; l < n_levels; ++l) fields[l] = stats[l].field_dev;
  launch_combine_step(fields.data(), dfac, n_levels, nc, denom, ctx->cfg.alpha, tau, !adaptive, z_dev,
                      adaptive ? gnew : grad_dev, gprev, partial, nblk, st);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(hb, partial + (size_t)rows * nblk, rows * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double hc = 1.0 / ctx->Nc(), hc3 = hc * hc * hc;
  const double g2 = hb[0] * hc3, ex2 = hb[1] * hc3, diff2 = hb[2] * hc3, gp2 = hb[3] * hc3, z2 = hb[4] * hc3;
  const double* ml = hb + 5;
  std::memset(rep, 0, sizeof(*rep));
  rep->grad_norm = std::sqrt(g2);
  rep->ey = ey;
  rep->shift = cstar;
  rep->truncated = ey < floor_y ? 1 : 0;
  rep->risk = ey > 0 ? cstar + std::log(ey) / theta : NAN;
  rep->z_norm = std::sqrt(z2);
  rep->objective = rep->risk + 0.5 * ctx->cfg.alpha * z2;
  if (!std::isfinite(rep->grad_norm)) return fail(ctx, MLSGD_ENONFINITE, "mlsgd_step: non-finite gradient");
  // ---- adaptive plan (eq:sec-order-sum .. eq:mse-estimate-mlmc; see the readings in the header)
  const int L = n_levels;
  const double C_hat = ex2 / (ey * ey);
  const double eps2 = (eta * rep->grad_norm) * (eta * rep->grad_norm);
  std::vector<double> v2(L), bias2(L), M(L), V, C;
  for (int l = 0; l < L; ++l) {
    const double* q = &sc[l * MLSGD_NSCALARS];
    const double f = std::exp(2.0 * theta * q[MLSGD_S_SHIFT]);
    v2[l] = f * (q[MLSGD_S_S2_DX] + C_hat * q[MLSGD_S_S2_DY]);
    bias2[l] = f * (ml[l] * hc3 + C_hat * q[MLSGD_S_MEAN_DY] * q[MLSGD_S_MEAN_DY]);
    M[l] = q[MLSGD_S_COUNT];
  }
  double err_sam = 0.0;
  for (int l = 0; l < L; ++l) err_sam += v2[l] / (M[l] * (M[l] - 1.0));
  double alpha_hat = 2.0;
  if (L - 1 >= 2) {
    std::vector<double> x, y;
    for (int l = 1; l < L; ++l) { x.push_back(l); y.push_back(std::log2(std::sqrt(bias2[l]))); }
    alpha_hat = -ls_slope(x, y);
  }
  double err_num = 0.0;
  for (int l = 1; l < L; ++l) {
    const double f = (std::pow(2.0, alpha_hat) - 1.0) * std::pow(std::pow(2.0, (double)(L - 1 - l)), alpha_hat);
    err_num = std::max(err_num, bias2[l] / (f * f));
  }
  for (int l = 0; l < L; ++l) { V.push_back(v2[l] / (M[l] - 1.0)); C.push_back(cost_model(ctx->cfg.n0, l)); }
  const int cap = std::min(max_levels, ctx->cfg.n_levels);
  const int Lnext = (err_num > eps2 / 2.0 && L < cap) ? L + 1 : L;
  if (Lnext > L) {
    double beta = 4.0;
    if (L - 1 >= 2) {
      std::vector<double> x, y;
      for (int l = 1; l < L; ++l) { x.push_back(l); y.push_back(std::log2(V[l])); }
      beta = -ls_slope(x, y);
    }
    V.push_back(V[L - 1] * std::pow(2.0, -beta));
    C.push_back(cost_model(ctx->cfg.n0, L));
  }
  double total = 0.0;
  for (int l = 0; l < Lnext; ++l) total += std::sqrt(V[l] * C[l]);
  rep->ex_norm2 = ex2;
  rep->c_hat = C_hat;
  for (int l = 0; l < L; ++l) {
    rep->mean_dx_norm2[l] = ml[l] * hc3;
    rep->v2[l] = v2[l];
  }
  rep->err_sam = err_sam;
  rep->err_num = err_num;
  rep->alpha_hat = alpha_hat;
  rep->eps2 = eps2;
  rep->next_levels = Lnext;
  for (int l = 0; l < Lnext && l < 16; ++l) {
    const double m = std::ceil(2.0 / eps2 * std::sqrt(V[l] / C[l]) * total);
    rep->next_counts[l] = (int64_t)std::max(2.0, std::min(m, 9.0e15));
  }
  // ---- rate diagnostics (eq:decayNum, eq:decayDenom, eq:weakerror2, eq:weakerror), log2 in the
  // shifted domain plus the shift so that large theta c does not overflow
  std::vector<double> lx(L), ly(L), lmx(L), lmy(L);
  const double log2e = 1.0 / std::log(2.0);
  for (int l = 0; l < L; ++l) {
    const double* q = &sc[l * MLSGD_NSCALARS];
    const double tc = theta * q[MLSGD_S_SHIFT] * log2e;  // log2 exp(theta c_l)
    const double sx = q[MLSGD_S_S2_DX] / M[l] + ml[l] * hc3;
    const double sy = q[MLSGD_S_S2_DY] / M[l] + q[MLSGD_S_MEAN_DY] * q[MLSGD_S_MEAN_DY];
    lx[l] = std::log2(sx) + 2.0 * tc;
    ly[l] = std::log2(sy) + 2.0 * tc;
    lmx[l] = 0.5 * std::log2(ml[l] * hc3) + tc;
    lmy[l] = std::log2(std::fabs(q[MLSGD_S_MEAN_DY])) + tc;
    rep->m2_dx[l] = std::exp2(lx[l]);
    rep->m2_dy[l] = std::exp2(ly[l]);
    rep->mean_dx_norm[l] = std::exp2(lmx[l]);
    rep->mean_dy_abs[l] = std::exp2(lmy[l]);
  }
  rep->beta_x = -diff_level_slope(lx);
  rep->beta_y = -diff_level_slope(ly);
  rep->alpha_x = -diff_level_slope(lmx);
  rep->alpha_y = -diff_level_slope(lmy);
  // ---- step size
  rep->l_hat = NAN;
  rep->tau = tau;
  if (adaptive) {
    if (gprev) {
      rep->l_hat = std::sqrt(diff2) / (tau_prev * std::sqrt(gp2));
      const double t = (g2 - err_sam) / (rep->l_hat * g2);
      if (std::isfinite(t) && t > 0) {
        rep->tau = t;
      } else {
        const bool lh = std::isfinite(rep->l_hat) && rep->l_hat > 0;
        rep->tau = lh ? std::min(tau_prev, 1.0 / rep->l_hat) : tau_prev;
        rep->tau_fallback = 1;
      }
    }
    launch_step_apply(nc, rep->tau, gnew, z_dev, grad_prev_dev, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  }
  return MLSGD_OK;
}

mlsgd_status mlsgd_step(mlsgd_ctx* ctx, const mlsgd_level_stats* stats, int n_levels, double tau, double eta,
                        int max_levels, double* z_dev, double* grad_dev, mlsgd_step_report* rep, void* stream) {
  if (!ctx) return MLSGD_EINVAL;
  return step_core(ctx, stats, n_levels, eta, max_levels, z_dev, grad_dev, false, tau, 0.0, nullptr, rep,
                   (cudaStream_t)stream);
}

mlsgd_status mlsgd_step_adaptive(mlsgd_ctx* ctx, const mlsgd_level_stats* stats, int n_levels, double tau0,
                                 double tau_prev, double eta, int max_levels, double* z_dev, double* grad_prev_dev,
                                 mlsgd_step_report* rep, void* stream) {
  if (!ctx) return MLSGD_EINVAL;
  return step_core(ctx, stats, n_levels, eta, max_levels, z_dev, nullptr, true, tau0, tau_prev, grad_prev_dev, rep,
                   (cudaStream_t)stream);
}

}  // extern "C"
