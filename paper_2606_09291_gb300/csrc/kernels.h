// kernels.h - host-visible declarations of the kernel launchers of libmlsgd.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stddef.h>
#include <stdint.h>

namespace mlsgd {

// KL mode table on the device (built on the host by kl_table.cpp)
struct ModeTable {
  const int* iy;        // [K] y-index of each 3D mode
  const int* iz;        // [K] z-index
  const double* scale;  // [K] sigma * sqrt(lambda_k)
  const int* order;     // [K] modes sorted by x-index
  const int* offs;      // [n1x+1] start of each x-index group in `order`
  int n1x;              // number of x-indices (max + 1)
  int n1d;              // number of 1D modes in the phi tables
};

// outputs of the field kernel (any may be null)
struct FieldOut {
  double* log_a;
  double* a64;
  float* a32;
  __nv_bfloat16* abf;
};

// half_width > 0: uniform xi on (-half_width, half_width] (the paper's field), else N(0, 1)
void launch_draw_xi(uint64_t seed, int iter, int level, long long first, int S, int K, double* xi, cudaStream_t st,
                    double half_width = 0.0);
cudaError_t launch_field(const double* xi, int K, const ModeTable& mt, const double* phi, int N, int S,
                         const FieldOut& out, cudaStream_t st);
size_t field_smem_bytes(const ModeTable& mt, int K, int N);
void launch_exp_field(const double* la, const FieldOut& out, long long n, cudaStream_t st);

// ---------------------------------------------------------------- solver
// per-sample scalar state of a (P)CG iteration
struct SolveScalars {
  double bb;     // ||b||^2 of the system being solved
  double rz;     // r . z
  double alpha;
  double beta;
  double rr;     // ||r||^2
  int active;    // 1 while iterating
  int iters;
  int status;    // 0 converged, 1 hit the iteration cap
  int pad;
};

__host__ __device__ inline long long nodes_of(int N) { return (long long)(N + 1) * (N + 1) * (N + 1); }
__host__ __device__ inline long long cells_of(int N) { return (long long)N * N * N; }
inline int node_blocks(int N) { return (int)((nodes_of(N) + 255) / 256); }
// block partials one level's statistics may write (control-cell blocks + level-cell
// blocks + slack); the buffer is sized with this and the kernels stay within it
inline long long level_partial_cap(int Nc, int Nf) {
  return (cells_of(Nc) + 255) / 256 + (cells_of(Nf) + 255) / 256 + 64;
}

// The samples one launch processes: a batch of S samples (the tile shapes and the
// per-sample partial-sum layout follow S), of which n are launched, sample act[t] for
// t < n (act null: samples 0..n-1, n == S).  The solver's host-checked modes compact
// the still-active samples into act, so retired samples start no blocks.
struct Batch {
  int S;
  int n;
  const int* act;
  int* err;      // device flag a kernel sets when one of its bounded waits runs out
  int stencil;   // 0: slab passes where supported, 1: z-marching tiles only
  int zchunks;   // z chunks per sample (0: chosen from S)
};

// Buffers of one batched solve on a grid with N cells per side.  Vectors are
// [S][nodes] (stride nodes_of(N)), coefficients [S][cells].
struct SolverBufs {
  int N, S, J;               // MG levels j = 0..J, N_j = N >> j, N_J = 2
  int n_act = 0;             // samples launched by the masked kernels (host-known)
  const int* actp = nullptr; // their indices (null: all S)
  int* act = nullptr;        // [S] device list the compaction writes
  int* err = nullptr;        // device error flag (bounded waits that ran out)
  int stencil = 0;           // see Batch
  int zchunks = 0;
  Batch batch() const { return Batch{S, n_act, actp, err, stencil, zchunks}; }
  // MG hierarchy (j >= 1 coarse; j = 0 uses the caller's operator coefficient)
  void* acoef[8];            // coefficient per MG level (j = 0: the V-cycle's own copy, may alias)
  void* vx[8];               // V-cycle iterate per level
  void* vt[8];               // V-cycle temporary / output per level
  void* vr[8];               // restricted residual (j >= 1)
  void* dinv[8];             // D^{-1} of levels run with the tiled passes (0 at boundary nodes), else null
  float2* bdf;               // mixed tiled solves: b as FP32 (hi, lo) pairs [S][nodes]; with the slab
                             // refinement step, the residual pairs of the step
  float2* bsh;               // the same for a b shared by every sample: [nodes]
  // Krylov vectors
  void* x;                   // solution / correction
  void* r;                   // residual
  void* r2;                  // second residual buffer (fused inner solve)
  void* p;
  void* q;                   // A p
  double* partial;           // [S][blocks]
  SolveScalars* sc;          // [S]
  int* count;                // device counter of active samples
  int* count_host;           // pinned host mirror
};

// FP64 batched PCG: solve A(a64) x = b for S samples (b may be shared: bstride 0)
struct PcgParams {
  double rtol;
  int max_iter;
  double omega;   // Jacobi damping of the smoother
  int check_every;
};
cudaError_t pcg_fp64(SolverBufs& B, const double* a64, const double* b, long long bstride, double* x_out,
                     const PcgParams& prm, cudaStream_t st);
// mixed: FP64 refinement around FP32 PCG (operator a32, V-cycle on abf)
// fixed_steps > 0: exactly that many refinement steps, no host synchronisation
// b_pair (tiled grids only): b given as FP32 (hi, lo) pairs instead of b (FP64)
// pair_out (tiled grids only): x_out's storage receives the solution as FP32 (hi, lo)
//   pairs (8 bytes per node, as the FP64 layout) instead of FP64 values
// inner_next: inner iterations of the steps after the first (0: inner_iters)
cudaError_t ir_mixed(SolverBufs& B, const float* a32, const __nv_bfloat16* abf, const double* b,
                     long long bstride, double* x_out, double* r64, const PcgParams& prm, int inner_iters,
                     cudaStream_t st, int fixed_steps = 0, const float2* b_pair = nullptr, bool pair_out = false,
                     int inner_next = 0);
// coefficient hierarchy for the V-cycle from the level-0 coefficient
// coarse coefficients and, per tiled level, omega D^-1 (omega: the smoother's damping)
void build_hierarchy_fp64(SolverBufs& B, const double* a64, double omega, cudaStream_t st);
void build_hierarchy_mixed(SolverBufs& B, const __nv_bfloat16* abf, double omega, cudaStream_t st);
// bytes the buffers need (elem = 8 for FP64, 4 for FP32 Krylov vectors)
size_t solver_bytes(int N, int S, int elem);
void carve_solver(SolverBufs& B, int N, int S, int elem, char*& ptr);

// tiled fine-grid kernels (tiled.cu); partial sums land in [S][blocks_per_sample], one
// entry per (xy tile, segment of 8 interior planes), independent of the z chunking
struct TiledShape { int bx, by, nzc, zc, nseg, blocks_per_sample; };
TiledShape tiled_shape(int N, int S, int rows_per_thread, int zchunks = 0);
// partial-sum entries per sample of the solver passes for elements of `elem` bytes
// (slab: the whole-row slab passes' geometry)
int tiled_blocks_per_sample(int N, int S, int elem, bool slab);
template <typename T, typename TA>
void tiled_apply(const T* z, const T* pold, T* pnew, const TA* a, T* q, double* partial, const SolveScalars* sc, int N,
                 const Batch& bt, int first, cudaStream_t st);
// PRE (and PREU): t = r - A x1 with x1 = omega D^-1 r (PREU: r <- r - alpha q first, stored
// in rnew).  True when the pass also restricted t to rc on grid N/2 (the slab passes;
// t is then not stored), false when t was stored for a separate restriction.
template <typename T, typename TA>
bool tiled_pre(const T* r, const TA* a, const T* wdinv, T* t, T* rc, const SolveScalars* sc, int N, const Batch& bt,
               cudaStream_t st);
template <typename T, typename TA>
void tiled_post(const T* r, const TA* a, const T* wdinv, const T* ec, T* z, double* partial, const SolveScalars* sc,
                int N, const Batch& bt, cudaStream_t st);
void tiled_apply_x(const float* z, const float* pold, float* pnew, const float* a, float* q, float* x, double* partial,
                   const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st, bool x_first);
bool tiled_pre_update(const float* r, const float* q, const __nv_bfloat16* a, const float* wdinv, float* t,
                      float* rnew, float* rc, const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st);
// r32 = (float)(b - A x) to FP64 accuracy with x, b as FP32 (hi, lo) pairs and error-free
// FP32 products and sums; partial r.r
void tiled_res64(const float2* b, long long bstride, const float2* x, const float* a, float* r32, double* partial,
                 const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st);
// Phi and the adjoint right-hand side; returns the partial-sum blocks per sample
int tiled_phi_df(const float2* y, int N, int S, const float2* gtab, const float2* mgtab, float2* badj,
                 double* partial, cudaStream_t st);
int tiled_phi(const double* y, int N, int S, const double* gtab, const double* mgtab, double* badj, double* partial,
              cudaStream_t st);
constexpr int kTiledMinN = 16;  // grids with at least this many cells per side use the tiled kernels

// whole-row slab passes (slab.cu) for the mixed path's FP32 vectors on 32^3 and 64^3
// grids; boundary nodes of the staged vectors are taken as 0 whatever they hold
bool slab_supported(int N);
TiledShape slab_shape(int N, int S, int zchunks = 0);
void slab_apply(const float* z, const float* pold, float* pnew, const float* a, float* q, float* x, double* partial,
                const SolveScalars* sc, int N, const Batch& bt, bool first, bool with_x, bool x_first, cudaStream_t st);
// PRE (q null) or PREU with the restriction of t fused: rc on grid N/2 (t not stored)
template <typename TA>
void slab_pre(const float* r, const float* q, const TA* a, const float* wdinv, float* rnew, float* rc,
              const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st);
template <typename TA>
void slab_post(const float* r, const TA* a, const float* wdinv, const float* ec, float* z, double* partial,
               const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st);
// the refinement step in one pass: inc = d + alpha p (alpha p when d_zero; alpha from
// sci), rr_out = rr_in - A inc and r32 = rr_out rounded (to FP64 accuracy in FP32 pair
// arithmetic; rr_in stride 0: one vector for every sample), partial r32.r32, and the
// solution pairs x (+)= inc (x = inc when assign; samples that take no step get x = 0
// on the first step); interior and x = N / y = N nodes only
void slab_res(const float* d, const float* p, bool d_zero, const SolveScalars* sci, const float2* rr_in,
              long long rr_stride, float2* rr_out, float2* x, bool assign, const float* a, float* r32,
              double* partial, const SolveScalars* sco, int N, const Batch& bt, cudaStream_t st);

// the V-cycle from a coarse 16^3 level (j >= 1 of a grid with N cells) down to 2^3 in one
// launch, one block per launched sample (coarse.cu): r16 the restricted residual, a the
// coefficients of the levels 16^3 .. 2^3, z16 the correction
bool coarse_vcycle_applies(int N, int j);
template <typename T>
void coarse_vcycle(const T* r16, const T* const a[4], T* z16, const SolveScalars* sc, const Batch& bt, double omega,
                   cudaStream_t st);

// tensor-core KL synthesis (kl_gemm.cu)
size_t kl_gemm_b_bytes(int N, int K);
size_t kl_gemm_a_bytes(int S, int K);
void kl_gemm_build_b(const double* phi, const int* ix, const int* iy, const int* iz, int N, int K, __nv_bfloat16* B,
                     cudaStream_t st);
cudaError_t kl_gemm(const double* xi, const double* scale, int S, int K, const __nv_bfloat16* B, int N,
                    __nv_bfloat16* A_scratch, __nv_bfloat16* abf, float* loga, int* err, cudaStream_t st);

// ---------------------------------------------------------------- estimator
void launch_rhs_state(const double* z, int Nc, int N, double* b, cudaStream_t st);
// Phi = 1/2 e^T M e, badj = M e (interior rows), e = y - g_h
void launch_phi_adjrhs(const double* y, int N, int S, double* badj, double* phi, double* partial,
                       const double* gtab, const double* mgtab, cudaStream_t st, int freq = 1);
// the same for a state stored as FP32 pairs on a tiled grid (tables and M e as pairs)
void launch_phi_adjrhs_df(const float2* y, int N, int S, float2* badj, double* phi, double* partial,
                          const float2* gtab, const float2* mgtab, cudaStream_t st);
// batch statistics of one level merged into stats (see mlsgd_level_stats)
// qf_pairs / qc_pairs: the adjoint solutions are stored as FP32 (hi, lo) pairs;
// work holds 4 + 4 S doubles; nodebuf (2 (Nf+1)^3 doubles, optional): when the
// level's grids are at least 4x coarser than the control grid the statistics are
// formed on the level grid (qf is then overwritten; partial needs cells(Nc)/256 +
// cells(Nf)/256 + 2 entries)
void launch_level_stats(const double* qf, const double* phif, int Nf, const double* qc, const double* phic,
                        int Ncoarse, int S, int Nc, double theta, double* field, double* scalars,
                        double* work, double* partial, const int* iters, const int* status, cudaStream_t st,
                        bool qf_pairs = false, bool qc_pairs = false, double* nodebuf = nullptr);
void launch_stats_reset(double* field, double* scalars, long long ncells, cudaStream_t st);
void launch_stats_merge(double* dfield, double* dsc, const double* sfield, const double* ssc, long long ncells,
                        double hc3, double theta, double* partial, cudaStream_t st);
// combine levels and (when `update`) step; partial gets [L + 5][blocks] sums and
// then the L + 5 totals; gprev (optional) is the previous gradient
void launch_combine_step(const double* const* fields, const double* factors, int L, long long ncells,
                         double denom, double alpha, double tau, bool update, double* z, double* grad,
                         const double* gprev, double* partial, int nblk, cudaStream_t st);
// z <- z - tau g; gout <- g
void launch_step_apply(long long ncells, double tau, const double* g, double* z, double* gout, cudaStream_t st);

}  // namespace mlsgd
