/*
 * mlsgd.h - C ABI of the GB300 multilevel entropic-risk gradient engine.
 *
 * The library evaluates the per-sample hot path of the multilevel stochastic
 * gradient method of Baumgarten, Guth, Schneiderhan and Vanzan ("Multilevel
 * Stochastic Gradient Descent for Risk-Averse PDE-Constrained
 * Optimization"): the random coefficient, the state and adjoint solves, the
 * entropic weights X = exp(theta Phi) B*q, Y = exp(theta Phi)
 * (eq:definition_Xell_Yell), the level differences (eq:delta-notation), the
 * per-level Chan statistics (Algorithm 1, PairwiseUpdate), the multilevel
 * gradient (eq:gradient_estimator) and the projected step
 * (eq:gradientdescentMLMC), on one GPU.
 *
 * Problem (Sec. 5): D = (0,1)^3, -div(a grad y) = z with y = 0 on the
 * boundary, a = exp(log a), log a = sigma sum_k sqrt(lambda_k) xi_k phi_k
 * with the K largest tensor-product KL modes of the exponential covariance
 * exp(-|x - x'| / corr_len) per coordinate, xi_k ~ N(0,1); target
 * g = sin(pi x) sin(pi y) sin(pi z); Phi = 1/2 ||y - g||^2_{L2} (eq:cost).
 * Discretisation: Q1 hexahedra on level l with N_l = n0 * 2^l cells per side,
 * coefficient constant per cell (value at the cell centre); the control z is
 * constant per cell of the control grid (level ctrl_level).  B z is exactly
 * int z phi_n dx (<Bu, v> = int u v, Sec. 5) and (B*q)_c is the average of q over
 * control cell c, for levels finer as well as coarser than the control grid.
 *
 * Conventions shared by every entry point
 *   - Every *_dev pointer is DEVICE memory owned by the caller (for example a
 *     torch tensor's data_ptr()).  The library never frees caller memory.  The
 *     library owns its scratch (grown on demand, freed by mlsgd_destroy).
 *   - Node vectors of a grid with N cells per side hold (N+1)^3 doubles per
 *     sample, node (i,j,k) at flat index i + (N+1)*(j + (N+1)*k), boundary
 *     nodes included (always 0).  Cell fields hold N^3 values per sample, cell
 *     (i,j,k) at i + N*(j + N*k).  Batched arrays are sample-major.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.
 *   - Every call returns a status and never aborts; mlsgd_last_error() gives
 *     a one-line description of the last failure on that context.
 *   - Sample identity is (seed, iteration, level, sample index): a sample's
 *     draw xi and every per-sample result are independent of how samples are
 *     grouped into calls.
 */
#ifndef MLSGD_H
#define MLSGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MLSGD_OK = 0,
  MLSGD_EINVAL = 1,      /* bad argument (sizes, levels, NULL pointers)          */
  MLSGD_ENOMEM = 2,      /* device scratch could not be allocated                 */
  MLSGD_ENOCONV = 3,     /* a solve hit max_iter; per-sample status flags say which */
  MLSGD_ENONFINITE = 4,  /* NaN/Inf in an input or a reduced result               */
  MLSGD_ECUDA = 5,       /* CUDA runtime error                                    */
  MLSGD_ENOTIMPL = 6
} mlsgd_status;

typedef enum { MLSGD_FP64 = 0, MLSGD_MIXED = 1 } mlsgd_precision;

/* Workload and solver configuration. */
typedef struct {
  int n_levels;     /* levels 0..n_levels-1                                          */
  int n0;           /* cells per side on level 0 (8 in every preset)                 */
  int ctrl_level;   /* level whose cells carry z (any level; solves on finer and
                       coarser grids both integrate z exactly)                      */
  int n_modes;      /* K, number of KL modes (even)                                  */
  double corr_len;  /* correlation length of the 1D exponential covariance           */
  double sigma;     /* standard-deviation factor of log a                           */
  double theta;     /* risk aversion (eq:entropic-risk)                              */
  double alpha;     /* control cost, the paper's lambda (eq:cost)                    */
  double rtol;      /* stop when ||b - A y||_2 <= rtol ||b||_2 (true residual, FP64) */
  int max_iter;     /* cap on PCG iterations (FP64) or refinement steps (MIXED)      */
  int precision;    /* mlsgd_precision                                               */
  int inner_iters;  /* MIXED only: FP32 PCG iterations per refinement step (0 = 6)   */
  int max_batch;    /* samples per internal chunk of mlsgd_level_gradient (0 = 256)  */
  int field_tc;     /* MIXED only: 1 = BF16 preconditioner coefficient synthesised on the
                       tensor cores (tcgen05 GEMM, BF16 in / FP32 accumulate); 0 = rounded
                       from the FP64 synthesis                                        */
  int ir_steps;     /* MIXED only: 0 = refine until converged, checking on the host after
                       each step (the samples still above rtol are compacted into a list and
                       only they are launched in the next step; the FP64 path does the same
                       at its host checks); k > 0 = exactly k refinement steps per solve with no host
                       synchronisation (per-sample masks; a sample still above rtol after k
                       steps gets status 1).  With k > 0 and the scratch already sized (one
                       earlier call of the same size), mlsgd_level_gradient enqueues only
                       stream work and can be captured into a CUDA graph.             */
  int field_model;  /* 0 = tensorised KL of exp(-|x-x'|/corr_len), xi ~ N(0,1);
                       1 = the paper's Sec. 5 field: modes cos(j pi x2) cos(k pi x3) cos(l pi x1),
                       j,k,l = 1..m, m^3 = n_modes (ordered j, k, l with l fastest),
                       lambda = exp(-pi (j+k+l) corr_len), xi ~ U(-4, 4), not normalised */
  int target_freq;  /* g = prod_i sin(f pi x_i): 1 for the workload, 2 for the paper (0 = 1) */
  uint64_t seed;
  /* kernel and smoother choices (none changes what a converged solve returns beyond
     the solver tolerance; an autotuner picks them per grid and batch) */
  int stencil;      /* MIXED only: 0 = whole-row slab passes on 32^3 and 64^3 grids,
                       z-marching tile passes elsewhere; 1 = z-marching tile passes only  */
  int z_chunks;     /* z chunks the fused passes split a sample into (0 = chosen from the
                       batch size); results do not depend on it                          */
  double omega;     /* damping of the Jacobi smoother in the V-cycle (0 = 0.6; (0, 1))    */
  int inner_iters_next; /* MIXED only: FP32 PCG iterations of the refinement steps after the
                           first, which start from a residual already reduced by it
                           (0 = inner_iters)                                               */
} mlsgd_config;

typedef struct mlsgd_ctx mlsgd_ctx;

/* Per-level statistics of the level differences, in device memory, mergeable
 * across calls (Algorithm 1, PairwiseUpdate; Sec. 4.2 b).
 *   field_dev   [n_ctrl_cells] FP64: sample mean of dX~ = X~_l - X~_{l-1}
 *   scalars_dev [MLSGD_NSCALARS] FP64, see the MLSGD_S_* indices.
 * X~ and Y~ carry the factor exp(-theta * shift): X~ = exp(theta (Phi - shift)) B*q. */
enum {
  MLSGD_S_COUNT = 0,   /* number of samples merged                                     */
  MLSGD_S_SHIFT = 1,   /* shift c of this level                                        */
  MLSGD_S_MEAN_DY = 2, /* mean of dY~                                                  */
  MLSGD_S_S2_DY = 3,   /* sum over samples of (dY~ - mean)^2                           */
  MLSGD_S_S2_DX = 4,   /* sum over samples of ||dX~ - mean||_U^2                       */
  MLSGD_S_PHI_MAX = 5, /* largest Phi seen on this level (either grid)                 */
  MLSGD_S_ITERS = 6,   /* total solver iterations spent (state + adjoint, both grids) */
  MLSGD_S_NOCONV = 7,  /* number of solves that hit max_iter                           */
  MLSGD_NSCALARS = 8
};
typedef struct {
  int level;
  double* field_dev;
  double* scalars_dev;
} mlsgd_level_stats;

/* Result of mlsgd_step (host memory). */
typedef struct {
  double grad_norm;   /* ||grad J^ML||_U                                               */
  double risk;        /* multilevel estimate of R_theta(Phi) = shift + log(E^ML[Y~])/theta */
  double ey;          /* E^ML[Y~] at the common shift                                  */
  double shift;       /* common shift c* = max_l c_l                                   */
  int truncated;      /* 1 if max{1, E^ML[Y]} took the value 1                         */
  double err_sam;     /* eq:mse-estimate-mlmc sampling part                            */
  double err_num;     /* eq:squared-bias-estimate-mlmc                                 */
  double alpha_hat;   /* fitted weak rate                                              */
  double eps2;        /* (eta ||grad||)^2                                              */
  int next_levels;    /* L_{k+1} (eq:optimal-level)                                    */
  int64_t next_counts[16]; /* M_{k+1,l} (eq:optimal-batch-size)                         */
  /* inputs of the plan, for inspection */
  double ex_norm2;         /* ||E^ML[X~]||_U^2 at the common shift                        */
  double c_hat;            /* ||E^ML[X]||^2 / E^ML[Y]^2                                   */
  double mean_dx_norm2[16];/* ||mean dX~_l||_U^2 (shift of level l)                       */
  double v2[16];           /* v^2_l in unshifted units (eq:sec-order-sum)                 */
  /* step size */
  double tau;              /* the step taken                                              */
  double l_hat;            /* L^ of eq:adaptive-step-size (NaN for a fixed or first step)  */
  int tau_fallback;        /* 1: the adaptive rule gave a non-positive or non-finite step
                              and min(tau_prev, 1/L^) was taken instead                   */
  /* rate diagnostics of this batch, unshifted, per level l (the difference samples) */
  double m2_dx[16];        /* (1/M_l) sum_m ||dX_l^(m)||_U^2, left side of eq:decayNum     */
  double m2_dy[16];        /* (1/M_l) sum_m |dY_l^(m)|^2, left side of eq:decayDenom       */
  double mean_dx_norm[16]; /* ||mean dX_l||_U (eq:weakerror2 through the level difference) */
  double mean_dy_abs[16];  /* |mean dY_l| (eq:weakerror)                                    */
  /* exponents from least-squares fits of log2 of the above against l over l >= 1:
     m2 ~ h_l^beta, means ~ h_l^alpha with h_l = h_0 2^-l (NaN with fewer than two
     difference levels) */
  double beta_x, beta_y, alpha_x, alpha_y;
  double z_norm;           /* ||u_k||_U, the control before the step                      */
  double objective;        /* J^ML(u_k) = risk + alpha/2 ||u_k||_U^2 (eq:cost)            */
} mlsgd_step_report;

/* Create a context on the current CUDA device.  Builds the KL mode table on
 * the host and uploads the 1D mode tables.  Returns MLSGD_EINVAL for an
 * inconsistent configuration (n_modes < 2, odd n_modes with field_model 0,
 * n_modes not a cube with field_model 1, ctrl_level outside [0, n_levels),
 * n_levels > 16, non-positive corr_len / rtol). */
mlsgd_status mlsgd_create(const mlsgd_config* cfg, mlsgd_ctx** out);
void mlsgd_destroy(mlsgd_ctx* ctx);
const char* mlsgd_last_error(const mlsgd_ctx* ctx);
const char* mlsgd_status_string(mlsgd_status s);

/* Number of control cells (n0 * 2^ctrl_level)^3 and of selected 1D KL modes. */
int64_t mlsgd_n_ctrl_cells(const mlsgd_ctx* ctx);
/* Bytes of library scratch one chunk of n_samples at `level` needs (both
 * grids of the level difference); used for admission by HBM footprint. */
size_t mlsgd_workspace_bytes(const mlsgd_ctx* ctx, int level, int n_samples);

/* Scratch owned by the caller: the context takes [ws_dev, ws_dev + bytes) (device
 * memory, 256-byte aligned, kept valid while the context uses it) as its workspace
 * instead of allocating its own, frees its own scratch if it had any (synchronising
 * the device first), and never grows, frees or reallocates the caller's range: a
 * call whose batch needs more (mlsgd_workspace_bytes) fails with MLSGD_ENOMEM.
 * Every call of the context until the next mlsgd_set_workspace reads and writes the
 * range, so a caller that hands disjoint ranges of one arena to several contexts can
 * run them concurrently on different streams and admit work by memory footprint.
 * ws_dev NULL with bytes 0 returns the context to allocating its own scratch.  The
 * per-level tensor-core mode tables are still allocated by the context on the first
 * call that needs them. */
mlsgd_status mlsgd_set_workspace(mlsgd_ctx* ctx, void* ws_dev, size_t bytes);

/* Copy the KL mode table to host arrays (each may be NULL):
 * idx [3*n_modes] 1D mode indices (x, y, z) of each 3D mode, lam [n_modes]
 * lambda_i lambda_j lambda_k.  Returns the number of 1D modes used. */
int mlsgd_mode_table(const mlsgd_ctx* ctx, int* idx, double* lam);

/* a1 + a2: draw xi^(m, level) for samples first_sample .. first_sample+n_samples-1
 * of optimisation step `iter` and write log a at the cell centres of grid
 * level `grid` (grid == level or level - 1: the same draw on both grids,
 * eq:shorthand-notation).  xi_dev (optional, may be NULL) receives
 * [n_samples][n_modes] normals; log_a_dev receives [n_samples][N_grid^3]. */
mlsgd_status mlsgd_sample_field(mlsgd_ctx* ctx, int iter, int level, int grid, int64_t first_sample,
                                int n_samples, double* xi_dev, double* log_a_dev, void* stream);

/* a2 on the tensor cores: log a[s, c] = sum_k (sigma sqrt(lambda_k) xi[s,k]) phi_k(x_c)
 * as a BF16 x BF16 -> FP32 GEMM (samples x modes) by (modes x cells) on the same
 * draws as mlsgd_sample_field.  log_a_f32_dev (optional) [n_samples][N^3] FP32;
 * a_bf16_dev (optional) [n_samples][N^3] BF16 exp(log a).  Requires n_modes % 64 == 0
 * and N^3 % 128 == 0; returns MLSGD_ENOTIMPL otherwise.  Synchronous (checks
 * the kernel's error flag). */
mlsgd_status mlsgd_sample_field_tc(mlsgd_ctx* ctx, int iter, int level, int grid, int64_t first_sample,
                                   int n_samples, float* log_a_f32_dev, void* a_bf16_dev, void* stream);

/* a3..a6: for each sample s, with a = exp(log_a_dev[s]) on grid level `grid`:
 * solve the state problem A y = B z (eq:sys), Phi = 1/2 (y - g_h)^T M (y - g_h)
 * (eq:cost with the nodal interpolant g_h and the Q1 mass M), and the adjoint
 * problem A q = M (y - g_h) (Sec. 2.2 adjoint equation; A is symmetric).
 * Inputs: log_a_dev [n_samples][N^3], z_dev [n_ctrl_cells].
 * Outputs: y_dev, q_dev [n_samples][(N+1)^3]; phi_dev [n_samples];
 * iters_dev [n_samples] PCG iterations (FP64) or inner iterations (MIXED),
 * state + adjoint; status_dev [n_samples] 0 = converged, bit 0 (1) = a solve hit
 * max_iter, bit 1 (2) = a solve went non-finite (NaN/Inf in z or the coefficient).
 * After writing every output, returns MLSGD_ENONFINITE if any sample has bit 1,
 * else MLSGD_ENOCONV if any has bit 0.  SYNCHRONOUS (reads the flags back). */
mlsgd_status mlsgd_solve_state_adjoint(mlsgd_ctx* ctx, int grid, int n_samples, const double* log_a_dev,
                                       const double* z_dev, double* y_dev, double* q_dev, double* phi_dev,
                                       int* iters_dev, int* status_dev, void* stream);

/* a1..a9 for one level: samples first_sample .. first_sample+n_samples-1 of
 * step `iter` on `level` (and level-1 on the same draw when level > 0):
 * fields, state and adjoint solves, B*q as control-cell averages, shifted
 * weights, dX~ = X~_l - X~_{l-1}, dY~, and the Chan merge of this batch into
 * *stats (which must have been reset with mlsgd_stats_reset or hold earlier
 * batches of the same level).  The shift becomes max(old shift, max Phi of the
 * batch) and older sums are rescaled to it. */
mlsgd_status mlsgd_level_gradient(mlsgd_ctx* ctx, int iter, int level, int64_t first_sample, int n_samples,
                                  const double* z_dev, mlsgd_level_stats* stats, void* stream);

/* Allocation-free variant of mlsgd_solve_state_adjoint.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory when they
 * need a solve, for example a latency-critical loop in which cudaMalloc's implicit
 * device-wide synchronisation is not acceptable, or an application whose own
 * allocator has reserved the device memory and does not let libraries call the
 * CUDA allocator.  Same arguments, layouts, results and status codes as
 * mlsgd_solve_state_adjoint, but every scratch buffer comes from one static device
 * array of MLSGD_NOALLOC_SCRATCH_BYTES compiled into the library, which each GPU
 * that loads the library holds until the process exits; the call makes no
 * cudaMalloc/cudaFree and calls no allocating library routine.  A batch whose
 * scratch would not fit is rejected with MLSGD_EINVAL and a message giving the
 * bytes it needs (about 6 samples of a 32^3 grid or 40 of a 16^3 grid in FP64).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  The call waits for its stream before it returns (it reads
 * back one status word).  All calls share the array and it keeps the last call's
 * contents: calls that overlap on the GPU (other streams, other threads, other
 * contexts) race, so serialise them.  Nothing in the array needs to start at
 * zero: the solve writes every buffer before it reads it. */
#define MLSGD_NOALLOC_SCRATCH_BYTES (16u << 20)
mlsgd_status mlsgd_solve_state_adjoint_noalloc(mlsgd_ctx* ctx, int grid, int n_samples, const double* log_a_dev,
                                               const double* z_dev, double* y_dev, double* q_dev, double* phi_dev,
                                               int* iters_dev, int* status_dev, void* stream);

/* Zero a statistics record (count 0, shift -inf). */
mlsgd_status mlsgd_stats_reset(mlsgd_ctx* ctx, mlsgd_level_stats* stats, void* stream);
/* Merge src into dst (both of the same level): Chan update with rescaling
 * to the larger shift.  dst and src may live on different contexts of the
 * same workload. */
mlsgd_status mlsgd_stats_merge(mlsgd_ctx* ctx, mlsgd_level_stats* dst, const mlsgd_level_stats* src,
                               void* stream);

/* a10 + a11: combine levels 0..n_levels-1 (stats[l] of level l) into
 * E^ML[X~], E^ML[Y~] at the common shift (eq:ml_estimator_numerator/denominator),
 * grad = E^ML[X~] / max{exp(-theta c*), E^ML[Y~]} + alpha z (eq:gradient_estimator
 * with its truncation), z <- z - tau grad (eq:gradientdescentMLMC; U_ad = U, so
 * the projection is the identity), and fill *rep including the adaptive plan
 * for the next step (eq:sec-order-sum .. eq:mse-estimate-mlmc) with eta and
 * the level cap `max_levels`.  grad_dev (optional) receives the gradient.
 * SYNCHRONOUS: returns after the report has been read back. */
mlsgd_status mlsgd_step(mlsgd_ctx* ctx, const mlsgd_level_stats* stats, int n_levels, double tau, double eta,
                        int max_levels, double* z_dev, double* grad_dev, mlsgd_step_report* rep, void* stream);

/* mlsgd_step with the adaptive step size of Sec. 5 (eq:adaptive-step-size):
 *   tau_k = (||g_k||^2 - err_sam_k) / (L^ ||g_k||^2),
 *   L^    = ||g_k - g_{k-1}||_U / ||tau_{k-1} g_{k-1}||_U,
 * g_k = grad J^ML(u_k) and err_sam_k as in *rep (the printed "t_{k-1}" is read as
 * tau_{k-1}).  Reading where the rule gives no positive finite step (sampling
 * error at or above ||g_k||^2, or g_k = g_{k-1}): tau_k = min(tau_{k-1}, 1/L^)
 * (tau_{k-1} if L^ is not positive and finite), and rep->tau_fallback = 1.
 *   tau0           step of the first iteration (> 0), used when tau_prev <= 0
 *   tau_prev       tau_{k-1} (<= 0 on the first iteration: grad_prev_dev is not read)
 *   grad_prev_dev  [n_ctrl_cells] FP64 device, IN g_{k-1}, OUT g_k (caller-owned,
 *                  kept between calls)
 * The step taken is rep->tau; z_dev <- z_dev - rep->tau g_k.  Same plan, report
 * and errors as mlsgd_step, plus MLSGD_EINVAL for a null grad_prev_dev, tau0 <= 0
 * or a non-finite tau_prev.  SYNCHRONOUS. */
mlsgd_status mlsgd_step_adaptive(mlsgd_ctx* ctx, const mlsgd_level_stats* stats, int n_levels, double tau0,
                                 double tau_prev, double eta, int max_levels, double* z_dev, double* grad_prev_dev,
                                 mlsgd_step_report* rep, void* stream);

/* ---------------------------------------------------------------- instrumentation
 * Process-wide.  Every kernel launch of the library is counted; when profiling
 * is on, launches of the named kernel class ("*" = all classes) are bracketed
 * by CUDA events recorded on their own stream, and the class's algorithmic
 * traffic (each input read once, each output written once) and flops are
 * summed.  Class names are listed in the launch sites (for example
 * "smooth_f32", "apply_f64", "resid64", "field", "level_field"). */
typedef struct {
  char cls[32];
  int64_t launches;
  double total_ms;
  double bytes;
  double flops;
} mlsgd_profile_entry;
int64_t mlsgd_launch_count(void);
/* start a profile (resets earlier records); kernel_class NULL turns profiling off */
int mlsgd_profile_start(const char* kernel_class);
/* stop, wait for the events, fill up to max_entries per-class totals; returns the
 * number of classes seen (may exceed max_entries) or -1 on a CUDA error */
int mlsgd_profile_stop(mlsgd_profile_entry* out, int max_entries);

#ifdef __cplusplus
}
#endif
#endif /* MLSGD_H */
