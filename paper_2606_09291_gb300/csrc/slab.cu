// slab.cu - fused fine-grid passes of the mixed-precision solver on 32^3 and 64^3
// grids, staged as whole-row slabs by bulk asynchronous copies (rows a4, a6).
//
// The passes compute what the z-marching passes of tiled.cu compute (APPLY,
// APPLYX, PRE, PREU, POST; FP32 vectors, BF16 or FP32 cell coefficient) with a
// layout chosen for fewer instructions per node:
//   * a block owns every node of TYT = 8 RY consecutive interior rows (all x) and
//     marches along z over a chunk of interior planes; warp w takes rows
//     RY w .. RY w + RY - 1 of the block, lane l the RX = N/32 nodes
//     x = 1 + RX l .. RX l + RX;
//   * node plane m of a staged vector, rows y0-1 .. y0+TYT (clamped to N), is one
//     contiguous span of memory (x fastest), so one thread copies it with a single
//     cp.async.bulk into a ring slot (the span is widened to 16-byte boundaries;
//     node (x, row) sits at delta + row (N+1) + x, delta = the span's offset modulo
//     4 floats); cell planes (rows y0-1 .. y0+TYT-1) and, for POST, the coarse
//     correction's planes are copied the same way; an mbarrier per ring slot counts
//     the bytes in;
//   * the operand plane is derived branch-free for every staged entry, boundary nodes
//     (and boundary values of the coarse correction) taken as 0 by a per-thread mask
//     whatever the staged vectors hold there, so the passes need no cleared
//     boundaries; they write the interior nodes and, branch-free, the nodes x = N and
//     y = N of a lane's window (as 0), never x = 0, y = 0 or the planes 0 and N;
//   * the derived operand plane has an even row stride N + 2, so a lane's window of
//     RX + 2 columns is read with 8-byte loads when RX = 2;
//   * all passes but RES sum the operator per operand plane: the window of plane
//     k + 1, read once, completes node plane k, adds the centre part of plane k + 1
//     and starts plane k + 2 (partial sums and the upper cell plane carried in
//     registers), so they need one block barrier per plane;
//   * the first APPLY of an inner solve may leave p unstored (p = z, out1 null) and
//     APPLYXL, the last APPLYX of an inner solve, stores no q (only p.q is needed).
// Partial sums (APPLY p.q, POST r.z, RES r.r) are formed per segment of kZSeg interior
// planes exactly as in tiled.cu (entry seg * by + tile_y per sample).
//
// PRE and PREU restrict their residual t = r - A x1 to the coarse grid N/2 in the same
// pass (t itself is never stored): rc(X, Y, Z) = sum over d in {-1, 0, 1}^3 of
// w(d_x) w(d_y) w(d_z) t(2X + d_x, 2Y + d_y, 2Z + d_z), w(0) = 1, w(+-1) = 1/2 (the
// transpose of trilinear interpolation).  A lane sums its rows over x with one shuffle,
// each warp combines its rows with the first row of the warp above (through shared
// memory, after the plane's last barrier), and the coarse planes are summed while
// marching in z.  A chunk computes t on one more plane than it owns (the first plane
// of the next chunk; nothing of it is stored) so that its last coarse plane is
// complete; the coarse row at the boundary of two row blocks takes exactly two atomic
// additions onto a zeroed row (k_zero_seams), so its value does not depend on their
// order.  Coarse boundary nodes are written 0.
//
// RES is the refinement step of the mixed solver in one pass: the operand is the inner
// solve's increment inc = d + alpha p, the stencil forms A inc to FP64 accuracy in
// FP32 arithmetic (exact cell-pair sums and FMA-split products, compensated sums), and
// each owned node updates the residual pair rr <- rr - A inc (rr = b before the first
// step), writes it rounded as the next inner solve's FP32 residual and updates the
// solution pair x (+)= inc.  Neither rr nor x is read at another block's nodes, so both
// are updated in place; the recursive residual equals b - A x up to the pair
// arithmetic's rounding (a few u^2 |A||x| per step, u = 2^-24).  The first step also
// writes x's boundary nodes (0) that the block's rows and planes own.
//
// Every wait on an mbarrier is bounded (about a second of SM clock); a wait that
// runs out sets *err, and the thread then skips its remaining waits and copies but
// still reaches every block barrier (its shared-memory work stays in bounds whatever
// the slots hold; its results are void), so the kernel ends and the host reads the
// flag.
#include <cstdio>

#include "internal.cuh"
#include "kernels.h"
#include "launch.h"

namespace mlsgd {

namespace {

// SL_APPLYXL: APPLYX as the inner solve's last pass, which needs p.q but not q
enum SlabMode { SL_APPLY = 0, SL_PRE = 1, SL_POST = 2, SL_PREU = 4, SL_APPLYX = 5, SL_RES = 6, SL_APPLYXL = 7 };
constexpr int kSegPlanes = 8;  // partial-sum segment (the same as tiled.cu's kZSeg)
// Raw plane slots: plane m of a chunk (j = m - (kbeg-1)) lives in slot j % 4 of the
// node vectors whose own-node values the epilogue reads, and in slot j % 3 of D^-1 in
// PRE and PREU (read only when deriving plane m, so three slots suffice: iteration k
// copies plane k + 3, whose D^-1 replaces that of plane k, derived one iteration
// earlier).  The shorter ring keeps PREU, which stages three node vectors, at three
// blocks per SM.
constexpr int kRing = 4;
constexpr int kAhead = 3;
constexpr int short_vec(int mode) { return mode == 1 ? 1 : (mode == 4 ? 2 : -1); }

struct SlabArgs {
  const float* in0;   // APPLY/APPLYX: z     PRE/PREU/POST: r
  const float* in1;   // APPLY/APPLYX: p_old PREU: q
  const float* dinv;  // PRE/PREU/POST: omega D^-1 (0 on the boundary)
  const float* ec;    // POST: coarse correction on grid N/2
  const void* a;      // cell coefficient (TA)
  float* out0;        // APPLY: q (not read by APPLYXL)   POST: z   RES: r32
  float* out1;        // APPLY: p_new (null on the first APPLY: p = z is not stored)   PREU: r_new
  float* x;           // APPLYX: solution updated with alpha_prev p_old
  double* partial;    // [S][by * nseg]
  const SolveScalars* sc;
  const int* act;
  int* err;           // set when a wait runs out
  int nzc, zc, nseg;
  int first, xfirst;
  float scale;
  // RES: the refinement step, see k_slab
  const SolveScalars* sci;  // inner solve's scalars (alpha of its last update)
  const float2* rr_in;      // residual pairs before the step (b on the first step)
  long long rr_stride;      // rr_in stride per sample (0: one shared vector)
  float2* rr_out;           // residual pairs after the step, [S][nodes]
  float2* xp;               // solution pairs, updated in place, [S][nodes]
  int assign, dzero;        // first step (x = inc); d never written (inc = alpha p)
  float* rc;                // PRE/PREU: the restricted residual on grid N/2, [S][(N/2+1)^3]
};

// ---- error-free FP32 arithmetic of the refinement step (RES)
// two_sum: s + e == a + b exactly (Knuth); a coefficient is an unevaluated pair (h, l)
struct P2 { float h, l; };
__device__ __forceinline__ P2 two_sum(float a, float b) {  // intrinsics: never contracted
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return P2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// (S, comp) += sgn (c.h + c.l) x for an FP32 operand x: the product c.h x is split
// exactly by the FMA, c.l x enters the compensation
template <bool NEG>
__device__ __forceinline__ void res_term(float& S, float& comp, P2 c, float x) {
  const float p = __fmul_rn(c.h, x);
  const float low = __fmaf_rn(c.l, x, __fmaf_rn(c.h, x, -p));
  const P2 t = two_sum(S, NEG ? -p : p);
  S = t.h;
  comp = __fadd_rn(comp, __fadd_rn(t.l, NEG ? -low : low));
}
// the same for a single FP32 coefficient c (a cell of the body diagonals)
template <bool NEG>
__device__ __forceinline__ void res_term1(float& S, float& comp, float c, float x) {
  const float p = __fmul_rn(c, x);
  const float low = __fmaf_rn(c, x, -p);
  const P2 t = two_sum(S, NEG ? -p : p);
  S = t.h;
  comp = __fadd_rn(comp, __fadd_rn(t.l, NEG ? -low : low));
}

template <int N>
struct SlabGeo {
  static constexpr int RX = N / 32;           // x nodes per lane
  static constexpr int RY = N == 64 ? 2 : 4;  // rows per warp
  static constexpr int TYT = 8 * RY;          // interior rows per block
  static constexpr int N1 = N + 1;
  static constexpr int NR = TYT + 2;          // staged node rows
  static constexpr int XS = N + 2;            // operand-plane row stride (even)
  static constexpr int RAWF = (NR * N1 + 3 + 3) / 4 * 4;  // raw node slab (floats), shift included
  static constexpr int XPL = NR * XS;         // operand plane (floats)
  static constexpr int CROWS = TYT + 1;       // staged cell rows
  static constexpr int NC = N / 2, NC1 = NC + 1;
  static constexpr int CNR = TYT / 2 + 2;     // staged coarse node rows
  static constexpr int CRAWF = (CNR * NC1 + 3 + 3) / 4 * 4;
  static constexpr int NE = (NR * N1 + 255) / 256;  // derived entries per thread
  static constexpr int NI = (NC1 * (CNR - 1) + 255) / 256;  // coarse interpolation items per thread
};

template <int N, typename TA, int MODE>
struct SlabSmem {
  using G = SlabGeo<N>;
  static constexpr int NV = (MODE == SL_PREU) ? 3 : 2;  // staged node vectors
  static constexpr bool kPost = MODE == SL_POST;
  static constexpr int SV = short_vec(MODE);             // the vector with a 3-slot ring (or -1)
  // RES reads its staged vectors only when deriving (its epilogue reads the operand
  // plane), so both of them take 3-slot rings
  static constexpr int slots(int v) { return (v == SV || MODE == SL_RES) ? kRing - 1 : kRing; }
  static constexpr int first_slot(int v) { return v == 0 ? 0 : first_slot(v - 1) + slots(v - 1); }
  static constexpr size_t raw = 0;
  static constexpr size_t cells = raw + sizeof(float) * first_slot(NV) * G::RAWF;
  static constexpr size_t cellb = (size_t)G::CROWS * N * sizeof(TA);  // one cell slab (a multiple of 16)
  static constexpr size_t craw = cells + kRing * cellb;
  static constexpr size_t xs = craw + (kPost ? sizeof(float) * 3 * G::CRAWF : 0);
  static constexpr size_t eps = xs + sizeof(float) * 3 * G::XPL;
  static constexpr size_t bar = eps + (kPost ? sizeof(float) * 2 * G::XPL : 0);
  // RES: x and the residual pairs rr_in of the thread's own nodes for the plane being
  // computed, copied ahead; APPLYX: x of the own nodes of the next plane
  static constexpr size_t xpre = (bar + 8 * kRing + 15) / 16 * 16;
  // PRE/PREU: the x-restricted first row of every warp, [plane parity][8 warps][32 lanes]
  static constexpr bool kRestr = MODE == SL_PRE || MODE == SL_PREU;
  static constexpr size_t hx =
      xpre + (MODE == SL_RES ? 2 * sizeof(float2) : (MODE == SL_APPLYX || MODE == SL_APPLYXL ? sizeof(float) : 0)) * 256 * G::RX * G::RY;
  static constexpr size_t total = hx + (kRestr ? sizeof(float) * 512 : 0);
  static_assert((sizeof(TA) == 4 && (MODE == SL_PREU || MODE == SL_POST)) || total + 1024 <= 228 * 1024 / 3,
                "three blocks per SM");
  static_assert(cells % 16 == 0 && craw % 16 == 0 && cellb % 16 == 0 && xs % 16 == 0 && bar % 8 == 0, "align");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// 8- and 4-byte asynchronous copies into shared memory (the thread waits for its own copies)
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait for phase `parity` of the barrier; false after about a second (the
// clock is read only when the first try finds the phase incomplete)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (clock64() - t0 > (2LL << 30)) return false;
  }
}

__device__ __forceinline__ float ld_cell(const float* c, int i) { return c[i]; }
__device__ __forceinline__ float ld_cell(const __nv_bfloat16* c, int i) { return __bfloat162float(c[i]); }
// two neighbouring cells from an 8-byte (FP32) or 4-byte (BF16) aligned address
__device__ __forceinline__ void ld_cell_pair(const float* c, float& a, float& b) {
  const float2 v = *reinterpret_cast<const float2*>(c);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ld_cell_pair(const __nv_bfloat16* c, float& a, float& b) {
  const uint32_t v = *reinterpret_cast<const uint32_t*>(c);
  a = __uint_as_float(v << 16);           // BF16 is the upper half of an FP32
  b = __uint_as_float(v & 0xffff0000u);
}

template <int N, typename TA, int MODE>
__global__ void __launch_bounds__(256, 3) k_slab(SlabArgs A) {
  using G = SlabGeo<N>;
  using L = SlabSmem<N, TA, MODE>;
  constexpr int RX = G::RX, RY = G::RY, TYT = G::TYT, N1 = G::N1, NR = G::NR, XS = G::XS;
  constexpr bool kX = MODE == SL_APPLYX || MODE == SL_APPLYXL;  // APPLY with the x update
  constexpr bool kApply = MODE == SL_APPLY || kX;
  constexpr bool kPost = MODE == SL_POST;
  constexpr bool kRes = MODE == SL_RES;
  constexpr int NV = L::NV;
  static_assert(N1 % 4 == 1 && G::NC1 % 4 == 1, "shift arithmetic assumes N + 1 = 1 mod 4");
  extern __shared__ __align__(16) unsigned char sm[];
  float* raw = (float*)(sm + L::raw);  // vector v, plane j: slot L::first_slot(v) + j % L::slots(v)
  TA* cs = (TA*)(sm + L::cells);       // [kRing][CROWS * N]
  float* craw = (float*)(sm + L::craw);  // [3][CRAWF]
  float* xs = (float*)(sm + L::xs);    // [3][XPL]
  float* eps = (float*)(sm + L::eps);  // [2][XPL]
  float2* xpre = (float2*)(sm + L::xpre) + threadIdx.x * (G::RX * G::RY);  // RES: this thread's nodes
  float2* rpre = (float2*)(sm + L::xpre) + (256 + threadIdx.x) * (G::RX * G::RY);  // RES: rr_in of them
  float* xq = (float*)(sm + L::xpre) + threadIdx.x * (G::RX * G::RY);    // APPLYX: this thread's nodes
  float* hx = (float*)(sm + L::hx);  // PRE/PREU: [plane parity][warp][lane]
  const uint32_t bar0 = smem_u32(sm + L::bar);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int chunk = blockIdx.z % A.nzc;
  const int s = A.act != nullptr ? A.act[blockIdx.z / A.nzc] : (int)(blockIdx.z / A.nzc);
  const int y0 = 1 + TYT * blockIdx.y;  // first interior row of the block
  const int kbeg = 1 + chunk * A.zc;
  const int kend0 = min(N - 1, kbeg + A.zc - 1);  // the chunk's last plane
  // PRE/PREU compute one more plane for the restriction (kend0 is even unless it is N-1)
  const int kend = (L::kRestr && kend0 < N - 1) ? kend0 + 1 : kend0;
  constexpr long long kNodes = (long long)N1 * N1 * N1;
  // RES, first step: the block also owns the boundary nodes of its rows and planes
  // (column x = 0; row 0 for the first row block; planes 0 and N for the first and
  // last z chunk), whose solution is 0
  const int rlo = blockIdx.y == 0 ? 0 : y0, rhi = min(N, y0 + TYT - 1);
  const int kl = kbeg == 1 ? 0 : kbeg, kh = kend == N - 1 ? N : kend;
  if (A.sc != nullptr && !A.sc[s].active) {
    if (kRes && A.assign) {  // a sample that takes no step: its solution is 0 (every owned node)
      float2* xo = A.xp + s * kNodes;
      const int per = (rhi - rlo + 1) * N1;
      for (int k = kl; k <= kh; ++k)
        for (int e = tid; e < per; e += 256)
          xo[(long long)k * N1 * N1 + (long long)(rlo + e / N1) * N1 + e % N1] = make_float2(0.f, 0.f);
    }
    return;
  }
  if (kRes && A.assign) {  // row 0 and planes 0, N here; column x = 0 in the epilogue
    float2* xo = A.xp + s * kNodes;
    if (rlo == 0)
      for (int e = tid; e < (kend - kbeg + 1) * N1; e += 256)
        xo[(long long)(kbeg + e / N1) * N1 * N1 + e % N1] = make_float2(0.f, 0.f);
    const int per = (rhi - rlo + 1) * N1;
    if (kl == 0)
      for (int e = tid; e < per; e += 256) xo[rlo * N1 + e] = make_float2(0.f, 0.f);
    if (kh == N)
      for (int e = tid; e < per; e += 256) xo[(long long)N * N1 * N1 + rlo * N1 + e] = make_float2(0.f, 0.f);
  }
  if (*(volatile int*)A.err != 0) return;  // an earlier wait ran out: the results are void anyway
  constexpr long long kCells = (long long)N * N * N;
  constexpr long long kCNodes = (long long)G::NC1 * G::NC1 * G::NC1;
  // node rows y0-1 .. y0+TYT and cell rows y0-1 .. y0+TYT-1 that exist
  const int rows = min(NR, N + 2 - y0);
  const int crows = min(G::CROWS, N + 1 - y0);
  const int cy0 = (y0 - 1) >> 1;  // first staged coarse row
  const int crows_c = min(G::CNR, G::NC1 - cy0);
  const float scale = A.scale;
  float beta = 0.f, alpha = 0.f;
  if (kApply && !A.first) beta = (float)A.sc[s].beta;
  if (kX || MODE == SL_PREU) alpha = (float)A.sc[s].alpha;
  if (kRes) alpha = (float)A.sci[s].alpha;
  auto vin = [&](int v) {
    return v == 0 ? A.in0 : (v == 1 && (MODE == SL_PREU || kApply || kRes) ? A.in1 : A.dinv);
  };
  bool dead = false;  // a wait of this thread ran out: skip the remaining waits and copies

  // ---- producers (threads 0 and 32): plane m into ring slot (m - first) % kRing
  const int first = kbeg - 1;
  // The node vectors by thread 0 (PREU on 64^3: the first one; its other two by thread
  // 64), the cells and coarse planes by thread 32; the APPLY passes on 32^3: all by
  // thread 0 (splitting them there, or more ways in the other passes, costs register
  // spills)
  constexpr bool kSplit = N == 64 || !kApply, kSplit3 = N == 64 && MODE == SL_PREU;
  auto producer = [&] { return tid == 0 || (kSplit && tid == 32) || (kSplit3 && tid == 64); };
  auto span = [&](long long off, int len, int& delta) {  // 16-byte aligned span covering [off, off + len)
    delta = (int)(off & 3);
    return (uint32_t)(4 * ((delta + len + 3) & ~3));
  };
  auto issue = [&](int m, bool extra_coarse) {
    const int j = m - first, slot = j % kRing;
    const uint32_t bar = bar0 + 8 * slot;
    const long long noff = (long long)s * kNodes + (long long)m * N1 * N1 + (long long)(y0 - 1) * N1;
    int d;
    const uint32_t nb = span(noff, rows * N1, d);
    const bool cell = m < N;
    const uint32_t cb = cell ? (uint32_t)(crows * N * sizeof(TA)) : 0u;
    const int nv = ((kApply && A.first) || (kRes && A.dzero)) ? 1 : NV;  // the first APPLY reads no old p
    uint32_t total = nv * nb + cb;
    // POST: coarse plane m/2 + 1 with every even fine plane (interpolated in derive(m)),
    // plane (kbeg-1)/2 as well with the first plane of the chunk
    const bool c0 = kPost && extra_coarse, c1 = kPost && !(m & 1) && (m >> 1) + 1 <= G::NC;
    const long long cbase = (long long)s * kCNodes + (long long)cy0 * G::NC1;
    const long long coff0 = cbase + (long long)(m >> 1) * G::NC1 * G::NC1;
    const long long coff1 = coff0 + (long long)G::NC1 * G::NC1;
    int dc;
    const uint32_t cb0 = c0 ? span(coff0, crows_c * G::NC1, dc) : 0u;  // spans differ with the offset mod 4
    const uint32_t cb1 = c1 ? span(coff1, crows_c * G::NC1, dc) : 0u;
    total += cb0 + cb1;
    if (!kSplit || tid == 0) {  // the byte count and the node vectors (PREU on 64^3: the first)
      mbar_expect(bar, total);
#pragma unroll
      for (int v = 0; v < (kSplit3 ? 1 : NV); ++v)
        if (v < nv)
          bulk_copy(smem_u32(raw + (L::first_slot(v) + j % L::slots(v)) * G::RAWF), vin(v) + (noff & ~3LL), nb, bar);
    }
    if constexpr (kSplit3) {
      if (tid == 64) {  // PREU on 64^3: q and omega D^-1
#pragma unroll
        for (int v = 1; v < NV; ++v)
          bulk_copy(smem_u32(raw + (L::first_slot(v) + j % L::slots(v)) * G::RAWF), vin(v) + (noff & ~3LL), nb, bar);
      }
    }
    if (!kSplit || tid == 32) {  // thread 32 (warp 1 derives no entry of the partial last round): cells, coarse
      if (cell) {
        const long long coff_c = (long long)s * kCells + (long long)m * N * N + (long long)(y0 - 1) * N;
        bulk_copy(smem_u32((unsigned char*)cs + slot * L::cellb), (const TA*)A.a + coff_c, cb, bar);
      }
      if (c0) bulk_copy(smem_u32(craw + ((m >> 1) % 3) * G::CRAWF), A.ec + (coff0 & ~3LL), cb0, bar);
      if (c1) bulk_copy(smem_u32(craw + (((m >> 1) + 1) % 3) * G::CRAWF), A.ec + (coff1 & ~3LL), cb1, bar);
    }
  };
  auto wait_plane = [&](int m) {
    const int j = m - first;
    if (!dead && !mbar_wait(bar0 + 8 * (j % kRing), (uint32_t)((j / kRing) & 1))) {
      dead = true;
      atomicOr(A.err, 1);
    }
  };
  // offset modulo 4 of node (0, y0-1, m) of sample s: N+1, (N+1)^2 and (N+1)^3 are 1 mod 4
  auto delta_of = [&](int m) { return (s + m + y0 - 1) & 3; };

  // ---- entries this thread derives: e = tid + 256 j, in the last, partial round
  // 256 j + 255 - tid (so that the last warps, not warp 0, which issues the copies, take
  // them); operand index e + e / N1 (stride N + 2)
  auto entry = [&](int j) { return j == G::NE - 1 ? 256 * j + 255 - tid : tid + 256 * j; };
  auto item = [&](int j) { return j == G::NI - 1 ? 256 * j + 255 - tid : tid + 256 * j; };
  // bnd bit j: entry j is a boundary node (x or y on the boundary; the planes 0 and N
  // are handled per plane), derived as 0 whatever the staged vector holds there
  int xo[G::NE];
  unsigned bnd = 0;
#pragma unroll
  for (int j = 0; j < G::NE; ++j) {
    const int e = entry(j);
    const int ly = e / N1, x = e - ly * N1, y = y0 - 1 + ly;
    xo[j] = e + ly;
    if (x == 0 || x == N || y == 0 || y >= N) bnd |= 1u << j;
  }
  // the same for the coarse interpolation items (a, b): bit 4j + (p + 2q) for coarse
  // node (a + p, cy0 + b + q) on the coarse boundary
  unsigned cbnd = 0;
  int ioff[G::NI];  // interpolation item j: offset 2a + 2b (N + 2) of its fine node (2a, 2b)
  if (kPost) {
#pragma unroll
    for (int j = 0; j < G::NI; ++j) {
      const int it = item(j);
      const int a = it % G::NC1, b = it / G::NC1;
      ioff[j] = 2 * a + 2 * XS * b;
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int ca = a + p, cb = cy0 + b + q;
          if (ca == 0 || ca >= G::NC || cb == 0 || cb >= G::NC) cbnd |= 1u << (4 * j + p + 2 * q);
        }
    }
  }

  // POST: interpolate staged coarse plane c (xy-bilinear) into eps[c & 1]: item
  // (a, b) of the coarse tile writes fine nodes (2a + p, 2b + q)
  // (coarse boundary values are taken as 0 whatever the staged vector holds there)
  // Every load stays inside the staged slot (its last item a = NC reads one value past
  // the row, still inside the slot), and the item a = NC writes column N + 1 of the
  // row, the padding of the even row stride; only items past the tile are skipped.
  auto interp = [&](int c) {
    const float* cp = craw + (c % 3) * G::CRAWF + ((s + c + cy0) & 3);
    float* ed = eps + (c & 1) * G::XPL;
    const unsigned all = (c == 0 || c == G::NC) ? ~0u : cbnd;
#pragma unroll
    for (int j = 0; j < G::NI; ++j) {
      const int it = item(j);
      if (j == G::NI - 1 && it >= G::NC1 * (G::CNR - 1)) break;
      const float* q = cp + it;  // coarse node (a, b) of item it = a + (N/2 + 1) b
      const unsigned mk = all >> (4 * j);
      const float e00 = (mk & 1u) ? 0.f : q[0], e10 = (mk & 2u) ? 0.f : q[1];
      const float e01 = (mk & 4u) ? 0.f : q[G::NC1], e11 = (mk & 8u) ? 0.f : q[G::NC1 + 1];
      float* o = ed + ioff[j];
      const float r0 = 0.5f * (e00 + e10), r1 = 0.5f * (e01 + e11);
      o[0] = e00;
      o[1] = r0;
      o[XS] = 0.5f * (e00 + e01);
      o[XS + 1] = 0.5f * (r0 + r1);
    }
  };

  // derive operand plane m into operand slot x3 = m % 3 (j3 = (m - first) % 3: the
  // slot of m in a 3-slot ring)
  auto raw_of = [&](int v, int m, int j3) {
    const int j = m - first;
    return raw + (L::first_slot(v) + (L::slots(v) == kRing ? (j & (kRing - 1)) : j3)) * G::RAWF + delta_of(m);
  };
  auto derive = [&](int m, int x3, int j3, bool interp_next) {
    const float* r0 = raw_of(0, m, j3);
    const float* r1 = raw_of(1, m, j3);
    const float* r2 = raw_of(NV - 1, m, j3);
    float* xp = xs + x3 * G::XPL;
    if (kPost && interp_next && !(m & 1) && (m >> 1) + 1 <= G::NC) interp((m >> 1) + 1);
    const float* e0 = eps + ((m >> 1) & 1) * G::XPL;
    const float* e1 = eps + (((m + 1) >> 1) & 1) * G::XPL;
    const unsigned mask = (m == 0 || m == N) ? ~0u : bnd;  // boundary entries of this plane
    auto each = [&](auto f) {
#pragma unroll
      for (int j = 0; j < G::NE; ++j) {
        const int e = entry(j);
        if (j == G::NE - 1 && e >= NR * N1) break;
        const float v = f(e, xo[j]);
        xp[xo[j]] = ((mask >> j) & 1u) ? 0.f : v;
      }
    };
    if (kApply) {
      if (A.first) each([&](int e, int) { return r0[e]; });
      else each([&](int e, int) { return fmaf(beta, r1[e], r0[e]); });
    } else if (kRes) {  // the inner solve's increment d + alpha p (alpha p when d is 0)
      if (A.dzero) each([&](int e, int) { return alpha * r0[e]; });
      else each([&](int e, int) { return fmaf(alpha, r1[e], r0[e]); });
    } else if (MODE == SL_PREU) {
      each([&](int e, int) { return fmaf(-alpha, r1[e], r0[e]) * r2[e]; });
    } else if (kPost) {  // coarse correction: one interpolated coarse plane (m even) or the mean of two
      if (m & 1) each([&](int e, int x) { return fmaf(r0[e], r1[e], 0.5f * (e0[x] + e1[x])); });
      else each([&](int e, int x) { return fmaf(r0[e], r1[e], e0[x]); });
    } else {
      each([&](int e, int) { return r0[e] * r1[e]; });
    }
  };

  // ---- prologue
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < kRing; ++q) mbar_init(bar0 + 8 * q);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  // planes first .. first+2 now, first+3 once the prologue has derived plane first
  // (whose D^-1 slot it may reuse); iteration k then copies plane k+3 into the slots of
  // plane k-1 (raw k-1 was last read by compute(k-1), its cells by compute(k))
  if (producer())
    for (int m = first; m <= min(first + kAhead - 1, kend + 1); ++m) issue(m, kPost && m == first);
  wait_plane(first);
  if (kPost) {
    interp(first >> 1);
    interp((first >> 1) + 1);
    __syncthreads();
  }
  // rotating slots of plane k: xk = k % 3 (operand ring), jk3 = (k - first) % 3
  int xk = kbeg % 3, jk3 = 1;
  const int xfirst3 = xk == 0 ? 2 : xk - 1;
  derive(first, xfirst3, 0, false);
  wait_plane(kbeg);
  derive(kbeg, xk, 1, false);
  __syncthreads();
  if (producer() && !dead && first + kAhead <= kend + 1) issue(first + kAhead, false);

  // ---- this thread's nodes: x = 1 + RX lane + i, rows y = y0 + RY warp + t
  const int ly0 = RY * warp;                // staged row of the window's first row
  const int xw = RX * lane;                 // window's first column
  const int own0 = (ly0 + 1) * N1 + xw + 1;  // raw index of node (i = 0, t = 0) without the shift
  const int cwin = ly0 * N + xw;             // cell slab index of the window's first cell
  float* out0 = L::kRestr ? nullptr : A.out0 + s * kNodes;
  // APPLY with out1 null: the first p equals z and is not stored (the caller reads z)
  float* out1 = ((kApply || MODE == SL_PREU) && A.out1 != nullptr) ? A.out1 + s * kNodes : nullptr;
  float* xg = kX ? A.x + s * kNodes : nullptr;
  // bit t RX + i: node (i, t) is interior (the others, x = N or y = N, are written 0)
  unsigned okb = 0;
#pragma unroll
  for (int t = 0; t < RY; ++t)
#pragma unroll
    for (int i = 0; i < RX; ++i)
      if (xw + 1 + i <= N - 1 && y0 + ly0 + t <= N - 1) okb |= 1u << (t * RX + i);
  const long long gown = (long long)(y0 + ly0) * N1 + xw + 1;  // node (i = 0, t = 0) of plane 0
  float red = 0.f;

  // ---- restriction (PRE/PREU): coarse column cx of the lane (RX = 1: odd lanes only),
  // the warp's coarse rows (y0 + RY warp + 2c + 1) / 2 and, warp 0, row (y0 - 1) / 2
  float zacc[RY / 2], zlow = 0.f;
#pragma unroll
  for (int c = 0; c < RY / 2; ++c) zacc[c] = 0.f;
  const int cx = RX == 2 ? lane + 1 : (lane + 1) >> 1;
  const bool has_cx = RX == 2 || (lane & 1);
  // coarse plane Zc of the block's rows: interior nodes stored (the row shared with
  // the neighbouring row block by atomic addition onto its zeroed value), boundary
  // nodes 0; zero: the whole plane is a boundary plane
  auto store_coarse = [&](int Zc, bool zero) {
    float* rz = A.rc + s * (long long)G::NC1 * G::NC1 * G::NC1 + (long long)Zc * G::NC1 * G::NC1;
#pragma unroll
    for (int c = 0; c < RY / 2; ++c) {
      const int Yc = (y0 + RY * warp + 2 * c + 1) >> 1;
      if (Yc > G::NC) continue;
      float* o = rz + Yc * G::NC1;
      if (lane == 0) o[0] = 0.f;
      if (!has_cx) continue;
      if (zero || cx == G::NC || Yc == G::NC) o[cx] = 0.f;
      else if (c == RY / 2 - 1 && warp == 7 && blockIdx.y + 1 < gridDim.y) atomicAdd(o + cx, zacc[c]);
      else o[cx] = zacc[c];
    }
    if (warp == 0) {
      const int Yl = (y0 - 1) >> 1;
      float* o = rz + Yl * G::NC1;
      if (lane == 0) o[0] = 0.f;
      if (has_cx) {
        if (zero || Yl == 0 || cx == G::NC) o[cx] = 0.f;
        else atomicAdd(o + cx, zlow);
      }
    }
  };

  // ---- the operator as contributions of one operand plane p (all modes but RES): to
  // node plane p - 1 and p + 1 through the cell plane between them (off_term), to node
  // plane p through the cell planes below and above it (centre_term).  Node (i, t) has
  // cells Cx[i + p][t + q] of a cell plane and operand neighbour (du, dv) of a plane at
  // window (i + 1 + du, t + 1 + dv).
  using Win = float[RX + 2][RY + 2];
  using Cel = float[RX + 1][RY + 1];
  using Acc = float[RY][RX];
  auto load_cells = [&](int cpl, Cel& Cx) {  // cell plane cpl, cell (xw + cc, row ly0 + cr)
    const TA* cp = cs + ((cpl - first) & (kRing - 1)) * (L::cellb / sizeof(TA)) + cwin;
#pragma unroll
    for (int cr = 0; cr < RY + 1; ++cr) {
      if constexpr (RX == 2) {  // cells xw, xw+1 as one aligned pair (xw and N even), then xw+2
        ld_cell_pair(cp + cr * N, Cx[0][cr], Cx[1][cr]);
        Cx[2][cr] = ld_cell(cp, cr * N + 2);
      } else {
#pragma unroll
        for (int cc = 0; cc < RX + 1; ++cc) Cx[cc][cr] = ld_cell(cp, cr * N + cc);
      }
    }
  };
  auto load_win = [&](int x3, Win& W) {  // the lane's (RX+2) x (RY+2) window of operand slot x3
    const float* xp = xs + x3 * G::XPL + ly0 * XS + xw;
#pragma unroll
    for (int rr = 0; rr < RY + 2; ++rr) {
      if constexpr (RX == 2) {
        const float2 a0 = *reinterpret_cast<const float2*>(xp + rr * XS);
        const float2 a1 = *reinterpret_cast<const float2*>(xp + rr * XS + 2);
        W[0][rr] = a0.x;
        W[1][rr] = a0.y;
        W[2][rr] = a1.x;
        W[3][rr] = a1.y;
      } else {
#pragma unroll
        for (int c = 0; c < RX + 2; ++c) W[c][rr] = xp[rr * XS + c];
      }
    }
  };
  auto off_term = [&](Acc& acc, const Win& W, const Cel& Cr) {
#pragma unroll
    for (int t = 0; t < RY; ++t)
#pragma unroll
      for (int i = 0; i < RX; ++i) {
        float a2 = acc[t][i];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          a2 -= (Cr[i + u][t] + Cr[i + u][t + 1]) * W[i + 2 * u][t + 1];  // xz face diagonals
          a2 -= (Cr[i][t + u] + Cr[i + 1][t + u]) * W[i + 1][t + 2 * u];  // yz face diagonals
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int p = 0; p < 2; ++p) a2 -= Cr[i + p][t + q] * W[i + 2 * p][t + 2 * q];  // body diagonals
        acc[t][i] = a2;
      }
  };
  auto centre_term = [&](Acc& acc, const Win& W, const Cel& Cl, const Cel& Ch) {
#pragma unroll
    for (int t = 0; t < RY; ++t)
#pragma unroll
      for (int i = 0; i < RX; ++i) {
        float pxy[2][2];  // in-plane face diagonals: pair sums over the two cell planes
#pragma unroll
        for (int v = 0; v < 2; ++v)
#pragma unroll
          for (int u = 0; u < 2; ++u) pxy[v][u] = Cl[i + u][t + v] + Ch[i + u][t + v];
        const float sum8 = (pxy[0][0] + pxy[0][1]) + (pxy[1][0] + pxy[1][1]);
        float a1 = fmaf(4.f * sum8, W[i + 1][t + 1], acc[t][i]);
#pragma unroll
        for (int v = 0; v < 2; ++v)
#pragma unroll
          for (int u = 0; u < 2; ++u) a1 -= pxy[v][u] * W[i + 2 * u][t + 2 * v];
        acc[t][i] = a1;
      }
  };
  // node planes k and k + 1 summed so far (below, then centre) and the operand of node
  // plane k at the own nodes, entering iteration k
  float accB[RY][RX], accC[RY][RX], ctrk[RY][RX];
  float Cn[RX + 1][RY + 1];  // cell plane k, loaded as the upper plane of iteration k - 1
  if constexpr (!kRes) {
    float W[RX + 2][RY + 2], Cl[RX + 1][RY + 1], Ch[RX + 1][RY + 1];
#pragma unroll
    for (int t = 0; t < RY; ++t)
#pragma unroll
      for (int i = 0; i < RX; ++i) accB[t][i] = accC[t][i] = 0.f;
    load_cells(first, Cl);
    load_cells(kbeg, Ch);
    load_win(xfirst3, W);
    off_term(accB, W, Cl);
    load_win(xk, W);
    centre_term(accB, W, Cl, Ch);
#pragma unroll
    for (int t = 0; t < RY; ++t)
#pragma unroll
      for (int i = 0; i < RX; ++i) ctrk[t][i] = W[i + 1][t + 1];
    off_term(accC, W, Ch);
#pragma unroll
    for (int c = 0; c < RX + 1; ++c)
#pragma unroll
      for (int r = 0; r < RY + 1; ++r) Cn[c][r] = Ch[c][r];
  }
  float ux[RY];  // PRE/PREU: x-restricted rows of the last computed plane
  // PRE/PREU: the coarse rows of this warp from plane k (fine rows t = 1, 3, .. of the
  // warp, the last one with the first row of the warp above) and, warp 0, row y0 for
  // coarse row (y0-1)/2; called after the barrier that follows plane k's epilogue
  auto restrict_plane = [&](int k) {
    const float hn = warp < 7 ? hx[(k & 1) * 256 + (warp + 1) * 32 + lane] : 0.f;
    float sv[RY / 2];
#pragma unroll
    for (int c = 0; c < RY / 2; ++c) sv[c] = fmaf(0.5f, ux[2 * c] + (2 * c + 2 < RY ? ux[2 * c + 2] : hn), ux[2 * c + 1]);
    const float sl = 0.5f * ux[0];
    if (k & 1) {  // plane k completes coarse plane (k-1)/2 (half weight) and starts (k+1)/2
#pragma unroll
      for (int c = 0; c < RY / 2; ++c) zacc[c] = fmaf(0.5f, sv[c], zacc[c]);
      zlow = fmaf(0.5f, sl, zlow);
      if (k > kbeg) store_coarse((k - 1) >> 1, false);
      else if (k == 1) store_coarse(0, true);
#pragma unroll
      for (int c = 0; c < RY / 2; ++c) zacc[c] = 0.5f * sv[c];
      zlow = 0.5f * sl;
      if (k == N - 1) store_coarse(G::NC, true);
    } else {
#pragma unroll
      for (int c = 0; c < RY / 2; ++c) zacc[c] += sv[c];
      zlow += sl;
    }
  };

  // APPLYX: x of the own interior nodes of plane m into xq, a plane ahead of its use
  // (the epilogue of plane m - 1 issues it after its last use of xq)
  auto prefetch_x = [&](int m) {
    const float* xm = xg + (long long)m * N1 * N1 + gown;
#pragma unroll
    for (int t = 0; t < RY; ++t)
#pragma unroll
      for (int i = 0; i < RX; ++i)
        if ((okb >> (t * RX + i)) & 1u) cp_async4(xq + t * RX + i, xm + t * N1 + i);
    cp_async_commit();
  };
  if (kX && !A.xfirst) prefetch_x(kbeg);
  // RES: x and rr_in of the own nodes of plane m into xpre, rpre, a plane ahead of their use
  auto prefetch_res = [&](int m) {
    const long long gm = (long long)m * N1 * N1 + gown;
    const float2* xs_g = A.xp + s * kNodes + gm;
    const float2* rr_g = A.rr_in + s * A.rr_stride + gm;
#pragma unroll
    for (int t = 0; t < RY; ++t)
#pragma unroll
      for (int i = 0; i < RX; ++i) {
        if (!A.assign) cp_async8(xpre + t * RX + i, xs_g + t * N1 + i);
        if ((okb >> (t * RX + i)) & 1u) cp_async8(rpre + t * RX + i, rr_g + t * N1 + i);
      }
    cp_async_commit();
  };
  if constexpr (kRes) prefetch_res(kbeg);

  for (int k = kbeg; k <= kend; ++k) {
    const long long gk = (long long)k * N1 * N1 + gown;
    const int xkp = xk == 2 ? 0 : xk + 1, xkm = xk == 0 ? 2 : xk - 1;
    const int jk3p = jk3 == 2 ? 0 : jk3 + 1;
    float tv[RY][RX];  // PRE/PREU: t of the own nodes
    if (k + 1 <= kend + 1) {
      wait_plane(k + 1);
      derive(k + 1, xkp, jk3p, true);
    }
    __syncthreads();
    // One barrier per plane for all modes but RES: compute(k) reads only operand plane
    // k + 1 (derived before this barrier; derive(k+2) overwrites plane k - 1, last read
    // by compute(k-2)) and cell planes k, k + 1, so plane k + 3 is copied now into the
    // slots of plane k - 1 (raw k - 1 was last read by compute(k-1), its cells too; a
    // 3-slot vector ring reuses the slot of plane k, last read by derive(k)).
    if constexpr (!kRes) {
      if (L::kRestr && k > kbeg) restrict_plane(k - 1);
      if (producer() && !dead && k + kAhead <= kend + 1) issue(k + kAhead, false);
    }
    {
      // RES: rr_new = rr - A inc to FP64 accuracy in FP32 arithmetic (exact cell-pair
      // sums and products, compensated sums, the scale h/12 and the subtraction as
      // pairs), r = rr_new rounded, x (+)= inc; node plane k from the windows of operand
      // planes k (first), k - 1 and k + 1 (the pair accumulators leave no registers to
      // carry partial sums from plane to plane)
      if constexpr (kRes) {
        // cells of the two cell planes around plane k: C[r][cc][cr], cell (xw + cc, row ly0 + cr)
        float C[2][RX + 1][RY + 1];
        load_cells(k - 1, C[0]);
        load_cells(k, C[1]);
        float Sa[RY][RX], Ca[RY][RX], ctr[RY][RX];
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
          const int order = pl == 0 ? 1 : (pl == 1 ? 0 : 2);  // centre plane first
          float W[RX + 2][RY + 2];
          load_win(order == 0 ? xkm : (order == 1 ? xk : xkp), W);
#pragma unroll
          for (int t = 0; t < RY; ++t)
#pragma unroll
            for (int i = 0; i < RX; ++i) {
              if (order == 1) {
                P2 pxy[2][2];
#pragma unroll
                for (int v = 0; v < 2; ++v)
#pragma unroll
                  for (int u = 0; u < 2; ++u) pxy[v][u] = two_sum(C[0][i + u][t + v], C[1][i + u][t + v]);
                float S8 = pxy[0][0].h, E8 = pxy[0][0].l;  // the first pair enters exactly
#pragma unroll
                for (int v = 0; v < 2; ++v)
#pragma unroll
                  for (int u = 0; u < 2; ++u) {
                    if (v == 0 && u == 0) continue;
                    const P2 q = two_sum(S8, pxy[v][u].h);
                    S8 = q.h;
                    E8 += q.l + pxy[v][u].l;
                  }
                ctr[t][i] = W[i + 1][t + 1];
                // the centre term starts the sum: its exact product split is (S, cmp)
                const float c8h = 4.f * S8, c8l = 4.f * E8;
                float S = __fmul_rn(c8h, W[i + 1][t + 1]);
                float cmp = __fmaf_rn(c8l, W[i + 1][t + 1], __fmaf_rn(c8h, W[i + 1][t + 1], -S));
#pragma unroll
                for (int v = 0; v < 2; ++v)
#pragma unroll
                  for (int u = 0; u < 2; ++u) res_term<true>(S, cmp, pxy[v][u], W[i + 2 * u][t + 2 * v]);
                Sa[t][i] = S;
                Ca[t][i] = cmp;
              } else {
                const int r = order >> 1;
                float S = Sa[t][i], cmp = Ca[t][i];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                  res_term<true>(S, cmp, two_sum(C[r][i + u][t], C[r][i + u][t + 1]), W[i + 2 * u][t + 1]);
                  res_term<true>(S, cmp, two_sum(C[r][i][t + u], C[r][i + 1][t + u]), W[i + 1][t + 2 * u]);
                }
#pragma unroll
                for (int q = 0; q < 2; ++q)
#pragma unroll
                  for (int p = 0; p < 2; ++p) res_term1<true>(S, cmp, C[r][i + p][t + q], W[i + 2 * p][t + 2 * q]);
                Sa[t][i] = S;
                Ca[t][i] = cmp;
              }
            }
        }
        constexpr double kH12 = 1.0 / (12.0 * N);
        const float sch = (float)kH12, scl = (float)(kH12 - (double)(float)kH12);  // h/12 as an FP32 pair

        float2* rro = A.rr_out + s * kNodes;
        float2* xo = A.xp + s * kNodes;
        cp_async_wait_all();
#pragma unroll
        for (int t = 0; t < RY; ++t) {
#pragma unroll
          for (int i = 0; i < RX; ++i) {
            const bool ok = (okb >> (t * RX + i)) & 1u;
            const long long g = gk + t * N1 + i;
            const P2 axs = two_sum(Sa[t][i], Ca[t][i]);
            const float pp = __fmul_rn(axs.h, sch);  // (A inc) as a pair (pp, pe)
            const float pe = __fmaf_rn(axs.h, scl, __fmaf_rn(axs.l, sch, __fmaf_rn(axs.h, sch, -pp)));
            const float2 bv = ok ? rpre[t * RX + i] : make_float2(0.f, 0.f);
            const P2 dd = two_sum(bv.x, -pp);
            const float e = dd.l + (bv.y - pe);
            const float rh = dd.h + e;  // renormalised pair (rh, rl)
            const float rl = e - (rh - dd.h);
            const float rv = ok ? rh : 0.f;
            out0[g] = rv;  // the next inner solve's FP32 residual
            rro[g] = ok ? make_float2(rh, rl) : make_float2(0.f, 0.f);
            red = fmaf(rv, rv, red);
            const float inc = ctr[t][i];  // 0 off the interior
            float2 xn = make_float2(inc, 0.f);
            if (!A.assign) {  // pair addition: two-sum of the head and inc, renormalised
              const float2 xv = xpre[t * RX + i];
              const float sh = xv.x + inc;
              const float bb = sh - xv.x;
              const float se = (xv.x - (sh - bb)) + (inc - bb);
              const float lo = xv.y + se;
              const float h = sh + lo;
              xn = make_float2(h, lo - (h - sh));
            }
            xo[g] = ok ? xn : make_float2(0.f, 0.f);
          }
          if (A.assign && lane == 0) xo[gk + t * N1 - 1] = make_float2(0.f, 0.f);  // column x = 0
        }
        if (k < kend) prefetch_res(k + 1);  // after the last use of xpre and rpre
      } else {
      // operand plane k + 1: completes node plane k (with cell plane k), adds the centre
      // part of node plane k + 1 and starts node plane k + 2 (with cell plane k + 1)
      float W[RX + 2][RY + 2];
      const Cel& Cl = Cn;
      load_win(xkp, W);
      off_term(accB, W, Cl);
      const Acc& acc = accB;
      const Acc& ctr = ctrk;
      float xv[RY][RX];  // APPLYX: x of the own nodes (0 where not interior or not read)
      if constexpr (kX) {
        if (!A.xfirst) cp_async_wait_all();
#pragma unroll
        for (int t = 0; t < RY; ++t)
#pragma unroll
          for (int i = 0; i < RX; ++i) xv[t][i] = (!A.xfirst && ((okb >> (t * RX + i)) & 1u)) ? xq[t * RX + i] : 0.f;
      }
      // every node of the window is written (nodes x = N or y = N with 0), so the
      // stores and the partial sum are branch-free
      const float* o0 = raw_of(0, k, jk3) + own0;
      const float* o1 = raw_of(1, k, jk3) + own0;
#pragma unroll
      for (int t = 0; t < RY; ++t) {
#pragma unroll
        for (int i = 0; i < RX; ++i) {
          const bool ok = (okb >> (t * RX + i)) & 1u;
          const float ax = scale * acc[t][i];
          const int own = t * N1 + i;
          const long long g = gk + t * N1 + i;
          if (kApply) {
            const float pv = ctr[t][i];  // 0 off the interior (derived with the mask)
            const float qv = ok ? ax : 0.f;
            if (MODE != SL_APPLYXL) out0[g] = qv;
            if (kX || out1 != nullptr) out1[g] = pv;
            red = fmaf(pv, qv, red);
            if (kX) xg[g] = ok ? xv[t][i] + alpha * o1[own] : 0.f;
          } else if (MODE == SL_PRE) {
            tv[t][i] = ok ? o0[own] - ax : 0.f;
          } else if (MODE == SL_PREU) {
            const float rn = ok ? fmaf(-alpha, o1[own], o0[own]) : 0.f;
            tv[t][i] = ok ? rn - ax : 0.f;
            if (k <= kend0) out1[g] = rn;
          } else {  // POST
            const float rv = ok ? o0[own] : 0.f;
            const float zv = ok ? fmaf(fmaf(-scale, acc[t][i], rv), o1[own], ctr[t][i]) : 0.f;
            out0[g] = zv;
            red = fmaf(rv, zv, red);
          }
        }
      }
      if constexpr (kX) {  // after the stores that used this plane's xq
        if (!A.xfirst && k < kend) prefetch_x(k + 1);
      }
      if constexpr (L::kRestr) {  // x-restriction of the thread's rows at coarse column cx
#pragma unroll
        for (int t = 0; t < RY; ++t) {
          if constexpr (RX == 2) {  // fine x = 2 cx - 1, 2 cx (this lane), 2 cx + 1 (the next)
            const float nb = __shfl_down_sync(0xffffffffu, tv[t][0], 1);
            ux[t] = fmaf(0.5f, tv[t][0] + nb, tv[t][1]);
          } else {  // fine x = lane + 1 (= 2 cx on odd lanes)
            const float lo = __shfl_up_sync(0xffffffffu, tv[t][0], 1);
            const float hi = __shfl_down_sync(0xffffffffu, tv[t][0], 1);
            ux[t] = fmaf(0.5f, lo + hi, tv[t][0]);
          }
        }
        hx[(k & 1) * 256 + warp * 32 + lane] = ux[0];
      }
      if (k < kend) {
        float Ch[RX + 1][RY + 1];
        load_cells(k + 1, Ch);
        centre_term(accC, W, Cl, Ch);
#pragma unroll
        for (int t = 0; t < RY; ++t)
#pragma unroll
          for (int i = 0; i < RX; ++i) {
            accB[t][i] = accC[t][i];
            accC[t][i] = 0.f;
            ctrk[t][i] = W[i + 1][t + 1];
          }
        off_term(accC, W, Ch);
#pragma unroll
        for (int c = 0; c < RX + 1; ++c)
#pragma unroll
          for (int r = 0; r < RY + 1; ++r) Cn[c][r] = Ch[c][r];
      }
      }  // not RES
    }
    if ((kApply || kPost || kRes) && (k == kend || (k - 1) % kSegPlanes == kSegPlanes - 1)) {
      const float b = block_sum(red);
      if (tid == 0) {
        const int per = gridDim.y * A.nseg;
        A.partial[(long long)s * per + ((k - 1) / kSegPlanes) * gridDim.y + blockIdx.y] = (double)b;
      }
      red = 0.f;
    }
    if constexpr (kRes) {  // RES reads operand planes k-1 .. k+1: a second barrier
      __syncthreads();
      if (producer() && !dead && k + kAhead <= kend + 1) issue(k + kAhead, false);
    }
    xk = xkp;
    jk3 = jk3p;
  }
  if constexpr (L::kRestr) {
    __syncthreads();
    restrict_plane(kend);
  }
  // the last copies of the chunk have been waited for (every issued plane is derived)
}

}  // namespace

// ---------------------------------------------------------------- host side
bool slab_supported(int N) { return N == 32 || N == 64; }

TiledShape slab_shape(int N, int S, int zchunks) {
  TiledShape t;
  const int tyt = N == 64 ? 16 : 32;
  t.bx = 1;
  t.by = (N - 1 + tyt - 1) / tyt;
  const int nseg = (N - 1 + kSegPlanes - 1) / kSegPlanes;
  const long long base = (long long)t.by * S;
  int nzc = 1;
  if (zchunks > 0) nzc = zchunks < nseg ? zchunks : nseg;
  else
    while (base * nzc < 3 * 152 * 4 && 2 * nzc <= nseg) nzc *= 2;
  const int spc = (nseg + nzc - 1) / nzc;
  t.nzc = (nseg + spc - 1) / spc;
  t.zc = spc * kSegPlanes;
  t.nseg = nseg;
  t.blocks_per_sample = t.by * nseg;
  return t;
}

template <int N, typename TA, int MODE>
static void run_slab(const char* cls, double bytes, SlabArgs args, const Batch& bt, cudaStream_t st,
                     double ops = 0.0) {
  const TiledShape t = slab_shape(N, bt.S, bt.zchunks);
  args.nzc = t.nzc;
  args.zc = t.zc;
  args.nseg = t.nseg;
  args.act = bt.act;
  args.scale = (float)(1.0 / (12.0 * N));
  const size_t smem = SlabSmem<N, TA, MODE>::total;
  static bool smem_set = false;  // once per instantiation (capture-friendly)
  if (!smem_set) {
    cudaFuncSetAttribute(k_slab<N, TA, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_slab<N, TA, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    smem_set = true;
  }
  launch_flops(cls, bytes, ops, k_slab<N, TA, MODE>, dim3(1, t.by, (unsigned)(bt.n * t.nzc)), dim3(256), smem, st,
               args);
}

template <typename TA, int MODE>
static void dispatch(int N, const char* cls, double bytes, SlabArgs args, const Batch& bt, cudaStream_t st,
                     double ops = 0.0) {
  if (N == 64) run_slab<64, TA, MODE>(cls, bytes, args, bt, st, ops);
  else run_slab<32, TA, MODE>(cls, bytes, args, bt, st, ops);
}

static double sbytes(int N, int n, double vec, double coef, size_t ta) {
  return (double)n * (vec * (double)nodes_of(N) * 4 + coef * (double)cells_of(N) * ta);
}

void slab_apply(const float* z, const float* pold, float* pnew, const float* a, float* q, float* x, double* partial,
                const SolveScalars* sc, int N, const Batch& bt, bool first, bool with_x, bool x_first, cudaStream_t st) {
  SlabArgs A{};
  A.in0 = z; A.in1 = pold; A.a = a; A.out0 = q; A.out1 = pnew; A.x = x; A.partial = partial; A.sc = sc;
  A.err = bt.err;
  A.first = first ? 1 : 0;
  A.xfirst = x_first ? 1 : 0;
  if (with_x && q == nullptr)  // the last pass of an inner solve: q not stored
    dispatch<float, SL_APPLYXL>(N, "apply_f32", sbytes(N, bt.n, x_first ? 4 : 5, 1, 4), A, bt, st);
  else if (with_x)
    dispatch<float, SL_APPLYX>(N, "apply_f32", sbytes(N, bt.n, x_first ? 5 : 6, 1, 4), A, bt, st);
  else
    dispatch<float, SL_APPLY>(N, "apply_f32", sbytes(N, bt.n, (first ? 3 : 4) - (pnew ? 0 : 1), 1, 4), A, bt, st);
}

// FP32 operations per interior node of the refinement step as written (no sharing
// between nodes): 12 exact cell-pair sums (6 each), the 8-cell sum (21), the centre
// product that starts the sum (4), 12 compensated products with a pair coefficient (11
// each) and 8 with a single cell (10 each), the scaling and subtraction (16), r.r and the
// pair update of x (10)
constexpr double kResOpsPerNode = 12 * 6 + 21 + 4 + 12 * 11 + 8 * 10 + 16 + 10;

void slab_res(const float* d, const float* p, bool d_zero, const SolveScalars* sci, const float2* rr_in,
              long long rr_stride, float2* rr_out, float2* x, bool assign, const float* a, float* r32,
              double* partial, const SolveScalars* sco, int N, const Batch& bt, cudaStream_t st) {
  SlabArgs A{};
  A.in0 = d_zero ? p : d; A.in1 = p; A.a = a; A.out0 = r32; A.partial = partial; A.sc = sco; A.err = bt.err;
  A.sci = sci; A.rr_in = rr_in; A.rr_stride = rr_stride; A.rr_out = rr_out; A.xp = x;
  A.assign = assign ? 1 : 0;
  A.dzero = d_zero ? 1 : 0;
  const double nodes = (double)nodes_of(N);
  // d (unless 0), p, the cells; the residual pairs in (once when shared) and out, r; x in (unless
  // assigned) and out
  const double bytes = sbytes(N, bt.n, d_zero ? 1 : 2, 1, 4) + (rr_stride ? bt.n : 1) * nodes * 8 +
                       bt.n * nodes * (8 + 4 + (assign ? 8 : 16));
  dispatch<float, SL_RES>(N, "resid64", bytes, A, bt, st, (double)bt.n * (N - 1) * (N - 1) * (N - 1) * kResOpsPerNode);
}

// the coarse rows shared by two row blocks, 0 before the blocks add their parts
template <int N>
__global__ void __launch_bounds__(256) k_zero_seams(float* __restrict__ rc, const int* __restrict__ act,
                                                    const SolveScalars* __restrict__ sc) {
  using G = SlabGeo<N>;
  const int s = act != nullptr ? act[blockIdx.x] : (int)blockIdx.x;
  if (sc != nullptr && !sc[s].active) return;
  constexpr int kBy = (N - 1 + G::TYT - 1) / G::TYT;
  constexpr int kPer = (kBy - 1) * G::NC1 * G::NC1;  // (seam, Z, X)
  float* r = rc + s * (long long)G::NC1 * G::NC1 * G::NC1;
  for (int e = threadIdx.x; e < kPer; e += 256) {
    const int x = e % G::NC1, rest = e / G::NC1, z = rest % G::NC1, b = 1 + rest / G::NC1;
    r[(long long)z * G::NC1 * G::NC1 + (b * G::TYT / 2) * G::NC1 + x] = 0.f;
  }
}

template <typename TA>
void slab_pre(const float* r, const float* q, const TA* a, const float* dinv, float* rnew, float* rc,
              const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st) {
  SlabArgs A{};
  A.in0 = r; A.in1 = q; A.a = a; A.dinv = dinv; A.out1 = rnew; A.rc = rc; A.sc = sc; A.err = bt.err;
  if (N == 64) {  // four row blocks per sample (32^3: one)
    const double zb = (double)bt.n * 4.0 * 33 * 33 * 3;
    launch("seams", zb, k_zero_seams<64>, dim3((unsigned)bt.n), dim3(256), 0, st, rc, bt.act, sc);
  }
  // r (and q), omega D^-1 and the cells in; r_new (PREU) and the coarse residual out
  const double coarse = (double)bt.n * nodes_of(N / 2) * 4;
  if (q)
    dispatch<TA, SL_PREU>(N, "pre_f32", sbytes(N, bt.n, 4, 1, sizeof(TA)) + coarse, A, bt, st);
  else
    dispatch<TA, SL_PRE>(N, "pre_f32", sbytes(N, bt.n, 2, 1, sizeof(TA)) + coarse, A, bt, st);
}

template <typename TA>
void slab_post(const float* r, const TA* a, const float* dinv, const float* ec, float* z, double* partial,
               const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st) {
  SlabArgs A{};
  A.in0 = r; A.a = a; A.dinv = dinv; A.ec = ec; A.out0 = z; A.partial = partial; A.sc = sc; A.err = bt.err;
  dispatch<TA, SL_POST>(N, "post_f32", sbytes(N, bt.n, 3, 1, sizeof(TA)) + (double)bt.n * nodes_of(N / 2) * 4, A, bt,
                        st);
}

template void slab_pre<__nv_bfloat16>(const float*, const float*, const __nv_bfloat16*, const float*, float*, float*,
                                      const SolveScalars*, int, const Batch&, cudaStream_t);
template void slab_pre<float>(const float*, const float*, const float*, const float*, float*, float*,
                              const SolveScalars*, int, const Batch&, cudaStream_t);
template void slab_post<__nv_bfloat16>(const float*, const __nv_bfloat16*, const float*, const float*, float*,
                                       double*, const SolveScalars*, int, const Batch&, cudaStream_t);
template void slab_post<float>(const float*, const float*, const float*, const float*, float*, double*,
                               const SolveScalars*, int, const Batch&, cudaStream_t);

}  // namespace mlsgd
