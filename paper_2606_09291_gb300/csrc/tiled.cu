// tiled.cu - z-marching shared-memory kernels for the fine-grid passes of the
// solver (rows a4, a6) and for Phi / the adjoint right-hand side (row a5).
//
// Layout: a block of 32 x 8 threads owns a 32 x 8 RY tile of interior nodes (RY
// rows per thread: 4 for FP32 vectors, 2 for FP64; x0 = 1 + 32 bx, y0 = 1 + 8 RY by)
// and marches along z over a chunk of interior planes.  Each node plane of an
// input vector is staged once into shared memory with a one-node halo
// (34 x (8 RY + 2)), each cell plane with a two-cell halo (36 x (8 RY + 3), from an
// even x start), with cp.async into a five-plane ring that keeps two planes in
// flight ahead of the stencil; the operand planes derived from them (three
// planes) are kept in their own ring.  So every value is read from HBM about
// once per pass (halos come from L2) and there is no integer division in the
// index arithmetic.  Node (lx, ly) of the staged plane is the global node
// (x0 - 1 + lx, y0 - 1 + ly); its eight surrounding cells are the staged cells
// (lx + p, ly + q), p, q in {0, 1}, of two cell planes.
//
// Fused passes (FE operator A: see q1_row in internal.cuh; D = (h/3) sum_8 a, whose
// inverse is precomputed per coefficient hierarchy and staged like a vector):
//   APPLY : pn = z + beta p (pn = z on the first iteration); q = A pn;
//           writes p = pn, q; partial p.q
//   PRE   : x1 = omega D^{-1} r computed on the fly; t = r - A x1
//   POST  : x2 = omega D^{-1} r + P e_c on the fly;
//           z = x2 + omega D^{-1} (r - A x2); partial r.z
//   (omega D^{-1} is precomputed per coefficient hierarchy and staged like a vector)
//   RES64 : r = b - A x to FP64 accuracy in FP32 arithmetic: x and b are FP32 (hi, lo)
//           pairs (staged as 8-byte words), a is FP32; writes r rounded to FP32 and the
//           partial r.r
// The fused passes write only interior nodes and zero-fill boundary nodes at staging
// (like nodes outside the grid), so they never read a buffer's boundary values.
#include <cstdio>
#include <type_traits>

#include "internal.cuh"
#include "kernels.h"
#include "launch.h"

namespace mlsgd {

constexpr int TX = 32, TY = 8;
constexpr int NPX = TX + 2;                     // staged node row: 34 nodes
constexpr int NPY = TY + 2, NP = NPX * NPY;      // the Phi kernels' staged plane (one row per thread): 34 x 10
constexpr int NT = TX * TY;

enum TiledMode { TM_APPLY = 0, TM_PRE = 1, TM_POST = 2, TM_RES64 = 3, TM_PREU = 4, TM_APPLYX = 5 };
// TM_PREU  : PRE with the CG residual update fused in: r_new = r - alpha q (staged from
//            both), t = r_new - A x1, x1 = omega D^{-1} r_new; writes t and r_new
// TM_APPLYX: APPLY with the previous iteration's x += alpha_prev p_old fused in

struct TiledArgs {
  const void* in0;   // APPLY: z   PRE/POST: r    RES64: x (FP64)
  const void* in1;   // APPLY: p (old)                RES64: b (FP64)
  const void* ec;    // POST: coarse correction (grid N/2)
  const void* a;     // cell coefficient
  const void* dinv;  // PRE/PREU/POST: omega D^{-1} per node (0 on the boundary)
  void* out0;        // APPLY: q   PRE: t   POST: z   RES64: r
  void* out1;        // APPLY: p (new)   PREU: r (new)
  const void* q;     // PREU: A p of the current iteration
  void* x;           // APPLYX: solution updated in place with alpha_prev * p_old
  double* partial;   // [S][blocks per sample]
  const SolveScalars* sc;
  const int* act;    // launched samples (null: blockIdx.z / nzc itself)
  long long bstride; // RES64: b stride per sample (0 = shared)
  int N;
  int nzc;           // z chunks per sample
  int zc;            // planes per chunk (a multiple of kZSeg)
  int nseg;          // partial-sum segments per sample column
  int first;         // APPLY: first iteration (pn = z)
  int xfirst;        // APPLYX: x not yet written (x = alpha_prev p_old)
};

__device__ __forceinline__ int ring3(int m) { return (m + 3) % 3; }

// ---------------------------------------------------------------- async staging
// cp.async (4- or 8-byte, zero-filled when the source is outside the grid)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int src = valid ? BYTES : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(BYTES), "r"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Partial sums (dot products of the fused passes, Phi) are formed per segment of
// kZSeg interior planes, whatever z chunk the block marches: partial entry
// (seg * by + tile_y) * bx + tile_x of a sample holds the segment's block sum, so
// the reduction order, and with it every sample's iterates, is independent of the
// batch size that chose the z chunking.
constexpr int kZSeg = 8;

constexpr int RING = 5;   // raw planes resident: k-1, k, k+1 + two in flight
constexpr double kRes64OpsPerNode = 12 * 6 + 28 + 21 * 12 + 20;  // = 372 (see tiled_res64)
constexpr int ERING = 4;  // coarse planes
constexpr int CW = TX + 4;  // staged cell row: 36 cells from x0 - 3 (even start)
constexpr int EWX = TX / 2 + 2;

// Tile geometry for RY nodes per thread in y (block 32 x 8 threads, tile 32 x 8*RY nodes).
template <int RY>
struct Geo {
  static constexpr int TYT = TY * RY;
  static constexpr int NPYT = TYT + 2, NPL = NPX * NPYT;  // staged node plane (34 x (TYT+2))
  static constexpr int CPYT = TYT + 3, CPL = CW * CPYT;   // staged cell plane (36 x (TYT+3))
  static constexpr int EWYT = TYT / 2 + 2, EPL = EWX * EWYT;  // staged coarse plane
};

template <typename T> struct RowsPerThread { static constexpr int value = 4; };
template <> struct RowsPerThread<double> { static constexpr int value = 2; };

template <typename T, typename TA, int MODE>
struct TiledSmem {
  static constexpr int RY = RowsPerThread<T>::value;
  using G = Geo<RY>;
  static constexpr bool kPre = (MODE == TM_PRE || MODE == TM_POST || MODE == TM_PREU);
  static constexpr bool kApply = (MODE == TM_APPLY || MODE == TM_APPLYX);
  static constexpr bool kRaw1 = kApply || MODE == TM_PREU;
  static constexpr size_t raw0 = 0;
  static constexpr size_t raw1 = raw0 + sizeof(T) * RING * G::NPL;
  static constexpr size_t xs = raw1 + (kRaw1 ? sizeof(T) * RING * G::NPL : 0);
  static constexpr size_t dv = xs + sizeof(T) * 3 * G::NPL;
  static constexpr size_t ec = dv + (kPre ? sizeof(T) * RING * G::NPL : 0);
  static constexpr size_t ep = ec + (MODE == TM_POST ? sizeof(T) * ERING * G::EPL : 0);
  static constexpr size_t cells = ep + (MODE == TM_POST ? sizeof(T) * 2 * G::NPL : 0);
  static constexpr size_t total = cells + sizeof(TA) * RING * G::CPL;
};


// ---- error-free FP32 arithmetic for the refinement residual (TM_RES64)
// two_sum: s + e == a + b exactly (Knuth); products use the FMA to split
// c * x into p + pe exactly.  A coefficient is an unevaluated pair (h, l).
struct F2 { float h, l; };
__device__ __forceinline__ F2 two_sum(float a, float b) {  // intrinsics: never contracted
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return F2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// (S, comp) += sgn * (c.h + c.l) * (x.x + x.y), sgn = +1 or -1
template <bool NEG>
__device__ __forceinline__ void df_term(float& S, float& comp, F2 c, float2 x) {
  const float p = __fmul_rn(c.h, x.x);
  const float pe = __fmaf_rn(c.h, x.x, -p);
  const float low = __fmaf_rn(c.h, x.y, __fmaf_rn(c.l, x.x, pe));
  const float q = NEG ? -p : p;
  const F2 t = two_sum(S, q);
  S = t.h;
  comp = __fadd_rn(comp, __fadd_rn(t.l, NEG ? -low : low));
}

template <typename T, typename TA, int MODE>
__global__ void __launch_bounds__(NT) k_tiled(TiledArgs A) {
  using L = TiledSmem<T, TA, MODE>;
  constexpr int RY = L::RY;
  using G = typename L::G;
  constexpr int NPL = G::NPL, CPL = G::CPL, EPL = G::EPL;
  constexpr bool kPre = L::kPre;
  constexpr bool kPairs = sizeof(TA) == 2;                 // BF16 cells staged as 4-byte pairs
  constexpr int NCE = kPairs ? CPL / 2 : CPL;              // cell staging entries per plane
  constexpr int MN = (NPL + NT - 1) / NT, MC = (NCE + NT - 1) / NT, ME = (EPL + NT - 1) / NT;
  // staging entries j < M - 1 always exist (only the last one per thread may not)
  static_assert((MN - 1) * NT < NPL && (MC - 1) * NT < NCE && (ME - 1) * NT < EPL, "staging entries");
  extern __shared__ __align__(16) unsigned char smraw[];
  T* raw0 = (T*)(smraw + L::raw0);
  T* raw1 = (T*)(smraw + L::raw1);
  T* xs = (T*)(smraw + L::xs);
  T* dvs = (T*)(smraw + L::dv);
  T* ecs = (T*)(smraw + L::ec);
  T* eps = (T*)(smraw + L::ep);  // POST: two coarse planes interpolated in x and y to this tile's nodes
  TA* cs = (TA*)(smraw + L::cells);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int N = A.N, n1 = N + 1;
  const int chunk = blockIdx.z % A.nzc;
  const int s = A.act != nullptr ? A.act[blockIdx.z / A.nzc] : (int)(blockIdx.z / A.nzc);
  if (A.sc != nullptr && !A.sc[s].active) return;
  const int x0 = 1 + TX * blockIdx.x, y0 = 1 + G::TYT * blockIdx.y;
  const long long nodes = (long long)n1 * n1 * n1, cells = (long long)N * N * N;
  const int kbeg = 1 + chunk * A.zc;
  const int kend = min(N - 1, kbeg + A.zc - 1);
  const T scale = T(1.0 / (12.0 * N));
  const T* in0 = (const T*)A.in0 + s * nodes;
  constexpr bool kApply = L::kApply;
  const T* in1 = kApply ? (const T*)A.in1 + s * nodes : (MODE == TM_PREU ? (const T*)A.q + s * nodes : in0);
  const bool stage1 = (kApply && !A.first) || MODE == TM_PREU;  // raw1 holds p_old or q
  const TA* a = (const TA*)A.a + s * cells;
  const T* dvg = kPre ? (const T*)A.dinv + s * nodes : in0;
  const int nc1 = N / 2 + 1;
  const T* e0 = (MODE == TM_POST) ? (const T*)A.ec + s * (long long)nc1 * nc1 * nc1 : in0;
  const int ex0 = (x0 - 1) / 2, ey0 = (y0 - 1) / 2;  // coarse tile origin
  const long long pn = (long long)n1 * n1, pc = (long long)N * N, pe = (long long)nc1 * nc1;
  T beta = T(0), alpha = T(0);
  if (kApply && !A.first) beta = (T)A.sc[s].beta;
  if (MODE == TM_APPLYX || MODE == TM_PREU) alpha = (T)A.sc[s].alpha;  // APPLYX: previous iteration's

  // ---- per-thread staging entries, fixed for the whole march (only the plane offset moves)
  int noff[MN], deb[MN];
  unsigned char nflag[MN];  // bit0: entry exists, bit1: inside grid, bit2: interior (x,y), bit3/4: gi/gj odd
#pragma unroll
  for (int j = 0; j < MN; ++j) {
    const int e = tid + j * NT;
    const int lx = e % NPX, ly = e / NPX;
    const int gi = x0 - 1 + lx, gj = y0 - 1 + ly;
    const bool has = e < NPL, in = has && gi <= N && gj <= N;
    const bool inter = has && gi > 0 && gj > 0 && gi < N && gj < N;
    nflag[j] = (has ? 1 : 0) | (in ? 2 : 0) | (inter ? 4 : 0) | ((gi & 1) ? 8 : 0) | ((gj & 1) ? 16 : 0);
    noff[j] = in ? gi + n1 * gj : 0;
    deb[j] = ((gi >> 1) - ex0) + EWX * ((gj >> 1) - ey0);
  }
  int coff[MC], cdst[MC];
  bool cok[MC], chas[MC];
#pragma unroll
  for (int j = 0; j < MC; ++j) {
    const int e = tid + j * NT;
    const int cx = kPairs ? 2 * (e % (CW / 2)) : e % CW;
    const int cy = kPairs ? e / (CW / 2) : e / CW;
    const int gi = x0 - 3 + cx, gj = y0 - 2 + cy;
    chas[j] = e < NCE;
    cok[j] = chas[j] && gi >= 0 && gj >= 0 && gi + (kPairs ? 1 : 0) < N && gj < N;
    coff[j] = cok[j] ? gi + N * gj : 0;
    cdst[j] = cx + CW * cy;
  }
  int eoff[ME];
  bool eok[ME], ehas[ME];
#pragma unroll
  for (int j = 0; j < ME; ++j) {
    const int e = tid + j * NT;
    const int ci = ex0 + e % EWX, cj = ey0 + e / EWX;
    ehas[j] = (MODE == TM_POST) && e < EPL;
    eok[j] = ehas[j] && ci > 0 && cj > 0 && ci < nc1 - 1 && cj < nc1 - 1;  // coarse interior
    eoff[j] = eok[j] ? ci + nc1 * cj : 0;
  }
  // POST: coarse plane c is staged once, by issue(2c - 2), and interpolated in x and y
  // by derive(2c - 2), one fine plane before derive(2c - 1) first reads it (the
  // barrier after each derive separates the two); the prologue stages and
  // interpolates the planes of the first derived plane
  auto stage_coarse = [&](int c) {
    const bool cok2 = c > 0 && c < nc1 - 1;
    const T* eb = e0 + (cok2 ? c * pe : 0);  // a plane inside the buffer; invalid entries are zero-filled
#pragma unroll
    for (int j = 0; j < ME; ++j) {
      if (j == ME - 1 && !ehas[j]) continue;
      cp_async<sizeof(T)>(ecs + (c & (ERING - 1)) * EPL + tid + j * NT, eb + eoff[j], cok2 && eok[j]);
    }
  };

  auto issue = [&](int m, int slot) {
    // every node vector here is zero on the Dirichlet boundary: boundary nodes are
    // zero-filled like nodes outside the grid, so no buffer's boundary is ever read
    const bool mok = m > 0 && m < N;
    // plane bases inside the buffers (plane 0 when m is outside); every staged offset
    // lies inside a plane, so each source address is valid and the flag alone decides
    // between a copy and a zero fill
    const long long mo = mok ? (long long)m * pn : 0;
    const T* b0 = in0 + mo;
    const T* b1 = in1 + mo;
    const T* bd = dvg + mo;
#pragma unroll
    for (int j = 0; j < MN; ++j) {
      if (j == MN - 1 && !(nflag[j] & 1)) continue;
      const int e = tid + j * NT;
      const bool ok = mok && (nflag[j] & 4);
      cp_async<sizeof(T)>(raw0 + slot * NPL + e, b0 + noff[j], ok);
      if (stage1) cp_async<sizeof(T)>(raw1 + slot * NPL + e, b1 + noff[j], ok);
      if (kPre) cp_async<sizeof(T)>(dvs + slot * NPL + e, bd + noff[j], ok);
    }
    const bool cmok = m >= 0 && m < N;
    const TA* ab = a + (cmok ? (long long)m * pc : 0);
#pragma unroll
    for (int j = 0; j < MC; ++j) {
      if (j == MC - 1 && !chas[j]) continue;
      cp_async<kPairs ? 4 : sizeof(TA)>(cs + slot * CPL + cdst[j], ab + coff[j], cmok && cok[j]);
    }
    if (MODE == TM_POST && !(m & 1)) stage_coarse((m >> 1) + 1);
    cp_async_commit();
  };

  // POST: eps[c & 1] holds coarse plane c interpolated bilinearly in x and y at this
  // tile's staged nodes; a fine plane m takes plane m/2 (m even) or the mean of planes
  // (m-1)/2 and (m+1)/2 (m odd), so each coarse plane is interpolated once for two
  // fine planes.  The tile origin is even (x0 - 1 = 32 bx, y0 - 1 = TYT by), so staged
  // node (2a + p, 2b + q) lies in coarse cell (a, b) of the staged coarse tile: one
  // work item per coarse cell writes its four nodes (odd index: halfway between two
  // coarse nodes), every staged entry included.
  auto interp_xy = [&](int c) {
    const T* cp = ecs + (c & (ERING - 1)) * EPL;
    T* ed = eps + (c & 1) * NPL;
    constexpr int AX = EWX - 1, AY = G::EWYT - 1;  // 17 x (TYT/2 + 1) cells cover 34 x (TYT+2) nodes
    // items NT.. go to the last threads (their warps stage one entry fewer in derive)
    static_assert(AX * AY <= 2 * NT, "two rounds at most");
#pragma unroll
    for (int rd = 0; rd < 2; ++rd) {
      const int wi = rd == 0 ? tid : 2 * NT - 1 - tid;
      if (wi >= AX * AY || (rd == 1 && wi < NT)) continue;
      const int ca = wi % AX, cb = wi / AX;
      const T* q = cp + ca + EWX * cb;
      const T e00 = q[0], e10 = q[1], e01 = q[EWX], e11 = q[EWX + 1];
      const T r0 = (e00 + e10) * T(0.5), r1 = (e01 + e11) * T(0.5);
      T* o = ed + 2 * ca + NPX * (2 * cb);
      o[0] = e00;
      o[1] = r0;
      o[NPX] = (e00 + e01) * T(0.5);
      o[NPX + 1] = (r0 + r1) * T(0.5);
    }
  };

  // operand plane m from its staged raw plane (slot: its raw ring slot, r3: its xs slot)
  auto derive = [&](int m, int slot, int r3) {
    T* xp = xs + r3 * NPL;
    const T* r0 = raw0 + slot * NPL;
    if (kApply) {
      const T* r1 = raw1 + slot * NPL;
#pragma unroll
      for (int j = 0; j < MN; ++j) {
        if (j == MN - 1 && !(nflag[j] & 1)) continue;
        const int e = tid + j * NT;
        xp[e] = A.first ? r0[e] : r0[e] + beta * r1[e];
      }
    } else if (MODE == TM_RES64) {
      // x is already an (hi, lo) pair: copy the 8-byte word
#pragma unroll
      for (int j = 0; j < MN; ++j)
        if (j < MN - 1 || (nflag[j] & 1)) xp[tid + j * NT] = r0[tid + j * NT];
    } else {
      const T* dvp = dvs + slot * NPL;
      const bool mint = m > 0 && m < N;
      const int dk = m & 1, c0 = m >> 1;
      // even m: coarse plane m/2 + 1 for the next (odd) plane, into the other eps slot
      if (MODE == TM_POST && !dk) interp_xy(c0 + 1);
      const T* e0p = eps + (c0 & 1) * NPL;
      const T* e1p = eps + ((c0 + 1) & 1) * NPL;
#pragma unroll
      for (int j = 0; j < MN; ++j) {
        if (j == MN - 1 && !(nflag[j] & 1)) continue;
        const int e = tid + j * NT;
        // branch-free: D^-1 is 0 on the boundary and zero-filled outside the grid (and
        // so is r outside 0 < m < N), so only the coarse correction needs a mask
        const T rn = (MODE == TM_PREU) ? r0[e] - alpha * raw1[slot * NPL + e] : r0[e];
        T v = rn * dvp[e];
        if (MODE == TM_POST) {
          const T mk = (mint && (nflag[j] & 4)) ? T(1) : T(0);
          v += mk * (dk ? (e0p[e] + e1p[e]) * T(0.5) : e0p[e]);
        }
        xp[e] = v;
      }
    }
  };

  // prologue: derive the planes before kbeg, keep two planes in flight
  const int first_plane = kPre ? kbeg - 2 : kbeg - 1;
  auto mod5 = [](int m) { return (m + 2 * RING) % RING; };
  if (MODE == TM_POST) {  // committed with the first issue below
    stage_coarse(first_plane >> 1);
    if (first_plane & 1) stage_coarse((first_plane >> 1) + 1);
  }
  for (int m = first_plane; m <= kbeg + 2; ++m) issue(m, mod5(m));
  cp_async_wait<2>();
  __syncthreads();
  if (MODE == TM_POST) {
    interp_xy(first_plane >> 1);
    if (first_plane & 1) interp_xy((first_plane >> 1) + 1);
    __syncthreads();
  }
  for (int m = first_plane; m <= kbeg; ++m) {
    derive(m, mod5(m), ring3(m));
    __syncthreads();
  }

  // this thread's column: gi, rows gj = y0 + RY*ty + t (t < RY); staged node rows RY*ty + 1 + t
  T red = T(0);
  const int gi = x0 + tx;
  const int gj0 = y0 + RY * ty;
  const bool colok = gi < N;
  const int xb = tx + NPX * (RY * ty);        // staged node (tx, RY*ty): top-left of the 3 x (RY+2) window
  const int cbn = (tx + 2) + CW * (RY * ty + 1);  // staged cell (gi-1, gj0-1)
  T* out0 = (T*)A.out0 + s * nodes + gi + (long long)n1 * gj0;
  T* out1 = (kApply || MODE == TM_PREU) ? (T*)A.out1 + s * nodes + gi + (long long)n1 * gj0 : nullptr;
  T* xio = (MODE == TM_APPLYX) ? (T*)A.x + s * nodes + gi + (long long)n1 * gj0 : nullptr;
  const T* bptr = (MODE == TM_RES64) ? (const T*)A.in1 + s * A.bstride + gi + (long long)n1 * gj0 : nullptr;
  float* r32o = (MODE == TM_RES64) ? (float*)A.out0 + s * nodes + gi + (long long)n1 * gj0 : nullptr;
  float redf = 0.f;  // RES64: r.r of this thread in FP32
  const double scd = 1.0 / (12.0 * N);
  const float sch = (float)scd, scl = (float)(scd - (double)sch);  // h/12 as an FP32 pair
  // ring slots of plane k, maintained incrementally: s5 in the RING-plane raw/cell
  // rings, r3 in the three-plane operand ring
  int s5 = mod5(kbeg), r3 = ring3(kbeg);
  for (int k = kbeg; k <= kend; ++k) {
    const int s5p1 = s5 + 1 == RING ? 0 : s5 + 1;
    const int s5p3 = s5 + 3 >= RING ? s5 + 3 - RING : s5 + 3;
    const int s5m1 = s5 == 0 ? RING - 1 : s5 - 1;
    const int r3p1 = r3 == 2 ? 0 : r3 + 1;
    const int r3m1 = r3 == 0 ? 2 : r3 - 1;
    const int r3s[3] = {r3m1, r3, r3p1};
    const int c5s[2] = {s5m1, s5};
    // APPLYX: fetch this plane's x early so the load overlaps the staging below
    T xv[RY];
    if (MODE == TM_APPLYX) {
#pragma unroll
      for (int t = 0; t < RY; ++t)
        xv[t] = (colok && gj0 + t < N && !A.xfirst) ? xio[pn * k + n1 * t] : T(0);
    }
    issue(k + 3, s5p3);
    cp_async_wait<2>();
    __syncthreads();
    derive(k + 1, s5p1, r3p1);
    __syncthreads();
    if constexpr (MODE == TM_RES64) {
      if (colok) {
        // b - A x with x = hi + lo (FP32 pairs) and FP32 cells, error-free products and
        // compensated sums: exact pair sums of cells, exact products, one rounding of the
        // unevaluated sum (S, comp) per term; the scale h/12 and the subtraction from b are
        // done in the same pair arithmetic, so no FP64 instruction is executed.
        float2 X[3][3][RY + 2];
        float C[2][2][RY + 1];
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
          const float2* xp = reinterpret_cast<const float2*>(xs + r3s[pl] * NPL) + xb;
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int rr = 0; rr < RY + 2; ++rr) X[pl][c][rr] = xp[c + NPX * rr];
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const TA* cp = cs + c5s[r] * CPL + cbn;
#pragma unroll
          for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int cr = 0; cr < RY + 1; ++cr) C[r][p][cr] = (float)cp[p + CW * cr];
        }
#pragma unroll
        for (int t = 0; t < RY; ++t) {
          if (gj0 + t >= N) break;
          F2 pxy[2][2], pxz[2][2], pyz[2][2];
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              pxy[v][u] = two_sum(C[0][u][t + v], C[1][u][t + v]);
              pxz[v][u] = two_sum(C[v][u][t], C[v][u][t + 1]);
              pyz[v][u] = two_sum(C[v][0][t + u], C[v][1][t + u]);
            }
          float S8 = 0.f, E8 = 0.f;
#pragma unroll
          for (int v = 0; v < 2; ++v)
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const F2 q = two_sum(S8, pxy[v][u].h);
              S8 = q.h;
              E8 += q.l + pxy[v][u].l;
            }
          float S = 0.f, comp = 0.f;
          df_term<false>(S, comp, F2{4.f * S8, 4.f * E8}, X[1][1][t + 1]);
#pragma unroll
          for (int v = 0; v < 2; ++v)
#pragma unroll
            for (int u = 0; u < 2; ++u) df_term<true>(S, comp, pxy[v][u], X[1][2 * u][t + 2 * v]);
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const int pl = 2 * r;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              df_term<true>(S, comp, pxz[r][u], X[pl][2 * u][t + 1]);
              df_term<true>(S, comp, pyz[r][u], X[pl][1][t + 2 * u]);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
              for (int p = 0; p < 2; ++p) df_term<true>(S, comp, F2{C[r][p][t + q], 0.f}, X[pl][2 * p][t + 2 * q]);
          }
          // ax = (S + comp) (sch + scl), a pair (p, pe)
          const F2 axs = two_sum(S, comp);
          const float p = __fmul_rn(axs.h, sch);
          const float pe = __fmaf_rn(axs.h, scl, __fmaf_rn(axs.l, sch, __fmaf_rn(axs.h, sch, -p)));
          const long long o = pn * k + n1 * t;
          const float2 bv = reinterpret_cast<const float2*>(bptr)[o];
          const F2 d = two_sum(bv.x, -p);
          const float rv = d.h + (d.l + (bv.y - pe));
          r32o[o] = rv;  // the inner solve's FP32 residual
          redf = __fmaf_rn(rv, rv, redf);
        }
      }
    } else if (colok) {
      // registers: operand window X[plane][col][row] (3 x 3 x (RY+2)), cells C[r][p][row] (2 x 2 x (RY+1))
      T X[3][3][RY + 2];
      T C[2][2][RY + 1];
#pragma unroll
      for (int pl = 0; pl < 3; ++pl) {
        const T* xp = xs + r3s[pl] * NPL + xb;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int rr = 0; rr < RY + 2; ++rr) X[pl][c][rr] = xp[c + NPX * rr];
      }
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const TA* cp = cs + c5s[r] * CPL + cbn;
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int cr = 0; cr < RY + 1; ++cr) C[r][p][cr] = smem_coef<T>(cp[p + CW * cr]);
      }
      const T* rk = raw0 + s5 * NPL + xb + 1 + NPX;
#pragma unroll
      for (int t = 0; t < RY; ++t) {
        if (gj0 + t >= N) break;
        // cells of node t: c[r][q][p] = C[r][p][t + q]; neighbour (du, dv) in plane pl: X[pl][1 + du][t + 1 + dv]
        T pxy[2][2], pxz[2][2], pyz[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            pxy[v][u] = C[0][u][t + v] + C[1][u][t + v];   // cells (u, v, 0), (u, v, 1)
            pxz[v][u] = C[v][u][t] + C[v][u][t + 1];       // cells (u, 0, v), (u, 1, v)
            pyz[v][u] = C[v][0][t + u] + C[v][1][t + u];   // cells (0, u, v), (1, u, v)
          }
        const T sum8 = (pxy[0][0] + pxy[0][1]) + (pxy[1][0] + pxy[1][1]);
        // three independent partial sums (centre plane, plane k-1, plane k+1): shorter
        // dependency chains than one running accumulator
        T accp[3];
        accp[1] = T(4) * sum8 * X[1][1][t + 1];
#pragma unroll
        for (int v = 0; v < 2; ++v)
#pragma unroll
          for (int u = 0; u < 2; ++u) accp[1] -= pxy[v][u] * X[1][2 * u][t + 2 * v];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int pl = 2 * r;  // plane k-1 (r = 0) or k+1 (r = 1)
          T a2 = T(0);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            a2 -= pxz[r][u] * X[pl][2 * u][t + 1];
            a2 -= pyz[r][u] * X[pl][1][t + 2 * u];
          }
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int p = 0; p < 2; ++p) a2 -= C[r][p][t + q] * X[pl][2 * p][t + 2 * q];
          accp[pl] = a2;
        }
        const T ax = scale * (accp[1] + (accp[0] + accp[2]));
        const long long o = pn * k + n1 * t;
        if (kApply) {
          const T pv = X[1][1][t + 1];
          out0[o] = ax;
          out1[o] = pv;
          red += pv * ax;
          if (MODE == TM_APPLYX) xio[o] = xv[t] + alpha * raw1[s5 * NPL + xb + 1 + NPX * (t + 1)];  // xv = 0 when A.xfirst
        } else if (MODE == TM_PRE) {
          out0[o] = rk[NPX * t] - ax;
        } else if (MODE == TM_PREU) {
          const T rn = rk[NPX * t] - alpha * raw1[s5 * NPL + xb + 1 + NPX * (t + 1)];
          out0[o] = rn - ax;
          out1[o] = rn;
        } else if (MODE == TM_POST) {
          const T rv = rk[NPX * t];
          const T dk = dvs[s5 * NPL + xb + 1 + NPX * (t + 1)];
          const T zv = X[1][1][t + 1] + (rv - ax) * dk;
          out0[o] = zv;
          red += rv * zv;
        }
      }
    }
    if (MODE != TM_PRE && MODE != TM_PREU && (k == kend || (k - 1) % kZSeg == kZSeg - 1)) {
      // end of a partial-sum segment (block-uniform condition)
      const T b = block_sum(MODE == TM_RES64 ? (T)redf : red);
      if (tid == 0) {
        const int per = gridDim.x * gridDim.y * A.nseg;
        const int bid = (((k - 1) / kZSeg) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        A.partial[(long long)s * per + bid] = (double)b;
      }
      red = T(0);
      redf = 0.f;
    }
    __syncthreads();
    s5 = s5p1;
    r3 = r3p1;
  }
  cp_async_wait<0>();
}

// Phi = 1/2 e^T M e and badj = M e on interior rows, e = y - g_h (row a5).
// The consistent Q1 mass is (h/6)^3 [1 4 1] x [1 4 1] x [1 4 1]: a staged plane of
// y is summed along x, then y, into the tile; three such planes combine along z.
// g_h = gx(i) gx(j) gx(k) and M g_h = mg(i) mg(j) mg(k) are separable, so they
// come from the 1D tables gtab[i] = sin(pi i / N) (0 at i = 0, N) and
// mgtab[i] = (h/6)(g[i-1] + 4 g[i] + g[i+1]).
__global__ void __launch_bounds__(NT) k_phi_tiled(const double* __restrict__ y, int N, const double* __restrict__ gtab,
                                                  const double* __restrict__ mgtab, double* __restrict__ badj,
                                                  double* __restrict__ partial, int nzc, int zc, int nseg) {
  __shared__ double ys[NP];
  __shared__ double xsum[NPY][TX];
  __shared__ double mxy[3][NT];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int n1 = N + 1;
  const int s = blockIdx.z / nzc, chunk = blockIdx.z % nzc;
  const int x0 = 1 + TX * blockIdx.x, y0 = 1 + TY * blockIdx.y;
  const long long nodes = (long long)n1 * n1 * n1;
  const double* yb = y + s * nodes;
  const int kbeg = 1 + chunk * zc;
  const int kend = min(N - 1, kbeg + zc - 1);
  const int gi = x0 + tx, gj = y0 + ty;
  const bool mine = gi < N && gj < N;
  double ycen[3] = {0.0, 0.0, 0.0};
  auto advance = [&](int m) {
    for (int e = tid; e < NP; e += NT) {
      const int lx = e % NPX, ly = e / NPX;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      ys[e] = (m >= 0 && m <= N && i <= N && j <= N) ? yb[i + (long long)n1 * (j + (long long)n1 * m)] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < NPY * TX; e += NT) {
      const int ly = e / TX, lx = e % TX;
      const double* row = ys + NPX * ly + lx;
      xsum[ly][lx] = row[0] + 4.0 * row[1] + row[2];
    }
    ycen[(m + 3) % 3] = ys[(tx + 1) + NPX * (ty + 1)];
    __syncthreads();
    mxy[(m + 3) % 3][tid] = xsum[ty][tx] + 4.0 * xsum[ty + 1][tx] + xsum[ty + 2][tx];
    __syncthreads();
  };
  const double h6 = 1.0 / (6.0 * N), h63 = h6 * h6 * h6;
  double red = 0.0;
  advance(kbeg - 1);
  advance(kbeg);
  for (int k = kbeg; k <= kend; ++k) {
    advance(k + 1);
    if (mine) {
      const double my = mxy[(k + 2) % 3][tid] + 4.0 * mxy[k % 3][tid] + mxy[(k + 1) % 3][tid];
      const double me = h63 * my - mgtab[gi] * mgtab[gj] * mgtab[k];
      const double e = ycen[k % 3] - gtab[gi] * gtab[gj] * gtab[k];
      badj[s * nodes + gi + (long long)n1 * (gj + (long long)n1 * k)] = me;
      red += e * me;
    }
    if (k == kend || (k - 1) % kZSeg == kZSeg - 1) {  // end of a partial-sum segment
      const double b = block_sum(red);
      if (tid == 0)
        partial[(long long)s * (gridDim.x * gridDim.y * nseg) + (((k - 1) / kZSeg) * gridDim.y + blockIdx.y) * gridDim.x +
                blockIdx.x] = b;
      red = 0.0;
      __syncthreads();
    }
  }
}

// k_phi_tiled for a state given as FP32 (hi, lo) pairs (the mixed level gradient):
// the same separable sums in pair arithmetic (no FP64 instruction), the 1D tables as
// pairs, M e written as pairs (the adjoint solve's right-hand side), the partial
// e.M e of each block returned in FP64.  Each thread takes kPhiRows rows of a
// 32 x (8 kPhiRows) tile, so the three block barriers of a plane serve four nodes;
// the staged plane is double-buffered and plane m + 1 is copied asynchronously while
// plane m is summed.
constexpr int kPhiRows = 4;
constexpr int kPhiTY = TY * kPhiRows;                        // tile rows
constexpr int kPhiNPY = kPhiTY + 2, kPhiNP = NPX * kPhiNPY;  // staged plane with halo
constexpr size_t kPhiSmem = sizeof(float2) * (2 * kPhiNP + kPhiNPY * TX + 3 * kPhiTY * TX);
__global__ void __launch_bounds__(NT) k_phi_tiled_df(const float2* __restrict__ y, int N, const float2* __restrict__ gtab,
                                                     const float2* __restrict__ mgtab, float2* __restrict__ badj,
                                                     double* __restrict__ partial, int nzc, int zc, int nseg) {
  extern __shared__ __align__(16) unsigned char smp[];
  float2* ysb = reinterpret_cast<float2*>(smp);  // [2][kPhiNP]: plane m in buffer m & 1
  float2(*xsum)[TX] = reinterpret_cast<float2(*)[TX]>(ysb + 2 * kPhiNP);                   // [kPhiNPY][TX]
  float2(*mxy)[kPhiTY][TX] = reinterpret_cast<float2(*)[kPhiTY][TX]>(ysb + 2 * kPhiNP + kPhiNPY * TX);  // [3]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int n1 = N + 1;
  const int s = blockIdx.z / nzc, chunk = blockIdx.z % nzc;
  const int x0 = 1 + TX * blockIdx.x, y0 = 1 + kPhiTY * blockIdx.y;
  const long long nodes = (long long)n1 * n1 * n1;
  const float2* yb = y + s * nodes;
  const int kbeg = 1 + chunk * zc;
  const int kend = min(N - 1, kbeg + zc - 1);
  const int gi = x0 + tx;
  const int ly0 = kPhiRows * ty;  // the thread's first tile row
  DF yc[kPhiRows], yn[kPhiRows];  // y at the thread's nodes of planes k and k + 1
  auto four = [](DF a) { return DF{4.f * a.h, 4.f * a.l}; };  // exact
  auto load = [&](int m) {  // plane m into buffer m & 1 (zeros outside the grid)
    float2* ys = ysb + (m & 1) * kPhiNP;
    for (int e = tid; e < kPhiNP; e += NT) {
      const int lx = e % NPX, ly = e / NPX;
      const int i = x0 - 1 + lx, j = y0 - 1 + ly;
      const bool ok = m >= 0 && m <= N && i <= N && j <= N;
      cp_async<8>(ys + e, ok ? yb + i + (long long)n1 * (j + (long long)n1 * m) : yb, ok);
    }
    cp_async_commit();
  };
  // plane m (copied by load(m)) into the x and xy sums; copies plane m + 1 meanwhile
  // (into the buffer of plane m - 1, whose last reads precede the first barrier)
  auto advance = [&](int m, DF* ycen) {
    const int r3 = (m + 3) % 3;
    const float2* ys = ysb + (m & 1) * kPhiNP;
    cp_async_wait<0>();
    __syncthreads();
    if (m + 1 <= kend + 1) load(m + 1);
    for (int e = tid; e < kPhiNPY * TX; e += NT) {
      const int ly = e / TX, lx = e % TX;
      const float2* row = ys + NPX * ly + lx;
      xsum[ly][lx] = df_f2(df_add(df_add(df_make(row[0]), df_make(row[2])), four(df_make(row[1]))));
    }
#pragma unroll
    for (int t = 0; t < kPhiRows; ++t) ycen[t] = df_make(ys[(tx + 1) + NPX * (ly0 + t + 1)]);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kPhiRows; ++t) {
      const int ly = ly0 + t;
      mxy[r3][ly][tx] =
          df_f2(df_add(df_add(df_make(xsum[ly][tx]), df_make(xsum[ly + 2][tx])), four(df_make(xsum[ly + 1][tx]))));
    }
    __syncthreads();
  };
  const double h6 = 1.0 / (6.0 * N);
  const DF h63 = df_make(df_split(h6 * h6 * h6));
  DF red{0.f, 0.f};
  load(kbeg - 1);
  advance(kbeg - 1, yn);
  advance(kbeg, yc);
  const DF mgi = gi < N ? df_make(mgtab[gi]) : DF{0.f, 0.f}, ggi = gi < N ? df_make(gtab[gi]) : DF{0.f, 0.f};
  for (int k = kbeg; k <= kend; ++k) {
    advance(k + 1, yn);
    const DF mgk = df_make(mgtab[k]), ggk = df_make(gtab[k]);
#pragma unroll
    for (int t = 0; t < kPhiRows; ++t) {
      const int gj = y0 + ly0 + t;
      if (gi < N && gj < N) {
        const DF my = df_add(df_add(df_make(mxy[(k + 2) % 3][ly0 + t][tx]), df_make(mxy[(k + 1) % 3][ly0 + t][tx])),
                             four(df_make(mxy[k % 3][ly0 + t][tx])));
        const DF mg3 = df_mul(df_mul(mgi, df_make(mgtab[gj])), mgk);
        const DF g3 = df_mul(df_mul(ggi, df_make(gtab[gj])), ggk);
        const DF me = df_add(df_mul(h63, my), df_neg(mg3));
        const DF e = df_add(yc[t], df_neg(g3));
        badj[s * nodes + gi + (long long)n1 * (gj + (long long)n1 * k)] = df_f2(me);
        red = df_add(red, df_mul(e, me));
      }
    }
#pragma unroll
    for (int t = 0; t < kPhiRows; ++t) yc[t] = yn[t];
    if (k == kend || (k - 1) % kZSeg == kZSeg - 1) {  // end of a partial-sum segment
      const double b = block_sum(df_to_double(red));
      if (tid == 0)
        partial[(long long)s * (gridDim.x * gridDim.y * nseg) + (((k - 1) / kZSeg) * gridDim.y + blockIdx.y) * gridDim.x +
                blockIdx.x] = b;
      red = DF{0.f, 0.f};
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- host side

TiledShape tiled_shape(int N, int S, int ry, int zchunks) {
  TiledShape t;
  t.bx = (N - 1 + TX - 1) / TX;
  t.by = (N - 1 + TY * ry - 1) / (TY * ry);
  // enough blocks to fill the GPU: split z into chunks of whole partial-sum segments
  // when the batch is small (the partial-sum layout does not depend on the split)
  const int nseg = (N - 1 + kZSeg - 1) / kZSeg;
  const long long base = (long long)t.bx * t.by * S;
  int nzc = 1;
  if (zchunks > 0) nzc = zchunks < nseg ? zchunks : nseg;
  else
    while (base * nzc < 4 * 152 * 4 && 2 * nzc <= nseg) nzc *= 2;
  const int spc = (nseg + nzc - 1) / nzc;  // segments per chunk
  t.nzc = (nseg + spc - 1) / spc;
  t.zc = spc * kZSeg;
  t.nseg = nseg;
  t.blocks_per_sample = t.bx * t.by * nseg;  // partial-sum entries per sample
  return t;
}

// The tile shape follows the batch size bt.S (not the number of samples launched),
// so a sample's partial sums, and with them its iterates, do not depend on how many
// other samples are still active.
template <typename T, typename TA, int MODE>
static void run_tiled(const char* cls, double bytes, TiledArgs args, const Batch& bt, cudaStream_t st,
                      double ops = 0.0) {
  const TiledShape t = tiled_shape(args.N, bt.S, RowsPerThread<T>::value, bt.zchunks);
  args.nzc = t.nzc;
  args.zc = t.zc;
  args.nseg = t.nseg;
  args.act = bt.act;
  const size_t smem = TiledSmem<T, TA, MODE>::total;  // up to ~91 KB (FP64): opt in above 48 KB
  static bool smem_set = false;  // once per instantiation (capture-friendly)
  if (smem > 48 * 1024 && !smem_set) {
    cudaFuncSetAttribute(k_tiled<T, TA, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    smem_set = true;
  }
  launch_flops(cls, bytes, ops, k_tiled<T, TA, MODE>, dim3(t.bx, t.by, (unsigned)(bt.n * t.nzc)), dim3(TX, TY), smem,
               st, args);
}

template <typename T, typename TA>
static double vbytes(int N, int S, double vec, double coef) {
  return (double)S * (vec * (double)nodes_of(N) * sizeof(T) + coef * (double)cells_of(N) * sizeof(TA));
}

template <typename T> const char* tag();
template <> const char* tag<double>() { return "f64"; }
template <> const char* tag<float>() { return "f32"; }
static const char* name(const char* base, const char* t) {
  static thread_local char buf[64];
  snprintf(buf, sizeof(buf), "%s_%s", base, t);
  return buf;
}

// p is double-buffered: neighbouring tiles read the old p in their halos while
// this tile writes the new one.
// FP32 vectors on 32^3 and 64^3 grids go to the whole-row slab passes (slab.cu)
template <typename T, typename TA>
void tiled_apply(const T* z, const T* pold, T* pnew, const TA* a, T* q, double* partial, const SolveScalars* sc, int N,
                 const Batch& bt, int first, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value && std::is_same<TA, float>::value) {
    if (bt.stencil == 0 && slab_supported(N)) {
      slab_apply(z, pold, pnew, a, q, nullptr, partial, sc, N, bt, first != 0, false, false, st);
      return;
    }
  }
  TiledArgs A{};
  A.in0 = z; A.in1 = pold; A.a = a; A.out0 = q; A.out1 = pnew; A.partial = partial; A.sc = sc; A.N = N;
  A.first = first;
  run_tiled<T, TA, TM_APPLY>(name("apply", tag<T>()), vbytes<T, TA>(N, bt.n, first ? 3 : 4, 1), A, bt, st);
}
// fused variants of the mixed inner solve (see TM_PREU / TM_APPLYX)
void tiled_apply_x(const float* z, const float* pold, float* pnew, const float* a, float* q, float* x, double* partial,
                   const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st, bool x_first) {
  if (bt.stencil == 0 && slab_supported(N)) {
    slab_apply(z, pold, pnew, a, q, x, partial, sc, N, bt, false, true, x_first, st);
    return;
  }
  TiledArgs A{};
  A.in0 = z; A.in1 = pold; A.a = a; A.out0 = q; A.out1 = pnew; A.x = x; A.partial = partial; A.sc = sc; A.N = N;
  A.xfirst = x_first ? 1 : 0;
  run_tiled<float, float, TM_APPLYX>("apply_f32", vbytes<float, float>(N, bt.n, x_first ? 5 : 6, 1), A, bt, st);
}
bool tiled_pre_update(const float* r, const float* q, const __nv_bfloat16* a, const float* dinv, float* t,
                      float* rnew, float* rc, const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st) {
  if (bt.stencil == 0 && slab_supported(N)) {
    slab_pre<__nv_bfloat16>(r, q, a, dinv, rnew, rc, sc, N, bt, st);
    return true;
  }
  TiledArgs A{};
  A.in0 = r; A.q = q; A.a = a; A.dinv = dinv; A.out0 = t; A.out1 = rnew; A.sc = sc; A.N = N;
  run_tiled<float, __nv_bfloat16, TM_PREU>("pre_f32", vbytes<float, __nv_bfloat16>(N, bt.n, 5, 1), A, bt, st);
  return false;
}

template <typename T, typename TA>
bool tiled_pre(const T* r, const TA* a, const T* dinv, T* t, T* rc, const SolveScalars* sc, int N, const Batch& bt,
               cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (bt.stencil == 0 && slab_supported(N)) {
      slab_pre<TA>(r, nullptr, a, dinv, nullptr, rc, sc, N, bt, st);
      return true;
    }
  }
  TiledArgs A{};
  A.in0 = r; A.a = a; A.dinv = dinv; A.out0 = t; A.sc = sc; A.N = N;
  run_tiled<T, TA, TM_PRE>(name("pre", tag<T>()), vbytes<T, TA>(N, bt.n, 3, 1), A, bt, st);
  return false;
}
template <typename T, typename TA>
void tiled_post(const T* r, const TA* a, const T* dinv, const T* ec, T* z, double* partial, const SolveScalars* sc,
                int N, const Batch& bt, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (bt.stencil == 0 && slab_supported(N)) {
      slab_post<TA>(r, a, dinv, ec, z, partial, sc, N, bt, st);
      return;
    }
  }
  TiledArgs A{};
  A.in0 = r; A.a = a; A.dinv = dinv; A.ec = ec; A.out0 = z; A.partial = partial; A.sc = sc; A.N = N;
  run_tiled<T, TA, TM_POST>(name("post", tag<T>()), vbytes<T, TA>(N, bt.n, 3, 1) + vbytes<T, T>(N / 2, bt.n, 1, 0), A,
                            bt, st);
}
void tiled_res64(const float2* b, long long bstride, const float2* x, const float* a, float* r32, double* partial,
                 const SolveScalars* sc, int N, const Batch& bt, cudaStream_t st) {
  TiledArgs A{};
  A.in0 = x; A.in1 = b; A.bstride = bstride; A.a = a; A.out0 = r32; A.partial = partial; A.sc = sc; A.N = N;
  const double bb = (double)(bstride ? bt.n : 1) * nodes_of(N) * 8;
  // FP32 operations per interior node as written (no sharing between nodes): 12 exact
  // cell-pair sums (6 each), the 8-cell sum (28), 21 compensated product terms (12
  // each), the scaling, the subtraction from b and r.r (20)
  const double ops = (double)bt.n * (N - 1) * (N - 1) * (N - 1) * kRes64OpsPerNode;
  run_tiled<double, float, TM_RES64>("resid64", bb + vbytes<double, float>(N, bt.n, 1, 1) + (double)bt.n * nodes_of(N) * 4,
                                     A, bt, st, ops);
}

int tiled_phi_df(const float2* y, int N, int S, const float2* gtab, const float2* mgtab, float2* badj,
                 double* partial, cudaStream_t st) {
  const TiledShape t = tiled_shape(N, S, kPhiRows);
  static bool smem_set = false;  // once (capture-friendly)
  if (!smem_set) {
    cudaFuncSetAttribute(k_phi_tiled_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPhiSmem);
    smem_set = true;
  }
  launch("phi_adjrhs", (double)S * nodes_of(N) * 16, k_phi_tiled_df, dim3(t.bx, t.by, (unsigned)(S * t.nzc)),
         dim3(TX, TY), kPhiSmem, st, y, N, gtab, mgtab, badj, partial, t.nzc, t.zc, t.nseg);
  return t.blocks_per_sample;
}

int tiled_phi(const double* y, int N, int S, const double* gtab, const double* mgtab, double* badj, double* partial,
              cudaStream_t st) {
  const TiledShape t = tiled_shape(N, S, 1);
  launch("phi_adjrhs", (double)S * nodes_of(N) * 16, k_phi_tiled, dim3(t.bx, t.by, (unsigned)(S * t.nzc)),
         dim3(TX, TY), 0, st, y, N, gtab, mgtab, badj, partial, t.nzc, t.zc, t.nseg);
  return t.blocks_per_sample;
}

template void tiled_apply<float, float>(const float*, const float*, float*, const float*, float*, double*,
                                        const SolveScalars*, int, const Batch&, int, cudaStream_t);
template void tiled_apply<double, double>(const double*, const double*, double*, const double*, double*, double*,
                                          const SolveScalars*, int, const Batch&, int, cudaStream_t);
template bool tiled_pre<float, __nv_bfloat16>(const float*, const __nv_bfloat16*, const float*, float*, float*,
                                              const SolveScalars*, int, const Batch&, cudaStream_t);
template bool tiled_pre<float, float>(const float*, const float*, const float*, float*, float*, const SolveScalars*,
                                      int, const Batch&, cudaStream_t);
template void tiled_post<float, float>(const float*, const float*, const float*, const float*, float*, double*,
                                       const SolveScalars*, int, const Batch&, cudaStream_t);
template bool tiled_pre<double, double>(const double*, const double*, const double*, double*, double*,
                                        const SolveScalars*, int, const Batch&, cudaStream_t);
template void tiled_post<float, __nv_bfloat16>(const float*, const __nv_bfloat16*, const float*, const float*, float*,
                                               double*, const SolveScalars*, int, const Batch&, cudaStream_t);
template void tiled_post<double, double>(const double*, const double*, const double*, const double*, double*, double*,
                                         const SolveScalars*, int, const Batch&, cudaStream_t);

}  // namespace mlsgd

namespace mlsgd {
int tiled_blocks_per_sample(int N, int S, int elem, bool slab) {
  if (elem == 4 && slab && slab_supported(N)) return slab_shape(N, S).blocks_per_sample;
  return tiled_shape(N, S, elem == 8 ? RowsPerThread<double>::value : RowsPerThread<float>::value).blocks_per_sample;
}
}  // namespace mlsgd
