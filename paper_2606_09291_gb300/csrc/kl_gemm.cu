// kl_gemm.cu - KL synthesis of the BF16 coefficient on the tensor cores (row a2).
//
// log a[s, c] = sum_k (sigma sqrt(lambda_k) xi[s, k]) * phi_k(x_c)  (Sec. 5 field
// model) is a dense (samples x modes) by (modes x cells) product.  It runs as a
// tcgen05 GEMM: BF16 operands staged by TMA into 128-byte-swizzled shared memory,
// FP32 accumulator in tensor memory, one elected thread issuing
// tcgen05.mma.cta_group::1.kind::f16 (M = 128 samples, N = 128 cells, K = 16 per
// instruction), and an epilogue that reads the accumulator with tcgen05.ld,
// applies exp and stores the BF16 coefficient (optionally also FP32 log a).
// The BF16 field feeds only the multigrid preconditioner; the accurate
// coefficient of the operator comes from the FP64 synthesis in field.cu.
//
// Every wait on an mbarrier is bounded: on timeout the kernel records an error
// code, waits (bounded) for the copies it issued, frees its tensor memory and
// returns.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "kernels.h"
#include "launch.h"

namespace mlsgd {

// K is short here (the mode count, 256 for the workload: four chunks), so two stages
// suffice; 66 KB of shared memory and 128 TMEM columns per CTA let three CTAs share
// an SM, so one CTA's epilogue (exp, BF16 stores) overlaps the others' loads and MMAs.
constexpr int GBM = 128, GBN = 128, GBK = 64, GSTAGES = 2;
constexpr int kGemmCtasPerSm = 3;
constexpr uint32_t GSTAGE_A = GBM * GBK * 2;  // 16 KB
constexpr uint32_t GSTAGE_B = GBN * GBK * 2;  // 16 KB
constexpr uint32_t kWaitLimit = 1u << 22;  // bounded polls of mbarrier.try_wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
// bounded wait: true when the phase completed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_try(bar, phase)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
// shared-memory matrix descriptor, K-major operand in the 128-byte swizzle layout:
// rows of 64 BF16 (128 B), 8-row atoms of 1024 B (stride byte offset), version 1
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;           // descriptor version
  d |= (uint64_t)2 << 61;           // SWIZZLE_128B
  return d;
}
// instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = GBN
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GBN >> 3) << 17) |
                            ((uint32_t)(GBM >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__global__ void __launch_bounds__(128, kGemmCtasPerSm)
    k_kl_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int S, int cells, int K,
              __nv_bfloat16* __restrict__ abf, float* __restrict__ loga, int* __restrict__ err) {
  extern __shared__ unsigned char gsm_raw[];
  // 1024-byte aligned base for the swizzled stages
  const uint32_t raw = su32(gsm_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t sA = base, sB = base + GSTAGES * GSTAGE_A;
  const uint32_t bars = sB + GSTAGES * GSTAGE_B;  // full[4], empty[4], done
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (GSTAGES + s); };
  const uint32_t done = bars + 8u * (2 * GSTAGES);
  const uint32_t tslot = done + 8u;
  unsigned char* gsm = gsm_raw + (base - raw);
  volatile uint32_t* tslot_ptr = (volatile uint32_t*)(gsm + (tslot - base));
  __shared__ int s_bad;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = (S + GBM - 1) / GBM;
  const int m0 = (blockIdx.x % mt) * GBM, n0 = (blockIdx.x / mt) * GBN;
  const int nch = K / GBK;

  if (tid == 0) {
    s_bad = 0;
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tslot), "r"(GBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot_ptr;

  int issued = 0;  // chunks whose TMA was issued (thread 0)
  if (tid == 0) {
    auto issue = [&](int c) {
      const int st = c % GSTAGES;
      mbar_expect_tx(full(st), GSTAGE_A + GSTAGE_B);
      tma_load_2d(sA + st * GSTAGE_A, &tmA, full(st), c * GBK, m0);
      tma_load_2d(sB + st * GSTAGE_B, &tmB, full(st), c * GBK, n0);
    };
    for (int c = 0; c < nch && c < GSTAGES; ++c) issue(c), ++issued;
    bool ok = true;
    for (int c = 0; c < nch && ok; ++c) {
      const int st = c % GSTAGES;
      const uint32_t ph = (c / GSTAGES) & 1;
      if (!mbar_wait(full(st), ph)) { ok = false; break; }
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < GBK / 16; ++ks) {
        const uint64_t ad = sw128_desc(sA + st * GSTAGE_A + ks * 32);
        const uint64_t bd = sw128_desc(sB + st * GSTAGE_B + ks * 32);
        const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty(st))
                   : "memory");
      if (c + GSTAGES < nch) {
        if (!mbar_wait(empty(st), ph)) { ok = false; break; }
        issue(c + GSTAGES);
        ++issued;
      }
    }
    if (ok)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                   : "memory");
    else
      s_bad = 1;
  }
  __syncthreads();
  bool good = s_bad == 0;
  if (good && !mbar_wait(done, 0)) good = false;
  const bool bad = __syncthreads_or(!good) != 0;
  if (bad) {
    if (tid == 0) {
      atomicExch(err, 1);
      // let the copies already issued land before the shared memory is released
      for (int c = 0; c < issued; ++c) (void)mbar_wait(full(c % GSTAGES), (c / GSTAGES) & 1);
    }
  } else {
    tc_fence_after();
    const int row = warp * 32 + lane;  // accumulator lane = sample row of the tile
    const int s = m0 + row;
#pragma unroll 1
    for (int cc = 0; cc < GBN; cc += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (s < S) {
        const long long o = (long long)s * cells + n0 + cc;
        if (loga) {
          float4* dst = reinterpret_cast<float4*>(loga + o);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                                 __uint_as_float(r[4 * q + 3]));
        }
        if (abf) {
          uint32_t packed[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const __nv_bfloat162 v =
                __floats2bfloat162_rn(expf(__uint_as_float(r[2 * q])), expf(__uint_as_float(r[2 * q + 1])));
            packed[q] = *reinterpret_cast<const uint32_t*>(&v);
          }
          uint4* dst = reinterpret_cast<uint4*>(abf + o);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(GBN) : "memory");
}

// A operand: A[s][k] = bf16(scale_k * xi[s][k])
__global__ void k_gemm_a(const double* __restrict__ xi, const double* __restrict__ scale, int S, int K,
                         __nv_bfloat16* __restrict__ A) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (long long)S * K) A[i] = __float2bfloat16_rn((float)(scale[i % K] * xi[i]));
}
// B operand (cells x K, K contiguous): phi_ix(x) phi_iy(y) phi_iz(z) at the cell centres
__global__ void k_gemm_b(const double* __restrict__ phi, const int* __restrict__ ix, const int* __restrict__ iy,
                         const int* __restrict__ iz, int N, int K, __nv_bfloat16* __restrict__ B) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long cells = (long long)N * N * N;
  if (i >= cells * K) return;
  const int k = (int)(i % K);
  const long long c = i / K;
  const int x = (int)(c % N), y = (int)((c / N) % N), z = (int)(c / ((long long)N * N));
  B[i] = __float2bfloat16_rn((float)(phi[ix[k] * N + x] * phi[iy[k] * N + y] * phi[iz[k] * N + z]));
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

static bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t K, uint32_t box_rows) {
  auto enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {K, rows};
  const cuuint64_t strides[1] = {K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)GBK, box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t kl_gemm_b_bytes(int N, int K) { return (size_t)N * N * N * K * 2; }
size_t kl_gemm_a_bytes(int S, int K) { return (size_t)S * K * 2; }

void kl_gemm_build_b(const double* phi, const int* ix, const int* iy, const int* iz, int N, int K, __nv_bfloat16* B,
                     cudaStream_t st) {
  const long long n = (long long)N * N * N * K;
  launch("gemm_b", (double)n * 2, k_gemm_b, dim3((unsigned)((n + 255) / 256)), 256, 0, st, phi, ix, iy, iz, N, K, B);
}

cudaError_t kl_gemm(const double* xi, const double* scale, int S, int K, const __nv_bfloat16* B, int N,
                    __nv_bfloat16* A_scratch, __nv_bfloat16* abf, float* loga, int* err, cudaStream_t st) {
  if (S == 0) return cudaSuccess;
  const long long cells = (long long)N * N * N;
  if (K % GBK != 0 || cells % GBN != 0) return cudaErrorInvalidValue;
  const long long na = (long long)S * K;
  launch("gemm_a", (double)na * 10, k_gemm_a, dim3((unsigned)((na + 255) / 256)), 256, 0, st, xi, scale, S, K,
         A_scratch);
  CUtensorMap ta, tb;
  if (!make_map(&ta, A_scratch, (uint64_t)S, (uint64_t)K, GBM) || !make_map(&tb, B, (uint64_t)cells, (uint64_t)K, GBN))
    return cudaErrorInvalidValue;
  const size_t smem = 1024 + GSTAGES * (GSTAGE_A + GSTAGE_B) + 8 * (2 * GSTAGES + 1) + 16;
  static bool smem_set = false;  // once per process (capture-friendly)
  if (!smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_kl_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = true;
  }
  const long long mt = (S + GBM - 1) / GBM, nt = cells / GBN;
  const double out_bytes = (double)S * cells * ((abf ? 2 : 0) + (loga ? 4 : 0));
  launch_flops("kl_gemm", out_bytes + (double)S * K * 2 + (double)cells * K * 2, 2.0 * S * (double)cells * K,
               k_kl_gemm, dim3((unsigned)(mt * nt)), 128, smem, st, ta, tb, S, (int)cells, K, abf, loga, err);
  return cudaGetLastError();
}

}  // namespace mlsgd
