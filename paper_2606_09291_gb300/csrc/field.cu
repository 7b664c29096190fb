// field.cu - random input xi and the log-normal coefficient field (rows a1, a2).
//
// xi^(m,l) ~ N(0,1) iid over modes, samples and levels (Sec. 2.2, after
// eq:delta-notation); the coefficient is exp of the truncated KL sum
// log a(x) = sigma sum_k sqrt(lambda_k) xi_k phi_ix(x) phi_iy(y) phi_iz(z)
// (Sec. 5 field model, with the exponential-covariance modes of this
// workload) evaluated at the cell centres of the requested grid.
#include "internal.cuh"
#include "kernels.h"
#include "launch.h"

namespace mlsgd {

// one thread per (sample, mode pair): counter = (pair, sample, level, iteration),
// key = seed; Box-Muller on two 53-bit uniforms.
// half_width > 0: xi uniform on (-half_width, half_width] from the same uniforms
__global__ void k_draw_xi(uint32_t key0, uint32_t key1, uint32_t iter, uint32_t level, long long first,
                          int S, int K, double half_width, double* __restrict__ xi) {
  const int pairs = (K + 1) / 2;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)S * pairs) return;
  const int s = (int)(idx / pairs), p = (int)(idx % pairs);
  const uint64_t sample = (uint64_t)(first + s);
  const U4 w = philox4x32_10(U4{(uint32_t)p, (uint32_t)sample, level, iter}, key0, key1);
  const double u1 = uniform53(w.x, w.y), u2 = uniform53(w.z, w.w);
  double v0, v1;
  if (half_width > 0.0) {
    v0 = -half_width + 2.0 * half_width * u1;
    v1 = -half_width + 2.0 * half_width * u2;
  } else {
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    v0 = r * cs;
    v1 = r * sn;
  }
  xi[(long long)s * K + 2 * p] = v0;
  if (2 * p + 1 < K) xi[(long long)s * K + 2 * p + 1] = v1;
}

void launch_draw_xi(uint64_t seed, int iter, int level, long long first, int S, int K, double* xi, cudaStream_t st,
                    double half_width) {
  const long long n = (long long)S * ((K + 1) / 2);
  if (n == 0) return;
  launch("xi", (double)S * K * 8, k_draw_xi, dim3((unsigned)((n + kBlock - 1) / kBlock)), kBlock, 0, st,
         (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), (uint32_t)iter, (uint32_t)level, first, S, K,
         half_width, xi);
}

// exp(la) for an FP32 result: FP64 range reduction la = k ln2 + r, |r| <= ln2/2,
// then the FP32 exponential of r scaled by 2^k (about 1.5 ulp of FP32; the FP64
// exponential is reserved for the FP64 coefficient).
__device__ __forceinline__ float exp_to_f32(double la) {
  const double k = rint(la * 1.4426950408889634);
  const double r = fma(-k, 0.6931471805599453, la);
  return ldexpf(expf((float)r), (int)k);
}

// Sum-factorised synthesis.  One block per (z plane, sample):
//   T2[i][y] = sum_{k : ix_k = i} c_k phi_{iy_k}(y) phi_{iz_k}(z),  c_k = scale_k xi_k
//   log a(x, y, z) = sum_i T2[i][y] phi_i(x)
// costs K N^2 + n1x N^3 FMA per sample instead of K N^3.
// Dynamic shared memory: c[K], phi[n1d][N], T2[n1x][N] (doubles).
__global__ void k_field(const double* __restrict__ xi, int K, const ModeTable mt, const double* __restrict__ phi,
                        int N, FieldOut out) {
  extern __shared__ double sm[];
  double* c = sm;
  double* ph = c + K;
  double* T2 = ph + mt.n1d * N;
  const int z = blockIdx.x, s = blockIdx.y;
  for (int k = threadIdx.x; k < K; k += blockDim.x) c[k] = mt.scale[k] * xi[(long long)s * K + k];
  for (int e = threadIdx.x; e < mt.n1d * N; e += blockDim.x) ph[e] = phi[e];
  __syncthreads();
  for (int e = threadIdx.x; e < mt.n1x * N; e += blockDim.x) {
    const int i = e / N, y = e % N;
    double acc = 0.0;
    for (int t = mt.offs[i]; t < mt.offs[i + 1]; ++t) {
      const int k = mt.order[t];
      acc += c[k] * ph[mt.iy[k] * N + y] * ph[mt.iz[k] * N + z];
    }
    T2[e] = acc;
  }
  __syncthreads();
  const long long cs = (long long)N * N * N;
  const long long base = (long long)s * cs + (long long)z * N * N;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int x = e % N, y = e / N;
    double la = 0.0;
    for (int i = 0; i < mt.n1x; ++i) la += T2[i * N + y] * ph[i * N + x];
    const long long o = base + e;
    if (out.log_a) out.log_a[o] = la;
    if (out.a64) out.a64[o] = exp(la);
    if (out.a32 || out.abf) {
      const float a = exp_to_f32(la);
      if (out.a32) out.a32[o] = a;
      if (out.abf) out.abf[o] = __float2bfloat16_rn(a);
    }
  }
}

// FP32-coefficient synthesis (the mixed path needs only a = exp(log a) rounded to
// FP32 and BF16).  One block per (chunk of kFieldPlanes z planes, sample): the 1D
// tables and c_k are split into FP32 pairs once per block (the only FP64 work),
// then per plane c_k phi_{iz_k}(z) is a pair product and stage 1 (T2) runs in FP32
// pair arithmetic;
// stage 2 contracts over i in pair arithmetic (exact products by FMA, two-sum
// accumulation: about 44 significant bits, far below the FP32 rounding of a), four
// consecutive cells in x per thread; exp by a Cody-Waite reduction against ln 2 split
// into a 16-bit head (exact multiples for |k| < 256) and its remainder, then expf.
// Dynamic shared memory: c_k phi(z) pairs and c_k pairs [K rounded up to even each],
// then T2 hi/lo [n1x][N] and phi hi/lo [n1d][N] (floats; 16-byte aligned for the
// float4 reads since N % 4 == 0 is required).
constexpr int kFieldPlanes = 16;
constexpr float kLn2Hi = 0.693145751953125f;        // ln 2 truncated to 16 bits
constexpr float kLn2Lo = 1.4286068202862268e-06f;   // ln 2 - kLn2Hi
__global__ void k_field_df(const double* __restrict__ xi, int K, const ModeTable mt, const double* __restrict__ phi,
                           int N, float* __restrict__ a32, __nv_bfloat16* __restrict__ abf) {
  extern __shared__ __align__(16) unsigned char smf[];
  float2* cz = reinterpret_cast<float2*>(smf);  // c_k phi_{iz_k}(z) as pairs
  float2* ck = cz + ((K + 1) & ~1);             // c_k as pairs
  float* T2h = reinterpret_cast<float*>(ck + ((K + 1) & ~1));
  float* T2l = T2h + mt.n1x * N;
  float* Ph = T2l + mt.n1x * N;  // all 1D tables as pairs
  float* Pl = Ph + mt.n1d * N;
  const int s = blockIdx.y;
  for (int k = threadIdx.x; k < K; k += blockDim.x) ck[k] = df_split(mt.scale[k] * xi[(long long)s * K + k]);
  for (int e = threadIdx.x; e < mt.n1d * N; e += blockDim.x) {
    const double v = phi[e];
    const float h = (float)v;
    Ph[e] = h;
    Pl[e] = (float)(v - (double)h);
  }
  const int z0 = kFieldPlanes * blockIdx.x, z1 = min(N, z0 + kFieldPlanes);
  for (int z = z0; z < z1; ++z) {
    __syncthreads();  // the tables (first plane); the previous plane's T2 reads done
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      const int o = mt.iz[k] * N + z;
      const DF v = df_mul(df_make(ck[k]), DF{Ph[o], Pl[o]});
      cz[k] = make_float2(v.h, v.l);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < mt.n1x * N; e += blockDim.x) {
      const int i = e / N, y = e % N;
      DF acc{0.f, 0.f};
      for (int t = mt.offs[i]; t < mt.offs[i + 1]; ++t) {
        const int k = mt.order[t];
        const int o = mt.iy[k] * N + y;
        acc = df_add(acc, df_mul(df_make(cz[k]), DF{Ph[o], Pl[o]}));
      }
      T2h[e] = acc.h;
      T2l[e] = acc.l;
    }
    __syncthreads();
    const long long base = (long long)s * N * N * N + (long long)z * N * N;
    const int nq = N / 4;
    for (int e = threadIdx.x; e < N * nq; e += blockDim.x) {
      const int x0 = 4 * (e % nq), y = e / nq;
      float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
      for (int i = 0; i < mt.n1x; ++i) {
        const float th = T2h[i * N + y], tl = T2l[i * N + y];
        const float4 phv = *reinterpret_cast<const float4*>(Ph + i * N + x0);
        const float4 plv = *reinterpret_cast<const float4*>(Pl + i * N + x0);
        const float pv[4] = {phv.x, phv.y, phv.z, phv.w}, lv[4] = {plv.x, plv.y, plv.z, plv.w};
  #pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float p = __fmul_rn(th, pv[q]);
          const float pe = __fmaf_rn(th, lv[q], __fmaf_rn(tl, pv[q], __fmaf_rn(th, pv[q], -p)));
          const float sum = __fadd_rn(S[q], p);  // two-sum of S and p (intrinsics: never contracted)
          const float bb = __fsub_rn(sum, S[q]);
          C[q] = __fadd_rn(C[q], __fadd_rn(__fadd_rn(__fsub_rn(S[q], __fsub_rn(sum, bb)), __fsub_rn(p, bb)), pe));
          S[q] = sum;
        }
      }
      float av[4];
  #pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float kf = rintf(S[q] * 1.44269504f);
        const float r = ((S[q] - kf * kLn2Hi) - kf * kLn2Lo) + C[q];
        av[q] = ldexpf(expf(r), (int)kf);
      }
      const long long o = base + (long long)y * N + x0;
      if (a32) *reinterpret_cast<float4*>(a32 + o) = make_float4(av[0], av[1], av[2], av[3]);
      if (abf) {
  #pragma unroll
        for (int q = 0; q < 4; ++q) abf[o + q] = __float2bfloat16_rn(av[q]);
      }
    }
  }
}

size_t field_smem_bytes(const ModeTable& mt, int K, int N) {
  return sizeof(double) * ((size_t)K + (size_t)mt.n1d * N + (size_t)mt.n1x * N);
}

cudaError_t launch_field(const double* xi, int K, const ModeTable& mt, const double* phi, int N, int S,
                         const FieldOut& out, cudaStream_t st) {
  if (S == 0) return cudaSuccess;
  if (!out.log_a && !out.a64 && (out.a32 || out.abf) && N % 4 == 0) {
    const size_t smem = 2 * sizeof(float2) * (size_t)((K + 1) & ~1) +
                        sizeof(float) * (2 * (size_t)mt.n1x * N + 2 * (size_t)mt.n1d * N);
    static size_t smem_df = 48 * 1024;
    if (smem > smem_df) {
      cudaError_t e = cudaFuncSetAttribute(k_field_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      smem_df = smem;
    }
    const double cells = (double)S * N * N * N;
    launch_flops("field", (double)S * K * 8 + cells * ((out.a32 ? 4 : 0) + (out.abf ? 2 : 0)),
                 2.0 * cells * mt.n1x + 2.0 * (double)S * K * N * N, k_field_df,
                 dim3((unsigned)((N + kFieldPlanes - 1) / kFieldPlanes), S), kBlock, smem, st, xi, K,
                 mt, phi, N, out.a32, out.abf);
    return cudaGetLastError();
  }
  const size_t smem = field_smem_bytes(mt, K, N);
  static size_t smem_set = 48 * 1024;  // raised once per size (not on every enqueue: capture-friendly)
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  const double cells = (double)S * N * N * N;
  const double outb = cells * ((out.log_a ? 8 : 0) + (out.a64 ? 8 : 0) + (out.a32 ? 4 : 0) + (out.abf ? 2 : 0));
  launch_flops("field", (double)S * K * 8 + outb, 2.0 * cells * mt.n1x + 2.0 * (double)S * K * N * N, k_field,
               dim3(N, S), kBlock, smem, st, xi, K, mt, phi, N, out);
  return cudaGetLastError();
}

// exp of a stored log field (used when the caller passes log a)
template <typename TO>
__global__ void k_exp_field(const double* __restrict__ la, TO* __restrict__ a, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (TO)exp(la[i]);
}
__global__ void k_exp_field_mixed(const double* __restrict__ la, float* __restrict__ a32,
                                  __nv_bfloat16* __restrict__ abf, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double a = exp(la[i]);
    a32[i] = (float)a;
    abf[i] = __float2bfloat16_rn((float)a);
  }
}

void launch_exp_field(const double* la, const FieldOut& out, long long n, cudaStream_t st) {
  if (n == 0) return;
  const unsigned g = (unsigned)((n + kBlock - 1) / kBlock);
  if (out.a64) launch("expfield", (double)n * 16, k_exp_field<double>, dim3(g), kBlock, 0, st, la, out.a64, n);
  if (out.a32 && out.abf)
    launch("expfield", (double)n * 14, k_exp_field_mixed, dim3(g), kBlock, 0, st, la, out.a32, out.abf, n);
}

}  // namespace mlsgd
