// Conventional correlation of partial-WHT FP32 plans on the tensor cores.
//
// h = Phi^H r = A^H zf_Omega(r) (Algorithm 1.1 step 2) with A the Sylvester
// Walsh–Hadamard matrix scaled by 1/sqrt(N): the fast Hadamard transform of
// the zero-filled residual (the FHT whose cost Sec. III-B and Table I count,
// N log2 N additions).  H_N = H_16 (x) H_16 (x) ... (x) H_{2^r}, so every
// radix-16 stage multiplies each 16-point group of the vector (the 16 indices
// that differ only in one 4-bit digit) by the 16 x 16 matrix H_16 of +-1
// entries: a dense contraction, run here as tcgen05 MMAs.
//
//   A operand  the groups, 128 per MMA (M = 128, one group per row, K = 16),
//              FP32 data split into three BF16 parts hi + mid + lo that sum to
//              the FP32 value exactly (8 + 8 + 8 significant bits);
//   B operand  H_16 in BF16 (+-1, exact), N = 16;
//   D          FP32 accumulators in tensor memory: the three parts' products
//              accumulate into the same D (D = H x_hi, then += H x_mid,
//              += H x_lo), so the only rounding is the FP32 accumulation.
//
// One CTA of 128 threads (one warpgroup: thread t reads TMEM lane t, i.e.
// row t of every D tile) transforms V vectors at a time (V N = 4096 elements,
// up to 2 tiles of 128 groups per stage; about 41 KB of shared memory, so
// five CTAs share an SM).  Per stage: the threads write the
// split A tiles, one thread issues 3 MMAs per tile and commits them to an
// mbarrier, the threads wait on it (bounded), read D with tcgen05.ld and
// write the results back.  A last radix-2^r stage (r = log2 N mod 4) runs on
// the CUDA cores; its output goes straight to h and to the arg-max of step 3.
#include "cs_internal.h"
#include "cs_blocks.cuh"

#include <cuda_bf16.h>

namespace csf {

namespace {

constexpr int kTT = 128;            // threads per CTA: one warpgroup
constexpr int kElems = 4096;        // elements (V vectors x N) per CTA round
constexpr int kMaxTiles = kElems / 16 / 128;  // 128-row tiles per stage: 2
constexpr int kTileBytes = 4096;    // 128 rows x 16 BF16
constexpr int kTmemCols = 16 * kMaxTiles;     // one 16-column FP32 accumulator per tile
constexpr long long kSpinLimit = 1LL << 22;   // bound on the mbarrier wait (about a second)
// instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

// Physical position of element e of the round's buffer: the low 4 bits are
// XORed with bits 4-7, so that the 16-strided, 256-strided and contiguous
// group accesses of the three stages spread over the banks (at most 2-way).
__device__ __forceinline__ int phys(int e) { return e ^ ((e >> 4) & 15); }

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) in a canonical K-major tile without
// swizzle: 8 x 8 core matrices of 128 contiguous bytes (8 rows of 16 bytes),
// the two K halves 128 bytes apart (leading byte offset), row groups of 8
// 256 bytes apart (stride byte offset).
__device__ __forceinline__ int tile_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1 at bits 46-47, base
// offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 FP32 accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + mid + lo with three BF16 values (exact for normal FP32 x: each
// part takes the next 8 significant bits, the remainders are exact in FP32).
__device__ __forceinline__ void split3(float x, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(mid);
  lo = __float2bfloat16_rn(r2);
}

struct TcSmem {
  size_t vec, a, b, total;
};

__host__ __device__ inline TcSmem tc_layout() {
  TcSmem L;
  L.a = 0;                                              // kMaxTiles x 3 split tiles, 1024-aligned
  L.b = L.a + (size_t)kMaxTiles * 3 * kTileBytes;       // H_16, 512 bytes
  L.vec = L.b + 1024;                                   // the round's vectors, FP32
  L.total = L.vec + (size_t)kElems * sizeof(float);
  return L;
}

// In-register WHT of 2^R points (R <= 3), natural order.
template <int R>
__device__ __forceinline__ void wht_small(float* x) {
#pragma unroll
  for (int h = 1; h < (1 << R); h <<= 1) {
#pragma unroll
    for (int i = 0; i < (1 << R); ++i) {
      if (i & h) continue;
      const float a = x[i], b = x[i + h];
      x[i] = a + b;
      x[i + h] = a - b;
    }
  }
}

// The radix-2^R stage on index bits [sh, sh + R) of the V vectors (CUDA cores).
template <int R>
__device__ void tail_stage(float* vec, int V, int logN, int sh) {
  const int gbits = logN - R, Gr = 1 << gbits;
  for (int q = threadIdx.x; q < (V << gbits); q += kTT) {
    const int v = q >> gbits, gi = q & (Gr - 1);
    const int base = (v << logN) + (gi & ((1 << sh) - 1)) + ((gi >> sh) << (sh + R));
    float x[1 << R];
#pragma unroll
    for (int d = 0; d < (1 << R); ++d) x[d] = vec[phys(base + (d << sh))];
    wht_small<R>(x);
#pragma unroll
    for (int d = 0; d < (1 << R); ++d) vec[phys(base + (d << sh))] = x[d];
  }
}

__global__ void __launch_bounds__(kTT) wht_tc_kernel(PlanDev<float> P, const float* __restrict__ r, int64_t batch,
                                                     float* __restrict__ h, int32_t* __restrict__ amax,
                                                     int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int fail;
  const TcSmem L = tc_layout();
  float* vec = (float*)(sm + L.vec);
  unsigned char* A = sm + L.a;
  unsigned char* B = sm + L.b;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int N = P.N, logN = P.logN, S = logN >> 2, R = logN & 3;
  const int gbits = logN - 4;  // groups of 16 per vector: 2^gbits
  const int Vmax = kElems >> logN;
  const uint32_t mb = saddr(&mbar);

  // H_16 in BF16 (entries +-1, exact), the B operand of every MMA
  for (int i = t; i < 256; i += kTT) {
    const int n = i >> 4, k = i & 15;
    *(__nv_bfloat16*)(B + tile_off(n, k)) = __float2bfloat16_rn((__popc(n & k) & 1) ? -1.f : 1.f);
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t parity = 0;
  const float scl = inv_sqrt_pow2<float>(logN);
  const int64_t rounds = (batch + Vmax - 1) / Vmax;
  for (int64_t rd = blockIdx.x; rd < rounds; rd += gridDim.x) {
    const int64_t b0 = rd * Vmax;
    const int V = (int)((batch - b0) < Vmax ? (batch - b0) : Vmax);
    // zero-filled, scaled residuals (Algorithm 1.1 step 2: A^H zf_Omega(r))
    for (int e = t; e < (V << logN); e += kTT) {
      const int v = e >> logN, pos = e & (N - 1);
      const int m = __ldg(P.slot + pos);
      vec[phys(e)] = m >= 0 ? __ldg(r + (b0 + v) * P.M + m) * scl : 0.f;
    }
    __syncthreads();
    const int rows = V << gbits;
    const int tiles = (rows + 127) >> 7;
    for (int s = 0; s < S; ++s) {
      const int sh = 4 * s;
      // the split A tiles: row = one group of 16 points, K = the digit
      for (int c = 0; c < tiles; ++c) {
        const int row = (c << 7) + t;
        uint32_t w[3][8];
        if (row < rows) {
          const int v = row >> gbits, gi = row & ((1 << gbits) - 1);
          const int base = (v << logN) + (gi & ((1 << sh) - 1)) + ((gi >> sh) << (sh + 4));
#pragma unroll
          for (int d = 0; d < 16; d += 2) {
            __nv_bfloat16 h0, m0, l0, h1, m1, l1;
            split3(vec[phys(base + (d << sh))], h0, m0, l0);
            split3(vec[phys(base + ((d + 1) << sh))], h1, m1, l1);
            w[0][d >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            w[1][d >> 1] = (uint32_t)__bfloat16_as_ushort(m0) | ((uint32_t)__bfloat16_as_ushort(m1) << 16);
            w[2][d >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int i = 0; i < 8; ++i) w[q][i] = 0u;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          unsigned char* At = A + (size_t)(c * 3 + q) * kTileBytes;
          *(uint4*)(At + tile_off(t, 0)) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
          *(uint4*)(At + tile_off(t, 8)) = make_uint4(w[q][4], w[q][5], w[q][6], w[q][7]);
        }
      }
      // generic-proxy writes -> visible to the tensor cores' async proxy
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (t == 0) {
        const uint64_t bd = smem_desc(saddr(B));
        for (int c = 0; c < tiles; ++c) {
          const uint32_t a0 = saddr(A + (size_t)c * 3 * kTileBytes);
          const uint32_t d = tmem + 16 * c;
          mma_f16(d, smem_desc(a0), bd, 0u);                   // D  = H x_hi
          mma_f16(d, smem_desc(a0 + kTileBytes), bd, 1u);      // D += H x_mid
          mma_f16(d, smem_desc(a0 + 2 * kTileBytes), bd, 1u);  // D += H x_lo
        }
        mma_commit(mb);
      }
      // completion of this stage's MMAs (bounded wait)
      long long spins = 0;
      while (!mbar_try_wait(mb, parity)) {
        if (++spins > kSpinLimit) {
          fail = 1;
          break;
        }
      }
      parity ^= 1u;
      tc_fence_after();
      __syncthreads();
      if (fail) break;
      for (int c = 0; c < tiles; ++c) {
        float dv[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * c), dv);
        const int row = (c << 7) + t;
        if (row < rows) {
          const int v = row >> gbits, gi = row & ((1 << gbits) - 1);
          const int base = (v << logN) + (gi & ((1 << sh) - 1)) + ((gi >> sh) << (sh + 4));
#pragma unroll
          for (int d = 0; d < 16; ++d) vec[phys(base + (d << sh))] = dv[d];
        }
      }
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
    if (fail) break;
    if (R == 1) tail_stage<1>(vec, V, logN, 4 * S);
    else if (R == 2) tail_stage<2>(vec, V, logN, 4 * S);
    else if (R == 3) tail_stage<3>(vec, V, logN, 4 * S);
    __syncthreads();
    // h and the arg-max of step 3 (largest |h(j)|^2, lowest j on ties), one
    // warp per vector
    for (int v = warp; v < V; v += kTT / 32) {
      float bv = -1.f;
      int bj = 0x7fffffff;
      float* hb = h ? h + (b0 + v) * N : nullptr;
      for (int j = lane; j < N; j += 32) {
        const float x = vec[phys((v << logN) + j)];
        if (hb) hb[j] = x;
        const float a = x * x;
        if (better(a, j, bv, bj)) {
          bv = a;
          bj = j;
        }
      }
      warp_argmax(bv, bj);
      if (lane == 0 && amax) amax[b0 + v] = bj;
    }
    __syncthreads();
  }
  if (fail) {  // the MMAs did not complete in time: wait once more (bounded) before releasing TMEM
    long long spins = 0;
    while (!mbar_try_wait(mb, parity ^ 1u) && ++spins < kSpinLimit) {
    }
    if (t == 0) atomicOr(status, kStatusTcTimeout);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

// WHT FP32 plans take the tensor-core transform for 16 <= N <= 512 by
// default (measured on GB300: 2.3x the CUDA-core butterflies' throughput at
// N = 256, where one 256-thread CTA per vector leaves the butterfly kernel
// latency-bound), and up to N = 4096 when the plan asks for it
// (CS_PLAN_TENSOR_CORES; slower than the butterflies from N = 1024 on).
bool wht_tc_applies(const PlanView& P) {
  if (P.dft || !P.fp32 || P.large || P.logN < 4) return false;
  return P.logN <= (P.tc ? 12 : 9);
}

cudaError_t launch_correlate_wht_tc(const PlanView& P, const void* r, int64_t batch, void* h, int32_t* amax,
                                    cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  const size_t smem = tc_layout().total;
  cudaError_t e = raise_smem_limit((const void*)wht_tc_kernel, smem);
  if (e != cudaSuccess) return e;
  // as much of the unified L1 / shared memory as possible goes to shared
  // memory, so that several CTAs share an SM and hide each other's latency
  e = cudaFuncSetAttribute(wht_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  // CTAs per SM by shared memory (each also holds kTmemCols of the 512
  // tensor-memory columns, which allows up to 16)
  int per_sm = smem_sm / (int)(smem + 2048);
  per_sm = per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm);
  const int64_t vmax = kElems >> P.logN;
  const int64_t rounds = (batch + vmax - 1) / vmax;
  const int64_t cap = (int64_t)per_sm * sms;
  const int grid = (int)(rounds < cap ? rounds : cap);
  wht_tc_kernel<<<grid, kTT, smem, st>>>(plan_dev<float>(P), (const float*)r, batch, (float*)h, amax, P.status);
  return cudaGetLastError();
}

}  // namespace csf
