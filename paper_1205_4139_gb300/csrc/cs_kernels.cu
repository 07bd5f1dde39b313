// Kernels and their launchers.
//
// Element type E selects (kind, precision): float / double = Walsh-Hadamard
// (real), float2 / double2 = Fourier (complex).  W = FT<E>::W is the FP64
// element of the least-squares side.
#include "cs_blocks.cuh"
#include "cs_internal.h"

namespace csf {

template <class E>
static PlanDev<E> plan_dev(const PlanView& P) {
  PlanDev<E> d;
  d.N = P.N;
  d.logN = P.logN;
  d.M = P.M;
  d.slot = P.slot;
  constexpr bool f32 = sizeof(typename FT<E>::R) == 4;
  d.tw = (const E*)(f32 ? P.tw32 : P.tw64);
  d.c = (const E*)(f32 ? P.c32 : P.c64);
  d.c64 = (const typename FT<E>::W*)P.c64;
  return d;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// ------------------------------------------------------------ plan tables
// DIF twiddles W_{L_p}^{n q} = exp(-2 pi i n q / L_p) of every pass, FP64
// via sincospi (exact argument: L_p is a power of two) and rounded to FP32.
__global__ void twiddle_kernel(int logN, double2* tw64, float2* tw32) {
  const int N = 1 << logN, P = sched_passes(logN);
  for (int p = 0; p < P; ++p) {
    const int L = 1 << sched_logL(logN, p), R = 1 << sched_logR(logN, p), S = L / R, off = N - L;
    const int cnt = (R - 1) * S;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
      const int q = i / S + 1, n = i % S;
      double sn, cs;
      sincospi(-2.0 * (double)(n * q) / (double)L, &sn, &cs);
      tw64[off + i] = make_double2(cs, sn);
      if (tw32) tw32[off + i] = make_float2((float)cs, (float)sn);
    }
  }
}

// c = N^{-1/2} U^H S^T S U e_1 = N^{-1} F^H zf(1) (DFT) or N^{-1} H zf(1)
// (WHT) (Eq. kernelsum), computed with the FP64 block transform; the final
// scaling by N^{-1} is exact.
template <class W>
__global__ void kernel_vector_kernel(PlanDev<W> P, W* c64) {
  extern __shared__ __align__(16) unsigned char sm[];
  W* buf = (W*)sm;
  for (int pos = threadIdx.x; pos < P.N; pos += blockDim.x) {
    const int m = P.slot[pos];
    buf[swz<W>(pos)] = m >= 0 ? make_w<W>(1.0, 0.0) : zero<W>();
  }
  __syncthreads();
  transform_adjoint<W, FT<W>::C>(buf, P);
  const double inv = 1.0 / (double)P.N;
  for (int j = threadIdx.x; j < P.N; j += blockDim.x) c64[j] = scale(buf[swz<W>(j)], inv);
}

template <class W, class E>
__global__ void round_kernel(const W* a, E* b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = from_w<E>(a[i]);
}

cudaError_t launch_twiddles(const PlanView& P, void* tw64, void* tw32, cudaStream_t st) {
  twiddle_kernel<<<64, kThreads, 0, st>>>(P.logN, (double2*)tw64, (float2*)tw32);
  return cudaGetLastError();
}

template <class W>
static cudaError_t kv_impl(const PlanView& P, void* c64, cudaStream_t st) {
  const size_t smem = (size_t)P.N * sizeof(W);
  cudaError_t e = cudaFuncSetAttribute(kernel_vector_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel_vector_kernel<W><<<1, kThreads, smem, st>>>(plan_dev<W>(P), (W*)c64);
  return cudaGetLastError();
}

cudaError_t launch_kernel_vector(const PlanView& P, void* c64, void* c32, cudaStream_t st) {
  cudaError_t e = P.dft ? kv_impl<double2>(P, c64, st) : kv_impl<double>(P, c64, st);
  if (e != cudaSuccess || !c32) return e;
  if (P.dft) round_kernel<double2, float2><<<16, kThreads, 0, st>>>((const double2*)c64, (float2*)c32, P.N);
  else round_kernel<double, float><<<16, kThreads, 0, st>>>((const double*)c64, (float*)c32, P.N);
  return cudaGetLastError();
}

// ---------------------------------------------------- conventional correlation
template <class E>
__global__ void __launch_bounds__(kThreads) correlate_kernel(PlanDev<E> P, const E* __restrict__ r, int64_t batch,
                                                             E* h, int32_t* amax) {
  using V = typename NormT<E>::V;
  extern __shared__ __align__(16) unsigned char sm[];
  E* buf = (E*)sm;
  V* rv = (V*)(sm + align16((size_t)P.N * sizeof(E)));
  int* rj = (int*)(rv + 34);
  for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
    correlate_transform<E, FT<E>::C>(buf, P, r + b * P.M);
    const int j = argmax_buffer(buf, P.N, nullptr, h ? h + b * P.N : nullptr, rv, rj);
    if (amax && threadIdx.x == 0) amax[b] = j;
  }
}

template <class E>
static cudaError_t corr_impl(const PlanView& P, const void* r, int64_t batch, void* h, int32_t* amax,
                             cudaStream_t st) {
  using V = typename NormT<E>::V;
  const size_t smem = align16((size_t)P.N * sizeof(E)) + 34 * sizeof(V) + 34 * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(correlate_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = batch < (int64_t)sms * 8 ? batch : (int64_t)sms * 8;
  correlate_kernel<E><<<(int)grid, kThreads, smem, st>>>(plan_dev<E>(P), (const E*)r, batch, (E*)h, amax);
  return cudaGetLastError();
}

cudaError_t launch_correlate(const PlanView& P, const void* r, int64_t batch, void* h, int32_t* amax,
                             cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (P.dft) return P.fp32 ? corr_impl<float2>(P, r, batch, h, amax, st) : corr_impl<double2>(P, r, batch, h, amax, st);
  return P.fp32 ? corr_impl<float>(P, r, batch, h, amax, st) : corr_impl<double>(P, r, batch, h, amax, st);
}

// ------------------------------------------------------------ fast correlation
template <class E>
__global__ void __launch_bounds__(kThreads) fast_kernel(PlanDev<E> P, const E* __restrict__ h0,
                                                        const int32_t* __restrict__ supp,
                                                        const E* __restrict__ x, int s, int64_t batch,
                                                        E* h, int32_t* amax) {
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = P.N;
  const bool dbl = kernel_doubled<E>(N);
  E* cb = (E*)sm;
  size_t off = align16((size_t)(dbl ? 2 * N : N) * sizeof(E));
  E* xw = (E*)(sm + off);
  off = align16(off + (size_t)s * sizeof(E));
  int* lam = (int*)(sm + off);
  off = align16(off + (size_t)s * sizeof(int));
  uint32_t* bits = (uint32_t*)(sm + off);
  const int nbits = (N + 31) >> 5;
  off = align16(off + (size_t)nbits * sizeof(uint32_t));
  V* rv = (V*)(sm + off);
  int* rj = (int*)(rv + 34);
  load_kernel_vector<E, DFT>(cb, P, dbl);
  for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
    for (int i = threadIdx.x; i < nbits; i += blockDim.x) bits[i] = 0u;
    // indices are reduced mod N so that no input can address outside c
    for (int k = threadIdx.x; k < s; k += blockDim.x) { lam[k] = supp[b * s + k] & (N - 1); xw[k] = x[b * s + k]; }
    __syncthreads();
    for (int k = threadIdx.x; k < s; k += blockDim.x) atomicOr(bits + (lam[k] >> 5), 1u << (lam[k] & 31));
    __syncthreads();
    const int j = correlate_fast<E, DFT>(cb, h0 + b * N, lam, xw, s, N, bits, h ? h + b * N : nullptr, rv, rj, dbl);
    if (amax && threadIdx.x == 0) amax[b] = j;
  }
}

template <class E>
static cudaError_t fast_impl(const PlanView& P, const void* h0, const int32_t* supp, const void* x, int s,
                             int64_t batch, void* h, int32_t* amax, cudaStream_t st) {
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  const int N = P.N;
  size_t smem = align16((size_t)(kernel_doubled<E>(N) ? 2 * N : N) * sizeof(E));
  smem = align16(smem + (size_t)s * sizeof(E));
  smem = align16(smem + (size_t)s * sizeof(int));
  smem = align16(smem + (size_t)((N + 31) >> 5) * sizeof(uint32_t));
  smem += 34 * sizeof(V) + 34 * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(fast_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = batch < (int64_t)sms * 4 ? batch : (int64_t)sms * 4;
  fast_kernel<E><<<(int)grid, kThreads, smem, st>>>(plan_dev<E>(P), (const E*)h0, supp, (const E*)x, s, batch,
                                                    (E*)h, amax);
  return cudaGetLastError();
}

cudaError_t launch_correlate_fast(const PlanView& P, const void* h0, const int32_t* supp, const void* x, int s,
                                  int64_t batch, void* h, int32_t* amax, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (P.dft) return P.fp32 ? fast_impl<float2>(P, h0, supp, x, s, batch, h, amax, st)
                           : fast_impl<double2>(P, h0, supp, x, s, batch, h, amax, st);
  return P.fp32 ? fast_impl<float>(P, h0, supp, x, s, batch, h, amax, st)
                : fast_impl<double>(P, h0, supp, x, s, batch, h, amax, st);
}

// ------------------------------------------------------------------- OMP
enum { PATH_FAST = 0, PATH_CONV = 1, PATH_HYBRID = 2 };

template <class E>
struct OmpArgs {
  PlanDev<E> P;
  const E* __restrict__ y;
  int64_t batch;
  int K;
  double rel_tol;
  int path, t_switch;
  typename FT<E>::W* x_out;
  int* supp_out;
  int* iters_out;
  double* res_out;
  E* h0_ws;
  typename FT<E>::W* B_ws;
  int* counter;
};

template <class E>
struct OmpSmem {
  size_t regA, z, x, g, part, xw, red, rv, rj, lam, bits, total;
};

template <class E>
__host__ __device__ inline OmpSmem<E> omp_layout(int N, int K, int path, int T) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  OmpSmem<E> L;
  size_t o = 0;
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const int Kc = K > 0 ? K : 1;
  L.regA = o; o = a16(o + (size_t)((path != PATH_CONV && kernel_doubled<E>(N)) ? 2 * N : N) * sizeof(E));
  L.z = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.x = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.g = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.part = o; o = a16(o + (size_t)(T > Kc ? T : Kc) * sizeof(W));
  L.xw = o;   o = a16(o + (size_t)Kc * sizeof(E));
  L.red = o;  o = a16(o + (size_t)(32 * 4 + 4) * sizeof(double));
  L.rv = o;   o = a16(o + 34 * sizeof(V));
  L.rj = o;   o = a16(o + 34 * sizeof(int));
  L.lam = o;  o = a16(o + (size_t)Kc * sizeof(int));
  L.bits = o; o = a16(o + (size_t)((N + 31) >> 5) * sizeof(uint32_t));
  L.total = o;
  return L;
}

template <class E>
__global__ void __launch_bounds__(kThreads, (sizeof(E) > 8 ? 2 : 3)) omp_kernel(OmpArgs<E> a) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = a.P.N, M = a.P.M, K = a.K, T = blockDim.x, tid = threadIdx.x;
  const OmpSmem<E> Ls = omp_layout<E>(N, K, a.path, T);
  E* regA = (E*)(sm + Ls.regA);
  W* z = (W*)(sm + Ls.z);
  W* x = (W*)(sm + Ls.x);
  W* g = (W*)(sm + Ls.g);
  W* part = (W*)(sm + Ls.part);
  E* xw = (E*)(sm + Ls.xw);
  double* red = (double*)(sm + Ls.red);
  V* rv = (V*)(sm + Ls.rv);
  int* rj = (int*)(sm + Ls.rj);
  int* lam = (int*)(sm + Ls.lam);
  uint32_t* bits = (uint32_t*)(sm + Ls.bits);
  __shared__ int s_inst, s_state;
  __shared__ double s_rn2, s_invd;
  __shared__ W s_zeta;
  const int nbits = (N + 31) >> 5;
  const bool dbl = kernel_doubled<E>(N);

  E* h0 = a.h0_ws + (size_t)blockIdx.x * N;
  W* B = a.B_ws + (size_t)blockIdx.x * (((size_t)K * (K + 1)) >> 1);
  const double c0 = re(a.P.c64[0]);                       // c(0) = M/N
  const double dep = 1e-10 * ((double)M / (double)N);     // dependence threshold on d^2
  const double tol2 = a.rel_tol * a.rel_tol;

  for (;;) {
    if (tid == 0) s_inst = atomicAdd(a.counter, 1);
    __syncthreads();
    const int64_t b = s_inst;
    __syncthreads();
    if (b >= a.batch) break;
    const E* y = a.y + b * M;
    for (int i = tid; i < nbits; i += T) bits[i] = 0u;

    // t = 1: h_0 = Phi^H y by one transform (Eq. kernelsumOMP, first case)
    double yy[1] = {correlate_transform<E, DFT, true>(regA, a.P, y)};
    block_sum(yy, red);
    const double ynorm2 = yy[0];
    int p = 0;
    if (tid == 0) s_rn2 = ynorm2;
    if (ynorm2 > 0.0 && K > 0) {
      int lnew = argmax_buffer(regA, N, nullptr, h0, rv, rj);  // step 3, and h_0 kept for later
      bool c_in_smem = false;
      while (lnew >= 0) {
        // ---- step 6: least squares, one more column ----
        for (int k = tid; k < p; k += T) {
          const int d = DFT ? ((lam[k] - lnew) & (N - 1)) : (lam[k] ^ lnew);
          g[k] = a.P.c64[d];                                 // G(lambda_k, lambda_new)
        }
        __syncthreads();
        tri_matvec(B, g, part, p);                           // g <- u = B g
        // Scalar FP64 work by one warp only: on this part every FP64 warp
        // instruction costs the same whatever its active lanes, so the other
        // warps wait at the barrier instead of repeating it.
        if (tid < 32) {
          double an = 0.0, ar = 0.0, ai = 0.0;
          for (int k = tid; k < p; k += 32) {
            an += norm2(g[k]);
            const W t = cmul(g[k], z[k]);
            ar += re(t);
            ai += im(t);
          }
          an = warp_sum(an);
          ar = warp_sum(ar);
          if constexpr (DFT) ai = warp_sum(ai);
          if (tid == 0) {
            const double d2 = c0 - an;
            int st = 0;
            if (!(d2 > dep)) {
              st = 1;                                        // column dependent on Lambda
            } else {
              const double invd = 1.0 / sqrt(d2);
              const W bp = to_w(h0[lnew]);                    // (Phi^H y)(lambda_new)
              const W zeta = scale(sub(bp, make_w<W>(ar, ai)), invd);
              const double r2 = s_rn2 - norm2(zeta);
              s_rn2 = r2;
              s_invd = invd;
              s_zeta = zeta;
              if (p + 1 >= K || r2 < tol2 * ynorm2) st = 2;  // step 8 after this column
            }
            s_state = st;
          }
        }
        __syncthreads();
        const int st = s_state;
        if (st == 1) break;
        const double invd = s_invd;
        const W zeta = s_zeta;
        tri_vecmat_row(B, g, part, p, -invd);                // row p of B (part[0..p))
        for (int k = tid; k < p; k += T) {
          const W xk = fmacv(x[k], part[k], zeta);
          x[k] = xk;
          xw[k] = from_w<E>(xk);
        }
        if (tid == 0) {
          B[pidx(p) + p] = make_w<W>(invd, 0.0);
          z[p] = zeta;
          const W xp = scale(zeta, invd);
          x[p] = xp;
          xw[p] = from_w<E>(xp);
          lam[p] = lnew;
          bits[lnew >> 5] |= 1u << (lnew & 31);
        }
        __syncthreads();
        ++p;
        // ---- step 8: halting ----
        if (st == 2) break;
        // ---- steps 2-3 at t = p + 1 ----
        const int t = p + 1;
        const bool fast = a.path == PATH_FAST || (a.path == PATH_HYBRID && t <= a.t_switch);
        if (fast) {
          if (!c_in_smem) { load_kernel_vector<E, DFT>(regA, a.P, dbl); c_in_smem = true; }
          lnew = correlate_fast<E, DFT>(regA, h0, lam, xw, p, N, bits, nullptr, rv, rj, dbl);
        } else {
          c_in_smem = false;
          correlate_residual<E, DFT>(regA, a.P, y, lam, xw, p);
          lnew = argmax_buffer<E>(regA, N, bits, nullptr, rv, rj);
        }
      }
    }
    // outputs
    for (int k = tid; k < K; k += T) {
      if (a.x_out) a.x_out[b * K + k] = k < p ? x[k] : W{};
      a.supp_out[b * K + k] = k < p ? lam[k] : -1;   // K > 0 here, so supp_out is set
    }
    if (tid == 0) {
      if (a.iters_out) a.iters_out[b] = p;
      if (a.res_out) a.res_out[b] = ynorm2 > 0.0 ? sqrt(fmax(s_rn2, 0.0) / ynorm2) : 0.0;
    }
    __syncthreads();
  }
}

template <class E>
static size_t omp_smem_t(const PlanView& P, int K, int path) {
  return omp_layout<E>(P.N, K, path, kThreads).total;
}

size_t omp_smem_bytes(const PlanView& P, int K, int path) {
  if (P.dft) return P.fp32 ? omp_smem_t<float2>(P, K, path) : omp_smem_t<double2>(P, K, path);
  return P.fp32 ? omp_smem_t<float>(P, K, path) : omp_smem_t<double>(P, K, path);
}

template <class E>
static int omp_grid_t(const PlanView& P, int K, int path, int64_t batch, int* err) {
  const size_t smem = omp_smem_t<E>(P, K, path);
  *err = 0;
  cudaError_t e = cudaFuncSetAttribute(omp_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) { *err = (int)e; return 0; }
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, omp_kernel<E>, kThreads, smem);
  if (e != cudaSuccess) { *err = (int)e; return 0; }
  if (occ < 1) { *err = (int)cudaErrorInvalidConfiguration; return 0; }
  const int64_t cap = (int64_t)occ * sms;
  return (int)(batch < cap ? batch : cap);
}

int omp_grid(const PlanView& P, int K, int path, int64_t batch, int* err) {
  if (P.dft) return P.fp32 ? omp_grid_t<float2>(P, K, path, batch, err) : omp_grid_t<double2>(P, K, path, batch, err);
  return P.fp32 ? omp_grid_t<float>(P, K, path, batch, err) : omp_grid_t<double>(P, K, path, batch, err);
}

static size_t esize(const PlanView& P) { return (P.dft ? 2 : 1) * (P.fp32 ? 4 : 8); }
static size_t wsize(const PlanView& P) { return P.dft ? 16 : 8; }

size_t omp_workspace_bytes(const PlanView& P, int K, int grid) {
  const size_t h0 = align16((size_t)grid * P.N * esize(P));
  const size_t B = align16((size_t)grid * (((size_t)K * (K + 1)) / 2) * wsize(P));
  return 16 + h0 + B;
}

template <class E>
static cudaError_t omp_impl(const PlanView& P, const OmpLaunch& L, void* ws, int grid, cudaStream_t st) {
  using W = typename FT<E>::W;
  OmpArgs<E> a;
  a.P = plan_dev<E>(P);
  a.y = (const E*)L.y;
  a.batch = L.batch;
  a.K = L.K;
  a.rel_tol = L.rel_tol;
  a.path = L.path;
  a.t_switch = L.t_switch;
  a.x_out = (W*)L.x_out;
  a.supp_out = L.supp_out;
  a.iters_out = L.iters_out;
  a.res_out = L.res_out;
  char* w = (char*)ws;
  a.counter = (int*)w;
  a.h0_ws = (E*)(w + 16);
  a.B_ws = (W*)(w + 16 + align16((size_t)grid * P.N * sizeof(E)));
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const size_t smem = omp_smem_t<E>(P, L.K, L.path);
  omp_kernel<E><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_omp(const PlanView& P, const OmpLaunch& a, void* ws, int grid, cudaStream_t st) {
  if (a.batch <= 0) return cudaSuccess;
  if (P.dft) return P.fp32 ? omp_impl<float2>(P, a, ws, grid, st) : omp_impl<double2>(P, a, ws, grid, st);
  return P.fp32 ? omp_impl<float>(P, a, ws, grid, st) : omp_impl<double>(P, a, ws, grid, st);
}

}  // namespace csf
