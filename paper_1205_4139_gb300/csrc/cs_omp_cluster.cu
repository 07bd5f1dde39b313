// OMP (Algorithm 1.1) for small batches: one thread-block cluster of kCL
// CTAs per instance.
//
// The persistent kernel (cs_omp.cu) puts one instance on one SM; with only a
// few instances the GPU sits idle and each instance is bound by one SM's FP64
// and shared-memory pipes.  Here the kCL CTAs of a cluster share an
// instance: each computes the kernel-sum correlation of Eq. kernelsumOMP on
// 1/kCL of the outputs and the arg-max of that slice (step 3); the kCL
// candidates are exchanged through distributed shared memory after a cluster
// barrier, and every CTA takes the same column.  The rest — the initial
// transform, the transform-path correlation, the FP64 least squares of step 6
// and the halting test of step 8 — every CTA runs on its own copy of the
// state with the same thread groups and the same arithmetic as the persistent
// kernel, so all CTAs hold the same state and the results equal the
// persistent kernel's bit for bit.
#include <cooperative_groups.h>

#include "cs_internal.h"
#include "cs_ls.cuh"

namespace cg = cooperative_groups;

namespace csf {

namespace {

constexpr int kCL = 8;     // CTAs per instance (a portable cluster size)
constexpr int kQT = 256;   // threads per CTA: the persistent kernel's correlation group
constexpr int kQL = 128;   // the persistent kernel's least-squares group
constexpr int kH0R = (1 << 13) / kCL / kQT;  // outputs of h per thread at N = 8192: 4
enum { PATH_FAST = 0, PATH_CONV = 1, PATH_HYBRID = 2 };

__host__ __device__ inline size_t q16(size_t x) { return (x + 15) & ~(size_t)15; }

template <class E>
struct QArgs {
  using W = typename FT<E>::W;
  PlanDev<E> P;
  const E* __restrict__ y;
  int64_t batch;
  int K;
  double rel_tol;
  int path, t_switch;
  W* x_out;
  int* supp_out;
  int* iters_out;
  double* res_out;
  E* h0_ws;  // [batch][kCL][N]
  W* B_ws;   // [batch][kCL][K(K+1)/2]
};

template <class E>
struct QLayout {
  size_t regA, z, x, g, part, xw, lam, bits, kidx, red, rv, rj, total;
};

template <class E>
__host__ __device__ inline QLayout<E> q_layout(int N, int K, int path) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  QLayout<E> L;
  const int Kc = K > 0 ? K : 1;
  const int npart = (2 * kQL > Kc ? 2 * kQL : Kc) + (3 * Kc * (int)sizeof(double) + (int)sizeof(W) - 1) / (int)sizeof(W);
  size_t o = 0;
  L.regA = o; o = q16(o + (size_t)((path != PATH_CONV && kernel_doubled<E>(N)) ? 2 * N : N) * sizeof(E));
  L.z = o;    o = q16(o + (size_t)Kc * sizeof(W));
  L.x = o;    o = q16(o + (size_t)Kc * sizeof(W));
  L.g = o;    o = q16(o + (size_t)Kc * sizeof(W));
  L.part = o; o = q16(o + (size_t)npart * sizeof(W));
  L.xw = o;   o = q16(o + (size_t)Kc * sizeof(E));
  L.lam = o;  o = q16(o + (size_t)Kc * sizeof(int));
  L.bits = o; o = q16(o + (size_t)((N + 31) >> 5) * sizeof(uint32_t));
  L.kidx = o; o = q16(o + (size_t)N * sizeof(uint16_t));
  L.red = o;  o = q16(o + (size_t)(32 + 1) * sizeof(double));
  L.rv = o;   o = q16(o + 34 * sizeof(V));
  L.rj = o;   o = q16(o + 34 * sizeof(int));
  L.total = o;
  return L;
}

template <class E>
__device__ void q_outputs(const QArgs<E>& a, int64_t b, const typename FT<E>::W* x, const int* lam, int p,
                          double ynorm2, double rn2) {
  using W = typename FT<E>::W;
  const int K = a.K;
  for (int k = threadIdx.x; k < K; k += kQT) {
    if (a.x_out) a.x_out[b * K + k] = k < p ? x[k] : W{};
    a.supp_out[b * K + k] = k < p ? lam[k] : -1;
  }
  if (threadIdx.x == 0) {
    if (a.iters_out) a.iters_out[b] = p;
    if (a.res_out) a.res_out[b] = ynorm2 > 0.0 ? sqrt(fmax(rn2, 0.0) / ynorm2) : 0.0;
  }
}

template <class E>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kQT) omp_cluster_kernel(QArgs<E> a) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ V cand_v[2];
  __shared__ int cand_j[2];
  __shared__ LsShared<W> lsh;
  __shared__ double rn2_s;
  __shared__ int sel;
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const int64_t b = blockIdx.x / kCL;
  const int N = a.P.N, M = a.P.M, K = a.K;
  const QLayout<E> L = q_layout<E>(N, K, a.path);
  E* regA = (E*)(sm + L.regA);
  LsView<E> lv;
  lv.B = a.B_ws + (b * kCL + r) * (((int64_t)K * (K + 1)) >> 1);
  lv.z = (W*)(sm + L.z);
  lv.x = (W*)(sm + L.x);
  lv.g = (W*)(sm + L.g);
  lv.part = (W*)(sm + L.part);
  lv.terms = (double*)(lv.part + (2 * kQL > K ? 2 * kQL : K));
  lv.xw = (E*)(sm + L.xw);
  lv.lam = (int*)(sm + L.lam);
  lv.bits = (uint32_t*)(sm + L.bits);
  lv.kidx = (uint16_t*)(sm + L.kidx);
  double* red = (double*)(sm + L.red);
  V* rv = (V*)(sm + L.rv);
  int* rj = (int*)(sm + L.rj);
  E* h0 = a.h0_ws + (b * kCL + r) * (int64_t)N;
  const E* y = a.y + b * M;
  const Grp gA = whole_block();
  const Grp gL{(int)threadIdx.x - (kQT - kQL), kQL, 2};
  const bool inL = threadIdx.x >= kQT - kQL;
  const bool dbl = a.path != PATH_CONV && kernel_doubled<E>(N);

  for (int i = threadIdx.x; i < ((N + 31) >> 5); i += kQT) lv.bits[i] = 0u;
  __syncthreads();
  // t = 1: h_0 = Phi^H y by one transform (Eq. kernelsumOMP, first case),
  // with the arg-max and ||y||^2, in every CTA
  double yy[1] = {0.0};
  int l = correlate_transform<E, DFT, true>(gA, regA, a.P, y, h0, yy, rv, rj);
  group_sum(gA, yy, red);
  const double ynorm2 = yy[0];
  if (!(ynorm2 > 0.0) || K == 0) {  // zero measurement (or K = 0): no iteration
    if (r == 0) q_outputs(a, b, lv.x, lv.lam, 0, ynorm2, ynorm2);
    cl.sync();
    return;
  }
  if (threadIdx.x == 0) rn2_s = ynorm2;
  __syncthreads();
  // this CTA's slice of h_0 in registers (at most N / kCL / kQT = 4 outputs
  // per thread for N <= 8192): the kernel sums of every iteration start from
  // it without a global-memory round trip on their critical path
  // (complex FP64 keeps reading the workspace: the 128-register budget has
  // no room for it)
  constexpr bool kRegH0 = sizeof(E) <= 8;
  const int lo = (int)(((int64_t)N * r) / kCL), hi = (int)(((int64_t)N * (r + 1)) / kCL);
  E h0r[kH0R];
#pragma unroll
  for (int i = 0; i < kH0R; ++i) {
    const int j = lo + (int)threadIdx.x + i * kQT;
    h0r[i] = (kRegH0 && j < hi) ? h0[j] : zero<E>();
  }
  int p = 0, c_valid = 0;
  for (int it = 0;; ++it) {
    if (l < 0) {  // no candidate column left
      if (r == 0) q_outputs(a, b, lv.x, lv.lam, p, ynorm2, rn2_s);
      break;
    }
    if (inL) ls_append(gL, a.P, lv, h0, p, l, rn2_s, lsh);  // step 6
    __syncthreads();
    if (lsh.st == 1) {  // column dependent on Lambda
      if (r == 0) q_outputs(a, b, lv.x, lv.lam, p, ynorm2, rn2_s);
      break;
    }
    // step 8 (FP32 mode: a downdate near the tolerance defers the test to the
    // explicit residual, as in the persistent kernel)
    const bool chk = resid_check<E>(a.rel_tol) && rn2_s < kResidTrigger * ynorm2;
    if (!chk && (p + 1 >= K || rn2_s < a.rel_tol * a.rel_tol * ynorm2)) {
      if (r == 0) q_outputs(a, b, lv.x, lv.lam, p + 1, ynorm2, rn2_s);
      break;
    }
    __syncthreads();  // rn2_s read by every thread before the next append
    p += 1;
    const int t = p + 1;
    const bool fast = a.path == PATH_FAST || (a.path == PATH_HYBRID && t <= a.t_switch);
    if (chk) {  // every CTA forms the same residual and takes the same decision
      const bool last = p >= K;
      double r2;
      int lr = -1;
      if (!last && !fast) {
        lr = correlate_residual<E, DFT, true>(gA, regA, a.P, y, lv.bits, lv.kidx, lv.xw, rv, rj, nullptr, nullptr,
                                              &r2, red);
      } else {
        r2 = residual_on_omega<E, DFT, true>(gA, regA, a.P, y, lv.bits, lv.kidx, lv.xw, red);
      }
      c_valid = 0;
      if (last || r2 < a.rel_tol * a.rel_tol * ynorm2) {
        if (r == 0) q_outputs(a, b, lv.x, lv.lam, p, ynorm2, r2);
        break;
      }
      if (threadIdx.x == 0) rn2_s = r2;
      __syncthreads();
      if (!fast) {
        l = lr;
        continue;
      }
    }
    if (fast) {
      if (!c_valid) {
        load_kernel_vector<E, DFT>(gA, regA, a.P, dbl);
        c_valid = 1;
      }
      // this CTA's slice of h = h_0 - sum_k x_k c(j (-) lambda_k), same
      // arithmetic per output as the persistent kernel (the terms in k
      // order; the unrolled loop only issues the next atoms' loads early)
      V bv = (V)-1;
      int bj = 0x7fffffff;
#pragma unroll
      for (int i = 0; i < kH0R; ++i) {
        const int j = lo + (int)threadIdx.x + i * kQT;
        if (j >= hi) break;
        E acc = kRegH0 ? h0r[i] : h0[j];
#pragma unroll 4
        for (int k = 0; k < p; ++k) {
          const int lk = lv.lam[k];
          const E xv = lv.xw[k];
          const int d = DFT ? ((j - lk) & (N - 1)) : (j ^ lk);
          acc = fnms(acc, xv, regA[d]);
        }
        const V v = in_bits(lv.bits, j) ? (V)-1 : (V)norm2(acc);
        if (better(v, j, bv, bj)) {
          bv = v;
          bj = j;
        }
      }
      // the slice's candidate, then the cluster's (step 3)
      warp_argmax(bv, bj);
      if ((threadIdx.x & 31) == 0) {
        rv[threadIdx.x >> 5] = bv;
        rj[threadIdx.x >> 5] = bj;
      }
      __syncthreads();
      const int par = it & 1;
      if (threadIdx.x < 32) {
        V v = threadIdx.x < (kQT >> 5) ? rv[threadIdx.x] : (V)-1;
        int j = threadIdx.x < (kQT >> 5) ? rj[threadIdx.x] : 0x7fffffff;
        warp_argmax(v, j);
        if (threadIdx.x == 0) {
          cand_v[par] = v;
          cand_j[par] = j;
        }
      }
      cl.sync();
      if (threadIdx.x < 32) {
        V v = (V)-1;
        int j = 0x7fffffff;
        if (threadIdx.x < kCL) {
          v = *cl.map_shared_rank(&cand_v[par], (unsigned)threadIdx.x);
          j = *cl.map_shared_rank(&cand_j[par], (unsigned)threadIdx.x);
        }
        warp_argmax(v, j);
        if (threadIdx.x == 0) sel = v < (V)0 ? -1 : j;
      }
      __syncthreads();
      l = sel;
    } else {
      l = correlate_residual<E, DFT>(gA, regA, a.P, y, lv.bits, lv.kidx, lv.xw, rv, rj);
      c_valid = 0;
    }
  }
  // no CTA leaves while another may still read its candidates
  cl.sync();
}

template <class E>
size_t q_smem(const PlanView& P, int K, int path) {
  return q_layout<E>(P.N, K, path).total;
}

template <class E>
cudaError_t q_impl(const PlanView& P, const OmpLaunch& L, void* ws, cudaStream_t st) {
  using W = typename FT<E>::W;
  QArgs<E> a;
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
  a.h0_ws = (E*)ws;
  a.B_ws = (W*)((char*)ws + q16((size_t)L.batch * kCL * P.N * sizeof(E)));
  const size_t smem = q_smem<E>(P, L.K, L.path);
  cudaError_t e = raise_smem_limit((const void*)omp_cluster_kernel<E>, smem);
  if (e != cudaSuccess) return e;
  omp_cluster_kernel<E><<<(unsigned)(L.batch * kCL), kQT, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t omp_cluster_smem(const PlanView& P, int K, int path) {
  if (P.dft) return P.fp32 ? q_smem<float2>(P, K, path) : q_smem<double2>(P, K, path);
  return P.fp32 ? q_smem<float>(P, K, path) : q_smem<double>(P, K, path);
}

size_t omp_cluster_workspace_bytes(const PlanView& P, int K, int64_t batch) {
  const size_t eb = (P.dft ? 2 : 1) * (P.fp32 ? 4 : 8), wb = P.dft ? 16 : 8;
  return q16((size_t)batch * kCL * P.N * eb) + (size_t)batch * kCL * (((size_t)K * (K + 1)) / 2) * wb;
}

cudaError_t launch_omp_cluster(const PlanView& P, const OmpLaunch& a, void* ws, cudaStream_t st) {
  if (a.batch <= 0) return cudaSuccess;
  if (P.dft) return P.fp32 ? q_impl<float2>(P, a, ws, st) : q_impl<double2>(P, a, ws, st);
  return P.fp32 ? q_impl<float>(P, a, ws, st) : q_impl<double>(P, a, ws, st);
}

}  // namespace csf
