// Batched OMP (Algorithm 1.1) in one persistent kernel.
//
// Each CTA runs two instances at once in two "slots" and splits its warps
// into two groups that work on different slots in alternating phases:
//
//   correlation group (8 warps): the initial transform h_0 = Phi^H y, then per
//       iteration the correlation of step 2 (kernel sums of Eq. kernelsumOMP
//       or transforms of the zero-filled residual) fused with the
//       identification of step 3;
//   least-squares group (4 warps, one per SM sub-partition): the FP64
//       Cholesky append of step 6, the residual-norm downdate and the halting
//       test of step 8.
//
// Phase k: the correlation group serves slot k mod 2 while the
// least-squares group serves the other slot; a CTA-wide barrier ends the
// phase.  Per slot the two steps alternate exactly as Algorithm 1.1 orders
// them (identification of column t, then the least squares that adds it, then
// the next correlation), while the SM's FP32 / shared-memory pipes (correlation)
// and its FP64 pipe (least squares) stay busy at the same time.  The kernel
// vector c is staged once per CTA in shared memory and shared by both slots;
// the transform path uses the same region as its buffer, after which c is
// staged again before the next kernel sum.
#include "cs_internal.h"
#include "cs_ls.cuh"

namespace csf {

namespace {

constexpr int kCWarps = 8, kLWarps = 4;
constexpr int kOmpThreads = 32 * (kCWarps + kLWarps);
constexpr int kCThreads = 32 * kCWarps, kLThreads = 32 * kLWarps;
enum { PATH_FAST = 0, PATH_CONV = 1, PATH_HYBRID = 2 };
enum { NEED_INIT = 0, NEED_LS = 1, NEED_CORR = 2, RETIRED = 3 };

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

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
  E* h0_ws;                  // [grid][2][N]
  typename FT<E>::W* B_ws;   // [grid][2][K(K+1)/2]
  int* counter;
  int* status;
  long long max_phases;      // bound on the phase loop (see omp_kernel)
};

// Shared-memory layout (offsets in bytes).
template <class E>
struct OmpLayout {
  size_t regA, slot[2], z, x, g, part, xw, lam, bits, kidx, slot_bytes, redC, rvC, rjC, total;
};

template <class E>
__host__ __device__ inline OmpLayout<E> omp_layout(int N, int K, int path) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  OmpLayout<E> L;
  const int Kc = K > 0 ? K : 1;
  // chunk partials (max(2 n, K) elements), then 3 doubles per k of terms
  const int npart = (2 * kLThreads > Kc ? 2 * kLThreads : Kc) + (3 * Kc * (int)sizeof(double) + (int)sizeof(W) - 1) / (int)sizeof(W);
  // per-slot block, offsets relative to the slot base
  size_t o = 0;
  L.z = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.x = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.g = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.part = o; o = a16(o + (size_t)npart * sizeof(W));
  L.xw = o;   o = a16(o + (size_t)Kc * sizeof(E));
  L.lam = o;  o = a16(o + (size_t)Kc * sizeof(int));
  L.bits = o; o = a16(o + (size_t)((N + 31) >> 5) * sizeof(uint32_t));
  L.kidx = o; o = a16(o + (size_t)N * sizeof(uint16_t));
  L.slot_bytes = o;
  size_t t = 0;
  L.regA = t; t = a16(t + (size_t)((path != PATH_CONV && kernel_doubled<E>(N)) ? 2 * N : N) * sizeof(E));
  L.slot[0] = t; t += L.slot_bytes;
  L.slot[1] = t; t += L.slot_bytes;
  L.redC = t; t = a16(t + (size_t)(32 * 4 + 4) * sizeof(double));
  L.rvC = t;  t = a16(t + 34 * sizeof(V));
  L.rjC = t;  t = a16(t + 34 * sizeof(int));
  L.total = t;
  return L;
}

struct SlotState {
  int64_t b;
  int p, lnew, state, chk;  // chk: the next correlation step first checks the explicit residual
  double ynorm2, rn2;
};

template <class E>
struct SlotView {
  using W = typename FT<E>::W;
  W *z, *x, *g, *part;
  E* xw;
  int* lam;
  uint32_t* bits;
  uint16_t* kidx;  // position -> index in the support (valid where bits is set)
  E* h0;   // global workspace
  W* B;    // global workspace
};

template <class E>
__device__ __forceinline__ SlotView<E> slot_view(unsigned char* sm, const OmpLayout<E>& L, int s,
                                                 const OmpArgs<E>& a) {
  using W = typename FT<E>::W;
  SlotView<E> v;
  unsigned char* base = sm + L.slot[s];
  v.z = (W*)(base + L.z);
  v.x = (W*)(base + L.x);
  v.g = (W*)(base + L.g);
  v.part = (W*)(base + L.part);
  v.xw = (E*)(base + L.xw);
  v.lam = (int*)(base + L.lam);
  v.bits = (uint32_t*)(base + L.bits);
  v.kidx = (uint16_t*)(base + L.kidx);
  const size_t ls = (size_t)blockIdx.x * 2 + s;
  v.h0 = a.h0_ws + ls * a.P.N;
  v.B = a.B_ws + ls * (((size_t)a.K * (a.K + 1)) >> 1);
  return v;
}

// Writes instance b's outputs from the slot (any group; g is the writer).
template <class E>
__device__ void write_outputs(const Grp& g, const OmpArgs<E>& a, const SlotView<E>& v, int64_t b, int p,
                              double ynorm2, double rn2) {
  using W = typename FT<E>::W;
  const int K = a.K;
  for (int k = g.tid; k < K; k += g.n) {
    if (a.x_out) a.x_out[b * K + k] = k < p ? v.x[k] : W{};
    a.supp_out[b * K + k] = k < p ? v.lam[k] : -1;
  }
  if (g.tid == 0) {
    if (a.iters_out) a.iters_out[b] = p;
    if (a.res_out) a.res_out[b] = ynorm2 > 0.0 ? sqrt(fmax(rn2, 0.0) / ynorm2) : 0.0;
  }
}

// ------------------------------------------------------ correlation group
template <class E>
__device__ void corr_step(const Grp& g, const OmpArgs<E>& a, SlotState& S, const SlotView<E>& v, E* regA,
                          double* red, typename NormT<E>::V* rv, int* rj, int& c_valid) {
  constexpr bool DFT = FT<E>::C;
  const int N = a.P.N, M = a.P.M;
  const bool dbl = kernel_doubled<E>(N);
  const int state = S.state;
  if (state == NEED_INIT) {
    if (g.tid == 0) S.b = atomicAdd(a.counter, 1);
    g.sync();
    const int64_t b = S.b;
    if (b >= a.batch) {
      g.sync();
      if (g.tid == 0) S.state = RETIRED;
      return;
    }
    const E* y = a.y + b * M;
    for (int i = g.tid; i < ((N + 31) >> 5); i += g.n) v.bits[i] = 0u;
    // t = 1: h_0 = Phi^H y by one transform (Eq. kernelsumOMP, first case),
    // fused with the identification of step 3; h_0 is kept for later steps
    double yy[1] = {0.0};
    const int l = correlate_transform<E, DFT, true>(g, regA, a.P, y, v.h0, yy, rv, rj);
    group_sum(g, yy, red);
    if (g.tid == 0) c_valid = 0;
    if (!(yy[0] > 0.0) || a.K == 0) {  // zero measurement (or K = 0): no iteration
      write_outputs(g, a, v, b, 0, yy[0], yy[0]);
      g.sync();
      if (g.tid == 0) S.state = NEED_INIT;
      return;
    }
    if (g.tid == 0) {
      S.lnew = l;
      S.p = 0;
      S.chk = 0;
      S.ynorm2 = yy[0];
      S.rn2 = yy[0];
      S.state = NEED_LS;
    }
    return;
  }
  if (state != NEED_CORR) return;
  const int p = S.p, t = p + 1;
  const bool fast = a.path == PATH_FAST || (a.path == PATH_HYBRID && t <= a.t_switch);
  int l;
  // The residual y - Phi x is formed by the transform path's correlation,
  // and for the halting test of step 8 on the explicit residual (FP32 mode,
  // S.chk); one call site each for the residual, the adjoint transform and
  // the kernel sums keeps the kernel within its register budget.
  constexpr bool kChk = sizeof(typename FT<E>::R) == 4;  // FP64 mode never sets S.chk
  if ((kChk && S.chk) || !fast) {
    const bool chk = kChk && S.chk;
    const double r2 = residual_on_omega_rt<E, DFT>(g, regA, a.P, a.y + S.b * M, v.bits, v.kidx, v.xw, red, chk);
    if (g.tid == 0) c_valid = 0;
    if (chk) {
      const double ynorm2 = S.ynorm2;
      if (p >= a.K || r2 < a.rel_tol * a.rel_tol * ynorm2) {
        write_outputs(g, a, v, S.b, p, ynorm2, r2);
        g.sync();
        if (g.tid == 0) S.state = NEED_INIT;
        return;
      }
      g.sync();  // every thread has read S before it changes
      if (g.tid == 0) {
        S.rn2 = r2;
        S.chk = 0;
      }
    }
    if (!fast) {
      l = adjoint_argmax<E, DFT>(g, regA, a.P, v.bits, rv, rj);
      if (g.tid == 0) {
        S.lnew = l;
        S.state = NEED_LS;
      }
      return;
    }
  }
  if (!c_valid) {
    load_kernel_vector<E, DFT>(g, regA, a.P, dbl);
    if (g.tid == 0) c_valid = 1;
  }
  l = correlate_fast<E, DFT>(g, regA, v.h0, v.lam, v.xw, p, N, v.bits, nullptr, rv, rj, dbl);
  if (g.tid == 0) {
    S.lnew = l;
    S.state = NEED_LS;
  }
}

// -------------------------------------------------- least-squares group
template <class E>
__device__ void ls_step(const Grp& g, const OmpArgs<E>& a, SlotState& S, const SlotView<E>& v,
                        LsShared<typename FT<E>::W>& sh) {
  if (S.state != NEED_LS) return;
  const int K = a.K;
  const int64_t b = S.b;
  const int p = S.p, l = S.lnew;
  const double ynorm2 = S.ynorm2;
  if (l < 0) {  // no candidate column left
    write_outputs(g, a, v, b, p, ynorm2, S.rn2);
    g.sync();
    if (g.tid == 0) S.state = NEED_INIT;
    return;
  }
  LsView<E> lv;
  lv.B = v.B;
  lv.z = v.z;
  lv.x = v.x;
  lv.g = v.g;
  lv.part = v.part;
  lv.terms = (double*)(v.part + (2 * kLThreads > K ? 2 * kLThreads : K));
  lv.xw = v.xw;
  lv.lam = v.lam;
  lv.bits = v.bits;
  lv.kidx = v.kidx;
  ls_append(g, a.P, lv, v.h0, p, l, S.rn2, sh);          // step 6
  if (sh.st == 1) {                                       // column dependent on Lambda
    write_outputs(g, a, v, b, p, ynorm2, S.rn2);
    g.sync();
    if (g.tid == 0) S.state = NEED_INIT;
    return;
  }
  // step 8: in FP32 mode a downdate near the tolerance defers the test to
  // the explicit residual, which the next correlation step forms
  const bool chk = resid_check<E>(a.rel_tol) && S.rn2 < kResidTrigger * ynorm2;
  if (!chk && (p + 1 >= K || S.rn2 < a.rel_tol * a.rel_tol * ynorm2)) {
    write_outputs(g, a, v, b, p + 1, ynorm2, S.rn2);
    g.sync();
    if (g.tid == 0) S.state = NEED_INIT;
    return;
  }
  g.sync();  // every thread has read S.rn2 before it is next written
  if (g.tid == 0) {
    S.p = p + 1;
    S.chk = chk;
    S.state = NEED_CORR;
  }
}

template <class E>
__global__ void __launch_bounds__(kOmpThreads, (sizeof(E) > 8 ? 1 : 2)) omp_kernel(OmpArgs<E> a) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ SlotState S[2];
  __shared__ int c_valid;
  __shared__ LsShared<W> l_sh;
  const OmpLayout<E> L = omp_layout<E>(a.P.N, a.K, a.path);
  E* regA = (E*)(sm + L.regA);
  const SlotView<E> v0 = slot_view(sm, L, 0, a), v1 = slot_view(sm, L, 1, a);
  const bool isC = threadIdx.x < kCThreads;
  const Grp gC{(int)threadIdx.x, kCThreads, 1};
  const Grp gL{(int)threadIdx.x - kCThreads, kLThreads, 2};
  if (threadIdx.x == 0) {
    S[0].state = NEED_INIT;
    S[1].state = NEED_INIT;
    c_valid = 0;
  }
  for (long long phase = 0;; ++phase) {
    __syncthreads();
    const bool done = S[0].state == RETIRED && S[1].state == RETIRED;
    __syncthreads();  // every thread has read the states before any step changes them
    if (done) break;
    // Every instance needs at most 2K + 6 phases of its slot and a CTA serves
    // at most the whole batch, so reaching the bound means a broken state
    // machine: record it in the status word and stop instead of spinning.
    if (phase >= a.max_phases) {
      if (threadIdx.x == 0) atomicOr(a.status, kStatusPhaseBound);
      break;
    }
    const int sc = phase & 1;
    if (isC) {
      corr_step<E>(gC, a, S[sc], sc ? v1 : v0, regA, (double*)(sm + L.redC), (V*)(sm + L.rvC), (int*)(sm + L.rjC),
                   c_valid);
    } else {
      ls_step<E>(gL, a, S[sc ^ 1], sc ? v0 : v1, l_sh);
    }
  }
}

template <class E>
size_t smem_t(const PlanView& P, int K, int path) {
  return omp_layout<E>(P.N, K, path).total;
}

template <class E>
int grid_t(const PlanView& P, int K, int path, int64_t batch, int* err) {
  const size_t smem = smem_t<E>(P, K, path);
  *err = 0;
  cudaError_t e = raise_smem_limit((const void*)omp_kernel<E>, smem);
  if (e != cudaSuccess) { *err = (int)e; return 0; }
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, omp_kernel<E>, kOmpThreads, smem);
  if (e != cudaSuccess) { *err = (int)e; return 0; }
  if (occ < 1) { *err = (int)cudaErrorInvalidConfiguration; return 0; }
  const int64_t need = (batch + 1) / 2;  // two instances per CTA
  const int64_t cap = (int64_t)occ * sms;
  return (int)(need < cap ? need : cap);
}

size_t esize(const PlanView& P) { return (P.dft ? 2 : 1) * (P.fp32 ? 4 : 8); }
size_t wsize(const PlanView& P) { return P.dft ? 16 : 8; }

template <class E>
cudaError_t omp_impl(const PlanView& P, const OmpLaunch& L, void* ws, int grid, cudaStream_t st) {
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
  a.status = P.status;
  a.max_phases = 2 * (L.batch + 2) * (2LL * L.K + 10) + 16;
  a.h0_ws = (E*)(w + 16);
  a.B_ws = (W*)(w + 16 + a16((size_t)grid * 2 * P.N * sizeof(E)));
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  omp_kernel<E><<<grid, kOmpThreads, smem_t<E>(P, L.K, L.path), st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t omp_smem_bytes(const PlanView& P, int K, int path) {
  if (P.dft) return P.fp32 ? smem_t<float2>(P, K, path) : smem_t<double2>(P, K, path);
  return P.fp32 ? smem_t<float>(P, K, path) : smem_t<double>(P, K, path);
}

int omp_grid(const PlanView& P, int K, int path, int64_t batch, int* err) {
  if (P.dft) return P.fp32 ? grid_t<float2>(P, K, path, batch, err) : grid_t<double2>(P, K, path, batch, err);
  return P.fp32 ? grid_t<float>(P, K, path, batch, err) : grid_t<double>(P, K, path, batch, err);
}

size_t omp_workspace_bytes(const PlanView& P, int K, int grid) {
  const size_t h0 = a16((size_t)grid * 2 * P.N * esize(P));
  const size_t B = a16((size_t)grid * 2 * (((size_t)K * (K + 1)) / 2) * wsize(P));
  return 16 + h0 + B;
}

cudaError_t launch_omp(const PlanView& P, const OmpLaunch& a, void* ws, int grid, cudaStream_t st) {
  if (a.batch <= 0) return cudaSuccess;
  if (P.dft) return P.fp32 ? omp_impl<float2>(P, a, ws, grid, st) : omp_impl<double2>(P, a, ws, grid, st);
  return P.fp32 ? omp_impl<float>(P, a, ws, grid, st) : omp_impl<double>(P, a, ws, grid, st);
}

}  // namespace csf
