// OMP (Algorithm 1.1) on a batch of instances that each bring their own
// plan: their own row set Omega, N (up to 2^16), M and K.  One persistent
// launch per element type and residence runs all instances of that kind, in
// a list sorted by decreasing estimated work that the CTAs take from with an
// atomic counter (the instances that start last are short ones).
//
// Shared-memory residence (N <= 8192), omp_multi_kernel: the structure of
// the batched kernel of cs_omp.cu, two instances ("slots") per CTA, a
// correlation group of 8 warps (the initial transform, then per iteration
// the kernel sums of Eq. kernelsumOMP or the transforms of the zero-filled
// residual, fused with the identification of step 3) and a least-squares
// group of 4 warps (the FP64 Cholesky append of step 6, the residual
// downdate and the halting test of step 8) serving the two slots in
// alternating phases.  Each slot carries its instance's descriptor (plan
// tables, y, K, outputs) in shared memory, and c is staged again whenever
// the correlation group turns to a slot of another plan.
//
// Global-memory residence (8192 < N <= 2^16), omp_seq_kernel: one instance
// per CTA at a time and several CTAs per SM; the transform vector, support
// bitmap and position map live in a global workspace (mostly in L2), c is
// read straight from the plan, and the transforms are the same radix-16
// chains, two passes per round trip through a shared-memory tile
// (cs_gchain.cuh).
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "cs_gchain.cuh"
#include "cs_internal.h"
#include "cs_ls.cuh"

namespace csf {

namespace {

constexpr int kCWarps = 8, kLWarps = 4;
constexpr int kMThreads = 32 * (kCWarps + kLWarps);
constexpr int kCThreads = 32 * kCWarps, kLThreads = 32 * kLWarps;
enum { PATH_FAST = 0, PATH_CONV = 1, PATH_HYBRID = 2 };
enum { NEED_INIT = 0, NEED_LS = 1, NEED_CORR = 2, RETIRED = 3 };

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline size_t tri(int K) { return ((size_t)K * (K + 1)) >> 1; }

template <class E>
struct MInst {
  PlanDev<E> P;             // tables of the instance's plan (chain order)
  const E* y;               // [M]
  typename FT<E>::W* x;     // [K] FP64 coefficients (nullable)
  int* supp;                // [K]
  int K, t_switch, idx, pad;
};

template <class E>
struct MArgs {
  const MInst<E>* __restrict__ inst;  // longest first
  int64_t count;
  double rel_tol;
  int path;
  int Nsm;    // largest N of a shared-memory launch (0 in a global-memory one)
  int Nbig;   // largest N of a global-memory launch (0 in a shared-memory one)
  int Nmax, Kmax;
  int* iters_out;             // [count], by instance index (nullable)
  double* res_out;            // [count] (nullable)
  E* h0_ws;                   // [grid][2][Nmax]
  typename FT<E>::W* B_ws;    // [grid][2][Kmax(Kmax+1)/2]
  E* buf_ws;                  // global-memory launches: [grid][Nbig] transform vector
  uint32_t* bits_ws;          //   [grid][Nbig/32] support bitmap
  uint16_t* kidx_ws;          //   [grid][Nbig] position -> index in the support
  int* counter;
  int* status;
  long long max_phases;
};

// Shared-memory layout of omp_multi_kernel (byte offsets): the c / transform
// region, then two slot blocks sized for (Nsm, Kmax).
template <class E>
struct MLayout {
  size_t regA, regA_n, slot[2], z, x, g, part, xw, lam, bits, kidx, slot_bytes, redC, rvC, rjC, total;
};

template <class E>
__host__ __device__ inline MLayout<E> mlayout(int Nsm, int K, int path) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  MLayout<E> L;
  const int Kc = K > 0 ? K : 1;
  const int npart = (2 * kLThreads > Kc ? 2 * kLThreads : Kc) +
                    (3 * Kc * (int)sizeof(double) + (int)sizeof(W) - 1) / (int)sizeof(W);
  size_t o = 0;
  L.z = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.x = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.g = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.part = o; o = a16(o + (size_t)npart * sizeof(W));
  L.xw = o;   o = a16(o + (size_t)Kc * sizeof(E));
  L.lam = o;  o = a16(o + (size_t)Kc * sizeof(int));
  L.bits = o; o = a16(o + (size_t)((Nsm + 31) >> 5) * sizeof(uint32_t));
  L.kidx = o; o = a16(o + (size_t)Nsm * sizeof(uint16_t));
  L.slot_bytes = o;
  size_t t = 0;
  L.regA_n = (size_t)((path != PATH_CONV && kernel_doubled<E>(Nsm)) ? 2 * Nsm : Nsm);
  L.regA = t; t = a16(t + L.regA_n * sizeof(E));
  L.slot[0] = t; t += L.slot_bytes;
  L.slot[1] = t; t += L.slot_bytes;
  L.redC = t; t = a16(t + (size_t)(32 * 4 + 4) * sizeof(double));
  L.rvC = t;  t = a16(t + 34 * sizeof(V));
  L.rjC = t;  t = a16(t + 34 * sizeof(int));
  L.total = t;
  return L;
}

template <class E>
struct MSlot {
  MInst<E> I;
  int64_t b;
  int p, lnew, state, chk;  // chk: the next correlation step first checks the explicit residual
  double ynorm2, rn2;
};

template <class E>
struct MView {
  using W = typename FT<E>::W;
  W *z, *x, *g, *part;
  E* xw;
  int* lam;
  uint32_t* bits;
  uint16_t* kidx;
  E* h0;
  W* B;
  E* buf;  // transform buffer
};

template <class E>
__device__ __forceinline__ MView<E> mview(unsigned char* sm, const MLayout<E>& L, int s, const MArgs<E>& a) {
  using W = typename FT<E>::W;
  MView<E> v;
  unsigned char* base = sm + L.slot[s];
  v.z = (W*)(base + L.z);
  v.x = (W*)(base + L.x);
  v.g = (W*)(base + L.g);
  v.part = (W*)(base + L.part);
  v.xw = (E*)(base + L.xw);
  v.lam = (int*)(base + L.lam);
  const size_t ls = (size_t)blockIdx.x * 2 + s;
  v.bits = (uint32_t*)(base + L.bits);
  v.kidx = (uint16_t*)(base + L.kidx);
  v.h0 = a.h0_ws + ls * (size_t)a.Nmax;
  v.B = a.B_ws + ls * tri(a.Kmax);
  v.buf = (E*)(sm + L.regA);
  return v;
}

// Key of the c vector held in the shared region: the plan's storage.
template <class E>
__device__ __forceinline__ const void* c_key(const PlanDev<E>& P) {
  return P.cfmt == CFMT_INT ? (const void*)P.ci : (const void*)P.c;
}

template <class E>
__device__ void mwrite(const Grp& g, const MArgs<E>& a, const MInst<E>& I, const MView<E>& v, int p, double ynorm2,
                       double rn2) {
  using W = typename FT<E>::W;
  for (int k = g.tid; k < I.K; k += g.n) {
    if (I.x) I.x[k] = k < p ? v.x[k] : W{};
    I.supp[k] = k < p ? v.lam[k] : -1;
  }
  if (g.tid == 0) {
    if (a.iters_out) a.iters_out[I.idx] = p;
    if (a.res_out) a.res_out[I.idx] = ynorm2 > 0.0 ? sqrt(fmax(rn2, 0.0) / ynorm2) : 0.0;
  }
}

// ------------------------------------------------------ correlation group
template <class E>
__device__ void mcorr_step(const Grp& g, const MArgs<E>& a, MSlot<E>& S, int s, unsigned char* sm,
                           const MLayout<E>& L, double* red, typename NormT<E>::V* rv, int* rj, const void*& ckey) {
  constexpr bool DFT = FT<E>::C;
  if (S.state == NEED_INIT) {
    if (g.tid == 0) S.b = atomicAdd(a.counter, 1);
    g.sync();
    const int64_t b = S.b;
    if (b >= a.count) {
      g.sync();
      if (g.tid == 0) S.state = RETIRED;
      return;
    }
    if (g.tid == 0) S.I = a.inst[b];
    g.sync();
    const MInst<E>& I = S.I;
    const MView<E> v = mview(sm, L, s, a);
    for (int i = g.tid; i < ((I.P.N + 31) >> 5); i += g.n) v.bits[i] = 0u;
    // t = 1: h_0 = Phi^H y by one transform, fused with step 3
    double yy[1] = {0.0};
    const int l = correlate_transform<E, DFT, true>(g, v.buf, I.P, I.y, v.h0, yy, rv, rj);
    group_sum(g, yy, red);
    if (g.tid == 0) ckey = nullptr;  // the shared region held the transform
    if (!(yy[0] > 0.0) || I.K == 0) {
      mwrite(g, a, I, v, 0, yy[0], yy[0]);
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
  if (S.state != NEED_CORR) return;
  const MInst<E>& I = S.I;
  const MView<E> v = mview(sm, L, s, a);
  const int p = S.p, t = p + 1, N = I.P.N;
  const bool fast = a.path == PATH_FAST || (a.path == PATH_HYBRID && t <= I.t_switch);
  int l;
  if (S.chk) {  // halting test of step 8 on the explicit residual (FP32 mode), as in cs_omp
    const bool last = p >= I.K;
    double r2;
    if (!last && !fast) {
      l = correlate_residual<E, DFT, true>(g, v.buf, I.P, I.y, v.bits, v.kidx, v.xw, rv, rj, nullptr, nullptr, &r2,
                                           red);
    } else {
      r2 = residual_on_omega<E, DFT, true>(g, v.buf, I.P, I.y, v.bits, v.kidx, v.xw, red);
    }
    if (g.tid == 0) ckey = nullptr;
    const double ynorm2 = S.ynorm2;
    if (last || r2 < a.rel_tol * a.rel_tol * ynorm2) {
      mwrite(g, a, I, v, p, ynorm2, r2);
      g.sync();
      if (g.tid == 0) S.state = NEED_INIT;
      return;
    }
    g.sync();  // every thread has read S before it changes
    if (g.tid == 0) {
      S.rn2 = r2;
      S.chk = 0;
    }
    if (!fast) {
      if (g.tid == 0) {
        S.lnew = l;
        S.state = NEED_LS;
      }
      return;
    }
  }
  if (fast) {
    E* regA = (E*)(sm + L.regA);
    const bool dbl = DFT && kernel_doubled<E>(N) && 2 * (size_t)N <= L.regA_n;
    const void* key = c_key(I.P);
    if (ckey != key) {  // every thread reads ckey before the barrier that ends the load
      load_kernel_vector<E, DFT>(g, regA, I.P, dbl);
      if (g.tid == 0) ckey = key;
    }
    l = correlate_fast<E, DFT>(g, regA, v.h0, v.lam, v.xw, p, N, v.bits, nullptr, rv, rj, dbl);
  } else {
    l = correlate_residual<E, DFT>(g, v.buf, I.P, I.y, v.bits, v.kidx, v.xw, rv, rj);
    if (g.tid == 0) ckey = nullptr;
  }
  if (g.tid == 0) {
    S.lnew = l;
    S.state = NEED_LS;
  }
}

// -------------------------------------------------- least-squares group
template <class E>
__device__ void mls_step(const Grp& g, const MArgs<E>& a, MSlot<E>& S, int s, unsigned char* sm, const MLayout<E>& L,
                         LsShared<typename FT<E>::W>& sh) {
  if (S.state != NEED_LS) return;
  const MInst<E>& I = S.I;
  const MView<E> v = mview(sm, L, s, a);
  const int K = I.K, p = S.p, l = S.lnew;
  const double ynorm2 = S.ynorm2;
  if (l < 0) {  // no candidate column left
    mwrite(g, a, I, v, p, ynorm2, S.rn2);
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
  lv.terms = (double*)(v.part + (2 * kLThreads > a.Kmax ? 2 * kLThreads : a.Kmax));
  lv.xw = v.xw;
  lv.lam = v.lam;
  lv.bits = v.bits;
  lv.kidx = v.kidx;
  ls_append(g, I.P, lv, v.h0, p, l, S.rn2, sh);         // step 6
  if (sh.st == 1) {                                      // column dependent on Lambda
    mwrite(g, a, I, v, p, ynorm2, S.rn2);
    g.sync();
    if (g.tid == 0) S.state = NEED_INIT;
    return;
  }
  // step 8 (FP32 mode: a downdate near the tolerance defers the test to the
  // explicit residual, which the next correlation step forms)
  const bool chk = resid_check<E>(a.rel_tol) && S.rn2 < kResidTrigger * ynorm2;
  if (!chk && (p + 1 >= K || S.rn2 < a.rel_tol * a.rel_tol * ynorm2)) {
    mwrite(g, a, I, v, p + 1, ynorm2, S.rn2);
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
__global__ void __launch_bounds__(kMThreads, (sizeof(E) > 4 ? 1 : 2)) omp_multi_kernel(MArgs<E> a) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ MSlot<E> S[2];
  __shared__ const void* ckey;
  __shared__ LsShared<W> l_sh;
  const MLayout<E> L = mlayout<E>(a.Nsm, a.Kmax, a.path);
  const bool isC = threadIdx.x < kCThreads;
  const Grp gC{(int)threadIdx.x, kCThreads, 1};
  const Grp gL{(int)threadIdx.x - kCThreads, kLThreads, 2};
  if (threadIdx.x == 0) {
    S[0].state = NEED_INIT;
    S[1].state = NEED_INIT;
    ckey = nullptr;
  }
  for (long long phase = 0;; ++phase) {
    __syncthreads();
    const bool done = S[0].state == RETIRED && S[1].state == RETIRED;
    __syncthreads();  // every thread has read the states before any step changes them
    if (done) break;
    // Each instance needs at most 2K + 4 phases of its slot and a CTA serves
    // at most the whole batch: reaching the bound means a broken state
    // machine, recorded in the status word instead of spinning on.
    if (phase >= a.max_phases) {
      if (threadIdx.x == 0) atomicOr(a.status, kStatusPhaseBound);
      break;
    }
    const int sc = phase & 1;
    if (isC) {
      mcorr_step<E>(gC, a, S[sc], sc, sm, L, (double*)(sm + L.redC), (V*)(sm + L.rvC), (int*)(sm + L.rjC), ckey);
    } else {
      mls_step<E>(gL, a, S[sc ^ 1], sc ^ 1, sm, L, l_sh);
    }
  }
}

// ------------------------------------------------ global-memory residence
// One instance per CTA at a time, its 8 warps running the correlation and
// the least squares of each iteration in turn, several CTAs per SM.  These
// instances are bound by the latency of their round trips through L2, not by
// a pipe, so several independent instances per SM hide one another's waits
// better than one CTA whose warp groups alternate between two instances
// (measured: 151 ms against 183 ms for 1221 complex instances).
constexpr int kSThreads = 256;

template <class E>
constexpr int seq_min_blocks() {
  // measured: one more CTA per SM (48 / 64 registers) spills and runs slower
  return sizeof(E) == 4 ? 4 : (sizeof(E) == 8 ? 3 : 2);
}

template <class E>
struct SLayout {
  size_t tile, tws, z, x, g, part, xw, lam, red, rv, rj, total;
};

// The least-squares scratch (g, part) is dead outside the least squares and
// the stage tile outside the transforms, so the scratch lives in the tile
// when it fits there: a smaller footprint, more CTAs per SM.
template <class E>
__host__ __device__ inline SLayout<E> slayout(int K) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  SLayout<E> L;
  const int Kc = K > 0 ? K : 1;
  const int npart = (2 * kSThreads > Kc ? 2 * kSThreads : Kc) +
                    (3 * Kc * (int)sizeof(double) + (int)sizeof(W) - 1) / (int)sizeof(W);
  const size_t tile_b = a16((size_t)kGTile * sizeof(E));
  const size_t scratch_b = a16((size_t)Kc * sizeof(W)) + a16((size_t)npart * sizeof(W));
  size_t o = 0;
  L.tile = o; o += tile_b;
  if (scratch_b <= tile_b) {
    L.g = L.tile;
    L.part = L.tile + a16((size_t)Kc * sizeof(W));
  } else {
    L.g = o;    o = a16(o + (size_t)Kc * sizeof(W));
    L.part = o; o = a16(o + (size_t)npart * sizeof(W));
  }
  L.tws = o;  o = a16(o + (FT<E>::C ? 512 : 0) * sizeof(E));  // split twiddle tables (DFT)
  L.z = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.x = o;    o = a16(o + (size_t)Kc * sizeof(W));
  L.xw = o;   o = a16(o + (size_t)Kc * sizeof(E));
  L.lam = o;  o = a16(o + (size_t)Kc * sizeof(int));
  L.red = o;  o = a16(o + (size_t)(32 * 4 + 4) * sizeof(double));
  L.rv = o;   o = a16(o + 34 * sizeof(V));
  L.rj = o;   o = a16(o + 34 * sizeof(int));
  L.total = o;
  return L;
}

template <class E>
__global__ void __launch_bounds__(kSThreads, seq_min_blocks<E>()) omp_seq_kernel(MArgs<E> a) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ MInst<E> I;
  __shared__ long long b_s;
  __shared__ double rn2;
  __shared__ LsShared<W> sh;
  const SLayout<E> L = slayout<E>(a.Kmax);
  const Grp g = whole_block();
  E* tile = (E*)(sm + L.tile);
  E* tws = (E*)(sm + L.tws);
  double* red = (double*)(sm + L.red);
  V* rv = (V*)(sm + L.rv);
  int* rj = (int*)(sm + L.rj);
  const size_t cta = blockIdx.x;
  LsView<E> lv;
  lv.B = a.B_ws + cta * tri(a.Kmax);
  lv.z = (W*)(sm + L.z);
  lv.x = (W*)(sm + L.x);
  lv.g = (W*)(sm + L.g);
  lv.part = (W*)(sm + L.part);
  lv.terms = (double*)(lv.part + (2 * kSThreads > a.Kmax ? 2 * kSThreads : a.Kmax));
  lv.xw = (E*)(sm + L.xw);
  lv.lam = (int*)(sm + L.lam);
  lv.bits = a.bits_ws + cta * (size_t)(a.Nbig >> 5);
  lv.kidx = a.kidx_ws + cta * (size_t)a.Nbig;
  E* h0 = a.h0_ws + cta * (size_t)a.Nmax;
  E* buf = a.buf_ws + cta * (size_t)a.Nbig;
  // a CTA serves each instance at most once; the bound only guards the loop
  for (int64_t served = 0; served <= a.count; ++served) {
    __syncthreads();  // every thread is done with the previous descriptor
    if (g.tid == 0) {
      b_s = atomicAdd(a.counter, 1);
      if (b_s < a.count) I = a.inst[b_s];
    }
    __syncthreads();
    if (b_s >= a.count) break;
    const int N = I.P.N, K = I.K;
    for (int i = g.tid; i < ((N + 31) >> 5); i += g.n) lv.bits[i] = 0u;
    if constexpr (DFT) fill_split_twiddles(g, tws, N);
    // t = 1: h_0 = Phi^H y by one transform, fused with step 3
    double yy[1] = {0.0};
    int l = gcorrelate_transform<E, DFT>(g, buf, tile, tws, I.P, I.y, h0, yy, rv, rj);
    group_sum(g, yy, red);
    const double ynorm2 = yy[0];
    if (g.tid == 0) rn2 = ynorm2;
    g.sync();
    int p = 0;
    if (ynorm2 > 0.0 && K > 0) {
      for (;;) {
        if (l < 0) break;                                   // no candidate column left
        ls_append(g, I.P, lv, h0, p, l, rn2, sh);            // step 6
        if (sh.st == 1) break;                              // column dependent on Lambda
        ++p;
        // step 8 (FP32 mode: a downdate near the tolerance is decided on the
        // explicit residual instead)
        const bool chk = resid_check<E>(a.rel_tol) && rn2 < kResidTrigger * ynorm2;
        if (!chk && (p >= K || rn2 < a.rel_tol * a.rel_tol * ynorm2)) break;
        const bool fast = a.path == PATH_FAST || (a.path == PATH_HYBRID && p + 1 <= I.t_switch);
        if (chk) {
          double r2;
          if (p < K && !fast) {
            l = gcorrelate_residual<E, DFT, true>(g, buf, tile, tws, I.P, I.y, lv.bits, lv.kidx, lv.xw, rv, rj, &r2,
                                                  red);
          } else {
            r2 = gresidual_norm<E, DFT>(g, buf, tile, tws, I.P, I.y, lv.bits, lv.kidx, lv.xw, red);
          }
          if (g.tid == 0) rn2 = r2;  // every thread has read rn2 (the barriers of the chain)
          g.sync();
          if (p >= K || r2 < a.rel_tol * a.rel_tol * ynorm2) break;
          if (!fast) continue;
        }
        l = fast ? correlate_fast<E, DFT>(g, I.P.c, h0, lv.lam, lv.xw, p, N, lv.bits, nullptr, rv, rj, false)
                 : gcorrelate_residual<E, DFT>(g, buf, tile, tws, I.P, I.y, lv.bits, lv.kidx, lv.xw, rv, rj);
      }
    }
    for (int k = g.tid; k < K; k += g.n) {
      if (I.x) I.x[k] = k < p ? lv.x[k] : W{};
      I.supp[k] = k < p ? lv.lam[k] : -1;
    }
    if (g.tid == 0) {
      if (a.iters_out) a.iters_out[I.idx] = p;
      if (a.res_out) a.res_out[I.idx] = ynorm2 > 0.0 ? sqrt(fmax(rn2, 0.0) / ynorm2) : 0.0;
    }
  }
}

// ------------------------------------------------------------------ host
template <class E>
PlanDev<E> chain_dev(const PlanView& P) {
  PlanDev<E> d = plan_dev<E>(P);
  if (P.large) {
    constexpr bool f32 = sizeof(typename FT<E>::R) == 4;
    d.slot = P.slot_chain;
    d.tw = (const E*)(f32 ? P.ctw32 : P.ctw64);
  }
  return d;
}

struct Sizes {
  int Nsm = 0, Nbig = 0, Nmax = 0, Kmax = 0;
};

Sizes sizes_of(const MultiItem* it, int64_t n) {
  Sizes z;
  for (int64_t i = 0; i < n; ++i) {
    const int N = it[i].P->N;
    if (it[i].P->large) z.Nbig = std::max(z.Nbig, N);
    else z.Nsm = std::max(z.Nsm, N);
    z.Nmax = std::max(z.Nmax, N);
    z.Kmax = std::max(z.Kmax, it[i].K);
  }
  return z;
}

// Shared memory of a launch of one residence.
template <class E>
size_t smem_t(const Sizes& z, int path) {
  return z.Nsm == 0 ? slayout<E>(z.Kmax).total : mlayout<E>(z.Nsm, z.Kmax, path).total;
}

// CTAs per SM the launch of these instances can hold (shared memory,
// registers), for the kernel of their residence.
template <class E>
int occ_t(const MultiItem* it, int64_t n, int path, int* err) {
  const Sizes z = sizes_of(it, n);
  const bool seq = z.Nsm == 0;
  const size_t smem = smem_t<E>(z, path);
  const void* kfn = seq ? (const void*)omp_seq_kernel<E> : (const void*)omp_multi_kernel<E>;
  cudaError_t e = raise_smem_limit(kfn, smem);
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, seq ? kSThreads : kMThreads, smem);
  *err = (int)e;
  return e == cudaSuccess ? occ : 0;
}

template <class E>
cudaError_t multi_t(MultiItem* it, int64_t n, double rel_tol, int path, int ctas_per_sm, int* iters_out,
                    double* res_out, int* status, cudaStream_t st) {
  using W = typename FT<E>::W;
  std::stable_sort(it, it + n, [](const MultiItem& u, const MultiItem& v) { return u.cost > v.cost; });
  const Sizes z = sizes_of(it, n);
  if (z.Nsm > 0 && z.Nbig > 0) return cudaErrorInvalidValue;  // one residence per launch
  const bool seq = z.Nsm == 0;  // global-memory residence
  const size_t smem = smem_t<E>(z, path);
  const void* kfn = seq ? (const void*)omp_seq_kernel<E> : (const void*)omp_multi_kernel<E>;
  const int threads = seq ? kSThreads : kMThreads;
  cudaError_t e = raise_smem_limit(kfn, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, threads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // resident CTAs: all that fit, or the tuned number per SM (fewer CTAs keep
  // fewer instance vectors in flight, which can keep them in L2)
  if (ctas_per_sm > 0 && ctas_per_sm < occ) occ = ctas_per_sm;
  const int64_t need = seq ? n : (n + 1) / 2, cap = (int64_t)occ * sms;
  const int grid = (int)(need < cap ? need : cap);
  const int per = seq ? 1 : 2;  // instance slots per CTA

  std::vector<MInst<E>> d((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    MInst<E>& m = d[(size_t)i];
    m.P = chain_dev<E>(*it[i].P);
    m.y = (const E*)it[i].y;
    m.x = (W*)it[i].x;
    m.supp = it[i].supp;
    m.K = it[i].K;
    m.t_switch = it[i].t_switch;
    m.idx = it[i].idx;
    m.pad = 0;
  }
  // workspace, stream-ordered: counter | descriptors | h0 | B | vector | bits | kidx
  // (the last three in global-memory launches only: Nbig = 0 otherwise)
  const size_t g2 = (size_t)grid * per;
  const size_t o_inst = 16, o_h0 = a16(o_inst + (size_t)n * sizeof(MInst<E>));
  const size_t o_B = a16(o_h0 + g2 * z.Nmax * sizeof(E));
  const size_t o_buf = a16(o_B + g2 * tri(z.Kmax) * sizeof(W));
  const size_t o_bits = a16(o_buf + (size_t)grid * z.Nbig * sizeof(E));
  const size_t o_kidx = a16(o_bits + g2 * (size_t)(z.Nbig >> 5) * sizeof(uint32_t));
  const size_t total = a16(o_kidx + g2 * (size_t)z.Nbig * sizeof(uint16_t));
  char* ws = nullptr;
  if ((e = cudaMallocAsync((void**)&ws, total, st)) != cudaSuccess) return e;
  MArgs<E> a;
  a.inst = (const MInst<E>*)(ws + o_inst);
  a.count = n;
  a.rel_tol = rel_tol;
  a.path = path;
  a.Nsm = z.Nsm;
  a.Nbig = z.Nbig;
  a.Nmax = z.Nmax;
  a.Kmax = z.Kmax;
  a.iters_out = iters_out;
  a.res_out = res_out;
  a.h0_ws = (E*)(ws + o_h0);
  a.B_ws = (W*)(ws + o_B);
  a.buf_ws = (E*)(ws + o_buf);
  a.bits_ws = (uint32_t*)(ws + o_bits);
  a.kidx_ws = (uint16_t*)(ws + o_kidx);
  a.counter = (int*)ws;
  a.status = status;
  a.max_phases = 2 * (n + 2) * (2LL * z.Kmax + 10) + 16;
  e = cudaMemsetAsync(ws, 0, 16, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + o_inst, d.data(), (size_t)n * sizeof(MInst<E>), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    if (seq) omp_seq_kernel<E><<<grid, kSThreads, smem, st>>>(a);
    else omp_multi_kernel<E><<<grid, kMThreads, smem, st>>>(a);
    e = cudaGetLastError();
  }
  const cudaError_t e2 = cudaFreeAsync(ws, st);
  return e != cudaSuccess ? e : e2;
}

}  // namespace

cudaError_t chain_twiddles(int logN, cudaStream_t st, const void** tw64, const void** tw32) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, std::pair<void*, void*>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  std::pair<void*, void*>& t = cache[std::make_pair(dev, logN)];
  if (!t.first) {
    const size_t N = (size_t)1 << logN;
    void *a = nullptr, *b = nullptr;
    cudaError_t e = cudaMalloc(&a, N * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&b, N * sizeof(float2));
    if (e == cudaSuccess) e = launch_twiddles_log(logN, a, b, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      if (a) cudaFree(a);
      if (b) cudaFree(b);
      return e;
    }
    t = std::make_pair(a, b);
  }
  *tw64 = t.first;
  *tw32 = t.second;
  return cudaSuccess;
}

int multi_switch_big(int logN) { return logN <= kMaxLogN ? 64 : 32; }

// Work of one instance in FMA-like units: the correlation (kernel sums up to
// the switch, two transforms per iteration after it; global-memory buffers
// weigh more) or the FP64 least squares, whichever is longer.
double multi_cost(const PlanView& P, int K, int t_switch, int path) {
  const double N = P.N, lg = P.logN, w = P.dft ? 4.0 : 1.0;
  const int tf = path == PATH_FAST ? K : (path == PATH_CONV ? 0 : std::min(K, t_switch));
  double corr = N * w * (0.5 * tf * (double)tf + (double)(K - tf) * 2.0 * lg + lg);
  if (P.large) corr *= 4.0;
  const double ls = 40.0 * w * (double)K * K * K / 3.0;
  return std::max(corr, ls);
}

size_t omp_multi_smem(const MultiItem* it, int64_t n, int path) {
  const Sizes z = sizes_of(it, n);
  const PlanView& P = *it[0].P;
  if (P.dft) return P.fp32 ? smem_t<float2>(z, path) : smem_t<double2>(z, path);
  return P.fp32 ? smem_t<float>(z, path) : smem_t<double>(z, path);
}

cudaError_t launch_omp_multi(MultiItem* it, int64_t n, double rel_tol, int path, int ctas_per_sm, int* iters_out,
                             double* res_out, int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const PlanView& P = *it[0].P;
  if (P.dft)
    return P.fp32 ? multi_t<float2>(it, n, rel_tol, path, ctas_per_sm, iters_out, res_out, status, st)
                  : multi_t<double2>(it, n, rel_tol, path, ctas_per_sm, iters_out, res_out, status, st);
  return P.fp32 ? multi_t<float>(it, n, rel_tol, path, ctas_per_sm, iters_out, res_out, status, st)
                : multi_t<double>(it, n, rel_tol, path, ctas_per_sm, iters_out, res_out, status, st);
}

int omp_multi_occupancy(const MultiItem* it, int64_t n, int path, int* err) {
  *err = 0;
  if (n <= 0) return 0;
  const PlanView& P = *it[0].P;
  if (P.dft) return P.fp32 ? occ_t<float2>(it, n, path, err) : occ_t<double2>(it, n, path, err);
  return P.fp32 ? occ_t<float>(it, n, path, err) : occ_t<double>(it, n, path, err);
}

}  // namespace csf
