// Building blocks of the hot path, each run by one group of warps (`Grp`) on
// one instance:
//   * correlate_transform  h = A^H zf_Omega(v)         (Algorithm 1.1 step 2)
//   * correlate_residual   h = A^H zf(y - S A x_Lambda) (steps 7 and 2)
//   * correlate_fast       h = h_0 - sum_k x_k c(j (-) lambda_k)
//                                                      (Eq. kernelsumOMP)
//   * each followed by the identification of step 3 (arg-max of |h|^2 over j
//     not in Lambda, lowest j on ties)
//   * tri_matvec / tri_vecmat_row, the two FP64 triangular products of the
//     least-squares update of step 6 (Gram column read off c, Eq. kernelsum).
#pragma once
#include "cs_internal.h"
#include "cs_transform.cuh"

namespace csf {

// Static per-plan data every kernel reads.
template <class E>
struct PlanDev {
  int N, logN, M;
  const int* __restrict__ slot;  // [N]: m if position holds row Omega_m, else -1
  const E* __restrict__ tw;      // DIF twiddles in the working precision (DFT only)
  const E* __restrict__ c;       // correlation kernel vector, working precision (storage format cfmt)
  const typename FT<E>::W* __restrict__ c64;  // correlation kernel vector, FP64 (storage format cfmt)
  int cfmt;                      // CFMT_FULL, CFMT_HALF (DFT) or CFMT_INT (WHT)
  const int* __restrict__ ci;    // CFMT_INT: N c(d), exact integers
};

// v 2^-logN in T, exact for |v| < 2^24 (FP32) or 2^53 (FP64): the integer
// converts exactly and the power of two scales exactly
template <class T> __device__ __forceinline__ T int_scaled(int v, int logN);
template <> __device__ __forceinline__ float int_scaled<float>(int v, int logN) {
  return __int2float_rn(v) * __int_as_float((127 - logN) << 23);
}
template <> __device__ __forceinline__ double int_scaled<double>(int v, int logN) {
  return __int2double_rn(v) * __longlong_as_double((long long)(1023 - logN) << 52);
}
template <> __device__ __forceinline__ float2 int_scaled<float2>(int v, int logN) {
  return make_float2(int_scaled<float>(v, logN), 0.f);
}
template <> __device__ __forceinline__ double2 int_scaled<double2>(int v, int logN) {
  return make_double2(int_scaled<double>(v, logN), 0.0);
}

// c(d), 0 <= d < N, from a vector in storage format `fmt` (s: the full or
// half vector in T; ci: the integers N c(d); N = 2^logN).  For CFMT_INT the
// scaling by 2^-logN is exact.
template <class T>
__device__ __forceinline__ T c_entry(int fmt, const T* __restrict__ s, const int* __restrict__ ci, int N, int logN,
                                     int d) {
  if (fmt == CFMT_HALF) return d <= (N >> 1) ? __ldg(s + d) : conjv(__ldg(s + (N - d)));
  if (fmt == CFMT_INT) return int_scaled<T>(__ldg(ci + d), logN);
  return __ldg(s + d);
}
template <class E>
__device__ __forceinline__ typename FT<E>::W c64_at(const PlanDev<E>& P, int d) {
  return c_entry(P.cfmt, P.c64, P.ci, P.N, P.logN, d);
}
template <class E>
__device__ __forceinline__ E cw_at(const PlanDev<E>& P, int d) {
  return c_entry(P.cfmt, P.c, P.ci, P.N, P.logN, d);
}

template <class E>
inline PlanDev<E> plan_dev(const PlanView& P) {
  PlanDev<E> d;
  d.N = P.N;
  d.logN = P.logN;
  d.M = P.M;
  d.slot = P.slot;
  constexpr bool f32 = sizeof(typename FT<E>::R) == 4;
  d.tw = (const E*)(f32 ? P.tw32 : P.tw64);
  d.c = (const E*)(f32 ? P.c32 : P.c64);
  d.c64 = (const typename FT<E>::W*)P.c64;
  d.cfmt = P.cfmt;
  d.ci = P.ci;
  return d;
}

// |h|^2 type used for identification: the working precision.
template <class E> struct NormT { using V = typename FT<E>::R; };

// Selection keys: unsigned integers that order like |h|^2 (the bit pattern of
// a non-negative IEEE number orders like the number), with the top bit set
// for candidates and 0 for excluded positions, in the working precision's
// width (32 bits for FP32, 64 for FP64).
template <class E> struct KeyT;
template <> struct KeyT<float> { using U = uint32_t; };
template <> struct KeyT<float2> { using U = uint32_t; };
template <> struct KeyT<double> { using U = unsigned long long; };
template <> struct KeyT<double2> { using U = unsigned long long; };
__device__ __forceinline__ uint32_t sel_key(float v) { return __float_as_uint(v) | 0x80000000u; }
__device__ __forceinline__ unsigned long long sel_key(double v) {
  return (unsigned long long)__double_as_longlong(v) | 0x8000000000000000ull;
}

// Unnormalised transform of the kind: DFT uses F^H (adjoint chain) for the
// correlation and F (forward chain) for the synthesis; WHT uses H for both.
template <class E, bool DFT>
__device__ __forceinline__ void transform_adjoint(const Grp& g, E* buf, const PlanDev<E>& P) {
  if constexpr (DFT) dft_adjoint(g, buf, P.logN, P.tw);
  else wht(g, buf, P.logN);
}
template <class E, bool DFT>
__device__ __forceinline__ void transform_forward(const Grp& g, E* buf, const PlanDev<E>& P) {
  if constexpr (DFT) dft_forward(g, buf, P.logN, P.tw);
  else wht(g, buf, P.logN);
}

__device__ __forceinline__ bool in_bits(const uint32_t* bits, int j) { return (bits[j >> 5] >> (j & 31)) & 1u; }

// 1/sqrt(N) for N = 2^logN, exact to the working precision without FP64 math
template <class R>
__device__ __forceinline__ R inv_sqrt_pow2(int logN) {
  const R r = (R)1 / (R)(1 << (logN >> 1));
  return (logN & 1) ? r * (R)0.70710678118654752440 : r;
}

// buf <- scl * zf_Omega(v) in the position order the adjoint chain expects
// (unit stride over positions, so the slot-map reads coalesce); with NORM,
// returns sum |v_m|^2 over this thread's entries (FP64).
template <class E, bool NORM>
__device__ double load_zero_filled(const Grp& g, E* buf, const PlanDev<E>& P, const E* __restrict__ v,
                                   typename FT<E>::R scl) {
  double s = 0.0;
  for (int pos = g.tid; pos < P.N; pos += g.n) {
    const int m = __ldg(P.slot + pos);
    E e = zero<E>();
    if (m >= 0) {
      const E vm = v[m];
      if constexpr (NORM) s += norm2(to_w(vm));
      e = scale(vm, scl);
    }
    buf[swz<E>(pos)] = e;
  }
  g.sync();
  return s;
}

// First-pass loader of the forward synthesis: the zero-filled coefficient
// vector x_Lambda, read from the support bitmap and the position ->
// coefficient index map.  The first forward pass strides by N/16, so a warp
// reads 32 consecutive positions (one bitmap word, broadcast).
template <class E>
struct SparseLoader {
  const uint32_t* bits;
  const uint16_t* kidx;
  const E* xw;
  __device__ __forceinline__ E operator()(int pos) const {
    return in_bits(bits, pos) ? xw[kidx[pos]] : zero<E>();
  }
};

// Last-pass sink of a correlation: running arg-max of |h(j)|^2 over j not
// flagged in `bits` (NULL: none), lowest j on ties; optionally stores h.  The
// last adjoint pass strides by N/16, so a warp's outputs are consecutive.
template <class E>
struct ArgmaxSink {
  using V = typename NormT<E>::V;
  const uint32_t* bits;
  E* h_out;
  V bv;
  int bj;
  typename KeyT<E>::U* keys;  // selection keys (nullable)
  __device__ __forceinline__ void operator()(int j, const E& h) {
    if (h_out) h_out[j] = h;
    const bool ex = bits && in_bits(bits, j);
    const V v = ex ? (V)-1 : (V)norm2(h);
    if (keys) keys[j] = ex ? 0 : sel_key(v);
    if (better(v, j, bv, bj)) { bv = v; bj = j; }
  }
};

// h = A^H zf_Omega(v) by one adjoint transform, fused with the arg-max of
// step 3 (no exclusions) and an optional store of h; returns the arg-max
// (to every thread of g) and, with NORM, this thread's share of sum |v_m|^2
// in *norm (FP64; reduce it over g).
template <class E, bool DFT, bool NORM = false>
__device__ int correlate_transform(const Grp& g, E* buf, const PlanDev<E>& P, const E* __restrict__ v, E* h_out,
                                   double* norm, typename NormT<E>::V* rv, int* rj) {
  using R = typename FT<E>::R;
  using V = typename NormT<E>::V;
  const double s = load_zero_filled<E, NORM>(g, buf, P, v, inv_sqrt_pow2<R>(P.logN));
  ArgmaxSink<E> sk{nullptr, h_out, (V)-1, 0x7fffffff, nullptr};
  if constexpr (DFT) dft_adjoint(g, buf, P.logN, P.tw, NoLoad{}, sk);
  else wht(g, buf, P.logN, NoLoad{}, sk);
  if (norm) *norm = s;
  return group_argmax(g, sk.bv, sk.bj, rv, rj);
}

// Residual of step 7 on the buffer: forward transform of the zero-filled
// coefficients (the first pass assembles them from the support in
// (bits, kidx, xw)), then buf <- N^{-1/2} y - N^{-1} F x on Omega and zero
// elsewhere, i.e. N^{-1/2} zf_Omega(y - S_Omega A x_Lambda) in the adjoint
// chain's position order.  With NORM, returns to every thread of g
// ||y - Phi x||^2 (FP64 accumulation of the working-precision residual; red
// holds 33 doubles), else 0.
template <class E, bool DFT, bool NORM>
__device__ double residual_on_omega(const Grp& g, E* buf, const PlanDev<E>& P, const E* __restrict__ y,
                                    const uint32_t* bits, const uint16_t* kidx, const E* xw, double* red) {
  using R = typename FT<E>::R;
  const int N = P.N;
  const SparseLoader<E> sl{bits, kidx, xw};
  if constexpr (DFT) dft_forward(g, buf, P.logN, P.tw, sl, NoSink{});
  else wht(g, buf, P.logN, sl, NoSink{});
  // buf holds F x (unnormalised).  Write N^{-1/2} y - N^{-1} F x on Omega and
  // zero elsewhere; the unnormalised adjoint then yields
  // N^{-1/2} F^H zf(y) - N^{-1} F^H S^T S F x = A^H zf(y - S A x).
  const R sy = inv_sqrt_pow2<R>(P.logN), sx = (R)1 / (R)N;
  double acc[1] = {0.0};
  for (int pos = g.tid; pos < N; pos += g.n) {
    const int m = __ldg(P.slot + pos);
    const int a = swz<E>(pos);
    const E r = m >= 0 ? sub(scale(y[m], sy), scale(buf[a], sx)) : zero<E>();
    if constexpr (NORM) acc[0] += norm2(to_w(r));
    buf[a] = r;
  }
  if constexpr (NORM) {
    group_sum(g, acc, red);  // ends with a group barrier
    return acc[0] * (double)N;  // the entries are r_m / sqrt(N); N is a power of two
  } else {
    g.sync();
    return 0.0;
  }
}

// h = A^H zf(y - S_Omega A x_Lambda) for the support in (bits, kidx, xw):
// the residual on Omega (residual_on_omega), then one adjoint transform whose
// last pass feeds the arg-max over j not in Lambda.  Returns the arg-max to
// every thread of g; with NORM also ||y - Phi x||^2 in *r2 (red: 33 doubles).
template <class E, bool DFT, bool NORM = false>
__device__ int correlate_residual(const Grp& g, E* buf, const PlanDev<E>& P, const E* __restrict__ y,
                                  const uint32_t* bits, const uint16_t* kidx, const E* xw,
                                  typename NormT<E>::V* rv, int* rj, const uint32_t* excl = nullptr,
                                  typename KeyT<E>::U* keys = nullptr, double* r2 = nullptr,
                                  double* red = nullptr) {
  using V = typename NormT<E>::V;
  const double rr = residual_on_omega<E, DFT, NORM>(g, buf, P, y, bits, kidx, xw, red);
  if constexpr (NORM) *r2 = rr;
  // OMP excludes the support itself; the pursuits pass their own exclusion
  ArgmaxSink<E> sk{keys ? excl : bits, nullptr, (V)-1, 0x7fffffff, keys};
  if constexpr (DFT) dft_adjoint(g, buf, P.logN, P.tw, NoLoad{}, sk);
  else wht(g, buf, P.logN, NoLoad{}, sk);
  return group_argmax(g, sk.bv, sk.bj, rv, rj);
}

// residual_on_omega with the norm chosen at run time (one inlined copy of
// the forward transform where a caller needs both forms).
template <class E, bool DFT>
__device__ double residual_on_omega_rt(const Grp& g, E* buf, const PlanDev<E>& P, const E* __restrict__ y,
                                       const uint32_t* bits, const uint16_t* kidx, const E* xw, double* red,
                                       bool norm) {
  using R = typename FT<E>::R;
  const int N = P.N;
  const SparseLoader<E> sl{bits, kidx, xw};
  if constexpr (DFT) dft_forward(g, buf, P.logN, P.tw, sl, NoSink{});
  else wht(g, buf, P.logN, sl, NoSink{});
  const R sy = inv_sqrt_pow2<R>(P.logN), sx = (R)1 / (R)N;
  if (norm) {  // two loops: no FP64 instruction, even predicated off, in the plain one
    double acc[1] = {0.0};
    for (int pos = g.tid; pos < N; pos += g.n) {
      const int m = __ldg(P.slot + pos);
      const int a = swz<E>(pos);
      const E r = m >= 0 ? sub(scale(y[m], sy), scale(buf[a], sx)) : zero<E>();
      acc[0] += norm2(to_w(r));
      buf[a] = r;
    }
    group_sum(g, acc, red);  // ends with a group barrier
    return acc[0] * (double)N;
  }
  for (int pos = g.tid; pos < N; pos += g.n) {
    const int m = __ldg(P.slot + pos);
    const int a = swz<E>(pos);
    buf[a] = m >= 0 ? sub(scale(y[m], sy), scale(buf[a], sx)) : zero<E>();
  }
  g.sync();
  return 0.0;
}

// The second half of correlate_residual for OMP: the adjoint transform of
// the residual on the buffer, its last pass feeding the arg-max over j not
// in Lambda (bits).  Returns the arg-max to every thread of g.
template <class E, bool DFT>
__device__ int adjoint_argmax(const Grp& g, E* buf, const PlanDev<E>& P, const uint32_t* bits,
                              typename NormT<E>::V* rv, int* rj) {
  using V = typename NormT<E>::V;
  ArgmaxSink<E> sk{bits, nullptr, (V)-1, 0x7fffffff, nullptr};
  if constexpr (DFT) dft_adjoint(g, buf, P.logN, P.tw, NoLoad{}, sk);
  else wht(g, buf, P.logN, NoLoad{}, sk);
  return group_argmax(g, sk.bv, sk.bj, rv, rj);
}

// Explicit residual check of the halting test (step 8) in FP32 mode.  The
// FP64 downdate ||r_t||^2 = ||y||^2 - sum |zeta_k|^2 carries the FP32
// rounding of h_0 on its right-hand side (about 1e-7 ||y||^2), so it cannot
// resolve the tolerance (||r|| < 1e-6 ||y||, squared 1e-12).  When the
// downdate falls below kResidTrigger ||y||^2 (well above that floor and far
// below the residual of any noisy run at 40 dB or less), the next step forms
// r = y - Phi x explicitly by one forward transform and decides on its norm,
// which resolves ||r|| / ||y|| to a few 1e-7.
constexpr double kResidTrigger = 1e-5;
template <class E>
__host__ __device__ __forceinline__ bool resid_check(double rel_tol) {
  return sizeof(typename FT<E>::R) == 4 && rel_tol > 0.0;
}

// Whether the fast correlation stores c twice over (DFT, when 2N elements
// fit in 128 KB of shared memory).
template <class E>
__host__ __device__ inline bool kernel_doubled(int N) {
  return FT<E>::C && 2 * (size_t)N * sizeof(E) <= (size_t)128 * 1024;
}

// Load c into shared memory for the fast correlation.  With `doubled` (DFT
// only) c is stored twice over so that c[(j - l) mod N + T e] is read at an
// immediate offset without a wrap test; otherwise the index is masked.
template <class E, bool DFT>
__device__ void load_kernel_vector(const Grp& g, E* cb, const PlanDev<E>& P, bool doubled) {
  const int n = (DFT && doubled) ? 2 * P.N : P.N;
  for (int i = g.tid; i < n; i += g.n) cb[i] = cw_at(P, i & (P.N - 1));
  g.sync();
}

// One chunk of CH outputs per thread: j = j0 + T e, e < CH.
template <class E, bool DFT, bool DBL, int CH>
__device__ __forceinline__ void fast_chunks(const Grp& g, const E* cb, const E* h0, const int* lam,
                                            const E* xw, int s, int N, const uint32_t* bits, E* h_out,
                                            typename NormT<E>::V& bv, int& bj, typename KeyT<E>::U* keys) {
  using V = typename NormT<E>::V;
  const int T = g.n;
  for (int j0 = g.tid; j0 < N; j0 += T * CH) {
    E acc[CH];
#pragma unroll
    for (int e = 0; e < CH; ++e) acc[e] = h0[j0 + T * e];
    for (int k = 0; k < s; ++k) {
      const int l = lam[k];
      const E xv = xw[k];
      if constexpr (DFT && DBL) {
        const E* cp = cb + ((j0 - l) & (N - 1));
#pragma unroll
        for (int e = 0; e < CH; ++e) acc[e] = fnms(acc[e], xv, cp[T * e]);
      } else if constexpr (DFT) {
#pragma unroll
        for (int e = 0; e < CH; ++e) acc[e] = fnms(acc[e], xv, cb[(j0 + T * e - l) & (N - 1)]);
      } else {
#pragma unroll
        for (int e = 0; e < CH; ++e) acc[e] = fnms(acc[e], xv, cb[(j0 + T * e) ^ l]);
      }
    }
#pragma unroll
    for (int e = 0; e < CH; ++e) {
      const int j = j0 + T * e;
      if (h_out) h_out[j] = acc[e];
      const bool ex = bits && in_bits(bits, j);
      const V v = ex ? (V)-1 : (V)norm2(acc[e]);
      if (keys) keys[j] = ex ? 0 : sel_key(v);
      if (better(v, j, bv, bj)) { bv = v; bj = j; }
    }
  }
}

template <class E, bool DFT, bool DBL>
__device__ __forceinline__ void fast_dispatch(const Grp& g, const E* cb, const E* h0, const int* lam, const E* xw,
                                              int s, int N, const uint32_t* bits, E* h_out,
                                              typename NormT<E>::V& bv, int& bj, typename KeyT<E>::U* keys) {
  const int per = N / g.n;  // outputs per thread (power of two, or 0 when N < T)
  if (per >= 8) fast_chunks<E, DFT, DBL, 8>(g, cb, h0, lam, xw, s, N, bits, h_out, bv, bj, keys);
  else if (per >= 4) fast_chunks<E, DFT, DBL, 4>(g, cb, h0, lam, xw, s, N, bits, h_out, bv, bj, keys);
  else if (per >= 2) fast_chunks<E, DFT, DBL, 2>(g, cb, h0, lam, xw, s, N, bits, h_out, bv, bj, keys);
  else fast_chunks<E, DFT, DBL, 1>(g, cb, h0, lam, xw, s, N, bits, h_out, bv, bj, keys);
}

// h(j) = h0(j) - sum_{k<s} x_k c(j (-) lam_k) for all j (Eq. kernelsumOMP),
// then the arg-max over j not in `bits`.  cb is c in shared memory, stored
// twice over when `doubled` (DFT).
template <class E, bool DFT>
__device__ int correlate_fast(const Grp& g, const E* cb, const E* h0, const int* lam, const E* xw, int s, int N,
                              const uint32_t* bits, E* h_out, typename NormT<E>::V* rv, int* rj, bool doubled,
                              typename KeyT<E>::U* keys = nullptr) {
  using V = typename NormT<E>::V;
  V bv = (V)-1;
  int bj = 0x7fffffff;
  if (DFT && doubled) fast_dispatch<E, DFT, true>(g, cb, h0, lam, xw, s, N, bits, h_out, bv, bj, keys);
  else fast_dispatch<E, DFT, false>(g, cb, h0, lam, xw, s, N, bits, h_out, bv, bj, keys);
  return group_argmax(g, bv, bj, rv, rj);
}

// ------------------------------------------------------------------------
// FP64 least squares (Algorithm 1.1 step 6) by an explicit inverse Cholesky
// factor.  With G_p = Phi_p^H Phi_p = L L^H, the library keeps B = L^{-1}
// (packed lower triangle, row i at i(i+1)/2, in global memory), z = L^{-1} b
// with b_k = h_0(lambda_k) = (Phi^H y)(lambda_k), and x = B^H z.  Adding
// column lambda with Gram column g_k = c(lambda_k (-) lambda) (Eq. kernelsum):
//   u = B g,  d^2 = c(0) - ||u||^2,  zeta = (b_p - u^H z) / d,
//   row p of B = [-(u^H B) / d, 1 / d],   x += zeta * conj(row p of B),
//   ||r||^2 -= |zeta|^2.
__device__ __forceinline__ int pidx(int i) { return (i * (i + 1)) >> 1; }

// Layout of the paired, chunked triangular products: row (column) pairs
// i <-> p-1-i over lanes, so that every lane carries p + 1 terms; the
// concatenated pair split into `chunks` slices over the group's warps (in a
// 4-warp group, one warp per SM sub-partition carries the FP64 work).
// Partial sums take chunks * p <= max(2 n, p) elements.  With more pairs than
// threads each thread walks pairs with stride n and chunks = 1.
struct PairSplit {
  int P2, chunks, pair, chunk, stride;
  __device__ PairSplit(const Grp& g, int p) {
    P2 = (p + 1) >> 1;
    int lanes = ((P2 + 31) >> 5) << 5;
    if (lanes == 0) lanes = 32;
    chunks = lanes <= g.n ? g.n / lanes : 1;
    stride = lanes <= g.n ? lanes : g.n;
    pair = g.tid % stride;
    chunk = g.tid / stride;
  }
};

// u_i = sum_{k<=i} B[i][k] g_k, i < p; result overwrites gv.  part holds
// max(2 n, p) elements.  B is read with plain loads: it is written by the
// same kernel.
// u_i = sum_{k<=i} B[i][k] g_k, i < p; result overwrites gv.  part holds
// max(2 n, p) elements.  B is read with plain loads: it is written by the
// same kernel.  When `terms` is given, the thread that finishes u_k also
// writes the FP64 terms |u_k|^2 and conj(u_k) z_k there (3 doubles per k),
// for the caller's reductions.
template <class W>
__device__ void tri_matvec(const Grp& grp, const W* B, W* gv, W* part, int p, const W* z = nullptr,
                           double* terms = nullptr) {
  if (p == 0) return;
  PairSplit ps(grp, p);
  if (ps.chunk < ps.chunks) {
    for (int pr = ps.pair; pr < ps.P2; pr += ps.stride) {
      const int ra = pr, rb = p - 1 - pr;
      const int la = ra + 1, lc = (rb != ra) ? la + rb + 1 : la;
      const int q0 = (ps.chunk * lc) / ps.chunks, q1 = ((ps.chunk + 1) * lc) / ps.chunks;
      // One accumulator and one FMA per position, whichever row the position
      // falls in: the row switch is a register move, not a second FMA path.
      W acc = W{}, first = W{};
      const W* Bb = B + pidx(rb) - la;
      const W* gb = gv - la;
      const W* Ba = B + pidx(ra);
      for (int q = q0; q < q1; ++q) {
        const bool second = q >= la;
        if (q == la) { first = acc; acc = W{}; }
        acc = fmav(acc, second ? Bb[q] : Ba[q], second ? gb[q] : gv[q]);
      }
      const bool ended_in_b = q1 > la;
      const W pa = ended_in_b ? (q0 < la ? first : W{}) : acc;
      const W pb = ended_in_b ? acc : W{};
      part[ps.chunk * p + ra] = pa;
      if (rb != ra) part[ps.chunk * p + rb] = pb;
    }
  }
  grp.sync();
  for (int i = grp.tid; i < p; i += grp.n) {
    W s = part[i];
    for (int c = 1; c < ps.chunks; ++c) s = add(s, part[c * p + i]);
    gv[i] = s;
    if (terms) {
      const W t = cmul(s, z[i]);
      terms[3 * i] = norm2(s);
      terms[3 * i + 1] = re(t);
      terms[3 * i + 2] = im(t);
    }
  }
  grp.sync();
}

// w_k = scl * sum_{i=k}^{p-1} conj(u_i) B[i][k], k < p, written to row p of
// B and to part[0..p).
template <class W>
__device__ void tri_vecmat_row(const Grp& grp, W* B, const W* u, W* part, int p, double scl) {
  if (p == 0) return;
  PairSplit ps(grp, p);
  if (ps.chunk < ps.chunks) {
    for (int pr = ps.pair; pr < ps.P2; pr += ps.stride) {
      const int ka = pr, kb = p - 1 - pr;
      const int la = p - ka, lc = (kb != ka) ? la + (p - kb) : la;
      const int q0 = (ps.chunk * lc) / ps.chunks, q1 = ((ps.chunk + 1) * lc) / ps.chunks;
      W acc = W{}, first = W{};
      for (int q = q0; q < q1; ++q) {
        const bool second = q >= la;
        if (q == la) { first = acc; acc = W{}; }
        const int i = second ? kb + (q - la) : ka + q;
        acc = fmacv(acc, u[i], B[pidx(i) + (second ? kb : ka)]);
      }
      const bool ended_in_b = q1 > la;
      const W pa = ended_in_b ? (q0 < la ? first : W{}) : acc;
      const W pb = ended_in_b ? acc : W{};
      part[ps.chunk * p + ka] = pa;
      if (kb != ka) part[ps.chunk * p + kb] = pb;
    }
  }
  grp.sync();
  // part[k] (chunk 0) is only ever read by the thread that owns column k
  for (int k = grp.tid; k < p; k += grp.n) {
    W s = part[k];
    for (int c = 1; c < ps.chunks; ++c) s = add(s, part[c * p + k]);
    s = scale(s, scl);
    part[k] = s;
    B[pidx(p) + k] = s;
  }
  grp.sync();
}

}  // namespace csf
