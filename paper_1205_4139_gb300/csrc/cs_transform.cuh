// Block-level transforms in shared memory: the unnormalised N-point DFT as a
// decimation-in-frequency (DIF) forward chain and its exact adjoint, a
// decimation-in-time (DIT) inverse chain, and the Sylvester Walsh-Hadamard
// transform.  One CTA owns one length-N vector; every pass reads R elements
// per butterfly into registers, runs an in-register radix-R butterfly and
// writes them back to the same slots, so passes need one barrier each and no
// second buffer.
//
// Ordering.  The forward DIF chain takes natural order and leaves frequency k
// at position pos(k) (mixed-radix digit reversal of the pass schedule); the
// inverse DIT chain consumes that order and produces natural order.  The
// library therefore scatters a residual r_m straight to pos(Omega_m) and gets
// h = A^H zf(r) in natural order with no reordering pass (Algorithm 1.1
// step 2), and gathers A x at pos(Omega_m) after a forward chain (step 7).
//
// Pass schedule for N = 2^n: floor(n/4) radix-16 passes, then one pass of
// radix 2^(n mod 4) if n mod 4 != 0.  Pass p of the DIF chain works on
// sub-transforms of length L_p (L_0 = N, L_{p+1} = L_p / R_p) with stride
// S_p = L_p / R_p and post-multiplies output q of butterfly n by
// W_{L_p}^{n q}, W_L = exp(-2 pi i / L).  Those twiddles come from a per-plan
// table, pass after pass, laid out [q-1][n] so that neighbouring threads read
// neighbouring entries.
#pragma once
#include <type_traits>

#include "cs_common.cuh"

namespace csf {

// Pass p of the DIF chain: L_p = N >> 4p, radix 2^min(4, log2 L_p), and the
// twiddle-table offset sum_{q<p} (R_q - 1) L_q / R_q = N - L_p.
__host__ __device__ inline int sched_passes(int logN) { return (logN + 3) >> 2; }
__host__ __device__ inline int sched_logL(int logN, int p) { return logN - 4 * p; }
__host__ __device__ inline int sched_logR(int logN, int p) {
  const int l = logN - 4 * p;
  return l < 4 ? l : 4;
}

// Position of frequency k after the forward DIF chain (host and device).
__host__ __device__ inline int dif_position(int k, int logN) {
  int pos = 0;
  const int P = sched_passes(logN);
  for (int p = 0; p < P; ++p) {
    const int lr = sched_logR(logN, p);
    const int q = k & ((1 << lr) - 1);
    k >>= lr;
    pos += q << (sched_logL(logN, p) - lr);  // digit q has stride S_p = L_p / R_p
  }
  return pos;
}

template <class E> __device__ __forceinline__ E ldt(const E* p) { return __ldg(p); }

// Loaders and sinks let the first pass of a chain read its input from
// somewhere other than the buffer (a zero-filled vector assembled on the
// fly) and the last pass hand its outputs to a consumer (a masked residual,
// an arg-max) instead of, or as well as, storing them: that removes the
// separate zero-fill, scatter, masking and read-back passes and their
// barriers.  A sink receives (position, value) and stores what it wants.
struct NoLoad {};
struct NoSink {};

template <class LD, int R, class E>
__device__ __forceinline__ void pass_load(const LD& ld, const E* buf, int base, int S, E (&v)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if constexpr (std::is_same<LD, NoLoad>::value) v[r] = buf[swz<E>(base + r * S)];
    else v[r] = ld(base + r * S);
  }
}

template <class SK, class E>
__device__ __forceinline__ void pass_store(SK& sk, E* buf, int pos, const E& o) {
  if constexpr (std::is_same<SK, NoSink>::value) buf[swz<E>(pos)] = o;
  else sk(pos, o);
}

template <int R, class E, class LD, class SK>
__device__ __forceinline__ void dif_pass(const Grp& g, E* buf, int N, int L, const E* __restrict__ tw,
                                         const LD& ld, SK& sk) {
  constexpr int LR = ilog2c(R);
  const int S = L >> LR;
  const int logS = 31 - __clz(S);
  for (int b = g.tid; b < (N >> LR); b += g.n) {
    const int n = b & (S - 1);
    const int base = ((b >> logS) * L) + n;
    E v[R];
    pass_load<LD, R>(ld, buf, base, S, v);
    dft_reg<R, -1>(v);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      E o = v[bitrevc(q, LR)];
      if (q > 0 && S > 1) o = mul(o, ldt(tw + (q - 1) * S + n));
      pass_store(sk, buf, base + q * S, o);
    }
  }
  g.sync();
}

template <int R, class E, class LD, class SK>
__device__ __forceinline__ void dit_pass(const Grp& g, E* buf, int N, int L, const E* __restrict__ tw,
                                         const LD& ld, SK& sk) {
  constexpr int LR = ilog2c(R);
  const int S = L >> LR;
  const int logS = 31 - __clz(S);
  for (int b = g.tid; b < (N >> LR); b += g.n) {
    const int n = b & (S - 1);
    const int base = ((b >> logS) * L) + n;
    E u[R];
    pass_load<LD, R>(ld, buf, base, S, u);
    if (S > 1) {
#pragma unroll
      for (int q = 1; q < R; ++q) u[q] = mulc(u[q], ldt(tw + (q - 1) * S + n));
    }
    dft_reg<R, +1>(u);
#pragma unroll
    for (int r = 0; r < R; ++r) pass_store(sk, buf, base + r * S, u[bitrevc(r, LR)]);
  }
  g.sync();
}

template <int R, class E, class LD, class SK>
__device__ __forceinline__ void wht_pass(const Grp& g, E* buf, int N, int S, const LD& ld, SK& sk) {
  constexpr int LR = ilog2c(R);
  const int logS = 31 - __clz(S);
  for (int b = g.tid; b < (N >> LR); b += g.n) {
    const int n = b & (S - 1);
    const int base = ((b >> logS) << (logS + LR)) + n;
    E v[R];
    pass_load<LD, R>(ld, buf, base, S, v);
    wht_reg<R>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) pass_store(sk, buf, base + r * S, v[r]);
  }
  g.sync();
}

// N = 1: the transform is the identity; still route the single element
// through the loader and the sink.
template <class E, class LD, class SK>
__device__ __forceinline__ void pass_identity(const Grp& g, E* buf, const LD& ld, SK& sk) {
  if (g.tid == 0) {
    E v[1];
    pass_load<LD, 1>(ld, buf, 0, 1, v);
    pass_store(sk, buf, 0, v[0]);
  }
  g.sync();
}

// One DIF / DIT / WHT pass with the loader if it is the chain's first pass
// and the sink if it is the last.
template <int R, int KIND, class E, class LD, class SK>
__device__ __forceinline__ void pass_fl(const Grp& g, E* buf, int N, int LS, const E* tw, bool first, bool last,
                                        const LD& ld, SK& sk) {
  NoLoad nl;
  NoSink ns;
  if (first && last) {
    if constexpr (KIND == 0) dif_pass<R>(g, buf, N, LS, tw, ld, sk);
    else if constexpr (KIND == 1) dit_pass<R>(g, buf, N, LS, tw, ld, sk);
    else wht_pass<R>(g, buf, N, LS, ld, sk);
  } else if (first) {
    if constexpr (KIND == 0) dif_pass<R>(g, buf, N, LS, tw, ld, ns);
    else if constexpr (KIND == 1) dit_pass<R>(g, buf, N, LS, tw, ld, ns);
    else wht_pass<R>(g, buf, N, LS, ld, ns);
  } else if (last) {
    if constexpr (KIND == 0) dif_pass<R>(g, buf, N, LS, tw, nl, sk);
    else if constexpr (KIND == 1) dit_pass<R>(g, buf, N, LS, tw, nl, sk);
    else wht_pass<R>(g, buf, N, LS, nl, sk);
  } else {
    if constexpr (KIND == 0) dif_pass<R>(g, buf, N, LS, tw, nl, ns);
    else if constexpr (KIND == 1) dit_pass<R>(g, buf, N, LS, tw, nl, ns);
    else wht_pass<R>(g, buf, N, LS, nl, ns);
  }
}

template <int KIND, class E, class LD, class SK>
__device__ __forceinline__ void pass_radix(const Grp& g, E* buf, int N, int LS, const E* tw, int lr, bool first,
                                           bool last, const LD& ld, SK& sk) {
  switch (lr) {
    case 4: pass_fl<16, KIND>(g, buf, N, LS, tw, first, last, ld, sk); break;
    case 3: pass_fl<8, KIND>(g, buf, N, LS, tw, first, last, ld, sk); break;
    case 2: pass_fl<4, KIND>(g, buf, N, LS, tw, first, last, ld, sk); break;
    default: pass_fl<2, KIND>(g, buf, N, LS, tw, first, last, ld, sk); break;
  }
}

// Forward DFT F (exp(-2 pi i ...), unnormalised): natural order in,
// digit-reversed order out.  The first pass reads through `ld` (or buf), the
// last pass writes through `sk` (or to buf); every pass ends on g's barrier.
template <class E, class LD = NoLoad, class SK = NoSink>
__device__ void dft_forward(const Grp& g, E* buf, int logN, const E* __restrict__ tw, const LD& ld = LD{},
                            SK&& sk = SK{}) {
  const int N = 1 << logN, P = sched_passes(logN);
  if (P == 0) pass_identity(g, buf, ld, sk);
  for (int p = 0; p < P; ++p) {
    const int L = 1 << sched_logL(logN, p);
    pass_radix<0>(g, buf, N, L, tw + (N - L), sched_logR(logN, p), p == 0, p == P - 1, ld, sk);
  }
}

// Adjoint F^H (exp(+2 pi i ...), unnormalised): digit-reversed order in,
// natural order out.
template <class E, class LD = NoLoad, class SK = NoSink>
__device__ void dft_adjoint(const Grp& g, E* buf, int logN, const E* __restrict__ tw, const LD& ld = LD{},
                            SK&& sk = SK{}) {
  const int N = 1 << logN, P = sched_passes(logN);
  if (P == 0) pass_identity(g, buf, ld, sk);
  for (int p = P - 1; p >= 0; --p) {
    const int L = 1 << sched_logL(logN, p);
    pass_radix<1>(g, buf, N, L, tw + (N - L), sched_logR(logN, p), p == P - 1, p == 0, ld, sk);
  }
}

// Unnormalised Sylvester Hadamard transform H (symmetric, H H = N I),
// natural order in and out.
template <class E, class LD = NoLoad, class SK = NoSink>
__device__ void wht(const Grp& g, E* buf, int logN, const LD& ld = LD{}, SK&& sk = SK{}) {
  const int N = 1 << logN;
  int S = 1, rem = logN;
  if (rem == 0) pass_identity(g, buf, ld, sk);
  while (rem > 0) {
    const int lr = rem >= 4 ? 4 : rem;
    pass_radix<2>(g, buf, N, S, (const E*)nullptr, lr, S == 1, rem == lr, ld, sk);
    S <<= lr;
    rem -= lr;
  }
}

}  // namespace csf
