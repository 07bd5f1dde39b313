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

template <int R, class E>
__device__ __forceinline__ void dif_pass(E* buf, int N, int L, const E* __restrict__ tw) {
  constexpr int LR = ilog2c(R);
  const int S = L >> LR;
  const int logS = 31 - __clz(S);
  for (int b = threadIdx.x; b < (N >> LR); b += blockDim.x) {
    const int n = b & (S - 1);
    const int base = ((b >> logS) * L) + n;
    E v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = buf[swz<E>(base + r * S)];
    dft_reg<R, -1>(v);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      E o = v[bitrevc(q, LR)];
      if (q > 0 && S > 1) o = mul(o, ldt(tw + (q - 1) * S + n));
      buf[swz<E>(base + q * S)] = o;
    }
  }
  __syncthreads();
}

template <int R, class E>
__device__ __forceinline__ void dit_pass(E* buf, int N, int L, const E* __restrict__ tw) {
  constexpr int LR = ilog2c(R);
  const int S = L >> LR;
  const int logS = 31 - __clz(S);
  for (int b = threadIdx.x; b < (N >> LR); b += blockDim.x) {
    const int n = b & (S - 1);
    const int base = ((b >> logS) * L) + n;
    E u[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      E t = buf[swz<E>(base + q * S)];
      if (q > 0 && S > 1) t = mulc(t, ldt(tw + (q - 1) * S + n));
      u[q] = t;
    }
    dft_reg<R, +1>(u);
#pragma unroll
    for (int r = 0; r < R; ++r) buf[swz<E>(base + r * S)] = u[bitrevc(r, LR)];
  }
  __syncthreads();
}

template <int R, class E>
__device__ __forceinline__ void wht_pass(E* buf, int N, int S) {
  constexpr int LR = ilog2c(R);
  const int logS = 31 - __clz(S);
  for (int b = threadIdx.x; b < (N >> LR); b += blockDim.x) {
    const int n = b & (S - 1);
    const int base = ((b >> logS) << (logS + LR)) + n;
    E v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = buf[swz<E>(base + r * S)];
    wht_reg<R>(v);
#pragma unroll
    for (int r = 0; r < R; ++r) buf[swz<E>(base + r * S)] = v[r];
  }
  __syncthreads();
}

// Forward DFT F (exp(-2 pi i ...), unnormalised): natural order in,
// digit-reversed order out.  buf must be visible to all threads on entry.
template <class E>
__device__ void dft_forward(E* buf, int logN, const E* __restrict__ tw) {
  const int N = 1 << logN, P = sched_passes(logN);
  for (int p = 0; p < P; ++p) {
    const int L = 1 << sched_logL(logN, p);
    const E* t = tw + (N - L);
    switch (sched_logR(logN, p)) {
      case 4: dif_pass<16>(buf, N, L, t); break;
      case 3: dif_pass<8>(buf, N, L, t); break;
      case 2: dif_pass<4>(buf, N, L, t); break;
      default: dif_pass<2>(buf, N, L, t); break;
    }
  }
}

// Adjoint F^H (exp(+2 pi i ...), unnormalised): digit-reversed order in,
// natural order out.
template <class E>
__device__ void dft_adjoint(E* buf, int logN, const E* __restrict__ tw) {
  const int N = 1 << logN, P = sched_passes(logN);
  for (int p = P - 1; p >= 0; --p) {
    const int L = 1 << sched_logL(logN, p);
    const E* t = tw + (N - L);
    switch (sched_logR(logN, p)) {
      case 4: dit_pass<16>(buf, N, L, t); break;
      case 3: dit_pass<8>(buf, N, L, t); break;
      case 2: dit_pass<4>(buf, N, L, t); break;
      default: dit_pass<2>(buf, N, L, t); break;
    }
  }
}

// Unnormalised Sylvester Hadamard transform H (symmetric, H H = N I),
// natural order in and out.
template <class E>
__device__ void wht(E* buf, int logN) {
  const int N = 1 << logN;
  int S = 1, rem = logN;
  while (rem > 0) {
    const int lr = rem >= 4 ? 4 : rem;
    switch (lr) {
      case 4: wht_pass<16>(buf, N, S); break;
      case 3: wht_pass<8>(buf, N, S); break;
      case 2: wht_pass<4>(buf, N, S); break;
      default: wht_pass<2>(buf, N, S); break;
    }
    S <<= lr;
    rem -= lr;
  }
}

}  // namespace csf
