// Large plans (2^14 <= N <= 2^24): the hot path with its length-N vectors in
// global memory, one instance spread over many CTAs.
//
//   * Transforms are four-step.  With N = N1 N2 and the natural index split
//     as i = i2 + N2 i1 (a row-major N1 x N2 view), the DFT is
//         X(k1 + N1 k2) = sum_i2 w_N2^(i2 k2) w_N^(i2 k1) sum_i1 x(i2 + N2 i1) w_N1^(i1 k1)
//     and the Sylvester WHT is H_N = H_N1 (x) H_N2 (no twiddles, output index
//     k2 + N2 k1).  Pass 1 transforms the columns (length N1, stride N2) in
//     tiles of adjacent columns and applies w_N^(i2 k1); pass 2 transforms
//     the rows (length N2, contiguous) in tiles of adjacent rows and writes
//     natural order.  Both sub-transforms are the shared-memory chains of
//     cs_transform.cuh; each pass reads and writes N elements once.  Only F
//     is computed: the adjoint is read off it by negating the output index,
//     (F^H v)(j) = (F v)(-j mod N), in pass 2's sink.
//   * Pass 2 hands its outputs to a sink: store h and/or keep the CTA's
//     arg-max (Algorithm 1.1 steps 2-3), the residual y - Phi x on Omega
//     (step 7), or the kernel vector c (Eq. kernelsum).
//   * The fast correlation h(j) = h_0(j) - sum_k x_k c(j (-) lambda_k)
//     (Eq. kernelsumOMP) reads c from L2 (c of N = 2^22 complex64 is 32 MB),
//     2048 outputs per CTA, and keeps the CTA's arg-max.
//   * One CTA per instance reduces the arg-max partials, appends the column
//     with the FP64 inverse-factor update of cs_ls.cuh (step 6, Gram entries
//     read off c) and tests the halting rule (step 8).
// The host queues, per iteration t, the correlation (kernel sums, or the
// forward transform of zf(x), the residual on Omega and the adjoint
// transform) and then the least squares, all on the caller's stream; a
// finished instance makes every later kernel of that instance return at
// once.
#include <atomic>
#include <map>
#include <mutex>
#include <cmath>

#include "cs_blocks.cuh"
#include "cs_cg.cuh"
#include "cs_internal.h"
#include "cs_ls.cuh"
#include "cs_select.cuh"

namespace csf {

namespace {

constexpr int kLT = 256;                   // threads per CTA of every kernel here
constexpr int kFastMaxCH = 8;              // outputs per thread of the fast correlation, at most
constexpr int kMaxBatchY = 65535;          // instances ride on gridDim.y
constexpr int kU = 8;                      // independent accesses per thread in flight in the pass loops

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

template <class E>
struct LDev {
  using W = typename FT<E>::W;
  int N, logN, M, n1, n2, wsh;
  const int* __restrict__ slot;  // [N] natural order: m if j = Omega_m, else -1
  const int* __restrict__ om_off;   // Omega by pass-2 row: offsets [N1 + 1] (NULL if M = 0)
  const int2* __restrict__ om_ent;  //   entries (j, m), grouped by row
  const int* __restrict__ oc_off;   // Omega by pass-1 column: offsets [N2 + 1] (NULL if M = 0)
  const int2* __restrict__ oc_ent;  //   entries (j, m), grouped by column
  const E* __restrict__ tw1;     // DIF twiddles of the N1 chain
  const E* __restrict__ tw2;     // DIF twiddles of the N2 chain
  const E* __restrict__ wlo;     // w_N^m, m < 2^wsh
  const E* __restrict__ whi;     // w_N^(m 2^wsh), m < N / 2^wsh
  const E* __restrict__ c;       // kernel vector, working precision (storage format cfmt)
  const W* __restrict__ c64;     // kernel vector, FP64 (storage format cfmt)
  int cfmt;                      // CFMT_FULL, CFMT_HALF (DFT) or CFMT_INT (WHT)
  const int* __restrict__ ci;    // CFMT_INT: N c(d)
};

template <class E>
LDev<E> ldev(const PlanView& P) {
  LDev<E> d;
  d.N = P.N;
  d.logN = P.logN;
  d.M = P.M;
  d.n1 = P.n1;
  d.n2 = P.n2;
  d.wsh = P.wsh;
  d.slot = P.slot;
  d.om_off = P.om_off;
  d.om_ent = P.om_ent;
  d.oc_off = P.oc_off;
  d.oc_ent = P.oc_ent;
  constexpr bool f32 = sizeof(typename FT<E>::R) == 4;
  const E* t = (const E*)(f32 ? P.lt32 : P.lt64);
  const int N1 = 1 << P.n1, N2 = 1 << P.n2;
  d.tw1 = t;
  d.tw2 = t ? t + N1 : nullptr;
  d.wlo = t ? t + N1 + N2 : nullptr;
  d.whi = t ? t + N1 + N2 + (1 << P.wsh) : nullptr;
  d.c = (const E*)(f32 ? P.c32 : P.c64);
  d.c64 = (const typename FT<E>::W*)P.c64;
  d.cfmt = P.cfmt;
  d.ci = P.ci;
  return d;
}

// A pass tile is 32 bytes wide: C = 32 / sizeof(E) adjacent columns (pass 1)
// or rows (pass 2), one full DRAM sector per tile row.  In shared memory each
// column / row is a swizzled buffer of its own, 16 bytes apart from the next
// one's bank pattern.
template <class E> __host__ __device__ constexpr int tile_c() { return 32 / (int)sizeof(E); }
template <class E> __host__ __device__ constexpr int log_tile_c() { return ilog2c(32 / (int)sizeof(E)); }
template <class E> __host__ __device__ inline int lstride(int len) { return len + 16 / (int)sizeof(E); }

struct LState {  // per instance, in the workspace
  int p, done, pad0, pad1;
  double ynorm2, rn2;
  int ncols;  // distinct support columns of the four-step split registered so far
  int chk;    // FP32 mode: the halting test waits for the explicit residual (lchk_kernel)
};

// Compact input of pass 2 for a sparse vector (the forward transform of
// zf(x_Lambda)): Tc[b][k1][c] is pass 1's output at row k1 and the c-th
// distinct column cols[b][c] of the support; every other column is zero.
template <class E>
struct LSparse {
  const E* Tc;      // NULL: pass 2 reads the dense pass-1 output
  const int* cols;  // [batch][kc]
  int kc;
};

enum { LD_DENSE = 0, LD_ZF = 1, LD_ONES = 2 };
enum { SK_H = 0, SK_ARG = 1, SK_RES = 2, SK_KV = 3, SK_RESN = 4 };

template <class E> __device__ __forceinline__ E one_e();
template <> __device__ __forceinline__ float one_e<float>() { return 1.f; }
template <> __device__ __forceinline__ double one_e<double>() { return 1.0; }
template <> __device__ __forceinline__ float2 one_e<float2>() { return make_float2(1.f, 0.f); }
template <> __device__ __forceinline__ double2 one_e<double2>() { return make_double2(1.0, 0.0); }

// w_N^m = w_N^(m_hi 2^wsh) w_N^(m_lo), m < N
template <class E>
__device__ __forceinline__ E root(const LDev<E>& P, int m) {
  return mul(__ldg(P.whi + (m >> P.wsh)), __ldg(P.wlo + (m & ((1 << P.wsh) - 1))));
}

// Forward chain (DIF for DFT, natural order in, digit-reversed out; WHT
// natural in and out) on buffer gi of the tile, by a group of kLT / C threads.
template <class E, bool DFT>
__device__ __forceinline__ void tile_chain(E* buf, int len_log, int stride, const E* tw) {
  constexpr int C = tile_c<E>(), GS = kLT / C;
  const int gi = threadIdx.x / GS;
  const Grp g{(int)threadIdx.x % GS, GS, GS == 32 ? -1 : 1 + gi};
  E* col = buf + gi * stride;
  if constexpr (DFT) dft_forward(g, col, len_log, tw);
  else wht(g, col, len_log);
}

// CTA-wide arg-max (largest v, lowest j); thread 0 writes the partial.
template <class V>
__device__ __forceinline__ void block_partial(V v, int j, V* rv, int* rj, V* out_v, int* out_j) {
  warp_argmax(v, j);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    rv[w] = v;
    rj[w] = j;
  }
  __syncthreads();
  if (w == 0) {
    V vv = lane < (kLT >> 5) ? rv[lane] : (V)-1;
    int jj = lane < (kLT >> 5) ? rj[lane] : 0x7fffffff;
    warp_argmax(vv, jj);
    if (lane == 0) {
      *out_v = vv;
      *out_j = vv < (V)0 ? -1 : jj;
    }
  }
}

// ------------------------------------------------------- pass scaffolding
// Shared memory of a pass CTA: the C swizzled buffers, the digit-reversal
// table of the sub-transform (DFT), the arg-max scratch.
template <class E>
struct PassSmem {
  size_t tab, red, rv, rj, total;
};
template <class E>
__host__ __device__ inline PassSmem<E> pass_layout(int len) {
  using V = typename NormT<E>::V;
  PassSmem<E> L;
  L.tab = al16((size_t)tile_c<E>() * lstride<E>(len) * sizeof(E));
  L.red = L.tab + al16((size_t)len * sizeof(short));
  L.rv = L.red + al16((kLT / 32) * sizeof(double));
  L.rj = L.rv + al16(34 * sizeof(V));
  L.total = L.rj + 34 * sizeof(int);
  return L;
}

// CTA-wide FP64 sum; thread 0 gets the total (fixed order: deterministic).
__device__ __forceinline__ double block_sum0(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kLT / 32; ++w) t += red[w];
  return t;
}

// One element, global -> shared, without passing through registers
// (cp.async: 4, 8 or 16 bytes), so that a thread keeps all of its tile's
// copies in flight at once.
template <class E>
__device__ __forceinline__ void cp_async_elem(E* sdst, const E* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gsrc), "n"((int)sizeof(E)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// tab[k] = position of frequency k after the forward DIF chain of length 2^lg
__device__ __forceinline__ void build_position_table(short* tab, int lg) {
  for (int k = threadIdx.x; k < (1 << lg); k += kLT) tab[k] = (short)dif_position(k, lg);
}

// ----------------------------------------------------------------- pass 1
// out[b][k1 N2 + i2] = (w_N^(i2 k1) for DFT) * sum_i1 v(i2 + N2 i1) w_N1^(i1 k1)
// for the C columns i2 of this CTA, v = in (LD_DENSE, stride in_stride),
// zf_Omega(in) (LD_ZF, in has in_stride >= M entries per instance, indexed
// by m: the tile is cleared and Omega's entries in its columns placed, read
// from the plan's grouping of Omega by column) or zf_Omega(1) (LD_ONES).
// Only the forward transform F is computed here: the adjoint is read off it
// by index negation in pass 2.
template <class E, bool DFT, int LD>
__global__ void __launch_bounds__(kLT) lcol_kernel(LDev<E> P, const E* __restrict__ in, int64_t in_stride,
                                                   E* __restrict__ out, const LState* __restrict__ st) {
  constexpr int C = tile_c<E>(), LC = log_tile_c<E>();
  extern __shared__ __align__(16) unsigned char sm[];
  E* buf = (E*)sm;
  const int64_t b = blockIdx.y;
  if (st && st[b].done) return;
  const int n1 = P.n1, n2 = P.n2, N1 = 1 << n1;
  const int cs = lstride<E>(N1);
  const PassSmem<E> L = pass_layout<E>(N1);
  short* tab = (short*)(sm + L.tab);
  const int c0 = blockIdx.x * C;
  const E* src = in ? in + b * in_stride : nullptr;
  // C * N1 is a multiple of kLT, so every guard below is uniform per step
  const int tot = C * N1;
  if constexpr (LD == LD_DENSE) {
    for (int q = threadIdx.x; q < tot; q += kLT)
      cp_async_elem(buf + (q & (C - 1)) * cs + swz<E>(q >> LC), src + c0 + (q & (C - 1)) + ((q >> LC) << n2));
  } else if constexpr (LD == LD_ZF) {
    // clear the C buffers (C * cs * sizeof(E) is a multiple of 16 bytes)
    uint4* z4 = (uint4*)buf;
    const int n4 = (int)(((size_t)C * cs * sizeof(E)) >> 4);
    for (int q = threadIdx.x; q < n4; q += kLT) z4[q] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (P.oc_off) {  // Omega's entries in columns c0 .. c0 + C - 1, kU in flight per thread
      const int e0 = __ldg(P.oc_off + c0), e1 = __ldg(P.oc_off + c0 + C), msk = (1 << n2) - 1;
      for (int q0 = e0 + (int)threadIdx.x; q0 < e1; q0 += kU * kLT) {
        int2 jm[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) jm[u] = q0 + u * kLT < e1 ? __ldg(P.oc_ent + q0 + u * kLT) : make_int2(-1, 0);
        E v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) v[u] = jm[u].x >= 0 ? src[jm[u].y] : zero<E>();
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (jm[u].x >= 0) buf[((jm[u].x & msk) - c0) * cs + swz<E>(jm[u].x >> n2)] = v[u];
      }
    }
  } else {  // LD_ONES: zero-filled through the slot map, kU in flight per thread
    for (int q0 = threadIdx.x; q0 < tot; q0 += kU * kLT) {
      int m[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int q = q0 + u * kLT;
        m[u] = q < tot ? __ldg(P.slot + c0 + (q & (C - 1)) + ((q >> LC) << n2)) : -1;
      }
      E v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) v[u] = m[u] >= 0 ? one_e<E>() : zero<E>();
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int q = q0 + u * kLT;
        if (q < tot) buf[(q & (C - 1)) * cs + swz<E>(q >> LC)] = v[u];
      }
    }
  }
  if constexpr (DFT) build_position_table(tab, n1);
  if constexpr (LD == LD_DENSE) cp_async_wait_all();
  __syncthreads();
  tile_chain<E, DFT>(buf, n1, cs, P.tw1);
  __syncthreads();
  E* dst = out + b * (int64_t)P.N;
  for (int q0 = threadIdx.x; q0 < tot; q0 += kU * kLT) {
    E v[kU], w[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = q0 + u * kLT;
      const int c = q & (C - 1), k1 = q >> LC;
      if (q < tot) {
        if constexpr (DFT) {
          v[u] = buf[c * cs + swz<E>(tab[k1])];
          w[u] = root(P, (c0 + c) * k1);
        } else {
          v[u] = buf[c * cs + swz<E>(k1)];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int q = q0 + u * kLT;
      if (q < tot) dst[c0 + (q & (C - 1)) + ((q >> LC) << n2)] = DFT ? mul(v[u], w[u]) : v[u];
    }
  }
}

// ----------------------------------------------------------------- pass 2
// Transforms the C rows k1 of this CTA (T[b][k1 N2 + i2], contiguous): the
// forward output X(jf), jf natural, is the adjoint's output at j = -jf mod N
// when neg is set (F^H v (j) = F v (-j), DFT), else at j = jf.  Each output
// v = scl * X is handed to the sink:
//   SK_H    out[j] = v (if out), arg-max over all j      -> partial
//   SK_ARG  arg-max over j whose bit is clear in `bits` -> partial
//   SK_RES  out[m] = y[m] - v where j = Omega_m (the residual on Omega,
//           compact: M entries per instance)
//   SK_KV   out[j] = v
//   SK_RESN only for instances whose state asks for the explicit residual:
//           the CTA's FP64 share of sum |y[m] - v|^2 over Omega's members in
//           its rows -> rpart[b * gridDim.x + blockIdx.x] (nothing stored)
// A partial is written to part_v / part_j[b * nparts + blockIdx.x].
template <class E, bool DFT, int SK>
__global__ void __launch_bounds__(kLT) lrow_kernel(LDev<E> P, const E* __restrict__ T, int neg,
                                                   typename FT<E>::R scl, E* __restrict__ out,
                                                   const E* __restrict__ y, const uint32_t* __restrict__ bits,
                                                   typename NormT<E>::V* __restrict__ part_v,
                                                   int* __restrict__ part_j, int nparts,
                                                   const LState* __restrict__ st, LSparse<E> sp,
                                                   double* __restrict__ rpart) {
  using V = typename NormT<E>::V;
  constexpr int C = tile_c<E>(), LC = log_tile_c<E>();
  extern __shared__ __align__(16) unsigned char sm[];
  E* buf = (E*)sm;
  const int64_t b = blockIdx.y;
  if (st && st[b].done) return;
  if (SK == SK_RESN && !st[b].chk) return;
  const int n1 = P.n1, n2 = P.n2, N2 = 1 << n2, Nm = P.N - 1;
  const int cs = lstride<E>(N2);
  const PassSmem<E> L = pass_layout<E>(N2);
  short* tab = (short*)(sm + L.tab);
  V* rv = (V*)(sm + L.rv);
  int* rj = (int*)(sm + L.rj);
  const int r0 = blockIdx.x * C;
  const int tot = C * N2;  // a multiple of kLT
  if (sp.Tc) {
    // sparse input: zero rows, then the registered columns of rows r0 ..
    for (int q = threadIdx.x; q < tot; q += kLT) buf[(q >> n2) * cs + swz<E>(q & (N2 - 1))] = zero<E>();
    __syncthreads();
    const int nc = st[b].ncols;
    const E* tcb = sp.Tc + b * ((int64_t)1 << n1) * sp.kc;
    const int* cb = sp.cols + b * sp.kc;
    for (int i = threadIdx.x; i < C * nc; i += kLT) {
      const int r = i / nc, c = i - r * nc;
      buf[r * cs + swz<E>(cb[c])] = tcb[(int64_t)(r0 + r) * sp.kc + c];
    }
  } else {
    const E* src = T + b * (int64_t)P.N;
    for (int q = threadIdx.x; q < tot; q += kLT)
      cp_async_elem(buf + (q >> n2) * cs + swz<E>(q & (N2 - 1)), src + ((r0 + (q >> n2)) << n2) + (q & (N2 - 1)));
  }
  if constexpr (DFT) build_position_table(tab, n2);
  cp_async_wait_all();
  __syncthreads();
  tile_chain<E, DFT>(buf, n2, cs, P.tw2);
  __syncthreads();
  E* dst = out ? out + b * (int64_t)(SK == SK_RES ? P.M : P.N) : nullptr;
  const E* yb = y ? y + b * (int64_t)P.M : nullptr;
  const uint32_t* bb = bits ? bits + b * (int64_t)(P.N >> 5) : nullptr;
  if constexpr (SK == SK_RESN) {  // ||y - Phi x||^2, this CTA's share, FP64, fixed order
    __shared__ double red[kLT / 32];
    double acc = 0.0;
    if (P.om_off) {
      const int e0 = __ldg(P.om_off + r0), e1 = __ldg(P.om_off + r0 + C);
      for (int e = e0 + (int)threadIdx.x; e < e1; e += kLT) {
        const int2 jm = __ldg(P.om_ent + e);  // (j, m)
        const int j = jm.x;
        int c, pos;
        if constexpr (DFT) {
          c = (j & ((1 << n1) - 1)) - r0;
          pos = tab[j >> n1];
        } else {
          c = (j >> n2) - r0;
          pos = j & (N2 - 1);
        }
        acc += norm2(to_w(sub(yb[jm.y], scale(buf[c * cs + swz<E>(pos)], scl))));
      }
    }
    acc = block_sum0(acc, red);
    if (threadIdx.x == 0) rpart[b * gridDim.x + blockIdx.x] = acc;
    return;
  }
  if constexpr (SK == SK_RES) {
    // only Omega's outputs are wanted: visit the members of Omega in this
    // CTA's rows (grouped by row in the plan) instead of every output's slot
    if (!neg && P.om_off) {
      const int e0 = __ldg(P.om_off + r0), e1 = __ldg(P.om_off + r0 + C);
      for (int e = e0 + (int)threadIdx.x; e < e1; e += kLT) {
        const int2 jm = __ldg(P.om_ent + e);  // (j, m)
        const int j = jm.x;
        int c, pos;
        if constexpr (DFT) {  // row k1 = j mod N1, frequency k2 = j / N1 at its chain position
          c = (j & ((1 << n1) - 1)) - r0;
          pos = tab[j >> n1];
        } else {              // row j / N2, natural position j mod N2
          c = (j >> n2) - r0;
          pos = j & (N2 - 1);
        }
        dst[jm.y] = sub(yb[jm.y], scale(buf[c * cs + swz<E>(pos)], scl));
      }
      return;
    }
  }
  V bv = (V)-1;
  int bj = 0x7fffffff;
  for (int q0 = threadIdx.x; q0 < tot; q0 += kU * kLT) {
    E v[kU];
    int jj[kU], aux[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {  // shared reads and the per-output lookups, all issued first
      const int q = q0 + u * kLT;
      int c, pos, jf;
      if constexpr (DFT) {  // C adjacent outputs per k2: jf = k1 + N1 k2
        c = q & (C - 1);
        const int k2 = q >> LC;
        jf = r0 + c + (k2 << n1);
        pos = q < tot ? tab[k2] : 0;
      } else {              // contiguous rows: jf = k2 + N2 k1
        c = q >> n2;
        pos = q & (N2 - 1);
        jf = pos + ((r0 + c) << n2);
      }
      jj[u] = neg ? ((P.N - jf) & Nm) : jf;
      aux[u] = 0;
      if (q < tot) {
        v[u] = buf[c * cs + swz<E>(pos)];
        if constexpr (SK == SK_RES) aux[u] = __ldg(P.slot + jj[u]);
        if constexpr (SK == SK_H || SK == SK_ARG) aux[u] = bb ? (int)in_bits(bb, jj[u]) : 0;
      }
    }
    E yv[kU];
    if constexpr (SK == SK_RES) {
#pragma unroll
      for (int u = 0; u < kU; ++u) yv[u] = (q0 + u * kLT < tot && aux[u] >= 0) ? yb[aux[u]] : zero<E>();
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (q0 + u * kLT >= tot) continue;
      const E o = scale(v[u], scl);
      const int j = jj[u];
      if constexpr (SK == SK_H || SK == SK_ARG) {
        if (SK == SK_H && dst) dst[j] = o;
        if (!aux[u]) {
          const V a = norm2(o);
          if (better(a, j, bv, bj)) {
            bv = a;
            bj = j;
          }
        }
      } else if constexpr (SK == SK_RES) {
        if (aux[u] >= 0) dst[aux[u]] = sub(yv[u], o);
      } else {
        dst[j] = o;
      }
    }
  }
  if constexpr (SK == SK_H || SK == SK_ARG) {
    if (part_v) block_partial(bv, bj, rv, rj, part_v + b * nparts + blockIdx.x, part_j + b * nparts + blockIdx.x);
  }
}

// ------------------------------------------------- sparse pass 1
// Pass 1 of the forward transform of zf(x_Lambda) straight from the support:
// column i2 of the N1 x N2 view holds the support entries lambda = i2 + N2 i1
// and pass 1's output there is sum over them of x_lambda w_N^(lambda k1)
// (DFT: w_N1^(i1 k1) w_N^(i2 k1) = w_N^(lambda k1)) or of
// x_lambda (-1)^popcount(i1 & k1) (WHT: H_N1 on the columns).  One thread per
// (k1, registered column c); the entries of a column are summed in the order
// they joined the support.  Output Tc[b][k1][c] (row stride kc).
template <class E, bool DFT>
__global__ void __launch_bounds__(kLT) lsp1_kernel(LDev<E> P, const E* __restrict__ xw, const int* __restrict__ lam,
                                                   const int* __restrict__ chead, const int* __restrict__ cnext,
                                                   int K, int kc, int kcl, E* __restrict__ Tc,
                                                   const LState* __restrict__ st, int only_chk) {
  const int64_t b = blockIdx.y;
  if (st[b].done || (only_chk && !st[b].chk)) return;
  const int nc = st[b].ncols;
  const int N1 = 1 << P.n1;
  const int idx = blockIdx.x * kLT + threadIdx.x;
  if (idx >= N1 * kcl) return;
  const int k1 = idx / kcl, c = idx - k1 * kcl;
  if (c >= nc) return;
  const int* nx = cnext + b * K;
  const int* lm = lam + b * K;
  const E* xv = xw + b * K;
  E acc = zero<E>();
  for (int k = chead[b * kc + c]; k >= 0; k = nx[k]) {
    const int l = lm[k];
    if constexpr (DFT) {
      acc = add(acc, mul(xv[k], root(P, (int)(((unsigned)l * (unsigned)k1) & (unsigned)(P.N - 1)))));
    } else {
      acc = (__popc((l >> P.n2) & k1) & 1) ? sub(acc, xv[k]) : add(acc, xv[k]);
    }
  }
  Tc[b * (int64_t)N1 * kc + (int64_t)k1 * kc + c] = acc;
}

// ------------------------------------------------------ fast correlation
// h(j) = h0(j) - sum_{k<s} x_k c(j (-) lam_k) for the kLT * CH outputs of
// this CTA (Eq. kernelsumOMP); lam / x of instance b start at b * kstride.
// Stores h if h != NULL; the arg-max over j with a clear bit (all j if
// bits == NULL) goes to the partial.
template <class E, bool DFT, int CF, int CH>
__global__ void __launch_bounds__(kLT) lfast_kernel(LDev<E> P, const E* __restrict__ h0,
                                                    const int* __restrict__ lam, const E* __restrict__ xw, int s,
                                                    int64_t kstride, const uint32_t* __restrict__ bits,
                                                    E* __restrict__ h, typename NormT<E>::V* __restrict__ part_v,
                                                    int* __restrict__ part_j, int nparts,
                                                    const LState* __restrict__ st) {
  using V = typename NormT<E>::V;
  extern __shared__ __align__(16) unsigned char sm[];
  const int64_t b = blockIdx.y;
  if (st && st[b].done) return;
  const int N = P.N;
  E* xs = (E*)sm;
  int* ls = (int*)(sm + al16((size_t)s * sizeof(E)));
  V* rv = (V*)(sm + al16((size_t)s * sizeof(E)) + al16((size_t)s * sizeof(int)));
  int* rj = (int*)((unsigned char*)rv + al16(34 * sizeof(V)));
  for (int k = threadIdx.x; k < s; k += kLT) {
    ls[k] = lam[b * kstride + k] & (N - 1);  // reduced mod N: no index leaves c
    xs[k] = xw[b * kstride + k];
  }
  __syncthreads();
  const int j0 = blockIdx.x * (kLT * CH) + threadIdx.x;
  const E* hb = h0 + b * (int64_t)N;
  E acc[CH];
#pragma unroll
  for (int e = 0; e < CH; ++e) acc[e] = hb[j0 + e * kLT];
#pragma unroll 2
  for (int k = 0; k < s; ++k) {
    const int l = ls[k];
    const E xk = xs[k];
#pragma unroll
    for (int e = 0; e < CH; ++e) {
      const int j = j0 + e * kLT;
      const int d = DFT ? ((j - l) & (N - 1)) : (j ^ l);
      E cv;
      if constexpr (CF == CFMT_HALF) cv = d <= (N >> 1) ? __ldg(P.c + d) : conjv(__ldg(P.c + (N - d)));
      else if constexpr (CF == CFMT_INT) cv = int_scaled<E>(__ldg(P.ci + d), P.logN);
      else cv = __ldg(P.c + d);
      acc[e] = fnms(acc[e], xk, cv);
    }
  }
  const uint32_t* bb = bits ? bits + b * (int64_t)(N >> 5) : nullptr;
  E* hout = h ? h + b * (int64_t)N : nullptr;
  V bv = (V)-1;
  int bj = 0x7fffffff;
#pragma unroll
  for (int e = 0; e < CH; ++e) {
    const int j = j0 + e * kLT;
    if (hout) hout[j] = acc[e];
    if (!bb || !in_bits(bb, j)) {
      const V a = norm2(acc[e]);
      if (better(a, j, bv, bj)) {
        bv = a;
        bj = j;
      }
    }
  }
  if (part_v) block_partial(bv, bj, rv, rj, part_v + b * nparts + blockIdx.x, part_j + b * nparts + blockIdx.x);
}

// arg-max of each instance's partials -> amax[b]
template <class V>
__global__ void __launch_bounds__(kLT) lreduce_kernel(const V* __restrict__ part_v, const int* __restrict__ part_j,
                                                      int stride, int nparts, int32_t* __restrict__ amax) {
  __shared__ V rv[34];
  __shared__ int rj[34];
  __shared__ V ov;
  __shared__ int oj;
  const int64_t b = blockIdx.x;
  V bv = (V)-1;
  int bj = 0x7fffffff;
  for (int i = threadIdx.x; i < nparts; i += kLT) {
    const V v = part_v[b * stride + i];
    const int j = part_j[b * stride + i];
    if (v >= (V)0 && better(v, j, bv, bj)) {
      bv = v;
      bj = j;
    }
  }
  block_partial(bv, bj, rv, rj, &ov, &oj);
  __syncthreads();
  if (threadIdx.x == 0) amax[b] = oj;
}

// bits[b] <- the set {supp[b][k] mod N}
__global__ void lbits_kernel(const int32_t* __restrict__ supp, int s, int N, uint32_t* __restrict__ bits) {
  const int64_t b = blockIdx.x;
  uint32_t* bb = bits + b * (int64_t)(N >> 5);
  for (int k = threadIdx.x; k < s; k += blockDim.x) {
    const int l = supp[b * s + k] & (N - 1);
    atomicOr(bb + (l >> 5), 1u << (l & 31));
  }
}

// w_N^m (m < 2^wsh) and w_N^(m 2^wsh) (m < N / 2^wsh), FP64 by sincospi of an
// exact argument, rounded to FP32 where asked
__global__ void roots_kernel(int logN, int wsh, double2* lo64, double2* hi64, float2* lo32, float2* hi32) {
  const int nlo = 1 << wsh, nhi = 1 << (logN - wsh);
  const double invN = ldexp(1.0, -logN);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nlo + nhi; i += gridDim.x * blockDim.x) {
    const bool lo = i < nlo;
    const int m = lo ? i : (i - nlo);
    const double a = -2.0 * (lo ? (double)m : ldexp((double)m, wsh)) * invN;
    double sn, cs;
    sincospi(a, &sn, &cs);
    if (lo) {
      lo64[m] = make_double2(cs, sn);
      if (lo32) lo32[m] = make_float2((float)cs, (float)sn);
    } else {
      hi64[m] = make_double2(cs, sn);
      if (hi32) hi32[m] = make_float2((float)cs, (float)sn);
    }
  }
}

// --------------------------------------------------------- least squares
// The FP64 column append of step 6 (the update of cs_ls.cuh: u = B g,
// d^2 = c(0) - ||u||^2, zeta = (h_0(lambda) - u^H z)/d, new row
// w = -u^H B / d, x += zeta conj(w)) split over G CTAs per instance so that a
// single large instance uses the whole GPU's FP64 units:
//   lls_u_kernel  step 3 (every CTA reduces the arg-max partials the same
//                 way), then u_i for a block of rows of B with equal area,
//                 plus the CTA's share of ||u||^2 and u^H z;
//   lls_w_kernel  every CTA adds the G shares in the same order, so all take
//                 the same d, zeta and halting decision; then w_k and x_k for
//                 a block of columns of equal area; the last CTA to finish
//                 (a ticket counter, no waiting) applies step 8.
template <class E>
struct LOmpArgs {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  LDev<E> P;
  const E* __restrict__ y;
  int K;
  double rel_tol;
  W* x_out;
  int* supp_out;
  int* iters_out;
  double* res_out;
  E* h0;           // [batch][N]
  E* xz;           // [batch][N] zero-filled x in the working precision, or NULL (not kept)
  uint32_t* bits;  // [batch][N / 32] support bitmap
  W* B;            // [batch][K(K+1)/2]
  W* z;            // [batch][K]
  W* x;            // [batch][K]
  W* u;            // [batch][K]
  E* xw;           // [batch][K]
  int* lam;        // [batch][K]
  LState* st;      // [batch]
  V* part_v;       // [batch][nparts]
  int* part_j;
  int nparts;
  double* ypart;   // [batch][nyp] shares of ||y||^2 from the first pass
  int nyp;
  double* terms;   // [batch][gmax][3] per-CTA shares of ||u||^2 and u^H z
  int gmax;
  // support columns of the four-step split (NULL: not kept), for the sparse
  // pass 1: colmap[b][i2] = registered index or -1; cols / chead / ctail per
  // registered column (at most kc); cnext[b][k] the next support index in k's
  // column or -1
  int* colmap;
  int* cols;
  int* chead;
  int* ctail;
  int* cnext;
  int kc;
};

// Boundaries of G blocks of equal area over p rows of a lower triangle
// (row i has i + 1 entries): rows [row_cut(g), row_cut(g + 1)).  Columns
// (column k has p - k entries) use the mirror image.
__device__ __forceinline__ int row_cut(int p, int g, int G) {
  if (g >= G) return p;
  const int r = (int)((double)p * sqrt((double)g / (double)G) + 0.5);
  return r < p ? r : p;
}
__device__ __forceinline__ int col_cut(int p, int g, int G) { return p - row_cut(p, G - g, G); }

template <class E>
__device__ void lwrite_outputs(const LOmpArgs<E>& a, int64_t b, int p, double ynorm2, double rn2) {
  using W = typename FT<E>::W;
  const int K = a.K;
  const W* xb = a.x + b * K;
  const int* lb = a.lam + b * K;
  for (int k = threadIdx.x; k < K; k += kLT) {
    if (a.x_out) a.x_out[b * K + k] = k < p ? __ldcg(xb + k) : W{};
    a.supp_out[b * K + k] = k < p ? __ldcg(lb + k) : -1;
  }
  if (threadIdx.x == 0) {
    if (a.iters_out) a.iters_out[b] = p;
    if (a.res_out) a.res_out[b] = ynorm2 > 0.0 ? sqrt(fmax(rn2, 0.0) / ynorm2) : 0.0;
    a.st[b].done = 1;
  }
}

template <class V>
__device__ __forceinline__ int reduce_partials(const V* pv, const int* pj, int n, V* rv, int* rj, V* sv, int* sj) {
  V bv = (V)-1;
  int bj = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += kLT) {
    const V v = pv[i];
    const int j = pj[i];
    if (v >= (V)0 && better(v, j, bv, bj)) {
      bv = v;
      bj = j;
    }
  }
  block_partial(bv, bj, rv, rj, sv, sj);
  __syncthreads();
  return *sj;
}

// ||y||^2 shares: CTA g of instance b sums |y_m|^2 in FP64 over its chunk of m
template <class E>
__global__ void __launch_bounds__(kLT) lynorm_kernel(const E* __restrict__ y, int M, double* __restrict__ ypart,
                                                     int nyp) {
  __shared__ double red[kLT / 32];
  const int64_t b = blockIdx.y;
  const int m0 = (int)(((int64_t)M * blockIdx.x) / nyp), m1 = (int)(((int64_t)M * (blockIdx.x + 1)) / nyp);
  double t = 0.0;
  for (int m = m0 + threadIdx.x; m < m1; m += kLT) t += norm2(to_w(y[b * (int64_t)M + m]));
  t = block_sum0(t, red);
  if (threadIdx.x == 0) ypart[b * nyp + blockIdx.x] = t;
}

// Phase u of the append for CTA gi of G on instance b; returns false when the
// instance is finished (or was already), uniformly over the CTA.
// gk: K FP64 elements of shared memory (the Gram column g).
template <class E>
__device__ bool ls_u_phase(const LOmpArgs<E>& a, int nparts, int G, int gi, int64_t b,
                           typename FT<E>::W* gk) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  __shared__ V rv[34], sv;
  __shared__ int rj[34], sj;
  __shared__ double red[kLT / 32];
  LState* S = a.st + b;
  if (S->done) return false;
  const int N = a.P.N, K = a.K, p = S->p;
  // step 3: the column with the largest |h(j)|^2
  const int l = reduce_partials(a.part_v + b * a.nparts, a.part_j + b * a.nparts, nparts, rv, rj, &sv, &sj);
  double ynorm2 = S->ynorm2;
  if (p == 0) {  // ||y||^2 from the first pass's shares, in a fixed order
    double t = 0.0;
    for (int i = threadIdx.x; i < a.nyp; i += kLT) t += a.ypart[b * a.nyp + i];
    ynorm2 = block_sum0(t, red);
    __syncthreads();
    if (threadIdx.x == 0) red[0] = ynorm2;
    __syncthreads();
    ynorm2 = red[0];
    if (!(ynorm2 > 0.0) || K == 0) {  // zero measurement (or K = 0): no iteration
      if (gi == 0) lwrite_outputs(a, b, 0, ynorm2, ynorm2);
      return false;
    }
  }
  if (l < 0) {  // no candidate column left
    if (gi == 0) lwrite_outputs(a, b, p, ynorm2, p == 0 ? ynorm2 : S->rn2);
    return false;
  }
  if (gi == 0 && threadIdx.x == 0) {
    S->pad1 = l;
    if (p == 0) {
      S->ynorm2 = ynorm2;
      S->rn2 = ynorm2;
    }
  }
  // u_i = sum_{k<=i} B[i][k] g_k for this CTA's rows; g_k = c(lambda_k (-) lambda)
  const int r0 = row_cut(p, gi, G), r1 = row_cut(p, gi + 1, G);
  const int* lam = a.lam + b * K;
  for (int k = threadIdx.x; k < r1; k += kLT) {
    const int d = DFT ? ((lam[k] - l) & (N - 1)) : (lam[k] ^ l);
    gk[k] = c_entry(a.P.cfmt, a.P.c64, a.P.ci, N, a.P.logN, d);
  }
  __syncthreads();
  const W* B = a.B + b * (((int64_t)K * (K + 1)) >> 1);
  const W* z = a.z + b * K;
  W* u = a.u + b * K;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double an = 0.0, ar = 0.0, ai = 0.0;
  for (int i = r0 + w; i < r1; i += kLT / 32) {
    const W* Bi = B + pidx(i);
    W acc = W{}, acc2 = W{};  // two independent chains: FP64 latency, not issue, bounds one row
    int k = lane;
    for (; k + 32 <= i; k += 64) {
      acc = fmav(acc, Bi[k], gk[k]);
      acc2 = fmav(acc2, Bi[k + 32], gk[k + 32]);
    }
    if (k <= i) acc = fmav(acc, Bi[k], gk[k]);
    acc = add(acc, acc2);
    const double sr = warp_sum(re(acc));
    const double si = DFT ? warp_sum(im(acc)) : 0.0;
    if (lane == 0) {
      const W ui = make_w<W>(sr, si);
      u[i] = ui;
      const W t = cmul(ui, z[i]);  // conj(u_i) z_i
      an += norm2(ui);
      ar += re(t);
      ai += im(t);
    }
  }
  // the CTA's shares, fixed order
  double* tb = a.terms + (b * a.gmax + gi) * 3;
  const double s0 = block_sum0(an, red);
  __syncthreads();
  const double s1 = block_sum0(ar, red);
  __syncthreads();
  const double s2 = block_sum0(ai, red);
  if (threadIdx.x == 0) {
    tb[0] = s0;
    tb[1] = s1;
    tb[2] = s2;
  }
  return true;
}

// Phase w of the append for CTA gi of G on instance b (after phase u of all
// G CTAs).
template <class E>
__device__ void ls_w_phase(const LOmpArgs<E>& a, int G, int gi, int64_t b) {
  using W = typename FT<E>::W;
  __shared__ int ticket;
  LState* S = a.st + b;
  if (S->done) return;
  const int N = a.P.N, K = a.K, p = S->p, l = S->pad1;
  const double ynorm2 = S->ynorm2;
  double rn2 = S->rn2;
  // every CTA adds the G shares in the same order: identical d and zeta
  double an = 0.0, ar = 0.0, ai = 0.0;
  for (int g = 0; g < G; ++g) {
    const double* tb = a.terms + (b * a.gmax + g) * 3;
    an += tb[0];
    ar += tb[1];
    ai += tb[2];
  }
  const double d2 = re(c_entry(a.P.cfmt, a.P.c64, a.P.ci, N, a.P.logN, 0)) - an;
  if (!(d2 > 1e-10 * ((double)a.P.M / (double)N))) {  // column dependent on Lambda: not added
    if (gi == 0) lwrite_outputs(a, b, p, ynorm2, rn2);
    return;
  }
  const double invd = rsqrt(d2);
  const W bp = to_w(a.h0[b * (int64_t)N + l]);  // (Phi^H y)(lambda)
  const W zeta = scale(sub(bp, make_w<W>(ar, ai)), invd);
  rn2 -= norm2(zeta);
  W* B = a.B + b * (((int64_t)K * (K + 1)) >> 1);
  W* x = a.x + b * K;
  E* xw = a.xw + b * K;
  const W* u = a.u + b * K;
  const int* lam = a.lam + b * K;
  E* xz = a.xz ? a.xz + b * (int64_t)N : nullptr;
  // w_k = -invd sum_{i=k}^{p-1} conj(u_i) B[i][k] over strips of 32 columns:
  // the lanes of a warp take the strip's columns (one contiguous segment of
  // each row), the 8 warps take every 8th row, and the 8 partial sums of a
  // column are added in shared memory in a fixed order
  constexpr int RG = kLT / 32;
  __shared__ W wpart[RG][32];
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int k0 = col_cut(p, gi, G), k1 = col_cut(p, gi + 1, G);
  // the new row's entry and the coefficient update for column k
  auto finish = [&](int k, const W& sum) {
    const W wk = scale(sum, -invd);
    B[pidx(p) + k] = wk;
    const W xk = fmacv(x[k], wk, zeta);
    x[k] = xk;
    const E e = from_w<E>(xk);
    xw[k] = e;
    if (xz) xz[lam[k]] = e;
  };
  if (k1 - k0 >= 32 * RG) {
    // wide block: strips of 32 columns over the lanes (one contiguous segment
    // of each row), every 8th row per warp, the 8 partial sums of a column
    // added in shared memory in a fixed order
    for (int kw = k0; kw < k1; kw += 32) {
      const int k = kw + lane;
      W acc = W{};
      if (k < k1)
        for (int i = kw + rg; i < p; i += RG)
          if (i >= k) acc = fmacv(acc, u[i], B[pidx(i) + k]);
      wpart[rg][lane] = acc;
      __syncthreads();
      if (rg == 0 && k < k1) {
        W sum = wpart[0][lane];
        for (int r = 1; r < RG; ++r) sum = add(sum, wpart[r][lane]);
        finish(k, sum);
      }
      __syncthreads();
    }
  } else {
    // narrow block (a few long columns): one column per warp, the lanes over
    // its rows, so that no FP64 lane idles (a masked FP64 lane costs as much
    // as an active one)
    for (int k = k0 + rg; k < k1; k += RG) {
      W acc = W{}, acc2 = W{};
      int i = k + lane;
      for (; i + 32 < p; i += 64) {
        acc = fmacv(acc, u[i], B[pidx(i) + k]);
        acc2 = fmacv(acc2, u[i + 32], B[pidx(i + 32) + k]);
      }
      if (i < p) acc = fmacv(acc, u[i], B[pidx(i) + k]);
      acc = add(acc, acc2);
      const double sr = warp_sum(re(acc));
      const double si = FT<E>::C ? warp_sum(im(acc)) : 0.0;
      if (lane == 0) finish(k, make_w<W>(sr, si));
    }
  }
  if (gi == 0 && threadIdx.x == 0) {
    B[pidx(p) + p] = make_w<W>(invd, 0.0);
    a.z[b * K + p] = zeta;
    const W xp = scale(zeta, invd);
    x[p] = xp;
    const E e = from_w<E>(xp);
    xw[p] = e;
    if (xz) xz[l] = e;
    a.lam[b * K + p] = l;
    a.bits[b * (int64_t)(N >> 5) + (l >> 5)] |= 1u << (l & 31);
    if (a.colmap) {  // register l's column (append order within a column)
      const int n2 = a.P.n2, i2 = l & ((1 << n2) - 1);
      int* cm = a.colmap + (b << n2);
      int c = cm[i2];
      if (c < 0 && S->ncols < a.kc) {
        c = S->ncols;
        S->ncols = c + 1;
        cm[i2] = c;
        a.cols[b * a.kc + c] = i2;
        a.chead[b * a.kc + c] = p;
      } else if (c >= 0) {
        a.cnext[b * K + a.ctail[b * a.kc + c]] = p;
      }
      if (c >= 0) a.ctail[b * a.kc + c] = p;
      a.cnext[b * K + p] = -1;
    }
  }
  // the last CTA of this instance to get here applies step 8
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    ticket = atomicAdd(&S->pad0, 1);
  }
  __syncthreads();
  if (ticket != G - 1) return;
  __threadfence();
  // step 8; in FP32 mode a downdate near the tolerance leaves the decision to
  // lchk_kernel, which forms the explicit residual
  const bool chk = resid_check<E>(a.rel_tol) && rn2 < kResidTrigger * ynorm2;
  if (!chk && (p + 1 >= K || rn2 < a.rel_tol * a.rel_tol * ynorm2)) {
    lwrite_outputs(a, b, p + 1, ynorm2, rn2);
  } else if (threadIdx.x == 0) {
    S->p = p + 1;
    S->rn2 = rn2;
    S->chk = chk ? 1 : 0;
  }
  if (threadIdx.x == 0) S->pad0 = 0;
}

// The halting test on the explicit residual (FP32 mode), one CTA per
// instance after the SK_RESN pass: ||r||^2 from the pass's nparts shares in a
// fixed order; stop when ||r|| < rel_tol ||y|| or K columns are in, else
// continue from the explicit value.
template <class E>
__global__ void __launch_bounds__(kLT) lchk_kernel(LOmpArgs<E> a, const double* __restrict__ rpart, int nparts) {
  __shared__ double red[kLT / 32];
  const int64_t b = blockIdx.y;
  LState* S = a.st + b;
  if (S->done || !S->chk) return;
  double t = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kLT) t += rpart[b * nparts + i];
  t = block_sum0(t, red);
  __syncthreads();
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  const double r2 = red[0], ynorm2 = S->ynorm2;
  const int p = S->p;
  __syncthreads();  // every thread has read the state
  if (p >= a.K || r2 < a.rel_tol * a.rel_tol * ynorm2) {
    lwrite_outputs(a, b, p, ynorm2, r2);
  } else if (threadIdx.x == 0) {
    S->rn2 = r2;
    S->chk = 0;
  }
}

// grid (G, batch); dynamic smem: K FP64 elements (the Gram column g)
template <class E>
__global__ void __launch_bounds__(kLT) lls_u_kernel(LOmpArgs<E> a, int nparts) {
  extern __shared__ __align__(16) unsigned char sm[];
  ls_u_phase(a, nparts, (int)gridDim.x, (int)blockIdx.x, (int64_t)blockIdx.y, (typename FT<E>::W*)sm);
}

// grid (G, batch), same G as the lls_u_kernel launch before it
template <class E>
__global__ void __launch_bounds__(kLT) lls_w_kernel(LOmpArgs<E> a) {
  ls_w_phase(a, (int)gridDim.x, (int)blockIdx.x, (int64_t)blockIdx.y);
}

// G = 1: both phases in one launch (one CTA per instance)
template <class E>
__global__ void __launch_bounds__(kLT) lls_one_kernel(LOmpArgs<E> a, int nparts) {
  extern __shared__ __align__(16) unsigned char sm[];
  if (!ls_u_phase(a, nparts, 1, 0, (int64_t)blockIdx.y, (typename FT<E>::W*)sm)) return;
  __syncthreads();  // u, the shares and the state written by phase u are visible to the whole CTA
  ls_w_phase(a, 1, 0, (int64_t)blockIdx.y);
}

// CTAs per instance for the least squares at p columns: about 2048 complex
// FP64 multiply-adds each (a few microseconds of one SM's FP64 pipe), at most
// gmax
inline int ls_ctas(int p, int gmax) {
  const int64_t work = (int64_t)p * (p + 1) / 2;
  int64_t g = (work + 2047) / 2048;
  if (g < 1) g = 1;
  return (int)(g < gmax ? g : gmax);
}


// ------------------------------------------------------------- launchers
template <class K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  return raise_smem_limit((const void*)kernel, bytes);
}

// Pass tiles of more than 48 KB (N >= 2^21 complex64): ask for a shared-
// memory carve-out of two CTAs per SM instead of three, which leaves the L1
// cache room for the twiddle tables every element reads (measured at
// N = 2^22: h_0 125 -> 115 us, an OMP iteration by transforms 5 % faster);
// smaller tiles keep the CUDA default.  The attribute is set only when it changes,
// so calls captured into a device-side loop make no runtime call.
template <class K>
cudaError_t pass_carveout(K kernel, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> cur;  // (device, kernel) -> carve-out set
  const int want = smem > 48 * 1024 ? 66 : (int)cudaSharedmemCarveoutDefault;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cur.find(std::make_pair(dev, (const void*)kernel));
  if (it == cur.end()) it = cur.emplace(std::make_pair(dev, (const void*)kernel), (int)cudaSharedmemCarveoutDefault).first;
  int& c = it->second;
  if (c == want) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, want);
  if (e == cudaSuccess) c = want;
  return e;
}

template <class E, bool DFT, int LD>
cudaError_t run_col(const LDev<E>& P, const E* in, int64_t in_stride, E* out, const LState* st, int64_t batch,
                    cudaStream_t s) {
  const size_t smem = pass_layout<E>(1 << P.n1).total;
  cudaError_t e = allow_smem(lcol_kernel<E, DFT, LD>, smem);
  if (e == cudaSuccess) e = pass_carveout(lcol_kernel<E, DFT, LD>, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((1u << P.n2) / tile_c<E>(), (unsigned)batch);
  lcol_kernel<E, DFT, LD><<<grid, kLT, smem, s>>>(P, in, in_stride, out, st);
  return cudaGetLastError();
}

template <class E, bool DFT, int SK>
cudaError_t run_row(const LDev<E>& P, const E* T, int neg, double scl, E* out, const E* y, const uint32_t* bits,
                    typename NormT<E>::V* pv, int* pj, int nparts, const LState* st, int64_t batch,
                    cudaStream_t s, LSparse<E> sp = LSparse<E>{nullptr, nullptr, 0}, double* rpart = nullptr) {
  const size_t smem = pass_layout<E>(1 << P.n2).total;
  cudaError_t e = allow_smem(lrow_kernel<E, DFT, SK>, smem);
  if (e == cudaSuccess) e = pass_carveout(lrow_kernel<E, DFT, SK>, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((1u << P.n1) / tile_c<E>(), (unsigned)batch);
  lrow_kernel<E, DFT, SK><<<grid, kLT, smem, s>>>(P, T, neg, (typename FT<E>::R)scl, out, y, bits, pv, pj,
                                                  nparts, st, sp, rpart);
  return cudaGetLastError();
}

// Outputs per thread of the kernel sums: the most (up to 8) that still give
// about two CTAs per SM over the batch (small N needs small tiles to use the
// GPU; large N needs several outputs per thread to keep loads in flight).
inline int fast_ch(int N, int64_t batch) {
  for (int ch = kFastMaxCH; ch > 1; ch >>= 1)
    if ((int64_t)(N / (kLT * ch)) * batch >= 2 * 152) return ch;
  return 1;
}

template <class E, bool DFT, int CF, int CH>
cudaError_t run_fast_t(const LDev<E>& P, const E* h0, const int* lam, const E* xw, int s, int64_t kstride,
                       const uint32_t* bits, E* h, typename NormT<E>::V* pv, int* pj, int nparts, const LState* st,
                       int64_t batch, size_t smem, cudaStream_t strm) {
  const cudaError_t e = allow_smem(lfast_kernel<E, DFT, CF, CH>, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(P.N / (kLT * CH), (unsigned)batch);
  lfast_kernel<E, DFT, CF, CH><<<grid, kLT, smem, strm>>>(P, h0, lam, xw, s, kstride, bits, h, pv, pj, nparts, st);
  return cudaGetLastError();
}

template <class E, bool DFT, int CF>
cudaError_t run_fast_cf(const LDev<E>& P, const E* h0, const int* lam, const E* xw, int s, int64_t kstride,
                        const uint32_t* bits, E* h, typename NormT<E>::V* pv, int* pj, int nparts, const LState* st,
                        int64_t batch, size_t smem, int ch, cudaStream_t strm) {
  switch (ch) {
    case 8: return run_fast_t<E, DFT, CF, 8>(P, h0, lam, xw, s, kstride, bits, h, pv, pj, nparts, st, batch, smem, strm);
    case 4: return run_fast_t<E, DFT, CF, 4>(P, h0, lam, xw, s, kstride, bits, h, pv, pj, nparts, st, batch, smem, strm);
    case 2: return run_fast_t<E, DFT, CF, 2>(P, h0, lam, xw, s, kstride, bits, h, pv, pj, nparts, st, batch, smem, strm);
    default: return run_fast_t<E, DFT, CF, 1>(P, h0, lam, xw, s, kstride, bits, h, pv, pj, nparts, st, batch, smem, strm);
  }
}

// Launches the kernel sums; *np receives the number of arg-max partials per
// instance (one per CTA).
template <class E, bool DFT>
cudaError_t run_fast(const LDev<E>& P, const E* h0, const int* lam, const E* xw, int s, int64_t kstride,
                     const uint32_t* bits, E* h, typename NormT<E>::V* pv, int* pj, int nparts, const LState* st,
                     int64_t batch, cudaStream_t strm, int* np = nullptr) {
  using V = typename NormT<E>::V;
  const size_t smem = al16((size_t)s * sizeof(E)) + al16((size_t)s * sizeof(int)) + al16(34 * sizeof(V)) +
                      34 * sizeof(int);
  const int ch = fast_ch(P.N, batch);
  if (np) *np = P.N / (kLT * ch);
  if (DFT && P.cfmt == CFMT_HALF)
    return run_fast_cf<E, DFT, CFMT_HALF>(P, h0, lam, xw, s, kstride, bits, h, pv, pj, nparts, st, batch, smem, ch,
                                          strm);
  if (!DFT && P.cfmt == CFMT_INT)
    return run_fast_cf<E, DFT, CFMT_INT>(P, h0, lam, xw, s, kstride, bits, h, pv, pj, nparts, st, batch, smem, ch,
                                         strm);
  return run_fast_cf<E, DFT, CFMT_FULL>(P, h0, lam, xw, s, kstride, bits, h, pv, pj, nparts, st, batch, smem, ch,
                                        strm);
}

template <class E>
int row_parts(const LDev<E>& P) { return (1 << P.n1) / tile_c<E>(); }
// arg-max partials per instance the kernel sums can leave (one per CTA, at
// the smallest tile)
template <class E>
int fast_parts(const LDev<E>& P) { return P.N / kLT; }

inline double inv_sqrt_n(int logN) { return 1.0 / std::sqrt(std::ldexp(1.0, logN)); }

// ------------------------------------------------ standalone correlations
template <class E>
size_t corr_ws_t(const PlanView& Pv, int64_t batch) {
  using V = typename NormT<E>::V;
  const LDev<E> P = ldev<E>(Pv);
  const int np = row_parts(P);
  return al16((size_t)batch * P.N * sizeof(E)) + al16((size_t)batch * np * sizeof(V)) +
         al16((size_t)batch * np * sizeof(int));
}

template <class E>
cudaError_t corr_t(const PlanView& Pv, const void* r, int64_t batch, void* h, int32_t* amax, void* ws,
                   cudaStream_t s) {
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  const LDev<E> P = ldev<E>(Pv);
  const int np = row_parts(P);
  unsigned char* w = (unsigned char*)ws;
  E* T = (E*)w;
  V* pv = (V*)(w + al16((size_t)batch * P.N * sizeof(E)));
  int* pj = (int*)((unsigned char*)pv + al16((size_t)batch * np * sizeof(V)));
  cudaError_t e = run_col<E, DFT, LD_ZF>(P, (const E*)r, P.M, T, nullptr, batch, s);
  if (e != cudaSuccess) return e;
  e = run_row<E, DFT, SK_H>(P, T, DFT, inv_sqrt_n(P.logN), (E*)h, nullptr, nullptr, amax ? pv : nullptr,
                            amax ? pj : nullptr, np, nullptr, batch, s);
  if (e != cudaSuccess || !amax) return e;
  lreduce_kernel<V><<<(unsigned)batch, kLT, 0, s>>>(pv, pj, np, np, amax);
  return cudaGetLastError();
}

template <class E>
size_t fast_ws_t(const PlanView& Pv, int64_t batch) {
  using V = typename NormT<E>::V;
  const LDev<E> P = ldev<E>(Pv);
  const int np = fast_parts(P);
  return al16((size_t)batch * (P.N >> 5) * sizeof(uint32_t)) + al16((size_t)batch * np * sizeof(V)) +
         al16((size_t)batch * np * sizeof(int));
}

template <class E>
cudaError_t fast_t(const PlanView& Pv, const void* h0, const int32_t* supp, const void* x, int s, int64_t batch,
                   void* h, int32_t* amax, void* ws, cudaStream_t st) {
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  const LDev<E> P = ldev<E>(Pv);
  const int np = fast_parts(P);
  unsigned char* w = (unsigned char*)ws;
  uint32_t* bits = (uint32_t*)w;
  V* pv = (V*)(w + al16((size_t)batch * (P.N >> 5) * sizeof(uint32_t)));
  int* pj = (int*)((unsigned char*)pv + al16((size_t)batch * np * sizeof(V)));
  cudaError_t e = cudaMemsetAsync(bits, 0, (size_t)batch * (P.N >> 5) * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (s > 0) {
    lbits_kernel<<<(unsigned)batch, kLT, 0, st>>>(supp, s, P.N, bits);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  int used = np;
  e = run_fast<E, DFT>(P, (const E*)h0, supp, (const E*)x, s, s, bits, (E*)h, amax ? pv : nullptr,
                       amax ? pj : nullptr, np, nullptr, batch, st, &used);
  if (e != cudaSuccess || !amax) return e;
  lreduce_kernel<V><<<(unsigned)batch, kLT, 0, st>>>(pv, pj, np, used, amax);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- OMP
template <class E>
struct LOmpWs {
  size_t st, h0, T, Z, xz, bits, B, z, x, u, xw, lam, pv, pj, yp, tm, cm, cl, ch, ct, cn, Tc, rp, total;
  int nparts, nyp, gmax, kc;
};

template <class E>
LOmpWs<E> lomp_ws(const PlanView& Pv, int K, int path, int64_t batch) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  const LDev<E> P = ldev<E>(Pv);
  const bool conv = path != 0;  // CS_PATH_FAST == 0
  LOmpWs<E> L;
  const int rp = row_parts(P), fp = fast_parts(P);
  L.nparts = rp > fp ? rp : fp;
  const size_t Nv = (size_t)batch * P.N * sizeof(E);
  const size_t Kc = (size_t)(K > 0 ? K : 1);
  size_t o = 0;
  L.st = o;   o = al16(o + (size_t)batch * sizeof(LState));
  L.h0 = o;   o = al16(o + Nv);
  L.T = o;    o = al16(o + Nv);
  L.Z = o;    o = al16(o + (conv ? (size_t)batch * P.M * sizeof(E) : 0));  // the residual on Omega
  L.xz = o;
  L.bits = o; o = al16(o + (size_t)batch * (P.N >> 5) * sizeof(uint32_t));
  L.B = o;    o = al16(o + (size_t)batch * ((Kc * (Kc + 1)) / 2) * sizeof(W));
  L.z = o;    o = al16(o + (size_t)batch * Kc * sizeof(W));
  L.x = o;    o = al16(o + (size_t)batch * Kc * sizeof(W));
  L.u = o;    o = al16(o + (size_t)batch * Kc * sizeof(W));
  L.xw = o;   o = al16(o + (size_t)batch * Kc * sizeof(E));
  L.lam = o;  o = al16(o + (size_t)batch * Kc * sizeof(int));
  L.pv = o;   o = al16(o + (size_t)batch * L.nparts * sizeof(V));
  L.pj = o;   o = al16(o + (size_t)batch * L.nparts * sizeof(int));
  {  // CTAs of the ||y||^2 kernel: about 2048 entries each (its FP64 work spreads over the SMs)
    const int64_t g = ((int64_t)P.M + 2047) / 2048;
    L.nyp = (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g));
  }
  L.yp = o;   o = al16(o + (size_t)batch * L.nyp * sizeof(double));
  {  // CTAs per instance for the least squares: about two per SM over the
     // batch (more only adds per-CTA overhead, and concurrent calls from the
     // request runtime share the GPU)
    int64_t g = (2 * 152 + batch - 1) / batch;
    L.gmax = (int)(g < 1 ? 1 : (g > 256 ? 256 : g));
  }
  L.tm = o;   o = al16(o + (size_t)batch * L.gmax * 3 * sizeof(double));
  // the sparse pass 1 of the transform path (and of the explicit residual
  // of FP32 mode): registered support columns, kc = min(K, N2) of them (a
  // support never spans more than N2 columns)
  const bool fp32 = sizeof(typename FT<E>::R) == 4;
  L.kc = (conv || fp32) ? (K < (1 << P.n2) ? K : (1 << P.n2)) : 0;
  const size_t kcs = (size_t)L.kc;
  L.cm = o;   o = al16(o + (kcs ? (size_t)batch * ((size_t)1 << P.n2) * sizeof(int) : 0));
  L.cl = o;   o = al16(o + (size_t)batch * kcs * sizeof(int));
  L.ch = o;   o = al16(o + (size_t)batch * kcs * sizeof(int));
  L.ct = o;   o = al16(o + (size_t)batch * kcs * sizeof(int));
  L.cn = o;   o = al16(o + (kcs ? (size_t)batch * Kc * sizeof(int) : 0));
  L.Tc = o;   o = al16(o + (size_t)batch * ((size_t)1 << P.n1) * kcs * sizeof(E));
  L.rp = o;   o = al16(o + (fp32 ? (size_t)batch * row_parts(P) * sizeof(double) : 0));  // SK_RESN shares
  L.total = o;
  return L;
}

template <class E>
cudaError_t omp_t(const PlanView& Pv, const OmpLaunch& a, void* ws, cudaStream_t s) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  constexpr bool DFT = FT<E>::C;
  const LDev<E> P = ldev<E>(Pv);
  const int64_t batch = a.batch;
  const LOmpWs<E> L = lomp_ws<E>(Pv, a.K, a.path, batch);
  unsigned char* w = (unsigned char*)ws;
  LOmpArgs<E> A;
  A.P = P;
  A.y = (const E*)a.y;
  A.K = a.K;
  A.rel_tol = a.rel_tol;
  A.x_out = (W*)a.x_out;
  A.supp_out = a.supp_out;
  A.iters_out = a.iters_out;
  A.res_out = a.res_out;
  A.st = (LState*)(w + L.st);
  A.h0 = (E*)(w + L.h0);
  E* T = (E*)(w + L.T);
  E* Z = a.path != 0 ? (E*)(w + L.Z) : nullptr;
  A.xz = nullptr;  // the transform path builds pass 1 from the support's columns
  A.bits = (uint32_t*)(w + L.bits);
  A.B = (W*)(w + L.B);
  A.z = (W*)(w + L.z);
  A.x = (W*)(w + L.x);
  A.xw = (E*)(w + L.xw);
  A.lam = (int*)(w + L.lam);
  A.u = (W*)(w + L.u);
  A.part_v = (V*)(w + L.pv);
  A.part_j = (int*)(w + L.pj);
  A.nparts = L.nparts;
  A.ypart = (double*)(w + L.yp);
  A.nyp = L.nyp;
  A.terms = (double*)(w + L.tm);
  A.gmax = L.gmax;
  A.kc = L.kc;
  A.colmap = L.kc ? (int*)(w + L.cm) : nullptr;
  A.cols = (int*)(w + L.cl);
  A.chead = (int*)(w + L.ch);
  A.ctail = (int*)(w + L.ct);
  A.cnext = (int*)(w + L.cn);
  E* Tc = (E*)(w + L.Tc);
  double* rpart = (double*)(w + L.rp);
  const bool chk_mode = resid_check<E>(a.rel_tol) && a.K > 0;
  cudaError_t e;
  if ((e = cudaMemsetAsync(A.st, 0, (size_t)batch * sizeof(LState), s)) != cudaSuccess) return e;
  if (A.colmap &&
      (e = cudaMemsetAsync(A.colmap, 0xff, (size_t)batch * ((size_t)1 << P.n2) * sizeof(int), s)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(A.bits, 0, (size_t)batch * (P.N >> 5) * sizeof(uint32_t), s)) != cudaSuccess) return e;
  const size_t ls_smem = (size_t)(a.K > 0 ? a.K : 1) * sizeof(W);
  if ((e = allow_smem(lls_one_kernel<E>, ls_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(lls_u_kernel<E>, ls_smem)) != cudaSuccess) return e;
  const double isq = inv_sqrt_n(P.logN);
  const int rp = row_parts(P);
  const int T_end = a.K > 0 ? a.K : 1;
  for (int t = 1; t <= T_end; ++t) {
    int np;
    if (t == 1) {  // h_0 = Phi^H y by one transform (Eq. kernelsumOMP, first case)
      lynorm_kernel<E><<<dim3((unsigned)L.nyp, (unsigned)batch), kLT, 0, s>>>(A.y, P.M, A.ypart, L.nyp);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = run_col<E, DFT, LD_ZF>(P, A.y, P.M, T, A.st, batch, s)) != cudaSuccess) return e;
      if ((e = run_row<E, DFT, SK_H>(P, T, DFT, isq, A.h0, nullptr, nullptr, A.part_v, A.part_j, L.nparts, A.st,
                                     batch, s)) != cudaSuccess)
        return e;
      np = rp;
    } else if (a.path == 0 || (a.path == 2 && t <= a.t_switch)) {  // kernel sums over t - 1 atoms
      if ((e = run_fast<E, DFT>(P, A.h0, A.lam, A.xw, t - 1, a.K, A.bits, nullptr, A.part_v, A.part_j, L.nparts,
                                A.st, batch, s, &np)) != cudaSuccess)
        return e;
    } else {  // r = y - Phi x by a forward transform of zf(x), then h = A^H zf(r):
              // pass 1 from the support's columns, pass 2 from the compact result
      const int N1 = 1 << P.n1, kcl = (t - 1) < L.kc ? (t - 1) : L.kc;
      const dim3 g1((unsigned)(((int64_t)N1 * kcl + kLT - 1) / kLT), (unsigned)batch);
      lsp1_kernel<E, DFT><<<g1, kLT, 0, s>>>(P, A.xw, A.lam, A.chead, A.cnext, a.K, L.kc, kcl, Tc, A.st, 0);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = run_row<E, DFT, SK_RES>(P, nullptr, 0, isq, Z, A.y, nullptr, nullptr, nullptr, 0, A.st, batch, s,
                                       LSparse<E>{Tc, A.cols, L.kc})) != cudaSuccess)
        return e;
      if ((e = run_col<E, DFT, LD_ZF>(P, Z, P.M, T, A.st, batch, s)) != cudaSuccess) return e;
      if ((e = run_row<E, DFT, SK_ARG>(P, T, DFT, isq, nullptr, nullptr, A.bits, A.part_v, A.part_j, L.nparts,
                                       A.st, batch, s)) != cudaSuccess)
        return e;
      np = rp;
    }
    const dim3 lg((unsigned)ls_ctas(t - 1, L.gmax), (unsigned)batch);
    if (lg.x == 1) {
      lls_one_kernel<E><<<lg, kLT, ls_smem, s>>>(A, np);
    } else {
      lls_u_kernel<E><<<lg, kLT, ls_smem, s>>>(A, np);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      lls_w_kernel<E><<<lg, kLT, 0, s>>>(A);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (chk_mode) {  // the explicit residual of instances whose downdate neared the tolerance
      const int N1 = 1 << P.n1, kcl = t < L.kc ? t : L.kc;
      const dim3 g1((unsigned)(((int64_t)N1 * kcl + kLT - 1) / kLT), (unsigned)batch);
      lsp1_kernel<E, DFT><<<g1, kLT, 0, s>>>(P, A.xw, A.lam, A.chead, A.cnext, a.K, L.kc, kcl, Tc, A.st, 1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = run_row<E, DFT, SK_RESN>(P, nullptr, 0, isq, nullptr, A.y, nullptr, nullptr, nullptr, 0, A.st, batch,
                                        s, LSparse<E>{Tc, A.cols, L.kc}, rpart)) != cudaSuccess)
        return e;
      lchk_kernel<E><<<dim3(1, (unsigned)batch), kLT, 0, s>>>(A, rpart, rp);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <class W>
cudaError_t kv_t(const PlanView& Pv, void* c64, void* tmp, cudaStream_t s) {
  constexpr bool DFT = FT<W>::C;
  const LDev<W> P = ldev<W>(Pv);
  cudaError_t e = run_col<W, DFT, LD_ONES>(P, nullptr, 0, (W*)tmp, nullptr, 1, s);
  if (e != cudaSuccess) return e;
  // c = N^{-1} A^H 1_Omega scaled as in Eq. (kernelsum): N^{-1} F^H zf(1)
  return run_row<W, DFT, SK_KV>(P, (const W*)tmp, DFT, std::ldexp(1.0, -P.logN), (W*)c64, nullptr, nullptr,
                                nullptr, nullptr, 0, nullptr, 1, s);
}

// ------------------------------------------------------ SP and CoSaMP
// The pursuits of cs_pursuit.cu on large plans.  Per iteration the host
// queues: the correlation h over all N (kernel sums over the current support,
// padded with zero coefficients, or the four-step passes of the residual),
// the top-k selection (each tile of kLT * 8 outputs keeps its own top k, then
// one CTA per instance takes the top k of the tiles' candidates: a tile's
// (k+1)-th best can never be in the overall top k, and candidates are kept in
// ascending j, so ties still go to the lower index), and the step: least
// squares on the candidate set, pruning and the stop rules, one CTA per
// instance, as in the one-CTA kernel.
constexpr int kSelTile = kLT * 8;  // outputs per tile of the first stage, at least
// Outputs per tile: at least 8 times the candidates a tile keeps, so that the
// second stage (one CTA per instance) sees at most N/8 candidates.
__host__ __device__ inline int lp_tile(int N, int kmax) {
  int t = kSelTile;
  while (t < 8 * kmax && t < N) t <<= 1;
  return t < N ? t : N;
}

struct LPExtra {  // per instance, beside the LState done flag
  int ns, m, it, pad;
  double ynorm2, rn2, rn2_new, ls_rn2;
  // least squares by conjugate gradients (large K): the set Tq[0..mq), the
  // next solver call's mode (0 none, 1 solve, 2 quadratic form), whether xq
  // holds a start, the solver's iterations so far, the quadratic form
  int mq, cgmode, warm, cgit;
  double qf;
};

template <class E>
struct LPArgs {
  using W = typename FT<E>::W;
  using U = typename KeyT<E>::U;
  LDev<E> P;
  const E* __restrict__ y;
  int K, algo, max_iter;
  double rel_tol;
  W* x_out;
  int* supp_out;
  int* iters_out;
  double* res_out;
  E* h0;            // [batch][N]
  E* xz;            // [batch][N] zero-filled x (transform path) or NULL
  uint32_t* bits;   // [batch][N/32] the support (subspace pursuit excludes it)
  int* S;           // [batch][K] support, ascending, 0 past ns
  W* xs;            // [batch][K] coefficients
  E* xsw;           // [batch][K] coefficients in the working precision, 0 past ns
  U* ckey;          // [batch][ntiles][kmax] tile candidates
  int* cj;
  int ntiles, kmax, tile;  // tile: outputs per first-stage tile (lp_tile)
  int* sel;         // [batch][kmax] selection, ascending
  W* B;             // [batch][mm(mm+1)/2]
  LState* st;       // done flags
  LPExtra* ex;
  double* ypart;
  int nyp;
  // conjugate-gradient least squares (lq != 0): column set, right-hand side
  // h_0(T) and solution / start, [batch][mm] each
  int lq;
  int* Tq;
  W* rq;
  W* xq;
  int cg_max;
  double cg_tol;
  // FP32 plans: h_0 = Phi^H y once more in FP64 ([batch][N]), the right-hand
  // sides of the least squares (NULL: h0 is already FP64)
  const W* h64;
  int* ndone;  // instances finished so far (the device-side loop stops at batch)
};

// (Phi^H y)(j) in FP64 for the least squares
template <class E>
__device__ __forceinline__ typename FT<E>::W lp_rhs(const LPArgs<E>& a, int64_t b, int j) {
  return a.h64 ? a.h64[b * (int64_t)a.P.N + j] : to_w(a.h0[b * (int64_t)a.P.N + j]);
}

__host__ __device__ inline int lp_mmax(int K, int algo) { return algo == 0 ? 2 * K : 3 * K; }

// Each tile's top-k of |src(j)|^2 over j (excluding the support when excl).
template <class E>
__global__ void __launch_bounds__(kLT) lp_tile_kernel(LPArgs<E> a, const E* __restrict__ src, int k, int excl) {
  using U = typename KeyT<E>::U;
  using V = typename NormT<E>::V;
  extern __shared__ __align__(16) unsigned char sm[];
  U* keys = (U*)sm;
  const int tile = a.tile;
  int* out = (int*)(sm + al16((size_t)tile * sizeof(U)));
  int* hist = out + al16((size_t)k * sizeof(int)) / sizeof(int);
  int* scr = hist + 260;
  const int64_t b = blockIdx.y;
  if (a.st[b].done) return;
  const int N = a.P.N, j0 = blockIdx.x * tile;
  const E* hb = src + b * (int64_t)N;
  const uint32_t* bb = a.bits + b * (int64_t)(N >> 5);
  for (int i = threadIdx.x; i < tile; i += kLT) {
    const int j = j0 + i;
    keys[i] = (excl && in_bits(bb, j)) ? (U)0 : sel_key((V)norm2(hb[j]));
  }
  const Grp g = whole_block();
  g.sync();
  group_topk(g, keys, tile, k, out, hist, scr);
  U* ck = a.ckey + (b * a.ntiles + blockIdx.x) * (int64_t)a.kmax;
  int* cjj = a.cj + (b * a.ntiles + blockIdx.x) * (int64_t)a.kmax;
  for (int i = threadIdx.x; i < k; i += kLT) {
    ck[i] = keys[out[i]];
    cjj[i] = j0 + out[i];
  }
}

// The overall top-k of the tiles' candidates (tile-major, j ascending within
// a tile, so candidate order is j order) -> sel, ascending.
template <class E>
__global__ void __launch_bounds__(kLT) lp_merge_kernel(LPArgs<E> a, int k) {
  extern __shared__ __align__(16) unsigned char sm[];
  int* out = (int*)sm;
  int* hist = out + al16((size_t)k * sizeof(int)) / sizeof(int);
  int* scr = hist + 260;
  const int64_t b = blockIdx.x;
  if (a.st[b].done) return;
  const Grp g = whole_block();
  // k == kmax: the tiles' candidates are contiguous
  const int n = a.ntiles * k;
  const typename KeyT<E>::U* keys = a.ckey + b * (int64_t)a.ntiles * a.kmax;
  const int* cjb = a.cj + b * (int64_t)a.ntiles * a.kmax;
  group_topk(g, keys, n, k, out, hist, scr);
  for (int i = threadIdx.x; i < k; i += kLT) a.sel[b * (int64_t)a.kmax + i] = cjb[out[i]];
}

template <class E>
struct LPLayout {
  size_t z, x, g, part, lam, sk, T, sel2, hist, scr, red, total;
  int npart;
};

template <class E>
__host__ __device__ inline LPLayout<E> lp_layout(int K, int algo) {
  using W = typename FT<E>::W;
  LPLayout<E> L;
  const int mm = lp_mmax(K, algo);
  L.npart = 2 * kLT > mm ? 2 * kLT : mm;
  size_t o = 0;
  L.z = o;    o = al16(o + (size_t)mm * sizeof(W));
  L.x = o;    o = al16(o + (size_t)mm * sizeof(W));
  L.g = o;    o = al16(o + (size_t)mm * sizeof(W));
  L.part = o; o = al16(o + (size_t)L.npart * sizeof(W) + (size_t)3 * mm * sizeof(double));
  L.lam = o;  o = al16(o + (size_t)mm * sizeof(int));
  L.sk = o;   o = al16(o + (size_t)mm * sizeof(unsigned long long));
  L.T = o;    o = al16(o + (size_t)mm * sizeof(int));
  L.sel2 = o; o = al16(o + (size_t)mm * sizeof(int));
  L.hist = o; o = al16(o + 260 * sizeof(int));
  L.scr = o;  o = al16(o + 34 * sizeof(int));
  L.red = o;  o = al16(o + (32 * 2 + 2) * sizeof(double));
  L.total = o;
  return L;
}

template <class E>
__device__ void lp_outputs(const LPArgs<E>& a, int64_t b, const LPExtra& X) {
  using W = typename FT<E>::W;
  const int K = a.K, ns = X.ns;
  for (int k = threadIdx.x; k < K; k += kLT) {
    if (a.x_out) a.x_out[b * K + k] = k < ns ? a.xs[b * K + k] : W{};
    a.supp_out[b * K + k] = k < ns ? a.S[b * K + k] : -1;
  }
  if (threadIdx.x == 0) {
    if (a.iters_out) a.iters_out[b] = X.it;
    if (a.res_out) a.res_out[b] = X.ynorm2 > 0.0 ? sqrt(fmax(X.rn2, 0.0) / X.ynorm2) : 0.0;
    a.st[b].done = 1;
    atomicAdd(a.ndone, 1);
  }
}

// phase 0: ||y||^2, SP's first support (sel) and its least squares; phase 1:
// one iteration's candidate set (sel with the support), least squares,
// pruning and the stop rules.
template <class E>
__global__ void __launch_bounds__(kLT) lp_step_kernel(LPArgs<E> a, int phase) {
  using W = typename FT<E>::W;
  constexpr bool DFT = FT<E>::C;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ LPExtra X;
  __shared__ LsShared<W> sh;
  const int64_t b = blockIdx.x;
  if (a.st[b].done) return;
  const int N = a.P.N, K = a.K, mm = lp_mmax(K, a.algo);
  const LPLayout<E> L = lp_layout<E>(K, a.algo);
  const Grp g = whole_block();
  LsView<E> lv;
  lv.B = a.B + b * (((int64_t)mm * (mm + 1)) >> 1);
  lv.z = (W*)(sm + L.z);
  lv.x = (W*)(sm + L.x);
  lv.g = (W*)(sm + L.g);
  lv.part = (W*)(sm + L.part);
  lv.terms = (double*)(lv.part + L.npart);
  lv.xw = nullptr;
  lv.lam = (int*)(sm + L.lam);
  lv.bits = nullptr;
  lv.kidx = nullptr;
  unsigned long long* sk = (unsigned long long*)(sm + L.sk);
  int* T = (int*)(sm + L.T);
  int* sel2 = (int*)(sm + L.sel2);
  int* hist = (int*)(sm + L.hist);
  int* scr = (int*)(sm + L.scr);
  double* red = (double*)(sm + L.red);
  PlanDev<E> pd;
  pd.N = N;
  pd.logN = a.P.logN;
  pd.M = a.P.M;
  pd.slot = a.P.slot;
  pd.tw = nullptr;
  pd.c = a.P.c;
  pd.c64 = a.P.c64;
  pd.cfmt = a.P.cfmt;
  pd.ci = a.P.ci;
  const E* h0 = a.h0 + b * (int64_t)N;
  int* S = a.S + b * K;
  W* xs = a.xs + b * K;
  E* xsw = a.xsw + b * K;
  uint32_t* bb = a.bits + b * (int64_t)(N >> 5);
  E* xz = a.xz ? a.xz + b * (int64_t)N : nullptr;
  const int* sel = a.sel + b * (int64_t)a.kmax;
  if (threadIdx.x == 0) X = a.ex[b];
  g.sync();
  const double tol2 = a.rel_tol * a.rel_tol;

  // least squares on cols[0..m): append them to an empty factor
  auto ls_set = [&](const int* cols, int m) {
    if (threadIdx.x == 0) X.ls_rn2 = X.ynorm2;
    g.sync();
    int p = 0;
    for (int c = 0; c < m; ++c) {
      ls_append(g, pd, lv, h0, p, cols[c], X.ls_rn2, sh);
      if (sh.st == 0) ++p;
    }
    if (threadIdx.x == 0) X.m = p;
    g.sync();
  };
  // the accepted support and coefficients (ns entries, ascending columns)
  auto set_support = [&](const int* cols, const W* coef, int ns) {
    for (int k = threadIdx.x; k < X.ns; k += kLT) {  // the old support leaves bits and zf(x)
      const int j = S[k];
      if (xz) xz[j] = zero<E>();
      atomicAnd(bb + (j >> 5), ~(1u << (j & 31)));
    }
    g.sync();
    for (int k = threadIdx.x; k < K; k += kLT) {
      const int j = k < ns ? cols[k] : 0;
      const W v = k < ns ? coef[k] : W{};
      S[k] = j;
      xs[k] = v;
      xsw[k] = from_w<E>(v);
      if (k < ns) {
        if (xz) xz[j] = from_w<E>(v);
        atomicOr(bb + (j >> 5), 1u << (j & 31));
      }
    }
    g.sync();
    if (threadIdx.x == 0) X.ns = ns;
    g.sync();
  };

  bool stop = false;
  if (phase == 0) {
    double t = 0.0;
    for (int i = threadIdx.x; i < a.nyp; i += kLT) t += a.ypart[b * a.nyp + i];
    double tt[1] = {t};
    group_sum(g, tt, red);
    if (threadIdx.x == 0) {
      X.ynorm2 = tt[0];
      X.rn2 = tt[0];
      X.ns = 0;
      X.it = 0;
    }
    g.sync();
    if (!(X.ynorm2 > 0.0) || K == 0) {
      stop = true;
    } else if (a.algo == 0) {  // SP: T_0 = top_K(h_0), x = LS on T_0
      for (int i = threadIdx.x; i < K; i += kLT) T[i] = sel[i];
      g.sync();
      ls_set(T, K);
      for (int k = threadIdx.x; k < X.m; k += kLT) sel2[k] = lv.lam[k];
      g.sync();
      set_support(sel2, lv.x, X.m);
      if (threadIdx.x == 0) X.rn2 = X.ls_rn2;
      g.sync();
    }
  } else {
    const int ns = X.ns, kk = a.algo == 0 ? K : 2 * K;
    // T = support + selection (both ascending), without duplicates
    if (threadIdx.x == 0) {
      int i = 0, j = 0, o = 0;
      while (i < ns || j < kk) {
        int v;
        if (j >= kk || (i < ns && S[i] < sel[j])) v = S[i++];
        else if (i < ns && S[i] == sel[j]) { v = S[i++]; ++j; }
        else v = sel[j++];
        T[o++] = v;
      }
      X.m = o;
    }
    g.sync();
    ls_set(T, X.m);                         // b = LS on T (lv.lam, lv.x)
    const int m = X.m;
    for (int i = threadIdx.x; i < m; i += kLT) sk[i] = sel_key(norm2(lv.x[i]));
    g.sync();
    const int kp = K < m ? K : m;
    group_topk(g, sk, m, kp, sel2, hist, scr);  // prune: the K largest |b|, ascending positions
    for (int i = threadIdx.x; i < kp; i += kLT) T[i] = lv.lam[sel2[i]];
    if (a.algo == 1)
      for (int i = threadIdx.x; i < kp; i += kLT) lv.g[i] = lv.x[sel2[i]];
    g.sync();
    if (a.algo == 0) {
      // T_new equal to the accepted support (both ascending): the solve would
      // repeat the accepted one, so the iteration is rejected without it
      if (threadIdx.x == 0) {
        bool same = kp == X.ns;
        for (int i = 0; same && i < kp; ++i) same = T[i] == S[i];
        scr[0] = same;
      }
      g.sync();
      if (scr[0]) {
        if (threadIdx.x == 0) X.rn2_new = X.rn2;
        g.sync();
      } else {
        ls_set(T, kp);                        // x_new = LS on T_new
        if (threadIdx.x == 0) X.rn2_new = X.ls_rn2;
        g.sync();
      }
    } else {
      // ||y - Phi x||^2 = ||y||^2 - 2 Re x^H h_0(S) + x^H G_S x  (FP64)
      double acc[2] = {0.0, 0.0};
      for (int i = threadIdx.x; i < kp; i += kLT) {
        const W xi = lv.g[i];
        acc[0] += re(cmul(xi, to_w(h0[T[i]])));
        W gx = W{};
        for (int j = 0; j < kp; ++j) {
          const int d = DFT ? ((T[i] - T[j]) & (N - 1)) : (T[i] ^ T[j]);
          gx = fmav(gx, c64_at(pd, d), lv.g[j]);
        }
        acc[1] += re(cmul(xi, gx));
      }
      group_sum(g, acc, red);
      if (threadIdx.x == 0) {
        X.rn2_new = X.ynorm2 - 2.0 * acc[0] + acc[1];
        X.m = kp;
      }
      g.sync();
    }
    if (threadIdx.x == 0) X.it = X.it + 1;
    g.sync();
    if (!(X.rn2_new < X.rn2)) {
      stop = true;  // keep the previous iterate
    } else {
      if (a.algo == 0) {
        for (int k = threadIdx.x; k < X.m; k += kLT) sel2[k] = lv.lam[k];
        g.sync();
        set_support(sel2, lv.x, X.m);
      } else {
        set_support(T, lv.g, kp);
      }
      if (threadIdx.x == 0) X.rn2 = X.rn2_new;
      g.sync();
    }
  }
  if (!stop && (X.it >= a.max_iter || X.rn2 < tol2 * X.ynorm2)) stop = true;
  if (stop) lp_outputs(a, b, X);
  if (threadIdx.x == 0) a.ex[b] = X;
}

// ---------------------------------- SP and CoSaMP with large column sets
// The least squares of an iteration (on up to 2K or 3K columns) by the
// cluster conjugate-gradient solver of cs_cg.cuh instead of appending the
// columns one CTA at a time.  Per iteration the host queues, after the
// correlation and the top-k: lq_form (the set T and its right-hand side,
// the previous coefficients as the start), lq_cg (b = LS on T), lq_prune
// (the K largest |b|; SP: the second set T_new, CoSaMP: the pruned estimate),
// lq_cg again (SP: x_new = LS on T_new from b's values; CoSaMP: the
// quadratic form x^H G x of the pruned estimate) and lq_accept (the stop
// rules).  Same steps, order, tie rules and stop rules as lp_step_kernel.

// The accepted support and coefficients (ns entries, ascending columns).
template <class E>
__device__ void lp_set_support(const LPArgs<E>& a, int64_t b, LPExtra& X, const int* cols,
                               const typename FT<E>::W* coef, int ns) {
  using W = typename FT<E>::W;
  const int K = a.K;
  int* S = a.S + b * K;
  W* xs = a.xs + b * K;
  E* xsw = a.xsw + b * K;
  uint32_t* bb = a.bits + b * (int64_t)(a.P.N >> 5);
  E* xz = a.xz ? a.xz + b * (int64_t)a.P.N : nullptr;
  for (int k = threadIdx.x; k < X.ns; k += kLT) {  // the old support leaves bits and zf(x)
    const int j = S[k];
    if (xz) xz[j] = zero<E>();
    atomicAnd(bb + (j >> 5), ~(1u << (j & 31)));
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += kLT) {
    const int j = k < ns ? cols[k] : 0;
    const W v = k < ns ? coef[k] : W{};
    S[k] = j;
    xs[k] = v;
    xsw[k] = from_w<E>(v);
    if (k < ns) {
      if (xz) xz[j] = from_w<E>(v);
      atomicOr(bb + (j >> 5), 1u << (j & 31));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) X.ns = ns;
  __syncthreads();
}

// phase 0: ||y||^2 (and SP: T_0 = top_K(h_0) to solve); phase 1: T = the
// support joined with the selection (both ascending, no duplicates), the
// start = the support's coefficients, zero on the new columns.
template <class E>
__global__ void __launch_bounds__(kLT) lq_form_kernel(LPArgs<E> a, int phase) {
  using W = typename FT<E>::W;
  __shared__ LPExtra X;
  __shared__ double red[32 * 1 + 1];
  const int64_t b = blockIdx.x;
  if (a.st[b].done) return;
  const int K = a.K, mm = lp_mmax(K, a.algo);
  const Grp g = whole_block();
  if (threadIdx.x == 0) X = a.ex[b];
  __syncthreads();
  int* T = a.Tq + b * (int64_t)mm;
  W* rq = a.rq + b * (int64_t)mm;
  W* xq = a.xq + b * (int64_t)mm;
  const int* sel = a.sel + b * (int64_t)a.kmax;
  if (phase == 0) {
    double t = 0.0;
    for (int i = threadIdx.x; i < a.nyp; i += kLT) t += a.ypart[b * a.nyp + i];
    double tt[1] = {t};
    group_sum(g, tt, red);
    if (threadIdx.x == 0) {
      X.ynorm2 = tt[0];
      X.rn2 = tt[0];
      X.ns = 0;
      X.it = 0;
      X.cgmode = 0;
      X.cgit = 0;
    }
    __syncthreads();
    if (!(X.ynorm2 > 0.0) || K == 0) {
      lp_outputs(a, b, X);
    } else if (a.algo == 0) {
      for (int i = threadIdx.x; i < K; i += kLT) {
        T[i] = sel[i];
        rq[i] = lp_rhs(a, b, sel[i]);
      }
      if (threadIdx.x == 0) {
        X.mq = K;
        X.cgmode = 1;
        X.warm = 0;
      }
    }
  } else {
    const int ns = X.ns, kk = a.algo == 0 ? K : 2 * K;
    const int* S = a.S + b * K;
    const W* xs = a.xs + b * K;
    if (threadIdx.x == 0) {
      int i = 0, j = 0, o = 0;
      while (i < ns || j < kk) {
        if (j >= kk || (i < ns && S[i] < sel[j])) {
          T[o] = S[i];
          xq[o++] = xs[i++];
        } else if (i < ns && S[i] == sel[j]) {
          T[o] = S[i];
          xq[o++] = xs[i++];
          ++j;
        } else {
          T[o] = sel[j++];
          xq[o++] = W{};
        }
      }
      X.mq = o;
      X.cgmode = 1;
      X.warm = ns > 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < X.mq; i += kLT) rq[i] = lp_rhs(a, b, T[i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) a.ex[b] = X;
}

// One cluster of G CTAs per instance: the solve (mode 1) or the quadratic
// form (mode 2) of cs_cg.cuh on the instance's set.
template <class E, int G>
__global__ void __launch_bounds__(kLT) lq_cg_kernel(LPArgs<E> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  cgx::cluster_group cl = cgx::this_cluster();
  const int64_t b = blockIdx.x / G;
  // every CTA of the cluster reads the same flags: all leave or none
  if (a.st[b].done) return;
  const int mode = a.ex[b].cgmode;
  if (mode == 0) return;
  const int m = a.ex[b].mq, mm = lp_mmax(a.K, a.algo);
  PlanDev<E> pd;
  pd.N = a.P.N;
  pd.logN = a.P.logN;
  pd.M = a.P.M;
  pd.slot = a.P.slot;
  pd.tw = nullptr;
  pd.c = a.P.c;
  pd.c64 = a.P.c64;
  pd.cfmt = a.P.cfmt;
  pd.ci = a.P.ci;
  using W = typename FT<E>::W;
  W* xq = a.xq + b * (int64_t)mm;
  const CgResult r = cg_cluster<E, G>(cl, pd, a.Tq + b * (int64_t)mm, m, a.rq + b * (int64_t)mm,
                                      (mode == 2 || a.ex[b].warm) ? xq : nullptr, xq, mode, a.cg_tol,
                                      a.cg_max, sm, mm);
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    if (mode == 1) {
      a.ex[b].ls_rn2 = a.ex[b].ynorm2 - r.bh;
      a.ex[b].cgit += r.iters;
    } else {
      a.ex[b].qf = r.q;
    }
  }
}

// phase 0 (SP): the first support is T_0 with its solution.  phase 1: the K
// largest |b| (ties to the lower index) -> SP: T_new to solve from b's
// values, unless it repeats the accepted support; CoSaMP: the pruned
// estimate, its quadratic form to be taken next.
template <class E>
__global__ void __launch_bounds__(kLT) lq_prune_kernel(LPArgs<E> a, int phase) {
  using W = typename FT<E>::W;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ LPExtra X;
  __shared__ double red[32 * 1 + 1];
  __shared__ int hist[260];
  __shared__ int scr[34];
  __shared__ int same;
  const int64_t b = blockIdx.x;
  if (a.st[b].done) return;
  const int K = a.K, mm = lp_mmax(K, a.algo);
  const Grp g = whole_block();
  if (threadIdx.x == 0) X = a.ex[b];
  __syncthreads();
  int* T = a.Tq + b * (int64_t)mm;
  W* rq = a.rq + b * (int64_t)mm;
  W* xq = a.xq + b * (int64_t)mm;
  const double tol2 = a.rel_tol * a.rel_tol;
  if (phase == 0) {
    lp_set_support(a, b, X, T, xq, X.mq);
    if (threadIdx.x == 0) {
      X.rn2 = X.ls_rn2;
      X.cgmode = 0;
    }
    __syncthreads();
    if (X.it >= a.max_iter || X.rn2 < tol2 * X.ynorm2) lp_outputs(a, b, X);
    if (threadIdx.x == 0) a.ex[b] = X;
    return;
  }
  const int m = X.mq, kp = K < m ? K : m;
  unsigned long long* sk = (unsigned long long*)sm;
  int* pos = (int*)(sm + al16((size_t)mm * sizeof(unsigned long long)));
  int* tn = pos + kp;
  W* vn = (W*)(sm + al16((size_t)mm * sizeof(unsigned long long)) + al16((size_t)2 * K * sizeof(int)));
  for (int i = threadIdx.x; i < m; i += kLT) sk[i] = sel_key(norm2(xq[i]));
  __syncthreads();
  group_topk(g, sk, m, kp, pos, hist, scr);  // ascending positions
  for (int i = threadIdx.x; i < kp; i += kLT) {
    tn[i] = T[pos[i]];
    vn[i] = xq[pos[i]];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kp; i += kLT) {
    T[i] = tn[i];
    xq[i] = vn[i];
  }
  if (a.algo == 0) {
    if (threadIdx.x == 0) {
      const int* S = a.S + b * K;
      bool sm_ = kp == X.ns;
      for (int i = 0; sm_ && i < kp; ++i) sm_ = tn[i] == S[i];
      same = sm_;
    }
    __syncthreads();
    if (same) {
      if (threadIdx.x == 0) {
        X.rn2_new = X.rn2;
        X.cgmode = 0;
      }
    } else {
      for (int i = threadIdx.x; i < kp; i += kLT) rq[i] = lp_rhs(a, b, tn[i]);
      if (threadIdx.x == 0) {
        X.mq = kp;
        X.cgmode = 1;
        X.warm = 1;
        X.rn2_new = -1.0;  // taken from the solve
      }
    }
  } else {
    // ||y - Phi x||^2 = ||y||^2 - 2 Re x^H h_0(S) + x^H G_S x; the quadratic
    // form comes from the next solver call
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < kp; i += kLT) acc[0] += re(cmul(vn[i], lp_rhs(a, b, tn[i])));
    group_sum(g, acc, red);
    if (threadIdx.x == 0) {
      X.rn2_new = X.ynorm2 - 2.0 * acc[0];
      X.mq = kp;
      X.cgmode = 2;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) a.ex[b] = X;
}

template <class E>
__global__ void __launch_bounds__(kLT) lq_accept_kernel(LPArgs<E> a) {
  __shared__ LPExtra X;
  const int64_t b = blockIdx.x;
  if (a.st[b].done) return;
  const int mm = lp_mmax(a.K, a.algo);
  if (threadIdx.x == 0) {
    X = a.ex[b];
    if (X.cgmode == 1) X.rn2_new = X.ls_rn2;       // SP: LS on T_new
    else if (X.cgmode == 2) X.rn2_new += X.qf;      // CoSaMP: + x^H G x
    X.it = X.it + 1;
  }
  __syncthreads();
  const double tol2 = a.rel_tol * a.rel_tol;
  bool stop = false;
  if (!(X.rn2_new < X.rn2)) {
    stop = true;  // keep the previous iterate
  } else {
    lp_set_support(a, b, X, a.Tq + b * (int64_t)mm, a.xq + b * (int64_t)mm, X.mq);
    if (threadIdx.x == 0) X.rn2 = X.rn2_new;
    __syncthreads();
  }
  if (!stop && (X.it >= a.max_iter || X.rn2 < tol2 * X.ynorm2)) stop = true;
  if (stop) lp_outputs(a, b, X);
  if (threadIdx.x == 0) {
    X.cgmode = 0;
    a.ex[b] = X;
  }
}

template <class E>
__global__ void __launch_bounds__(kLT) widen_kernel(const E* __restrict__ in, int64_t n,
                                                    typename FT<E>::W* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)kLT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kLT) out[i] = to_w(in[i]);
}

template <class E>
struct LPWs {
  size_t st, ex, h0, H, T, Z, xz, bits, S, xs, xsw, ck, cj, sel, B, yp, Tq, rq, xq, h64, T64, y64, ctr, total;
  int ntiles, kmax, nyp, tile;
};

// Column sets larger than this take the conjugate-gradient least squares.
constexpr int kLqMin = 96;
__host__ __device__ inline bool lp_uses_cg(int K, int algo) { return lp_mmax(K, algo) > kLqMin; }

template <class E>
LPWs<E> lp_ws(const PlanView& Pv, int K, int algo, int fast, int64_t batch) {
  using W = typename FT<E>::W;
  using U = typename KeyT<E>::U;
  LPWs<E> L;
  const size_t N = (size_t)Pv.N, Nv = (size_t)batch * N * (Pv.dft ? 2 : 1) * (Pv.fp32 ? 4 : 8);
  const int mm = lp_mmax(K, algo);
  L.kmax = algo == 0 ? K : 2 * K;
  L.tile = lp_tile((int)N, L.kmax);
  L.ntiles = (int)(N / L.tile);
  {
    const int64_t g = ((int64_t)Pv.M + 2047) / 2048;
    L.nyp = (int)(g < 1 ? 1 : (g > 1024 ? 1024 : g));
  }
  size_t o = 0;
  L.st = o;   o = al16(o + (size_t)batch * sizeof(LState));
  L.ex = o;   o = al16(o + (size_t)batch * sizeof(LPExtra));
  L.h0 = o;   o = al16(o + Nv);
  L.H = o;    o = al16(o + Nv);
  L.T = o;    o = al16(o + Nv);
  L.Z = o;    o = al16(o + (fast ? 0 : (size_t)batch * Pv.M * (Pv.dft ? 2 : 1) * (Pv.fp32 ? 4 : 8)));
  L.xz = o;   o = al16(o + (fast ? 0 : Nv));
  L.bits = o; o = al16(o + (size_t)batch * (N >> 5) * sizeof(uint32_t));
  L.S = o;    o = al16(o + (size_t)batch * K * sizeof(int));
  L.xs = o;   o = al16(o + (size_t)batch * K * sizeof(W));
  L.xsw = o;  o = al16(o + (size_t)batch * K * sizeof(E));
  L.ck = o;   o = al16(o + (size_t)batch * L.ntiles * L.kmax * sizeof(U));
  L.cj = o;   o = al16(o + (size_t)batch * L.ntiles * L.kmax * sizeof(int));
  L.sel = o;  o = al16(o + (size_t)batch * L.kmax * sizeof(int));
  const bool lq = lp_uses_cg(K, algo);
  L.B = o;    o = al16(o + (lq ? 0 : (size_t)batch * (((size_t)mm * (mm + 1)) / 2) * sizeof(W)));
  L.yp = o;   o = al16(o + (size_t)batch * L.nyp * sizeof(double));
  L.Tq = o;   o = al16(o + (lq ? (size_t)batch * mm * sizeof(int) : 0));
  L.rq = o;   o = al16(o + (lq ? (size_t)batch * mm * sizeof(W) : 0));
  L.xq = o;   o = al16(o + (lq ? (size_t)batch * mm * sizeof(W) : 0));
  const bool h64 = lq && sizeof(E) != sizeof(W);
  L.h64 = o;  o = al16(o + (h64 ? (size_t)batch * N * sizeof(W) : 0));
  L.T64 = o;  o = al16(o + (h64 ? (size_t)batch * N * sizeof(W) : 0));
  L.y64 = o;  o = al16(o + (h64 ? (size_t)batch * Pv.M * sizeof(W) : 0));
  L.ctr = o;  o = al16(o + 2 * sizeof(int));  // instances done, loop iterations
  L.total = o;
  return L;
}

// ------------------------------------------------ device-side iteration loop
// The iterations of a large-plan pursuit are the same kernels every time,
// with all their state on the device, and most instances stop long before
// max_iter.  Instead of queuing max_iter copies of them from the host, the
// call runs one CUDA graph whose conditional while node repeats them: a
// one-thread kernel at the end of each pass counts it and lets the loop go on
// while an instance is unfinished and the count is below the limit, so the
// loop ends on the device as soon as the last instance does.

// Iterations after the first from which the device-side loop is used.
constexpr int kDeviceLoopMin = 64;

__global__ void loop_ctl_kernel(cudaGraphConditionalHandle h, int* ctr, const int* ndone, int64_t batch,
                                int limit) {
  const int it = ++*ctr;
  cudaGraphSetConditional(h, (*ndone < batch && it < limit) ? 1u : 0u);
}

// body(stream) enqueues one iteration.  Returns cudaErrorNotSupported, with
// nothing queued, when the graph cannot be built (the caller then queues the
// iterations itself).
template <class F>
cudaError_t device_loop(cudaStream_t s, int* ctr, const int* ndone, int64_t batch, int limit, F&& body) {
  if (limit <= 0) return cudaSuccess;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  bool capturing = false;
  cudaError_t rc = cudaSuccess;
  do {
    if (e != cudaSuccess) { rc = cudaErrorNotSupported; break; }
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
      rc = cudaErrorNotSupported;
      break;
    }
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) { rc = cudaErrorNotSupported; break; }
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { rc = cudaErrorNotSupported; break; }
    if (cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = cudaErrorNotSupported;
      break;
    }
    capturing = true;
    rc = body(cs);
    if (rc == cudaSuccess) {
      loop_ctl_kernel<<<1, 1, 0, cs>>>(h, ctr, ndone, batch, limit);
      rc = cudaGetLastError();
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &captured);
    capturing = false;
    if (rc != cudaSuccess) break;
    if (ee != cudaSuccess) { rc = ee; break; }
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = cudaErrorNotSupported;
      break;
    }
    if ((rc = cudaMemsetAsync(ctr, 0, sizeof(int), s)) != cudaSuccess) break;
    rc = cudaGraphLaunch(x, s);
  } while (0);
  if (capturing) {
    cudaGraph_t captured = nullptr;
    (void)cudaStreamEndCapture(cs, &captured);
  }
  if (x) cudaGraphExecDestroy(x);  // a launched graph is freed once it completes
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  return rc;
}

// Conjugate-gradient launches: one cluster of G CTAs per instance.  A CTA
// asks for more than half of an SM's shared memory when G >= 8, so that the
// cluster spreads over G SMs (the solver is bound by the FP64 pipe).
template <class E, int G>
cudaError_t lq_cg_launch(const LPArgs<E>& a, int64_t batch, cudaStream_t s, bool probe_only, int* ok) {
  using W = typename FT<E>::W;
  const int mm = lp_mmax(a.K, a.algo);
  size_t smem = cg_smem_bytes<W>(mm, G);
  if (G >= 8 && smem < (size_t)116 * 1024) smem = (size_t)116 * 1024;
  auto kern = lq_cg_kernel<E, G>;
  cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  // set once per device (the launches inside a device-side loop are
  // captured into a graph after the first iteration has set it)
  static std::atomic<unsigned long long> nonportable{0ull};  // one bit per device
  if (G > 8) {
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(nonportable.load() & bit)) {
      if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
        return e;
      nonportable.fetch_or(bit);
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(batch * G));
  cfg.blockDim = dim3(kLT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (probe_only) {
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      n = 0;
    }
    *ok = n > 0;
    return cudaSuccess;
  }
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class E>
cudaError_t lq_cg(const LPArgs<E>& a, int64_t batch, int G, cudaStream_t s) {
  int ok = 0;
  switch (G) {
    case 16: return lq_cg_launch<E, 16>(a, batch, s, false, &ok);
    case 8: return lq_cg_launch<E, 8>(a, batch, s, false, &ok);
    default: return lq_cg_launch<E, 4>(a, batch, s, false, &ok);
  }
}

// CTAs per cluster: 16 for large sets where the GPU can place such a
// cluster, else 8; 4 for small sets.
template <class E>
int lq_cluster_size(const LPArgs<E>& a, int64_t batch, cudaStream_t s) {
  const int mm = lp_mmax(a.K, a.algo);
  if (mm < 256) return 4;
  if (mm >= 768) {
    int ok = 0;
    if (lq_cg_launch<E, 16>(a, batch, s, true, &ok) == cudaSuccess && ok) return 16;
  }
  return 8;
}

template <class E>
cudaError_t lp_t(const PlanView& Pv, const PursuitLaunch& q, void* ws, cudaStream_t s) {
  using W = typename FT<E>::W;
  using U = typename KeyT<E>::U;
  constexpr bool DFT = FT<E>::C;
  const LDev<E> P = ldev<E>(Pv);
  const int64_t batch = q.batch;
  const LPWs<E> L = lp_ws<E>(Pv, q.K, q.algo, q.fast, batch);
  unsigned char* w = (unsigned char*)ws;
  LPArgs<E> a;
  a.P = P;
  a.y = (const E*)q.y;
  a.K = q.K;
  a.algo = q.algo;
  a.max_iter = q.max_iter;
  a.rel_tol = q.rel_tol;
  a.x_out = (W*)q.x_out;
  a.supp_out = q.supp_out;
  a.iters_out = q.iters_out;
  a.res_out = q.res_out;
  a.st = (LState*)(w + L.st);
  a.ex = (LPExtra*)(w + L.ex);
  a.h0 = (E*)(w + L.h0);
  E* H = (E*)(w + L.H);
  E* T = (E*)(w + L.T);
  E* Z = q.fast ? nullptr : (E*)(w + L.Z);
  a.xz = q.fast ? nullptr : (E*)(w + L.xz);
  a.bits = (uint32_t*)(w + L.bits);
  a.S = (int*)(w + L.S);
  a.xs = (W*)(w + L.xs);
  a.xsw = (E*)(w + L.xsw);
  a.ckey = (U*)(w + L.ck);
  a.cj = (int*)(w + L.cj);
  a.ntiles = L.ntiles;
  a.tile = L.tile;
  a.kmax = L.kmax;
  a.sel = (int*)(w + L.sel);
  a.B = (W*)(w + L.B);
  a.ypart = (double*)(w + L.yp);
  a.nyp = L.nyp;
  a.lq = lp_uses_cg(q.K, q.algo);
  a.Tq = a.lq ? (int*)(w + L.Tq) : nullptr;
  a.rq = a.lq ? (W*)(w + L.rq) : nullptr;
  a.xq = a.lq ? (W*)(w + L.xq) : nullptr;
  a.h64 = (a.lq && sizeof(E) != sizeof(W)) ? (const W*)(w + L.h64) : nullptr;
  a.ndone = (int*)(w + L.ctr);
  {
    const int mm = lp_mmax(q.K, q.algo);
    a.cg_max = 2 * mm < 64 ? 64 : (2 * mm > 4000 ? 4000 : 2 * mm);
    a.cg_tol = cg_tol<E>();
  }
  const size_t Nv = (size_t)batch * P.N * sizeof(E);
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.st, 0, (size_t)batch * sizeof(LState), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.ex, 0, (size_t)batch * sizeof(LPExtra), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.ndone, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.bits, 0, (size_t)batch * (P.N >> 5) * sizeof(uint32_t), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.S, 0, (size_t)batch * q.K * sizeof(int), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.xsw, 0, (size_t)batch * q.K * sizeof(E), s)) != cudaSuccess) return e;
  if (a.xz && (e = cudaMemsetAsync(a.xz, 0, Nv, s)) != cudaSuccess) return e;
  const size_t tile_smem = al16((size_t)a.tile * sizeof(U)) + al16((size_t)a.kmax * sizeof(int)) + 300 * sizeof(int);
  const size_t merge_smem = al16((size_t)a.kmax * sizeof(int)) + 300 * sizeof(int);
  const size_t step_smem = lp_uses_cg(q.K, q.algo) ? 0 : lp_layout<E>(q.K, q.algo).total;
  if ((e = allow_smem(lp_tile_kernel<E>, tile_smem)) != cudaSuccess) return e;
  if ((e = allow_smem(lp_merge_kernel<E>, merge_smem)) != cudaSuccess) return e;
  if (step_smem && (e = allow_smem(lp_step_kernel<E>, step_smem)) != cudaSuccess) return e;
  const double isq = inv_sqrt_n(P.logN);
  const dim3 tgrid((unsigned)L.ntiles, (unsigned)batch);
  // h_0 = Phi^H y by one transform, and ||y||^2
  lynorm_kernel<E><<<dim3((unsigned)L.nyp, (unsigned)batch), kLT, 0, s>>>(a.y, P.M, a.ypart, L.nyp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = run_col<E, DFT, LD_ZF>(P, a.y, P.M, T, a.st, batch, s)) != cudaSuccess) return e;
  if ((e = run_row<E, DFT, SK_H>(P, T, DFT, isq, a.h0, nullptr, nullptr, nullptr, nullptr, 0, a.st, batch, s)) !=
      cudaSuccess)
    return e;
  if (a.h64) {  // the same correlation in FP64 for the least squares' right-hand sides
    const LDev<W> P64 = ldev<W>(Pv);
    W* y64 = (W*)(w + L.y64);
    const int64_t ny = batch * (int64_t)P.M;
    if (ny > 0) {
      widen_kernel<E><<<(unsigned)((ny + kLT - 1) / kLT < 4096 ? (ny + kLT - 1) / kLT : 4096), kLT, 0, s>>>(a.y, ny,
                                                                                                        y64);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = run_col<W, DFT, LD_ZF>(P64, y64, P.M, (W*)(w + L.T64), a.st, batch, s)) != cudaSuccess) return e;
    if ((e = run_row<W, DFT, SK_H>(P64, (const W*)(w + L.T64), DFT, isq, (W*)a.h64, nullptr, nullptr, nullptr,
                                   nullptr, 0, a.st, batch, s)) != cudaSuccess)
      return e;
  }
  if (q.algo == 0) {  // SP's first support: top_K(h_0)
    lp_tile_kernel<E><<<tgrid, kLT, tile_smem, s>>>(a, a.h0, q.K, 0);
    lp_merge_kernel<E><<<(unsigned)batch, kLT, merge_smem, s>>>(a, q.K);
  }
  int G = 0;
  size_t prune_smem = 0;
  if (a.lq) {
    const int mm = lp_mmax(q.K, q.algo);
    G = lq_cluster_size<E>(a, batch, s);
    prune_smem = al16((size_t)mm * sizeof(unsigned long long)) + al16((size_t)2 * q.K * sizeof(int)) +
                 (size_t)q.K * sizeof(W);
    if ((e = allow_smem(lq_prune_kernel<E>, prune_smem)) != cudaSuccess) return e;
    lq_form_kernel<E><<<(unsigned)batch, kLT, 0, s>>>(a, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (q.algo == 0) {
      if ((e = lq_cg<E>(a, batch, G, s)) != cudaSuccess) return e;
      lq_prune_kernel<E><<<(unsigned)batch, kLT, prune_smem, s>>>(a, 0);
    }
  } else {
    lp_step_kernel<E><<<(unsigned)batch, kLT, step_smem, s>>>(a, 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int kk = q.algo == 0 ? q.K : 2 * q.K;
  // one iteration on stream st
  auto iteration = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    if (q.fast) {  // h = h_0 - sum over the support (zero-padded to K atoms)
      if ((e = run_fast<E, DFT>(P, a.h0, a.S, a.xsw, q.K, q.K, nullptr, H, nullptr, nullptr, 0, a.st, batch, st)) !=
          cudaSuccess)
        return e;
    } else {  // r = y - Phi x by a forward transform of zf(x), then h = A^H zf(r)
      if ((e = run_col<E, DFT, LD_DENSE>(P, a.xz, P.N, T, a.st, batch, st)) != cudaSuccess) return e;
      if ((e = run_row<E, DFT, SK_RES>(P, T, 0, isq, Z, a.y, nullptr, nullptr, nullptr, 0, a.st, batch, st)) !=
          cudaSuccess)
        return e;
      if ((e = run_col<E, DFT, LD_ZF>(P, Z, P.M, T, a.st, batch, st)) != cudaSuccess) return e;
      if ((e = run_row<E, DFT, SK_H>(P, T, DFT, isq, H, nullptr, nullptr, nullptr, nullptr, 0, a.st, batch, st)) !=
          cudaSuccess)
        return e;
    }
    lp_tile_kernel<E><<<tgrid, kLT, tile_smem, st>>>(a, H, kk, q.algo == 0);
    lp_merge_kernel<E><<<(unsigned)batch, kLT, merge_smem, st>>>(a, kk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.lq) {
      // every launch is checked at once: a kernel that failed to start
      // would leave the next one working on the previous step's state
      lq_form_kernel<E><<<(unsigned)batch, kLT, 0, st>>>(a, 1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = lq_cg<E>(a, batch, G, st)) != cudaSuccess) return e;
      lq_prune_kernel<E><<<(unsigned)batch, kLT, prune_smem, st>>>(a, 1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = lq_cg<E>(a, batch, G, st)) != cudaSuccess) return e;
      lq_accept_kernel<E><<<(unsigned)batch, kLT, 0, st>>>(a);
    } else {
      lp_step_kernel<E><<<(unsigned)batch, kLT, step_smem, st>>>(a, 1);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaSuccess;
  };
  // the first iteration from the host (it also sets the kernels' attributes),
  // the others in a device-side loop when there are many of them to save
  // (building and instantiating the graph costs host time on every call, and
  // with many solves at once on several streams, as in the request runtime,
  // the graphs slowed the whole mix: 65 -> 38 solves/s on the serving
  // workload, where CoSaMP has max_iter 50); the host queues them where the
  // graph is not worth it or cannot be built
  if (q.max_iter < 1) return cudaSuccess;
  if ((e = iteration(s)) != cudaSuccess) return e;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusActive;
  // (a stream under capture gets the iterations queued into its graph)
  if (q.max_iter - 1 >= kDeviceLoopMin && cap == cudaStreamCaptureStatusNone) {
    e = device_loop(s, a.ndone + 1, a.ndone, batch, q.max_iter - 1, iteration);
    if (e != cudaErrorNotSupported) return e;
    (void)cudaGetLastError();
  }
  for (int it = 1; it < q.max_iter; ++it)
    if ((e = iteration(s)) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

// ------------------------------------------------------------ entry points
cudaError_t large_tables(const PlanView& P, void* lt64, void* lt32, cudaStream_t st) {
  if (!P.dft) return cudaSuccess;
  const int N1 = 1 << P.n1, N2 = 1 << P.n2;
  double2* t64 = (double2*)lt64;
  float2* t32 = (float2*)lt32;
  cudaError_t e = launch_twiddles_log(P.n1, t64, t32, st);
  if (e != cudaSuccess) return e;
  e = launch_twiddles_log(P.n2, t64 + N1, t32 ? t32 + N1 : nullptr, st);
  if (e != cudaSuccess) return e;
  const int nlo = 1 << P.wsh;
  roots_kernel<<<64, kLT, 0, st>>>(P.logN, P.wsh, t64 + N1 + N2, t64 + N1 + N2 + nlo,
                                   t32 ? t32 + N1 + N2 : nullptr, t32 ? t32 + N1 + N2 + nlo : nullptr);
  return cudaGetLastError();
}

cudaError_t large_kernel_vector(const PlanView& P, void* c64_full, void* tmp, cudaStream_t st) {
  return P.dft ? kv_t<double2>(P, c64_full, tmp, st) : kv_t<double>(P, c64_full, tmp, st);
}

size_t large_correlate_ws(const PlanView& P, int64_t batch) {
  if (P.dft) return P.fp32 ? corr_ws_t<float2>(P, batch) : corr_ws_t<double2>(P, batch);
  return P.fp32 ? corr_ws_t<float>(P, batch) : corr_ws_t<double>(P, batch);
}

cudaError_t large_correlate(const PlanView& P, const void* r, int64_t batch, void* h, int32_t* amax, void* ws,
                            cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (batch > kMaxBatchY) return cudaErrorInvalidValue;
  if (P.dft) return P.fp32 ? corr_t<float2>(P, r, batch, h, amax, ws, st) : corr_t<double2>(P, r, batch, h, amax, ws, st);
  return P.fp32 ? corr_t<float>(P, r, batch, h, amax, ws, st) : corr_t<double>(P, r, batch, h, amax, ws, st);
}

size_t large_fast_ws(const PlanView& P, int64_t batch) {
  if (P.dft) return P.fp32 ? fast_ws_t<float2>(P, batch) : fast_ws_t<double2>(P, batch);
  return P.fp32 ? fast_ws_t<float>(P, batch) : fast_ws_t<double>(P, batch);
}

cudaError_t large_correlate_fast(const PlanView& P, const void* h0, const int32_t* supp, const void* x, int s,
                                 int64_t batch, void* h, int32_t* amax, void* ws, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (batch > kMaxBatchY) return cudaErrorInvalidValue;
  if (P.dft) return P.fp32 ? fast_t<float2>(P, h0, supp, x, s, batch, h, amax, ws, st)
                           : fast_t<double2>(P, h0, supp, x, s, batch, h, amax, ws, st);
  return P.fp32 ? fast_t<float>(P, h0, supp, x, s, batch, h, amax, ws, st)
                : fast_t<double>(P, h0, supp, x, s, batch, h, amax, ws, st);
}

size_t large_omp_ws(const PlanView& P, int K, int path, int64_t batch) {
  if (P.dft) return P.fp32 ? lomp_ws<float2>(P, K, path, batch).total : lomp_ws<double2>(P, K, path, batch).total;
  return P.fp32 ? lomp_ws<float>(P, K, path, batch).total : lomp_ws<double>(P, K, path, batch).total;
}

cudaError_t large_omp(const PlanView& P, const OmpLaunch& a, void* ws, cudaStream_t st) {
  if (a.batch <= 0) return cudaSuccess;
  if (a.batch > kMaxBatchY) return cudaErrorInvalidValue;
  if (P.dft) return P.fp32 ? omp_t<float2>(P, a, ws, st) : omp_t<double2>(P, a, ws, st);
  return P.fp32 ? omp_t<float>(P, a, ws, st) : omp_t<double>(P, a, ws, st);
}

}  // namespace csf

namespace csf {
size_t large_pursuit_ws(const PlanView& P, int K, int algo, int fast, int64_t batch) {
  if (P.dft) return P.fp32 ? lp_ws<float2>(P, K, algo, fast, batch).total : lp_ws<double2>(P, K, algo, fast, batch).total;
  return P.fp32 ? lp_ws<float>(P, K, algo, fast, batch).total : lp_ws<double>(P, K, algo, fast, batch).total;
}

cudaError_t large_pursuit(const PlanView& P, const PursuitLaunch& a, void* ws, cudaStream_t st) {
  if (a.batch <= 0) return cudaSuccess;
  if (a.batch > kMaxBatchY) return cudaErrorInvalidValue;
  if (P.dft) return P.fp32 ? lp_t<float2>(P, a, ws, st) : lp_t<double2>(P, a, ws, st);
  return P.fp32 ? lp_t<float>(P, a, ws, st) : lp_t<double>(P, a, ws, st);
}
}  // namespace csf
