// The one-CTA radix-16 chains of cs_transform.cuh for a vector held in
// global memory (N = 2^14 .. 2^16, four passes), two passes per round trip:
// every butterfly, twiddle and output position is that of the chain, but
// passes 0 and 1 run together on tiles of 16 groups of 256 elements at stride
// N/256 (the elements one group's two butterfly levels touch), and passes 2
// and 3 on contiguous tiles, in shared memory.  A transform then reads and
// writes the vector twice instead of four times, and the loader / sink of
// the chain's first / last pass fuse the zero-fill of a measurement and the
// masked residual of Algorithm 1.1 step 7 into it.
//
// Twiddles of passes 0 and 1 (W_N^e, e < N) would be read from a table as
// long as the vector; instead they are W_N^(256 hi) W_N^lo, e = 256 hi + lo,
// from two 256-entry tables in shared memory (`tws`, filled once per vector
// by fill_split_twiddles): one more complex product per twiddle, and no
// global-memory load.  Passes 2 and 3 use the chain's table (at most 256
// entries of it, which stay in L1).
//
// KIND 0: forward DIF chain (natural order in, chain positions out);
// KIND 1: adjoint DIT chain (chain positions in, natural order out);
// KIND 2: Sylvester Walsh-Hadamard transform (natural order in and out,
// its four digit levels applied in the DIF schedule's order).
#pragma once
#include <type_traits>

#include "cs_blocks.cuh"

namespace csf {

constexpr int kGTile = 4096;  // elements of one stage tile in shared memory

// Loader / sink adaptors from tile positions to vector positions.
template <class LD>
struct OffLoad {
  const LD& ld;
  int off;
  __device__ __forceinline__ auto operator()(int pos) const { return ld(off + pos); }
};
template <class SK>
struct OffSink {
  SK& sk;
  int off;
  template <class E>
  __device__ __forceinline__ void operator()(int pos, const E& v) { sk(off + pos, v); }
};

// scl * zf_Omega(v) at a position (the input of the correlation's adjoint).
template <class E>
struct ZeroFillLoad {
  const int* slot;
  const E* v;
  typename FT<E>::R scl;
  __device__ __forceinline__ E operator()(int pos) const {
    const int m = __ldg(slot + pos);
    return m >= 0 ? scale(v[m], scl) : zero<E>();
  }
};

// N^{-1/2} y - N^{-1} (F x) on Omega and 0 elsewhere, stored to the vector:
// the zero-filled residual of step 7 from the forward transform of x.
template <class E, bool NORM = false>
struct ResidualSink {
  const int* slot;
  const E* y;
  typename FT<E>::R sy, sx;
  E* out;
  double acc = 0.0;  // with NORM: this thread's share of sum |out|^2 (FP64)
  __device__ __forceinline__ void operator()(int pos, const E& fx) {
    const int m = __ldg(slot + pos);
    const E r = m >= 0 ? sub(scale(y[m], sy), scale(fx, sx)) : zero<E>();
    if constexpr (NORM) acc += norm2(to_w(r));
    out[pos] = r;
  }
};

// exp(-2 pi i e / N) in the working precision (sincospi of an exact
// argument: N is a power of two).
template <class E>
__device__ __forceinline__ E unit_root(int e, int N);
template <>
__device__ __forceinline__ float2 unit_root<float2>(int e, int N) {
  float sn, cs;
  sincospif(-2.0f * (float)e / (float)N, &sn, &cs);
  return make_float2(cs, sn);
}
template <>
__device__ __forceinline__ double2 unit_root<double2>(int e, int N) {
  double sn, cs;
  sincospi(-2.0 * (double)e / (double)N, &sn, &cs);
  return make_double2(cs, sn);
}

// tws[i] = W_N^i and tws[256 + i] = W_N^(256 i), i < 256 (DFT only).
template <class E>
__device__ void fill_split_twiddles(const Grp& g, E* tws, int N) {
  for (int i = g.tid; i < 256; i += g.n) {
    tws[i] = unit_root<E>(i, N);
    tws[256 + i] = unit_root<E>((256 * i) & (N - 1), N);
  }
  g.sync();
}

// Moves kGTile elements between a global vector and the tile: dst(i) =
// src(i) for i < kGTile, every thread issuing 8 loads before its 8 stores so
// that the loads overlap (one CTA per SM leaves little else to hide their
// latency).
template <class E, class SRC, class DST>
__device__ __forceinline__ void tile_move(const Grp& g, const SRC& src, const DST& dst) {
  constexpr int kPer = 8;
  for (int i0 = 0; i0 < kGTile; i0 += kPer * g.n) {
    E r[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int i = i0 + k * g.n + g.tid;
      r[k] = i < kGTile ? src(i) : zero<E>();
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int i = i0 + k * g.n + g.tid;
      if (i < kGTile) dst(i, r[k]);
    }
  }
  g.sync();
}

// Passes 0 and 1 on the groups c + m S1 (c < S1 = N/256, m < 256), 16
// groups (c0 .. c0 + 15) per tile, element m of group gg at tile[16 m + gg].
// Pass 0 (L = N, stride S0 = 16 S1) has butterflies (gg, u) over
// m = u + 16 r; pass 1 (L = N/16, stride S1) has butterflies (gg, v) over
// m = 16 v + r.  DIF and WHT run pass 0 then pass 1 and take the loader;
// DIT runs pass 1 then pass 0 and feeds the sink.
template <int KIND, class E, class LD, class SK>
__device__ void gstage_strided(const Grp& g, E* gbuf, E* tile, int logN, const E* tws, const LD& ld, SK& sk) {
  constexpr bool hasLD = !std::is_same<LD, NoLoad>::value;
  constexpr bool hasSK = !std::is_same<SK, NoSink>::value;
  static_assert(!(hasLD && KIND == 1) && !(hasSK && KIND != 1), "loader / sink on the wrong stage");
  const int N = 1 << logN, S1 = N >> 8;
  for (int c0 = 0; c0 < S1; c0 += 16) {
    if constexpr (!hasLD) {
      tile_move<E>(g, [&](int i) { return gbuf[c0 + (i & 15) + (i >> 4) * S1]; },
                   [&](int i, const E& v) { tile[i] = v; });
    }
    for (int half = 0; half < 2; ++half) {
      const bool outer = (KIND == 1) ? half == 1 : half == 0;  // pass 0 is the outer pass
      for (int bf = g.tid; bf < 256; bf += g.n) {
        const int gg = bf & 15, w = bf >> 4, c = c0 + gg;
        // element r of this butterfly: m = u + 16 r (outer) or 16 v + r (inner)
        const int m0 = outer ? w : 16 * w, mst = outer ? 16 : 1;
        E v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int m = m0 + r * mst;
          if constexpr (hasLD) v[r] = outer ? ld(c + m * S1) : tile[16 * m + gg];
          else v[r] = tile[16 * m + gg];
        }
        // output / input q of this butterfly carries W_N^(q e1): pass 0
        // (L = N) has W_N^(n q), n = c + w S1 its index within the
        // transform; pass 1 (L = N/16) has W_{N/16}^(c q) = W_N^(16 c q)
        const int e1 = outer ? c + w * S1 : 16 * c;
        if constexpr (KIND == 0) {
          dft_reg<16, -1>(v);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            E o = v[bitrevc(q, 4)];
            if (q > 0) {
              const int e = q * e1;
              o = mul(o, mul(tws[256 + (e >> 8)], tws[e & 255]));
            }
            tile[16 * (m0 + q * mst) + gg] = o;
          }
        } else if constexpr (KIND == 1) {
#pragma unroll
          for (int q = 1; q < 16; ++q) {
            const int e = q * e1;
            v[q] = mulc(v[q], mul(tws[256 + (e >> 8)], tws[e & 255]));
          }
          dft_reg<16, +1>(v);
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const int m = m0 + r * mst;
            if constexpr (hasSK) {
              if (outer) sk(c + m * S1, v[bitrevc(r, 4)]);
              else tile[16 * m + gg] = v[bitrevc(r, 4)];
            } else {
              tile[16 * m + gg] = v[bitrevc(r, 4)];
            }
          }
        } else {
          wht_reg<16>(v);
#pragma unroll
          for (int r = 0; r < 16; ++r) tile[16 * (m0 + r * mst) + gg] = v[r];
        }
      }
      g.sync();
    }
    if constexpr (!hasSK) {
      tile_move<E>(g, [&](int i) { return tile[i]; },
                   [&](int i, const E& v) { gbuf[c0 + (i & 15) + (i >> 4) * S1] = v; });
    }
  }
}

template <int KIND, class E, class L2, class S2>
__device__ __forceinline__ void contig_passes(const Grp& g, E* tile, int logN, const E* tw, const L2& ld, S2& sk,
                                              bool first, bool last) {
  const int N = 1 << logN;
  const int LA = 1 << sched_logL(logN, 2), LB = 1 << sched_logL(logN, 3);
  const int lrA = sched_logR(logN, 2), lrB = sched_logR(logN, 3);
  if constexpr (KIND == 1) {  // DIT: pass 3, then pass 2
    pass_radix<1>(g, tile, kGTile, LB, tw + (N - LB), lrB, first, false, ld, sk);
    pass_radix<1>(g, tile, kGTile, LA, tw + (N - LA), lrA, false, last, ld, sk);
  } else if constexpr (KIND == 0) {
    pass_radix<0>(g, tile, kGTile, LA, tw + (N - LA), lrA, first, false, ld, sk);
    pass_radix<0>(g, tile, kGTile, LB, tw + (N - LB), lrB, false, last, ld, sk);
  } else {  // WHT levels at strides L_2 / R_2 and 1
    pass_radix<2>(g, tile, kGTile, LA >> lrA, (const E*)nullptr, lrA, first, false, ld, sk);
    pass_radix<2>(g, tile, kGTile, 1, (const E*)nullptr, lrB, false, last, ld, sk);
  }
}

// Passes 2 and 3: sub-transforms of length L_2 <= 256, contiguous, kGTile
// elements per tile (the chain's swizzled tile layout).  DIT runs first in
// its chain and takes the loader; DIF and WHT run last and feed the sink.
template <int KIND, class E, class LD, class SK>
__device__ void gstage_contig(const Grp& g, E* gbuf, E* tile, int logN, const E* __restrict__ tw, const LD& ld,
                              SK& sk) {
  constexpr bool hasLD = !std::is_same<LD, NoLoad>::value;
  constexpr bool hasSK = !std::is_same<SK, NoSink>::value;
  static_assert(!(hasLD && KIND != 1) && !(hasSK && KIND == 1), "loader / sink on the wrong stage");
  const int N = 1 << logN;
  NoLoad nl;
  NoSink ns;
  for (int base = 0; base < N; base += kGTile) {
    if constexpr (!hasLD) {
      tile_move<E>(g, [&](int i) { return gbuf[base + i]; }, [&](int i, const E& v) { tile[swz<E>(i)] = v; });
    }
    if constexpr (hasLD && hasSK) {
      OffLoad<LD> ol{ld, base};
      OffSink<SK> os{sk, base};
      contig_passes<KIND>(g, tile, logN, tw, ol, os, true, true);
    } else if constexpr (hasLD) {
      OffLoad<LD> ol{ld, base};
      contig_passes<KIND>(g, tile, logN, tw, ol, ns, true, false);
    } else if constexpr (hasSK) {
      OffSink<SK> os{sk, base};
      contig_passes<KIND>(g, tile, logN, tw, nl, os, false, true);
    } else {
      contig_passes<KIND>(g, tile, logN, tw, nl, ns, false, false);
    }
    if constexpr (!hasSK) {
      tile_move<E>(g, [&](int i) { return tile[swz<E>(i)]; }, [&](int i, const E& v) { gbuf[base + i] = v; });
    }
  }
}

// Whole chain of the kind on gbuf (natural positions; the caller's group
// holds the tile).  `ld` feeds the chain's first pass, `sk` its last; tw is
// the chain's twiddle table, tws the split tables of passes 0 and 1.
template <int KIND, class E, class LD, class SK>
__device__ void gchain(const Grp& g, E* gbuf, E* tile, int logN, const E* tw, const E* tws, const LD& ld, SK& sk) {
  NoLoad nl;
  NoSink ns;
  if constexpr (KIND == 1) {
    gstage_contig<1>(g, gbuf, tile, logN, tw, ld, ns);
    gstage_strided<1>(g, gbuf, tile, logN, tws, nl, sk);
  } else {
    gstage_strided<KIND>(g, gbuf, tile, logN, tws, ld, ns);
    gstage_contig<KIND>(g, gbuf, tile, logN, tw, nl, sk);
  }
}

// h = A^H zf_Omega(v) for a vector in global memory (as correlate_transform),
// with the arg-max of step 3 and an optional store of h; *norm receives this
// thread's share of sum |v_m|^2 (FP64).
template <class E, bool DFT>
__device__ int gcorrelate_transform(const Grp& g, E* gbuf, E* tile, const E* tws, const PlanDev<E>& P,
                                    const E* __restrict__ v, E* h_out, double* norm, typename NormT<E>::V* rv,
                                    int* rj) {
  using R = typename FT<E>::R;
  using V = typename NormT<E>::V;
  double s = 0.0;
  for (int m = g.tid; m < P.M; m += g.n) s += norm2(to_w(v[m]));
  *norm = s;
  const ZeroFillLoad<E> ld{P.slot, v, inv_sqrt_pow2<R>(P.logN)};
  ArgmaxSink<E> sk{nullptr, h_out, (V)-1, 0x7fffffff, nullptr};
  gchain<DFT ? 1 : 2>(g, gbuf, tile, P.logN, P.tw, tws, ld, sk);
  return group_argmax(g, sk.bv, sk.bj, rv, rj);
}

// h = A^H zf(y - S_Omega A x_Lambda) for a vector in global memory (as
// correlate_residual): forward chain from the sparse coefficients whose last
// stage writes the masked residual, adjoint chain whose last stage feeds the
// arg-max over j not in Lambda.
// With NORM, *r2 receives ||y - Phi x||^2 (FP64 accumulation of the
// working-precision residual; red holds 33 doubles).
template <class E, bool DFT, bool NORM = false>
__device__ int gcorrelate_residual(const Grp& g, E* gbuf, E* tile, const E* tws, const PlanDev<E>& P,
                                   const E* __restrict__ y,
                                   const uint32_t* bits, const uint16_t* kidx, const E* xw,
                                   typename NormT<E>::V* rv, int* rj, double* r2 = nullptr, double* red = nullptr) {
  using R = typename FT<E>::R;
  using V = typename NormT<E>::V;
  const SparseLoader<E> sl{bits, kidx, xw};
  ResidualSink<E, NORM> rs{P.slot, y, inv_sqrt_pow2<R>(P.logN), (R)1 / (R)P.N, gbuf};
  gchain<DFT ? 0 : 2>(g, gbuf, tile, P.logN, P.tw, tws, sl, rs);
  if constexpr (NORM) {
    double acc[1] = {rs.acc};
    group_sum(g, acc, red);
    *r2 = acc[0] * (double)P.N;  // the entries are r_m / sqrt(N)
  }
  NoLoad nl;
  ArgmaxSink<E> sk{bits, nullptr, (V)-1, 0x7fffffff, nullptr};
  gchain<DFT ? 1 : 2>(g, gbuf, tile, P.logN, P.tw, tws, nl, sk);
  return group_argmax(g, sk.bv, sk.bj, rv, rj);
}

// ||y - Phi x||^2 for a vector in global memory: the forward chain of
// gcorrelate_residual with its residual sink, without the adjoint.
template <class E, bool DFT>
__device__ double gresidual_norm(const Grp& g, E* gbuf, E* tile, const E* tws, const PlanDev<E>& P,
                                 const E* __restrict__ y, const uint32_t* bits, const uint16_t* kidx, const E* xw,
                                 double* red) {
  using R = typename FT<E>::R;
  const SparseLoader<E> sl{bits, kidx, xw};
  ResidualSink<E, true> rs{P.slot, y, inv_sqrt_pow2<R>(P.logN), (R)1 / (R)P.N, gbuf};
  gchain<DFT ? 0 : 2>(g, gbuf, tile, P.logN, P.tw, tws, sl, rs);
  double acc[1] = {rs.acc};
  group_sum(g, acc, red);
  return acc[0] * (double)P.N;
}

}  // namespace csf
