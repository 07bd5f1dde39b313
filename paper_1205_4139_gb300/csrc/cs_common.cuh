// Shared device helpers: element arithmetic for the four element types, the
// shared-memory swizzle, in-register radix-R DFT / Hadamard butterflies and
// block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace csf {

// ------------------------------------------------------------ element traits
// E is the element type of the correlation side (float, double, float2,
// double2; complex types are interleaved re/im).  W is the FP64 element type
// of the least-squares side (double for the real Hadamard case, double2 for
// the complex Fourier case).
template <class E> struct FT;
template <> struct FT<float>   { using R = float;  using W = double;  static constexpr bool C = false; };
template <> struct FT<double>  { using R = double; using W = double;  static constexpr bool C = false; };
template <> struct FT<float2>  { using R = float;  using W = double2; static constexpr bool C = true; };
template <> struct FT<double2> { using R = double; using W = double2; static constexpr bool C = true; };

template <class E> __device__ __forceinline__ E zero();
template <> __device__ __forceinline__ float zero<float>() { return 0.f; }
template <> __device__ __forceinline__ double zero<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 zero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero<double2>() { return make_double2(0.0, 0.0); }

__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ float sub(float a, float b) { return a - b; }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 mul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float mulc(float a, float b) { return a * b; }
__device__ __forceinline__ double mulc(double a, double b) { return a * b; }
__device__ __forceinline__ float2 mulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 mulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ double cmul(double a, double b) { return a * b; }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}

__device__ __forceinline__ float scale(float a, float s) { return a * s; }
__device__ __forceinline__ double scale(double a, double s) { return a * s; }
__device__ __forceinline__ float2 scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

__device__ __forceinline__ float conjv(float a) { return a; }
__device__ __forceinline__ double conjv(double a) { return a; }
__device__ __forceinline__ float2 conjv(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ double2 conjv(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ float norm2(float a) { return a * a; }
__device__ __forceinline__ double norm2(double a) { return a * a; }
__device__ __forceinline__ float norm2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double norm2(double2 a) { return fma(a.x, a.x, a.y * a.y); }

// acc - x * c with one rounding per real FMA (4 FMAs for complex)
__device__ __forceinline__ float fnms(float acc, float x, float c) { return fmaf(-x, c, acc); }
__device__ __forceinline__ double fnms(double acc, double x, double c) { return fma(-x, c, acc); }
__device__ __forceinline__ float2 fnms(float2 acc, float2 x, float2 c) {
  return make_float2(fmaf(-x.x, c.x, fmaf(x.y, c.y, acc.x)), fmaf(-x.x, c.y, fmaf(-x.y, c.x, acc.y)));
}
__device__ __forceinline__ double2 fnms(double2 acc, double2 x, double2 c) {
  return make_double2(fma(-x.x, c.x, fma(x.y, c.y, acc.x)), fma(-x.x, c.y, fma(-x.y, c.x, acc.y)));
}
// acc + a * b
__device__ __forceinline__ double fmav(double acc, double a, double b) { return fma(a, b, acc); }
__device__ __forceinline__ double2 fmav(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc + conj(a) * b
__device__ __forceinline__ double fmacv(double acc, double a, double b) { return fma(a, b, acc); }
__device__ __forceinline__ double2 fmacv(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}

// conversions between the working element and the FP64 element
__device__ __forceinline__ double to_w(float a) { return (double)a; }
__device__ __forceinline__ double to_w(double a) { return a; }
__device__ __forceinline__ double2 to_w(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_w(double2 a) { return a; }
template <class E> __device__ __forceinline__ E from_w(typename FT<E>::W a);
template <> __device__ __forceinline__ float from_w<float>(double a) { return (float)a; }
template <> __device__ __forceinline__ double from_w<double>(double a) { return a; }
template <> __device__ __forceinline__ float2 from_w<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ double2 from_w<double2>(double2 a) { return a; }

__device__ __forceinline__ double re(double a) { return a; }
__device__ __forceinline__ double re(double2 a) { return a.x; }
__device__ __forceinline__ double im(double) { return 0.0; }
__device__ __forceinline__ double im(double2 a) { return a.y; }
template <class W> __device__ __forceinline__ W make_w(double r, double i);
template <> __device__ __forceinline__ double make_w<double>(double r, double) { return r; }
template <> __device__ __forceinline__ double2 make_w<double2>(double r, double i) { return make_double2(r, i); }

// ----------------------------------------------------------- smem swizzle
// Elements are stored at i ^ ((i >> G) & (2^G - 1)), G = log2(128 B / size):
// a row of 128 bytes is permuted by the row index, so that the strided
// accesses of every transform pass and the unit-stride element passes both
// spread over all 32 banks.
template <class E> __device__ __forceinline__ int swz(int i) {
  constexpr int G = sizeof(E) == 4 ? 5 : (sizeof(E) == 8 ? 4 : 3);
  return i ^ ((i >> G) & ((1 << G) - 1));
}

// ------------------------------------------------- in-register butterflies
__host__ __device__ constexpr int ilog2c(int r) { return r <= 1 ? 0 : 1 + ilog2c(r >> 1); }
__host__ __device__ constexpr int bitrevc(int q, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((q >> i) & 1) << (bits - 1 - i);
  return r;
}

// cos(pi k / 8) for any integer k, and sin(pi k / 8) = cos(pi (k - 4) / 8)
__device__ __forceinline__ double cos_pi8(int k) {
  constexpr double C1 = 0.92387953251128675613;  // cos(pi/8)
  constexpr double C2 = 0.70710678118654752440;  // cos(pi/4)
  constexpr double C3 = 0.38268343236508977173;  // cos(3 pi/8)
  switch (k & 15) {
    case 0: return 1.0;
    case 1: return C1;
    case 2: return C2;
    case 3: return C3;
    case 4: return 0.0;
    case 5: return -C3;
    case 6: return -C2;
    case 7: return -C1;
    case 8: return -1.0;
    case 9: return -C1;
    case 10: return -C2;
    case 11: return -C3;
    case 12: return 0.0;
    case 13: return C3;
    case 14: return C2;
    default: return C1;
  }
}
__device__ __forceinline__ double sin_pi8(int k) { return cos_pi8(k + 12); }

// t * exp(SIGN * i * pi * k / 8), k in [0, 8)
template <int SIGN, class E>
__device__ __forceinline__ E rot_pi8(E t, int k) {
  using R = typename FT<E>::R;
  if (k == 0) return t;
  if (k == 4) {  // multiply by SIGN * i
    E o;
    o.x = SIGN > 0 ? -t.y : t.y;
    o.y = SIGN > 0 ? t.x : -t.x;
    return o;
  }
  const R c = (R)cos_pi8(k);
  const R s = (R)(SIGN > 0 ? sin_pi8(k) : -sin_pi8(k));
  E o;
  o.x = t.x * c - t.y * s;
  o.y = t.x * s + t.y * c;
  return o;
}

// In-place radix-2 decimation-in-frequency DFT of R values held in
// registers: V_q = sum_r v_r exp(SIGN 2 pi i r q / R).  On return v[k] holds
// V_{bitrev(k)}.  Stages recurse on the half-span H at compile time so that
// every register index is a constant.
template <int R, int SIGN, int H, class E>
__device__ __forceinline__ void dft_stage(E (&v)[R]) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if ((i & H) == 0) {
      E a = v[i], b = v[i + H];
      v[i] = add(a, b);
      const int e = (i & (H - 1)) * (R / (2 * H));  // power of exp(SIGN 2 pi i / R)
      v[i + H] = rot_pi8<SIGN>(sub(a, b), (16 / R) * e);
    }
  }
  if constexpr (H > 1) dft_stage<R, SIGN, H / 2>(v);
}
template <int R, int SIGN, class E>
__device__ __forceinline__ void dft_reg(E (&v)[R]) {
  if constexpr (R > 1) dft_stage<R, SIGN, R / 2>(v);
}

// In-place Sylvester Hadamard butterflies (natural order in and out).
template <int R, int H, class E>
__device__ __forceinline__ void wht_stage(E (&v)[R]) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    if ((i & H) == 0) {
      E a = v[i], b = v[i + H];
      v[i] = add(a, b);
      v[i + H] = sub(a, b);
    }
  }
  if constexpr (H > 1) wht_stage<R, H / 2>(v);
}
template <int R, class E>
__device__ __forceinline__ void wht_reg(E (&v)[R]) {
  if constexpr (R > 1) wht_stage<R, R / 2>(v);
}

// ------------------------------------------------------------ thread groups
// A group of whole warps of one CTA working on one task: `tid` is the thread
// index within the group, `n` its size, `bar` the hardware barrier it
// synchronises on (0 = the CTA-wide barrier when the group is the whole CTA,
// -1 = a group of exactly one warp, which synchronises with __syncwarp).
// The compiler does not know that the inline named barrier is a barrier, so
// it would not reconverge a warp whose lanes took different paths before it:
// __syncwarp() reconverges the warp first, and the non-aligned form counts
// every thread's arrival on its own.
struct Grp {
  int tid, n, bar;
  __device__ __forceinline__ void sync() const {
    if (bar == 0) {
      __syncthreads();
    } else if (bar < 0) {  // a group of one warp
      __syncwarp();
    } else {
      __syncwarp();
      asm volatile("barrier.sync %0, %1;" ::"r"(bar), "r"(n) : "memory");
    }
  }
  __device__ __forceinline__ int lane() const { return tid & 31; }
  __device__ __forceinline__ int warp() const { return tid >> 5; }
  __device__ __forceinline__ int nwarps() const { return n >> 5; }
};

__device__ __forceinline__ Grp whole_block() { return Grp{(int)threadIdx.x, (int)blockDim.x, 0}; }

// --------------------------------------------------------------- reductions
template <class V>
__device__ __forceinline__ bool better(V av, int aj, V bv, int bj) {
  return av > bv || (av == bv && aj < bj);
}
// FP64 magnitudes compare as signed 64-bit integers: the bit pattern of a
// non-negative double orders like the double, and the negative sentinel
// (sign bit set) is below every one of them.  Integer compares run on the
// ALU pipe, FP64 compares on GB300's narrow FP64 pipe.
template <>
__device__ __forceinline__ bool better<double>(double av, int aj, double bv, int bj) {
  const long long a = __double_as_longlong(av), b = __double_as_longlong(bv);
  return a > b || (a == b && aj < bj);
}

template <class V>
__device__ __forceinline__ void warp_argmax(V& v, int& j) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    V ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oj = __shfl_xor_sync(0xffffffffu, j, o);
    if (better(ov, oj, v, j)) { v = ov; j = oj; }
  }
}

// Group-wide arg-max of (v, j): largest v, smallest j among equal v.  Entries
// with v < 0 are "no candidate".  Returns j (or -1) to every thread of g.
// rv, rj: 34 entries of group-private shared memory.
template <class V>
__device__ int group_argmax(const Grp& g, V v, int j, V* rv, int* rj) {
  warp_argmax(v, j);
  const int lane = g.lane(), w = g.warp(), nw = g.nwarps();
  if (lane == 0) { rv[w] = v; rj[w] = j; }
  g.sync();
  if (w == 0) {
    V vv = lane < nw ? rv[lane] : (V)-1;
    int jj = lane < nw ? rj[lane] : 0x7fffffff;
    warp_argmax(vv, jj);
    if (lane == 0) { rj[32] = vv < (V)0 ? -1 : jj; }
  }
  g.sync();
  const int r = rj[32];
  g.sync();
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Group-wide sums of NV doubles; every thread of g gets the totals.
// red: 32*NV + NV group-private doubles.
template <int NV>
__device__ void group_sum(const Grp& g, double (&v)[NV], double* red) {
  const int lane = g.lane(), w = g.warp(), nw = g.nwarps();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) red[w * NV + i] = v[i];
  }
  g.sync();
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double t = lane < nw ? red[lane * NV + i] : 0.0;
      t = warp_sum(t);
      if (lane == 0) red[32 * NV + i] = t;
    }
  }
  g.sync();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = red[32 * NV + i];
  g.sync();
}

}  // namespace csf
