// Group-wide selection of the k largest keys (the identification step of
// subspace pursuit and CoSaMP: the indices of the k largest |h(j)|, ties to
// the lower index), by an MSB-first radix select over 8-bit digits followed
// by an ordered compaction.  Output indices are in ascending order.
#pragma once
#include "cs_common.cuh"

namespace csf {

// Exclusive prefix over the group's warps of one int per warp (lane 0's v);
// every thread receives its warp's prefix, and *total the sum.
__device__ __forceinline__ int warp_prefix(const Grp& g, int v, int* scratch, int* total) {
  const int w = g.warp(), nw = g.nwarps();
  if (g.lane() == 0) scratch[w] = v;
  g.sync();
  if (g.tid == 0) {
    int s = 0;
    for (int i = 0; i < nw; ++i) {
      const int t = scratch[i];
      scratch[i] = s;
      s += t;
    }
    scratch[32] = s;
  }
  g.sync();
  const int r = scratch[w];
  *total = scratch[32];
  g.sync();
  return r;
}

// Selects the k largest keys[0..n) (ties to the lower index) and writes
// their indices, ascending, to out[0..k).  Requires 0 <= k <= n.  Each warp
// owns a contiguous segment of indices and reads it 32 at a time, so lane
// order is index order and the compaction is a ballot.  hist: 258 ints,
// scratch: 33 ints, both group-private shared memory.
template <class U>
__device__ void group_topk(const Grp& g, const U* keys, int n, int k, int* out, int* hist, int* scratch) {
  constexpr int BITS = (int)sizeof(U) * 8;
  if (k <= 0) return;
  U prefix = 0, mask = 0;
  int need = k;  // keys still to take among those matching prefix
  for (int shift = BITS - 8; shift >= 0; shift -= 8) {
    for (int i = g.tid; i < 256; i += g.n) hist[i] = 0;
    g.sync();
    for (int j = g.tid; j < n; j += g.n) {
      const U kk = keys[j];
      if ((kk & mask) == prefix) atomicAdd(&hist[(int)((kk >> shift) & (U)255)], 1);
    }
    g.sync();
    // the digit: the highest bucket b whose count with all higher buckets'
    // reaches `need` (bucket 0 if none of 255 .. 1 does), and how many keys
    // of it are still needed.  One warp: lane l holds buckets 255 - 8l down
    // to 248 - 8l, a shuffle scan gives every lane the keys above its chunk,
    // and the lane whose chunk crosses `need` walks its eight buckets.
    if (g.warp() == 0) {
      const int l = g.lane(), top = 255 - 8 * l;
      int c[8], sum = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        c[i] = hist[top - i];
        sum += c[i];
      }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += v;
      }
      const int excl = incl - sum;
      if (excl < need && (incl >= need || l == 31)) {  // exactly one lane
        int cum = excl, b = top - 7;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (top - i == 0 || cum + c[i] >= need) {
            b = top - i;
            break;
          }
          cum += c[i];
        }
        hist[256] = b;
        hist[257] = need - cum;
      }
    }
    g.sync();
    const int b = hist[256];
    need = hist[257];
    prefix |= (U)b << shift;
    mask |= (U)255 << shift;
    g.sync();
  }
  // every key > prefix is taken; among keys == prefix the `need` lowest indices
  const int nw = g.nwarps(), w = g.warp(), lane = g.lane();
  const int seg = (((n + nw - 1) / nw) + 31) & ~31;
  const int s0 = w * seg, s1 = min(n, s0 + seg);
  const unsigned lt = (1u << lane) - 1u;
  int eq_cnt = 0;
  for (int base = s0; base < s1; base += 32) {
    const int j = base + lane;
    const bool eq = j < s1 && keys[j] == prefix;
    eq_cnt += __popc(__ballot_sync(0xffffffffu, eq));
  }
  int tot;
  const int eq_before = warp_prefix(g, eq_cnt, scratch, &tot);
  int sel_cnt = 0, er = eq_before;
  for (int base = s0; base < s1; base += 32) {
    const int j = base + lane;
    const U kk = j < s1 ? keys[j] : (U)0;
    const bool eq = j < s1 && kk == prefix;
    const unsigned eqb = __ballot_sync(0xffffffffu, eq);
    const bool sel = j < s1 && (kk > prefix || (eq && er + __popc(eqb & lt) < need));
    sel_cnt += __popc(__ballot_sync(0xffffffffu, sel));
    er += __popc(eqb);
  }
  const int sel_before = warp_prefix(g, sel_cnt, scratch, &tot);
  int pos = sel_before;
  er = eq_before;
  for (int base = s0; base < s1; base += 32) {
    const int j = base + lane;
    const U kk = j < s1 ? keys[j] : (U)0;
    const bool eq = j < s1 && kk == prefix;
    const unsigned eqb = __ballot_sync(0xffffffffu, eq);
    const bool sel = j < s1 && (kk > prefix || (eq && er + __popc(eqb & lt) < need));
    const unsigned sb = __ballot_sync(0xffffffffu, sel);
    if (sel) out[pos + __popc(sb & lt)] = j;
    pos += __popc(sb);
    er += __popc(eqb);
  }
  g.sync();
}

}  // namespace csf
