// FP64 least squares (Algorithm 1.1 step 6) one column at a time.
//
// With G_p = Phi_p^H Phi_p = L L^H for the p columns chosen so far, the
// library keeps B = L^{-1} (packed lower triangle, row i at i(i+1)/2),
// z = L^{-1} b with b_k = (Phi^H y)(lambda_k) = h_0(lambda_k), and x = B^H z.
// Appending column lambda with Gram column g_k = c(lambda_k (-) lambda)
// (Eq. kernelsum applied to columns):
//   u = B g,  d^2 = c(0) - ||u||^2,  zeta = (b_p - u^H z) / d,
//   row p of B = [-(u^H B) / d, 1 / d],   x += zeta * conj(row p of B),
//   ||r||^2 -= |zeta|^2.
// OMP appends one column per iteration; subspace pursuit and CoSaMP solve on
// a fresh column set by appending its columns to an empty factor.
#pragma once
#include "cs_blocks.cuh"

namespace csf {

template <class E>
struct LsView {
  using W = typename FT<E>::W;
  W* B;            // packed inverse factor
  W* z;            // [K] L^{-1} b
  W* x;            // [K] coefficients, FP64
  W* g;            // [K] Gram column, then u
  W* part;         // partial sums, max(2 n, K) elements
  double* terms;   // 3 doubles per k
  E* xw;           // [K] x in the working precision (nullable)
  int* lam;        // [K] columns in append order
  uint32_t* bits;  // support bitmap (nullable)
  uint16_t* kidx;  // position -> index in lam (nullable)
};

template <class W>
struct LsShared {
  double invd;
  W zeta;
  int st;  // 0 appended, 1 column dependent on the others (not appended)
};

// Appends column l as the p-th column.  h0 holds (Phi^H y) in the working
// precision (the right-hand side entry is h0[l]); rn2 (shared) is ||r||^2,
// downdated by |zeta|^2.  Every thread of g returns with sh.st set.
template <class E>
__device__ void ls_append(const Grp& g, const PlanDev<E>& P, const LsView<E>& v, const E* h0, int p, int l,
                          double& rn2, LsShared<typename FT<E>::W>& sh) {
  using W = typename FT<E>::W;
  constexpr bool DFT = FT<E>::C;
  const int N = P.N;
  const double c0 = re(c64_at(P, 0));                    // c(0) = M/N
  const double dep = 1e-10 * ((double)P.M / (double)N);  // dependence threshold on d^2
  for (int k = g.tid; k < p; k += g.n) {
    const int d = DFT ? ((v.lam[k] - l) & (N - 1)) : (v.lam[k] ^ l);
    v.g[k] = c64_at(P, d);                                // G(lambda_k, lambda)
  }
  g.sync();
  // g <- u = B g; the finishing threads leave |u_k|^2 and conj(u_k) z_k in terms
  tri_matvec(g, v.B, v.g, v.part, p, v.z, v.terms);
  // d^2 and u^H z: the group's last warp adds the terms and one of its
  // threads runs the scalar FP64 work (an FP64 warp instruction costs the
  // same whatever its active lanes; the first warps carry the low-k combines)
  if (g.warp() == g.nwarps() - 1) {
    double an = 0.0, ar = 0.0, ai = 0.0;
    for (int k = g.lane(); k < p; k += 32) {
      an += v.terms[3 * k];
      ar += v.terms[3 * k + 1];
      ai += v.terms[3 * k + 2];
    }
    an = warp_sum(an);
    ar = warp_sum(ar);
    if constexpr (DFT) ai = warp_sum(ai);
    if (g.lane() == 0) {
      const double d2 = c0 - an;
      if (!(d2 > dep)) {
        sh.st = 1;
      } else {
        const double invd = rsqrt(d2);
        const W bp = to_w(h0[l]);                         // (Phi^H y)(lambda)
        const W zeta = scale(sub(bp, make_w<W>(ar, ai)), invd);
        rn2 -= norm2(zeta);
        sh.invd = invd;
        sh.zeta = zeta;
        sh.st = 0;
      }
    }
  }
  g.sync();
  if (sh.st == 1) return;
  const double invd = sh.invd;
  const W zeta = sh.zeta;
  tri_vecmat_row(g, v.B, v.g, v.part, p, -invd);         // row p of B (part[0..p))
  for (int k = g.tid; k < p; k += g.n) {
    const W xk = fmacv(v.x[k], v.part[k], zeta);
    v.x[k] = xk;
    if (v.xw) v.xw[k] = from_w<E>(xk);
  }
  if (g.tid == 0) {
    v.B[pidx(p) + p] = make_w<W>(invd, 0.0);
    v.z[p] = zeta;
    const W xp = scale(zeta, invd);
    v.x[p] = xp;
    if (v.xw) v.xw[p] = from_w<E>(xp);
    v.lam[p] = l;
    if (v.kidx) v.kidx[l] = (uint16_t)p;
    if (v.bits) v.bits[l >> 5] |= 1u << (l & 31);
  }
  g.sync();
}

}  // namespace csf
