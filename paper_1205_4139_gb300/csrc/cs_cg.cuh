// FP64 least squares on a column set by conjugate gradients, on a
// thread-block cluster.
//
// Subspace pursuit and CoSaMP solve the normal equations (Algorithm 1.1 step
// 6 applied to a column set T) G_T b = (Phi^H y)(T) = h_0(T) on sets of up to
// 2K and 3K columns, afresh every iteration.  Appending the columns one by
// one to an inverse Cholesky factor costs about (4/3) m^3 FP64 FMAs for m
// columns, 4e10 at m = 3072 (K = 1024).  Conjugate gradients needs only
// products G_T v, whose entries come from the correlation kernel vector
// (G(j, k) = c(j (-) k), Eq. kernelsum applied to columns): 4 m^2 FP64 FMAs
// each, and G_T is well conditioned when the columns are few against M (its
// eigenvalues cluster around c(0) = M/N).
//
// One cluster of G CTAs solves one system.  Every CTA keeps the whole search
// direction p and the column list in shared memory and owns a slice of the
// rows: its rows of G p, and its slices of b, of the residual and of p.  The
// two inner products of an iteration are summed over the cluster in a fixed
// order (each CTA adds its warps' partials, then reads the G CTA partials in
// rank order through distributed shared memory), so every CTA takes the same
// step lengths and the same stopping decision; after each p update the CTAs
// copy the other slices of p from one another.  Three cluster barriers per
// iteration (hardware barriers: no spinning).
#pragma once
#include <cooperative_groups.h>

#include "cs_blocks.cuh"

namespace csf {

namespace cgx = cooperative_groups;

// Cluster-wide FP64 sum of one value per thread; every thread of every CTA
// returns the same total.  red: 32 doubles of block scratch; slot: this
// call site's own shared double (read by the other CTAs after the barrier).
template <int G>
__device__ __forceinline__ double cl_sum(cgx::cluster_group& cl, double v, double* red, double* slot) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *slot = t;
  }
  cl.sync();
  double t = 0.0;
#pragma unroll
  for (int r = 0; r < G; ++r) t += *cl.map_shared_rank(slot, r);
  return t;
}

// out[a - lo] = sum_k G(T[a], T[k]) v[k] for lo <= a < hi, G(j, k) = c(j (-) k)
// from the FP64 kernel vector.  One warp per row, lanes over k (four
// independent loads in flight per lane), fixed summation order.
template <class E>
__device__ __forceinline__ void gram_rows(const PlanDev<E>& P, const int* T, int m,
                                          const typename FT<E>::W* v, int lo, int hi,
                                          typename FT<E>::W* out) {
  using W = typename FT<E>::W;
  constexpr bool DFT = FT<E>::C;
  const int N = P.N, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int a = lo + (int)(threadIdx.x >> 5); a < hi; a += nw) {
    const int ta = T[a];
    W acc[4] = {W{}, W{}, W{}, W{}};
    int k = lane;
    for (; k + 96 < m; k += 128) {
      W cv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int tk = T[k + 32 * u];
        cv[u] = c64_at(P, DFT ? ((ta - tk) & (N - 1)) : (ta ^ tk));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmav(acc[u], cv[u], v[k + 32 * u]);
    }
    for (; k < m; k += 32) {
      const int tk = T[k];
      acc[0] = fmav(acc[0], c64_at(P, DFT ? ((ta - tk) & (N - 1)) : (ta ^ tk)), v[k]);
    }
    double re_ = (re(acc[0]) + re(acc[1])) + (re(acc[2]) + re(acc[3]));
    double im_ = (im(acc[0]) + im(acc[1])) + (im(acc[2]) + im(acc[3]));
    re_ = warp_sum(re_);
    if constexpr (DFT) im_ = warp_sum(im_);
    if (lane == 0) out[a - lo] = make_w<W>(re_, im_);
  }
}

// Shared memory of the solver (bytes, 16-aligned parts): p [mmax], T [mmax],
// and the slices x, r, A p [ceil(mmax / G)] each.
template <class W>
__host__ __device__ inline size_t cg_smem_bytes(int mmax, int G) {
  const size_t sl = (size_t)((mmax + G - 1) / G);
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  return a16((size_t)mmax * sizeof(W)) + a16((size_t)mmax * sizeof(int)) + 3 * a16(sl * sizeof(W));
}

// Relative residual at which the solver stops: 1e-12 for FP64 plans; 1e-10
// for FP32 plans, whose data carry FP32 rounding (about 6e-8 relative) far
// above what the extra iterations would resolve.
template <class E>
__host__ __device__ constexpr double cg_tol() {
  return sizeof(typename FT<E>::R) == 4 ? 1e-10 : 1e-12;
}

struct CgResult {
  double bh;   // Re b^H rhs + Re b^H r: ||y||^2 - ||y - Phi_T b||^2 for the solution b
  double q;    // quadratic form v^H G v (mode 2)
  int iters;
};

// mode 1: solves G_T b = rhs (m columns T, FP64) from the start x0 (nullable:
// zero), to ||rhs - G b|| <= tol ||rhs|| or max_it iterations; b -> xout
// (this CTA's slice; xout may alias x0).  mode 2: q = v^H G_T v for v = x0.
// Every CTA of the cluster must call it with the same arguments.
template <class E, int G>
__device__ CgResult cg_cluster(cgx::cluster_group& cl, const PlanDev<E>& P, const int* Tg, const int m,
                               const typename FT<E>::W* rhs, const typename FT<E>::W* x0,
                               typename FT<E>::W* xout, int mode, double tol, int max_it,
                               unsigned char* sm, int mmax) {
  using W = typename FT<E>::W;
  __shared__ double red[32];
  __shared__ double s_pap, s_rs, s_h, s_fin;
  const int rank = (int)cl.block_rank();
  const int sl = (m + G - 1) / G, lo = rank * sl < m ? rank * sl : m, hi = lo + sl < m ? lo + sl : m;
  const int sla = (mmax + G - 1) / G;
  auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  W* pf = (W*)sm;
  int* T = (int*)(sm + a16((size_t)mmax * sizeof(W)));
  W* xs = (W*)((unsigned char*)T + a16((size_t)mmax * sizeof(int)));
  W* rs = (W*)((unsigned char*)xs + a16((size_t)sla * sizeof(W)));
  W* ap = (W*)((unsigned char*)rs + a16((size_t)sla * sizeof(W)));
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    T[i] = Tg[i];
    pf[i] = x0 ? x0[i] : W{};
  }
  __syncthreads();
  CgResult res{0.0, 0.0, 0};
  if (mode == 2) {  // q = v^H G v
    gram_rows<E>(P, T, m, pf, lo, hi, ap);
    __syncthreads();
    double t = 0.0;
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) t += re(cmul(pf[i], ap[i - lo]));
    res.q = cl_sum<G>(cl, t, red, &s_pap);
    cl.sync();  // no CTA leaves while another still reads its partial
    return res;
  }
  // r = rhs - G x0, x = x0 (slices)
  if (x0) {
    gram_rows<E>(P, T, m, pf, lo, hi, ap);
    __syncthreads();
  }
  double hh = 0.0, rr = 0.0;
  for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
    const W hv = rhs[i];
    const W r = x0 ? sub(hv, ap[i - lo]) : hv;
    xs[i - lo] = pf[i];
    rs[i - lo] = r;
    hh += norm2(hv);
    rr += norm2(r);
  }
  __syncthreads();
  for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) pf[i] = rs[i - lo];  // p = r (own slice)
  const double hn = cl_sum<G>(cl, hh, red, &s_h);
  double rsq = cl_sum<G>(cl, rr, red, &s_rs);
  // the other slices of p
  for (int r = 0; r < G; ++r) {
    if (r == rank) continue;
    const int l0 = r * sl < m ? r * sl : m, l1 = l0 + sl < m ? l0 + sl : m;
    const W* rp = cl.map_shared_rank(pf, r);
    for (int i = l0 + (int)threadIdx.x; i < l1; i += blockDim.x) pf[i] = rp[i];
  }
  __syncthreads();
  const double stop2 = tol * tol * hn;
  int it = 0;
  while (it < max_it && rsq > stop2) {
    gram_rows<E>(P, T, m, pf, lo, hi, ap);
    __syncthreads();
    double t = 0.0;
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) t += re(cmul(pf[i], ap[i - lo]));
    const double pap = cl_sum<G>(cl, t, red, &s_pap);
    if (!(pap > 0.0)) break;  // G_T numerically singular along p: keep the iterate
    const double alpha = rsq / pap;
    double rn = 0.0;
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
      const W pv = pf[i];
      xs[i - lo] = add(xs[i - lo], scale(pv, alpha));
      const W r = sub(rs[i - lo], scale(ap[i - lo], alpha));
      rs[i - lo] = r;
      rn += norm2(r);
    }
    const double rsq_new = cl_sum<G>(cl, rn, red, &s_rs);
    ++it;
    if (!(rsq_new > stop2)) {
      rsq = rsq_new;
      break;
    }
    const double beta = rsq_new / rsq;
    rsq = rsq_new;
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) pf[i] = add(rs[i - lo], scale(pf[i], beta));
    cl.sync();
    for (int r = 0; r < G; ++r) {
      if (r == rank) continue;
      const int l0 = r * sl < m ? r * sl : m, l1 = l0 + sl < m ? l0 + sl : m;
      const W* rp = cl.map_shared_rank(pf, r);
      for (int i = l0 + (int)threadIdx.x; i < l1; i += blockDim.x) pf[i] = rp[i];
    }
    __syncthreads();
  }
  // b -> xout, and Re b^H rhs + Re b^H r over the cluster
  double bh = 0.0;
  for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
    const W xv = xs[i - lo];
    xout[i] = xv;
    bh += re(cmul(xv, rhs[i])) + re(cmul(xv, rs[i - lo]));
  }
  res.bh = cl_sum<G>(cl, bh, red, &s_fin);
  res.iters = it;
  cl.sync();  // no CTA leaves while another still reads its shared memory
  return res;
}

}  // namespace csf
