// Subspace pursuit and CoSaMP on a batch of measurements sharing Omega.
//
// The paper applies its fast correlation to "almost all MPAs" (Sec. I) and
// reports a fast CoSaMP (Sec. IV, Fig. 3) without describing it.  Both
// algorithms here take their standard forms; the step that matters for the
// paper is the correlation h = Phi^H r of each iteration, computed either as
// kernel sums over the current estimate's support, h = h_0 - sum_k x_k
// c(j (-) lambda_k) (Eq. kernelsum: K atoms per iteration, hence the
// constant per-iteration cost the paper notes for CoSaMP), or by transforms.
// One CTA solves one instance at a time:
//   SP      T = top_K(h_0); x = LS_T; repeat: T' = T + top_K(h) over j not in
//           T; b = LS_T'; T_new = top_K(|b|); x_new = LS_T_new; stop, keeping
//           the previous iterate, when ||r_new|| >= ||r||;
//   CoSaMP  x = 0; repeat: T = top_2K(h) + supp(x); b = LS_T; x_new = b on its
//           K largest entries; stop, keeping the previous iterate, when
//           ||r_new|| >= ||r||;
// both also stop when ||r|| < rel_tol ||y|| or after max_iter iterations.
// Least squares on a column set appends its columns, in ascending order, to
// an empty FP64 inverse Cholesky factor (cs_ls.cuh).
#include "cs_cg.cuh"
#include "cs_internal.h"
#include "cs_ls.cuh"
#include "cs_select.cuh"

namespace csf {

namespace {

constexpr int kPThreads = 256;
enum { ALGO_SP = 0, ALGO_COSAMP = 1 };

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

template <class E>
struct PursuitArgs {
  PlanDev<E> P;
  const E* __restrict__ y;
  int64_t batch;
  int K, algo, max_iter, fast;
  double rel_tol;
  typename FT<E>::W* x_out;
  int* supp_out;
  int* iters_out;
  double* res_out;
  E* h0_ws;                  // [grid][N]
  typename FT<E>::W* B_ws;   // [grid][mmax(mmax+1)/2]
  int* counter;
};

__host__ __device__ inline int pursuit_mmax(int K, int algo) { return algo == ALGO_SP ? 2 * K : 3 * K; }
// Column sets larger than this are solved by conjugate gradients (cs_cg.cuh,
// a cluster of one CTA) instead of appending the columns to a factor.
constexpr int kPCgMin = 96;
__host__ __device__ inline bool pursuit_cg(int K, int algo) { return pursuit_mmax(K, algo) > kPCgMin; }

template <class E>
struct PLayout {
  size_t regA, keys, bits, kidx, S, T, sel, xs, xsw, z, x, g, part, lam, sk, hist, scr, red, rv, rj, total;
};

template <class E>
__host__ __device__ inline PLayout<E> pursuit_layout(int N, int K, int algo, int fast) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  using U = typename KeyT<E>::U;
  PLayout<E> L;
  const int Kc = K > 0 ? K : 1;
  const int mm = pursuit_mmax(Kc, algo);
  const int npart = (2 * kPThreads > mm ? 2 * kPThreads : mm);
  size_t o = 0;
  L.regA = o; o = a16(o + (size_t)((fast && kernel_doubled<E>(N)) ? 2 * N : N) * sizeof(E));
  L.keys = o; o = a16(o + (size_t)N * sizeof(U));
  L.bits = o; o = a16(o + (size_t)((N + 31) >> 5) * sizeof(uint32_t));
  L.kidx = o; o = a16(o + (size_t)N * sizeof(uint16_t));
  L.S = o;    o = a16(o + (size_t)Kc * sizeof(int));
  L.T = o;    o = a16(o + (size_t)mm * sizeof(int));
  L.sel = o;  o = a16(o + (size_t)mm * sizeof(int));
  L.xs = o;   o = a16(o + (size_t)Kc * sizeof(W));
  L.xsw = o;  o = a16(o + (size_t)Kc * sizeof(E));
  L.z = o;    o = a16(o + (size_t)mm * sizeof(W));
  L.x = o;    o = a16(o + (size_t)mm * sizeof(W));
  L.g = o;    o = a16(o + (size_t)mm * sizeof(W));
  {  // the append's partial sums, or the conjugate-gradient scratch
    const size_t part = (size_t)npart * sizeof(W) + (size_t)3 * mm * sizeof(double);
    const size_t cgs = cg_smem_bytes<W>(mm, 1);
    L.part = o; o = a16(o + (pursuit_cg(Kc, algo) && cgs > part ? cgs : part));
  }
  L.lam = o;  o = a16(o + (size_t)mm * sizeof(int));
  L.sk = o;   o = a16(o + (size_t)mm * sizeof(unsigned long long));
  L.hist = o; o = a16(o + 258 * sizeof(int));
  L.scr = o;  o = a16(o + 34 * sizeof(int));
  L.red = o;  o = a16(o + (32 * 4 + 4) * sizeof(double));
  L.rv = o;   o = a16(o + 34 * sizeof(V));
  L.rj = o;   o = a16(o + 34 * sizeof(int));
  L.total = o;
  return L;
}

struct PState {
  int ns;        // size of the accepted support S
  int m;         // size of the last column set solved
  int it;
  double ynorm2, rn2, rn2_new, ls_rn2;
};

// Least squares on cols[0..m) (ascending): appends them to an empty factor.
// Coefficients land in v.x[0..m) in the order of v.lam; returns through
// st.m the number actually appended (a column dependent on earlier ones is
// skipped) and ls_rn2 = ||y||^2 - sum |z|^2.
template <class E>
__device__ void ls_set(const Grp& g, const PlanDev<E>& P, const LsView<E>& v, const E* h0, const int* cols, int m,
                       PState& st, LsShared<typename FT<E>::W>& sh) {
  if (g.tid == 0) st.ls_rn2 = st.ynorm2;
  g.sync();
  int p = 0;
  for (int a = 0; a < m; ++a) {
    ls_append(g, P, v, h0, p, cols[a], st.ls_rn2, sh);
    if (sh.st == 0) ++p;
  }
  if (g.tid == 0) st.m = p;
  g.sync();
}

template <class E>
__global__ void __launch_bounds__(kPThreads) pursuit_kernel(PursuitArgs<E> a) {
  using W = typename FT<E>::W;
  using V = typename NormT<E>::V;
  using U = typename KeyT<E>::U;
  constexpr bool DFT = FT<E>::C;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ PState st;
  __shared__ LsShared<W> sh;
  __shared__ int s_inst;
  const int N = a.P.N, M = a.P.M, K = a.K;
  const PLayout<E> L = pursuit_layout<E>(N, K, a.algo, a.fast);
  E* regA = (E*)(sm + L.regA);
  U* keys = (U*)(sm + L.keys);
  uint32_t* bits = (uint32_t*)(sm + L.bits);
  uint16_t* kidx = (uint16_t*)(sm + L.kidx);
  int* S = (int*)(sm + L.S);
  int* T = (int*)(sm + L.T);
  int* sel = (int*)(sm + L.sel);
  W* xs = (W*)(sm + L.xs);
  E* xsw = (E*)(sm + L.xsw);
  unsigned long long* sk = (unsigned long long*)(sm + L.sk);  // FP64 keys of |b|
  int* hist = (int*)(sm + L.hist);
  int* scr = (int*)(sm + L.scr);
  double* red = (double*)(sm + L.red);
  V* rv = (V*)(sm + L.rv);
  int* rj = (int*)(sm + L.rj);
  const int mm = pursuit_mmax(K > 0 ? K : 1, a.algo);
  const int npart = (2 * kPThreads > mm ? 2 * kPThreads : mm);
  LsView<E> lv;
  lv.B = a.B_ws + (size_t)blockIdx.x * (((size_t)mm * (mm + 1)) >> 1);
  lv.z = (W*)(sm + L.z);
  lv.x = (W*)(sm + L.x);
  lv.g = (W*)(sm + L.g);
  lv.part = (W*)(sm + L.part);
  lv.terms = (double*)(lv.part + npart);
  lv.xw = nullptr;
  lv.lam = (int*)(sm + L.lam);
  lv.bits = nullptr;
  lv.kidx = nullptr;
  const Grp g = whole_block();
  const bool dbl = kernel_doubled<E>(N);
  E* h0 = a.h0_ws + (size_t)blockIdx.x * N;
  const double tol2 = a.rel_tol * a.rel_tol;
  const int nbits = (N + 31) >> 5;
  // Large column sets: least squares on cols[0..m) (ascending) by conjugate
  // gradients from lv.x (warm) or zero, right-hand side h_0(cols); results
  // in the append's places (lv.lam, lv.x, st.m, st.ls_rn2).  The scratch
  // takes the append's partial-sum region, the right-hand side its z.
  const bool cgm = pursuit_cg(K > 0 ? K : 1, a.algo);
  cgx::cluster_group cl = cgx::this_cluster();  // a cluster of this one CTA
  auto ls_cg = [&](const int* cols, int m, bool warm) {
    W* rhs = lv.z;
    for (int i = g.tid; i < m; i += g.n) {
      lv.lam[i] = cols[i];
      rhs[i] = to_w(h0[cols[i]]);
    }
    g.sync();
    const int max_it = 2 * m < 64 ? 64 : (2 * m > 4000 ? 4000 : 2 * m);
    const CgResult r = cg_cluster<E, 1>(cl, a.P, lv.lam, m, rhs, warm ? lv.x : nullptr, lv.x, 1, cg_tol<E>(), max_it,
                                        (unsigned char*)lv.part, mm);
    if (g.tid == 0) {
      st.m = m;
      st.ls_rn2 = st.ynorm2 - r.bh;
    }
    g.sync();
  };

  for (;;) {
    if (g.tid == 0) s_inst = atomicAdd(a.counter, 1);
    g.sync();
    const int64_t b = s_inst;
    g.sync();
    if (b >= a.batch) break;
    const E* y = a.y + b * M;
    double yy[1] = {0.0};
    correlate_transform<E, DFT, true>(g, regA, a.P, y, h0, yy, rv, rj);  // h_0 kept in the workspace
    group_sum(g, yy, red);
    if (g.tid == 0) {
      st.ynorm2 = yy[0];
      st.rn2 = yy[0];
      st.ns = 0;
      st.it = 0;
    }
    g.sync();
    if (yy[0] > 0.0 && K > 0) {
      if (a.algo == ALGO_SP) {
        // T_0 = top_K(h_0), x = LS on T_0
        for (int j = g.tid; j < N; j += g.n) keys[j] = sel_key((V)norm2(h0[j]));
        g.sync();
        group_topk(g, keys, N, K, S, hist, scr);
        if (cgm) ls_cg(S, K, false);
        else ls_set(g, a.P, lv, h0, S, K, st, sh);
        for (int k = g.tid; k < st.m; k += g.n) { S[k] = lv.lam[k]; xs[k] = lv.x[k]; }
        if (g.tid == 0) { st.ns = st.m; st.rn2 = st.ls_rn2; }
        g.sync();
      }
      bool c_loaded = false;
      while (st.it < a.max_iter && st.rn2 >= tol2 * st.ynorm2) {
        const int ns = st.ns;
        // correlation with the current estimate: keys over j (SP excludes S)
        for (int i = g.tid; i < nbits; i += g.n) bits[i] = 0u;
        g.sync();
        for (int k = g.tid; k < ns; k += g.n) {
          xsw[k] = from_w<E>(xs[k]);
          kidx[S[k]] = (uint16_t)k;
          atomicOr(bits + (S[k] >> 5), 1u << (S[k] & 31));
        }
        g.sync();
        const uint32_t* excl = a.algo == ALGO_SP ? bits : nullptr;
        if (a.fast) {
          if (!c_loaded) { load_kernel_vector<E, DFT>(g, regA, a.P, dbl); c_loaded = true; }
          correlate_fast<E, DFT>(g, regA, h0, S, xsw, ns, N, excl, nullptr, rv, rj, dbl, keys);
        } else {
          correlate_residual<E, DFT>(g, regA, a.P, y, bits, kidx, xsw, rv, rj, excl, keys);
        }
        // candidate set
        int m;
        if (a.algo == ALGO_SP) {
          group_topk(g, keys, N, K, sel, hist, scr);
          // T' = S + sel (both ascending, disjoint): merge
          if (g.tid == 0) {
            int i = 0, j = 0, o = 0;
            while (i < ns || j < K) T[o++] = (j >= K || (i < ns && S[i] < sel[j])) ? S[i++] : sel[j++];
            st.m = o;
          }
        } else {
          group_topk(g, keys, N, 2 * K, sel, hist, scr);
          // T = top_2K + S (both ascending): merge without duplicates
          if (g.tid == 0) {
            int i = 0, j = 0, o = 0;
            while (i < ns || j < 2 * K) {
              int v;
              if (j >= 2 * K || (i < ns && S[i] < sel[j])) v = S[i++];
              else if (i < ns && S[i] == sel[j]) { v = S[i++]; ++j; }
              else v = sel[j++];
              T[o++] = v;
            }
            st.m = o;
          }
        }
        g.sync();
        m = st.m;
        if (cgm) {  // b = LS on T from the support's coefficients (zero on the new columns)
          for (int i = g.tid; i < m; i += g.n) {
            const int j = T[i];
            lv.x[i] = in_bits(bits, j) ? xs[kidx[j]] : W{};
          }
          g.sync();
          ls_cg(T, m, true);
        } else {
          ls_set(g, a.P, lv, h0, T, m, st, sh);          // b = LS on T (lv.lam, lv.x)
        }
        m = st.m;
        // prune: the K entries of b with the largest |b| (ties to the lower column)
        for (int i = g.tid; i < m; i += g.n) sk[i] = sel_key(norm2(lv.x[i]));
        g.sync();
        const int kk = K < m ? K : m;
        group_topk(g, sk, m, kk, sel, hist, scr);
        // sel holds positions (ascending) in lv.lam, i.e. ascending columns
        for (int i = g.tid; i < kk; i += g.n) T[i] = lv.lam[sel[i]];
        if (a.algo == ALGO_COSAMP) {
          for (int i = g.tid; i < kk; i += g.n) lv.g[i] = lv.x[sel[i]];  // pruned coefficients
        }
        g.sync();
        if (a.algo == ALGO_SP) {
          // T_new equal to the accepted support (both ascending): x_new and
          // its residual are the accepted ones (the same solve in the same
          // column order), so the iteration is rejected without solving
          if (g.tid == 0) {
            bool same = kk == st.ns;
            for (int i = 0; same && i < kk; ++i) same = T[i] == S[i];
            scr[0] = same;
          }
          g.sync();
          if (scr[0]) {
            if (g.tid == 0) st.rn2_new = st.rn2;
            g.sync();
          } else {
            if (cgm) {  // x_new = LS on T_new from b's values there
              for (int i = g.tid; i < kk; i += g.n) lv.g[i] = lv.x[sel[i]];
              g.sync();
              for (int i = g.tid; i < kk; i += g.n) lv.x[i] = lv.g[i];
              g.sync();
              ls_cg(T, kk, true);
            } else {
              ls_set(g, a.P, lv, h0, T, kk, st, sh);        // x_new = LS on T_new
            }
            if (g.tid == 0) st.rn2_new = st.ls_rn2;
            g.sync();
          }
        } else {
          // ||y - Phi x||^2 = ||y||^2 - 2 Re x^H h_0(S) + x^H G_S x  (FP64)
          double acc[2] = {0.0, 0.0};
          for (int i = g.tid; i < kk; i += g.n) {
            const W xi = lv.g[i];
            const W hi = to_w(h0[T[i]]);
            acc[0] += re(cmul(xi, hi));
            W gx = W{};
            for (int j = 0; j < kk; ++j) {
              const int d = DFT ? ((T[i] - T[j]) & (N - 1)) : (T[i] ^ T[j]);
              gx = fmav(gx, c64_at(a.P, d), lv.g[j]);
            }
            acc[1] += re(cmul(xi, gx));
          }
          group_sum(g, acc, red);
          if (g.tid == 0) { st.rn2_new = st.ynorm2 - 2.0 * acc[0] + acc[1]; st.m = kk; }
          g.sync();
        }
        const bool accept = st.rn2_new < st.rn2;
        g.sync();
        if (g.tid == 0) st.it = st.it + 1;
        if (!accept) { g.sync(); break; }
        if (a.algo == ALGO_SP) {
          const int ms = st.m;
          for (int i = g.tid; i < ms; i += g.n) { S[i] = lv.lam[i]; xs[i] = lv.x[i]; }
          if (g.tid == 0) { st.ns = ms; st.rn2 = st.rn2_new; }
        } else {
          for (int i = g.tid; i < kk; i += g.n) { S[i] = T[i]; xs[i] = lv.g[i]; }
          if (g.tid == 0) { st.ns = kk; st.rn2 = st.rn2_new; }
        }
        g.sync();
      }
    }
    // outputs: support ascending, FP64 coefficients
    const int ns = st.ns;
    for (int k = g.tid; k < K; k += g.n) {
      if (a.x_out) a.x_out[b * K + k] = k < ns ? xs[k] : W{};
      a.supp_out[b * K + k] = k < ns ? S[k] : -1;
    }
    if (g.tid == 0) {
      if (a.iters_out) a.iters_out[b] = st.it;
      if (a.res_out) a.res_out[b] = st.ynorm2 > 0.0 ? sqrt(fmax(st.rn2, 0.0) / st.ynorm2) : 0.0;
    }
    g.sync();
  }
}

template <class E>
size_t psmem_t(const PlanView& P, int K, int algo, int fast) {
  return pursuit_layout<E>(P.N, K, algo, fast).total;
}

template <class E>
int pgrid_t(const PlanView& P, int K, int algo, int fast, int64_t batch, int* err) {
  const size_t smem = psmem_t<E>(P, K, algo, fast);
  *err = 0;
  cudaError_t e = raise_smem_limit((const void*)pursuit_kernel<E>, smem);
  if (e != cudaSuccess) { *err = (int)e; return 0; }
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pursuit_kernel<E>, kPThreads, smem);
  if (e != cudaSuccess) { *err = (int)e; return 0; }
  if (occ < 1) { *err = (int)cudaErrorInvalidConfiguration; return 0; }
  const int64_t cap = (int64_t)occ * sms;
  return (int)(batch < cap ? batch : cap);
}

size_t pes(const PlanView& P) { return (P.dft ? 2 : 1) * (P.fp32 ? 4 : 8); }
size_t pws(const PlanView& P) { return P.dft ? 16 : 8; }

template <class E>
cudaError_t pursuit_impl(const PlanView& P, const PursuitLaunch& L, void* ws, int grid, cudaStream_t st) {
  using W = typename FT<E>::W;
  PursuitArgs<E> a;
  a.P = plan_dev<E>(P);
  a.y = (const E*)L.y;
  a.batch = L.batch;
  a.K = L.K;
  a.algo = L.algo;
  a.max_iter = L.max_iter;
  a.fast = L.fast;
  a.rel_tol = L.rel_tol;
  a.x_out = (W*)L.x_out;
  a.supp_out = L.supp_out;
  a.iters_out = L.iters_out;
  a.res_out = L.res_out;
  char* w = (char*)ws;
  a.counter = (int*)w;
  a.h0_ws = (E*)(w + 16);
  a.B_ws = (W*)(w + 16 + a16((size_t)grid * P.N * sizeof(E)));
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  pursuit_kernel<E><<<grid, kPThreads, psmem_t<E>(P, L.K, L.algo, L.fast), st>>>(a);
  return cudaGetLastError();
}

}  // namespace

int pursuit_grid(const PlanView& P, int K, int algo, int fast, int64_t batch, int* err) {
  if (P.dft) return P.fp32 ? pgrid_t<float2>(P, K, algo, fast, batch, err) : pgrid_t<double2>(P, K, algo, fast, batch, err);
  return P.fp32 ? pgrid_t<float>(P, K, algo, fast, batch, err) : pgrid_t<double>(P, K, algo, fast, batch, err);
}

size_t pursuit_workspace_bytes(const PlanView& P, int K, int algo, int grid) {
  const size_t mm = (size_t)pursuit_mmax(K > 0 ? K : 1, algo);
  const size_t fac = pursuit_cg(K > 0 ? K : 1, algo) ? 0 : (mm * (mm + 1) / 2) * pws(P);
  return 16 + a16((size_t)grid * P.N * pes(P)) + a16((size_t)grid * fac);
}

cudaError_t launch_pursuit(const PlanView& P, const PursuitLaunch& a, void* ws, int grid, cudaStream_t st) {
  if (a.batch <= 0) return cudaSuccess;
  if (P.dft) return P.fp32 ? pursuit_impl<float2>(P, a, ws, grid, st) : pursuit_impl<double2>(P, a, ws, grid, st);
  return P.fp32 ? pursuit_impl<float>(P, a, ws, grid, st) : pursuit_impl<double>(P, a, ws, grid, st);
}

}  // namespace csf
