// Host-side interface between the C ABI (cs_api.cu) and the kernel
// launchers (cs_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace csf {

constexpr int kThreads = 256;
constexpr int kMaxLogN = 13;       // N <= 8192: one instance per CTA
constexpr int kMaxLogNLarge = 24;  // four-step transforms through global memory
constexpr int kMaxK = 1024;
constexpr int kMaxKLarge = 4096;       // large plans: the factor lives in global memory
constexpr int kMaxLargeBatch = 65535;  // large plans: instances per call
constexpr int kMaxPursuitK = 128;       // SP / CoSaMP, N <= 8192: one CTA appends the columns
constexpr int kMaxPursuitKLarge = 1024; // SP / CoSaMP, large plans: conjugate-gradient least squares
constexpr int kMaxLogNMulti = 16;      // cs_omp_batched: one CTA per instance up to N = 2^16

// Type-erased view of a plan's device tables.
struct PlanView {
  int N, logN, M;
  bool dft, fp32;
  const int* slot;
  const void* tw64;   // double2 [N] (DFT)
  const void* tw32;   // float2 [N]  (DFT, FP32)
  const void* c64;    // double / double2 [N]
  const void* c32;    // float / float2 [N] (FP32)
  int* status;        // device status word (kernel-detected errors), owned by the plan
  // large plans (logN > kMaxLogN): N = N1 N2 with N1 = 2^n1, N2 = 2^n2; the
  // slot map is in natural order and lt64 / lt32 hold, one after the other,
  // the DIF twiddles of the N1 chain, of the N2 chain, then w_N^m for
  // m < 2^wsh and w_N^(m 2^wsh) for m < N / 2^wsh (DFT only)
  bool large;
  int n1, n2, wsh;
  const void* lt64;
  const void* lt32;
  // storage of c: CFMT_FULL c64 / c32 hold c(0..N-1); CFMT_HALF (DFT) hold
  // c(0..N/2) and c(N - d) = conj(c(d)); CFMT_INT (WHT) ci holds the exact
  // integers N c(d) and c64 / c32 are unused
  int cfmt;
  const int* ci;
  // WHT FP32, 16 <= N <= 4096: cs_correlate runs the radix-16 Hadamard
  // stages on the tensor cores (CS_PLAN_TENSOR_CORES)
  bool tc;
  // the one-CTA radix-16 chains (N <= 2^16): slot map in the chains' position
  // order and, for DFT, the chains' twiddles (FP64 / FP32).  For N <= 8192
  // these are slot / tw64 / tw32; for 8192 < N <= 2^16 the slot map is the
  // plan's own and the twiddles are shared by all plans of that N; NULL above.
  const int* slot_chain;
  const void* ctw64;
  const void* ctw32;
  // large plans: Omega grouped by the row of the four-step view that pass 2
  // produces it in (DFT: j mod N1, WHT: j / N2): entries om_ent[om_off[r] ..
  // om_off[r + 1]) = (j, m) with j = Omega_m
  const int* om_off;
  const int2* om_ent;
  // large plans: Omega grouped by the pass-1 column of the four-step view
  // (j mod N2): entries oc_ent[oc_off[c] .. oc_off[c + 1]) = (j, m)
  const int* oc_off;
  const int2* oc_ent;
};

enum { CFMT_FULL = 0, CFMT_HALF = 1, CFMT_INT = 2 };

// Bits of the device status word.
constexpr int kStatusPhaseBound = 1;  // the OMP kernel's phase loop hit its bound
constexpr int kStatusTcTimeout = 2;   // a tensor-core transform's MMAs did not complete in time

struct OmpLaunch {
  const void* y;
  int64_t batch;
  int K;
  double rel_tol;
  int path, t_switch;
  void* x_out;
  int* supp_out;
  int* iters_out;
  double* res_out;
};

struct PursuitLaunch {
  const void* y;
  int64_t batch;
  int K, algo, max_iter, fast;  // algo: 0 subspace pursuit, 1 CoSaMP
  double rel_tol;
  void* x_out;
  int* supp_out;
  int* iters_out;
  double* res_out;
};

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device.  The limit is a property of the kernel shared by every
// thread of the process, so it only ever grows, under a lock: callers with
// different needs (the request runtime's workers) never lower it under one
// another between setting it and launching.
cudaError_t raise_smem_limit(const void* func, size_t bytes);
// Streams the library forks work onto (a few per device), created on first use.
cudaError_t fork_stream(int dev, int k, cudaStream_t* out);

// plan construction
cudaError_t launch_twiddles(const PlanView& P, void* tw64, void* tw32, cudaStream_t st);
cudaError_t launch_twiddles_log(int logN, void* tw64, void* tw32, cudaStream_t st);
cudaError_t launch_round(bool dft, const void* c64, void* c32, int n, cudaStream_t st);
// c from its full FP64 vector into the plan's storage format, and back
cudaError_t launch_compress_c(const PlanView& P, const void* full64, void* c64, void* c32, int* ci, cudaStream_t st);
cudaError_t launch_expand_c(const PlanView& P, void* out, bool fp32, cudaStream_t st);
cudaError_t launch_kernel_vector(const PlanView& P, void* c64_full, cudaStream_t st);

// transforms / correlations
// FP32 FMA-pipe probe (cs_fma_probe): queues the kernel, returns its flop count.
cudaError_t launch_fma_probe(int iters, float* sink, cudaStream_t st, double* flops);
// Conventional correlation of partial-WHT FP32 plans (16 <= N <= 4096) with
// the radix-16 Hadamard stages on the tensor cores (cs_wht_tc.cu), for plans
// created with CS_PLAN_TENSOR_CORES.
bool wht_tc_applies(const PlanView& P);
cudaError_t launch_correlate_wht_tc(const PlanView& P, const void* r, int64_t batch, void* h, int32_t* amax,
                                    cudaStream_t st);
cudaError_t launch_correlate(const PlanView& P, const void* r, int64_t batch, void* h, int32_t* amax,
                             cudaStream_t st);
cudaError_t launch_correlate_fast(const PlanView& P, const void* h0, const int32_t* supp, const void* x,
                                  int s, int64_t batch, void* h, int32_t* amax, cudaStream_t st);

// OMP: workspace sizing then launch
size_t omp_smem_bytes(const PlanView& P, int K, int path);
int omp_grid(const PlanView& P, int K, int path, int64_t batch, int* err);
size_t omp_workspace_bytes(const PlanView& P, int K, int grid);
cudaError_t launch_omp(const PlanView& P, const OmpLaunch& a, void* ws, int grid, cudaStream_t st);

// OMP on small batches, one cluster of CTAs per instance (cs_omp_cluster.cu)
constexpr int kClusterMaxBatch = 19;  // up to 152 CTAs: one wave of 8-CTA clusters
constexpr int kClusterMaxK = 256;     // every CTA keeps its own FP64 factor
size_t omp_cluster_smem(const PlanView& P, int K, int path);
size_t omp_cluster_workspace_bytes(const PlanView& P, int K, int64_t batch);
cudaError_t launch_omp_cluster(const PlanView& P, const OmpLaunch& a, void* ws, cudaStream_t st);

// OMP on instances with their own plans (cs_omp_multi.cu).  One item per
// instance; items of one element type go to one launch.
struct MultiItem {
  const PlanView* P;
  const void* y;
  void* x;
  int* supp;
  int K, t_switch, idx;
  double cost;  // estimated work, for the longest-first order
};
// Chain twiddles of the one-CTA radix-16 DFT chains for N = 2^logN, built on
// first use per device and kept until the process exits.
cudaError_t chain_twiddles(int logN, cudaStream_t st, const void** tw64, const void** tw32);
// Switch point of instances whose buffers live in global memory (N > 8192).
int multi_switch_big(int logN);
double multi_cost(const PlanView& P, int K, int t_switch, int path);
size_t omp_multi_smem(const MultiItem* it, int64_t n, int path);
// ctas_per_sm: resident CTAs per SM (0: as many as fit)
cudaError_t launch_omp_multi(MultiItem* it, int64_t n, double rel_tol, int path, int ctas_per_sm, int* iters_out,
                             double* res_out, int* status, cudaStream_t st);
// CTAs per SM a launch of these instances (one element type and residence) can hold
int omp_multi_occupancy(const MultiItem* it, int64_t n, int path, int* err);

// large plans (cs_large.cu)
cudaError_t large_tables(const PlanView& P, void* lt64, void* lt32, cudaStream_t st);
cudaError_t large_kernel_vector(const PlanView& P, void* c64_full, void* tmp, cudaStream_t st);
size_t large_correlate_ws(const PlanView& P, int64_t batch);
cudaError_t large_correlate(const PlanView& P, const void* r, int64_t batch, void* h, int32_t* amax, void* ws,
                            cudaStream_t st);
size_t large_fast_ws(const PlanView& P, int64_t batch);
cudaError_t large_correlate_fast(const PlanView& P, const void* h0, const int32_t* supp, const void* x, int s,
                                 int64_t batch, void* h, int32_t* amax, void* ws, cudaStream_t st);
size_t large_omp_ws(const PlanView& P, int K, int path, int64_t batch);
cudaError_t large_omp(const PlanView& P, const OmpLaunch& a, void* ws, cudaStream_t st);
size_t large_pursuit_ws(const PlanView& P, int K, int algo, int fast, int64_t batch);
cudaError_t large_pursuit(const PlanView& P, const PursuitLaunch& a, void* ws, cudaStream_t st);

// subspace pursuit / CoSaMP
int pursuit_grid(const PlanView& P, int K, int algo, int fast, int64_t batch, int* err);
size_t pursuit_workspace_bytes(const PlanView& P, int K, int algo, int grid);
cudaError_t launch_pursuit(const PlanView& P, const PursuitLaunch& a, void* ws, int grid, cudaStream_t st);

}  // namespace csf
