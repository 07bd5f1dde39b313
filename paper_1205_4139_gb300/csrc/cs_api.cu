// C ABI of libcsfast.so (declared in include/csfast.h): argument checks,
// plan tables, workspace management and launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/csfast.h"
#include "cs_internal.h"
#include "cs_transform.cuh"

using namespace csf;

struct cs_plan_s {
  PlanView v;
  int kind, prec;
  int device;
  int t_switch_default;
  int t_switch_tuned = -1;  // set by cs_plan_tune
  int* d_slot = nullptr;
  int* d_slot_chain = nullptr;  // 8192 < N <= 2^16, DFT: slot map in the one-CTA chains' order
  int* d_om_off = nullptr;      // large plans: Omega by pass-2 row (offsets)
  int2* d_om_ent = nullptr;     //   and entries (j, m)
  int* d_oc_off = nullptr;      // large plans: Omega by pass-1 column (offsets)
  int2* d_oc_ent = nullptr;     //   and entries (j, m)
  void* d_tw64 = nullptr;
  void* d_tw32 = nullptr;
  void* d_c64 = nullptr;
  void* d_c32 = nullptr;
  int* d_ci = nullptr;      // CFMT_INT: N c(d)
  size_t table_bytes = 0;   // device bytes of the plan's tables (cs_plan_memory)
  void* d_lt64 = nullptr;   // large plans: four-step tables (FP64)
  void* d_lt32 = nullptr;   // large plans: four-step tables (FP32)
  int* d_status = nullptr;  // kernel-detected errors (cs_plan_status)
  void* ws = nullptr;       // OMP workspace (grows on demand, stream-ordered)
  size_t ws_bytes = 0;
  bool ordered = false;     // every buffer stream-ordered on `home` (request runtime)
  cudaStream_t home = nullptr;
};

static thread_local char g_err[256] = "";

static cs_status cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? CS_ERR_NOMEM : CS_ERR_CUDA;
}

#define CS_CUDA(call, what)                       \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

static size_t elem_bytes(int kind, int prec) { return (kind == CS_DFT ? 2 : 1) * (prec == CS_FP32 ? 4 : 8); }

extern "C" const char* cs_status_string(cs_status s) {
  switch (s) {
    case CS_OK: return "ok";
    case CS_ERR_INVALID: return "invalid argument";
    case CS_ERR_NOMEM: return "device allocation failed";
    case CS_ERR_CUDA: return "CUDA error";
    case CS_ERR_UNSUPPORTED: return "size beyond the kernels' limits";
  }
  return "unknown status";
}

extern "C" const char* cs_last_error(void) { return g_err; }

namespace csf {
cudaError_t raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit, static_bytes;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, func);
  // without the attribute a launch may use 48 KB of shared memory in all,
  // the kernel's static shared memory included
  auto it = static_bytes.find(key);
  if (it == static_bytes.end()) {
    cudaFuncAttributes fa;
    const cudaError_t ea = cudaFuncGetAttributes(&fa, func);
    if (ea != cudaSuccess) return ea;
    it = static_bytes.emplace(key, fa.sharedSizeBytes).first;
  }
  if (bytes + it->second <= 48 * 1024) return cudaSuccess;
  size_t& cur = limit[key];
  if (cur >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// Streams the library forks work onto (a few per device), created on first
// use and kept until the process exits.
cudaError_t fork_stream(int dev, int k, cudaStream_t* out) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, cudaStream_t> pool;
  std::lock_guard<std::mutex> lk(mu);
  cudaStream_t& s = pool[std::make_pair(dev, k)];
  if (!s) {
    const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      s = nullptr;
      return e;
    }
  }
  *out = s;
  return cudaSuccess;
}

// accessors for the other translation units of the library
const PlanView* plan_view(cs_plan_t plan) { return &plan->v; }
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
}  // namespace csf

// Crossover of the two correlations measured on GB300 (python -m
// switch_curves.py: OMP per-iteration cost of kernel sums
// and of transforms versus t, M = N/4, partial DFT and WHT): the t above
// which transforms are cheaper per iteration, by log2 N.  One-CTA plans
// (batches of instances in shared memory) cross near 64.  A large plan (one
// instance spread over the GPU) measured alone crosses late for N <= 2^18,
// where the least squares and the launches shared by both paths dominate an
// iteration, and near 100 from N = 2^20 on; the default switches earlier for
// N <= 2^19 (128 to 160), because several solves at once (the request
// runtime) share L2, which the kernel sums stream c through, and the
// transform path's cost does not grow with t.
static int gb300_switch(int logN) {
  if (logN <= kMaxLogN) return 64;
  static const int table[] = {160, 128, 128, 128, 128, 128, 96, 96, 96, 96, 96};  // log2 N = 14 .. 24
  const int i = logN - 14;
  return table[i < 0 ? 0 : (i > 10 ? 10 : i)];
}

// Switch point used when a call passes t_switch < 0: the one cs_plan_tune
// measured for this plan, else the GB300 crossover table.
static int plan_switch(const cs_plan_s* p) {
  return p->t_switch_tuned >= 0 ? p->t_switch_tuned : gb300_switch(p->v.logN);
}

namespace csf {
// the switch point of calls with t_switch < 0, for the other translation units
int plan_switch_point(cs_plan_t plan) { return plan_switch(plan); }
}  // namespace csf

// Launch shapes of the uneven-batch launches that cs_omp_batched_tune
// measured, per device and launch group (element type and residence):
// resident CTAs per SM (0: as many as fit) and the switch point of calls with
// t_switch < 0 (-1: the plan's, or 32 in global memory).
namespace {
struct BatchShape {
  int ctas_per_sm = 0, t_switch = -1;
};
std::mutex g_shape_mu;
std::map<std::pair<int, int>, BatchShape> g_shape;
BatchShape batch_shape(int dev, int group) {
  std::lock_guard<std::mutex> lk(g_shape_mu);
  auto it = g_shape.find(std::make_pair(dev, group));
  return it == g_shape.end() ? BatchShape{} : it->second;
}
void set_batch_shape(int dev, int group, BatchShape s) {
  std::lock_guard<std::mutex> lk(g_shape_mu);
  g_shape[std::make_pair(dev, group)] = s;
}
// launch group of a plan: DFT 4, FP64 2, global-memory residence 1
size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
int batch_group(const csf::PlanView& v) { return (v.dft ? 4 : 0) + (v.fp32 ? 0 : 2) + (v.large ? 1 : 0); }
}  // namespace

static void plan_free(cs_plan_s* p) {
  if (!p) return;
  void* bufs[] = {p->d_slot, p->d_slot_chain, p->d_om_off, p->d_om_ent, p->d_oc_off, p->d_oc_ent, p->d_tw64, p->d_tw32,
                  p->d_c64,  p->d_c32,        p->d_ci,     p->d_lt64,   p->d_lt32, p->d_status, p->ws};
  for (void* b : bufs) {
    if (!b) continue;
    if (p->ordered) cudaFreeAsync(b, p->home);
    else cudaFree(b);
  }
  delete p;
}

// Device allocation for a plan: plain, or stream-ordered on its home stream
// (no device-wide synchronisation when it is released).
static cudaError_t plan_alloc(cs_plan_s* p, void** ptr, size_t bytes) {
  p->table_bytes += bytes;
  return p->ordered ? cudaMallocAsync(ptr, bytes, p->home) : cudaMalloc(ptr, bytes);
}

// Grows the plan's workspace to `need` bytes (stream-ordered).
static cs_status ensure_ws(cs_plan_s* plan, size_t need, cudaStream_t st) {
  if (need <= plan->ws_bytes) return CS_OK;
  if (plan->ws) CS_CUDA(cudaFreeAsync(plan->ws, st), "cudaFreeAsync workspace");
  plan->ws = nullptr;
  plan->ws_bytes = 0;
  CS_CUDA(cudaMallocAsync(&plan->ws, need, st), "cudaMallocAsync workspace");
  plan->ws_bytes = need;
  return CS_OK;
}

static cs_status plan_create_impl(int64_t N, const int32_t* omega_host, int64_t M, int32_t kind, int32_t prec,
                                  uint32_t flags, void* stream, bool ordered, cs_plan_t* out) {
  if (!out) return CS_ERR_INVALID;
  *out = nullptr;
  if (flags & ~(uint32_t)(CS_PLAN_C_HALF | CS_PLAN_C_INT | CS_PLAN_TENSOR_CORES)) return CS_ERR_INVALID;
  if ((flags & CS_PLAN_TENSOR_CORES) && (kind != CS_WHT || prec != CS_FP32)) return CS_ERR_INVALID;
  if ((flags & CS_PLAN_C_HALF) && kind != CS_DFT) return CS_ERR_INVALID;
  if ((flags & CS_PLAN_C_INT) && kind != CS_WHT) return CS_ERR_INVALID;
  if (kind != CS_WHT && kind != CS_DFT) return CS_ERR_INVALID;
  if (prec != CS_FP64 && prec != CS_FP32) return CS_ERR_INVALID;
  if (N < 1 || (N & (N - 1))) return CS_ERR_INVALID;
  if (M < 0 || M > N) return CS_ERR_INVALID;
  if (M > 0 && !omega_host) return CS_ERR_INVALID;
  for (int64_t m = 0; m < M; ++m) {
    if (omega_host[m] < 0 || omega_host[m] >= N) return CS_ERR_INVALID;
    if (m > 0 && omega_host[m] <= omega_host[m - 1]) return CS_ERR_INVALID;
  }
  int logN = 0;
  while ((int64_t(1) << logN) < N) ++logN;
  if (logN > kMaxLogNLarge) return CS_ERR_UNSUPPORTED;
  const bool large = logN > kMaxLogN;

  cs_plan_s* p = new (std::nothrow) cs_plan_s();
  if (!p) return CS_ERR_NOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  p->ordered = ordered;
  p->home = st;
  p->kind = kind;
  p->prec = prec;
  cudaGetDevice(&p->device);
  p->v.N = (int)N;
  p->v.logN = logN;
  p->v.M = (int)M;
  p->v.dft = kind == CS_DFT;
  p->v.fp32 = prec == CS_FP32;
  p->v.large = large;
  p->v.n1 = large ? logN / 2 : 0;
  p->v.n2 = large ? logN - logN / 2 : 0;
  p->v.wsh = large ? (logN + 1) / 2 : 0;
  p->v.cfmt = (flags & CS_PLAN_C_HALF) ? CFMT_HALF : ((flags & CS_PLAN_C_INT) ? CFMT_INT : CFMT_FULL);
  p->v.tc = (flags & CS_PLAN_TENSOR_CORES) != 0;
  // Sec. IV excessive point under the Table I flop model
  p->t_switch_default = kind == CS_DFT ? 1 + (5 * logN) / 6 : 1 + logN;

  // slot map: position -> m.  DFT positions of one-CTA plans are those of
  // the forward DIF chain (the adjoint chain's input order); WHT positions
  // and those of large plans are natural.
  std::vector<int32_t> slot((size_t)N, -1);
  for (int64_t m = 0; m < M; ++m) {
    const int pos = (kind == CS_DFT && !large) ? dif_position(omega_host[m], logN) : omega_host[m];
    slot[(size_t)pos] = (int32_t)m;
  }
  const size_t wb = kind == CS_DFT ? 16 : 8;
  cudaError_t e;
#define PLAN_TRY(call, what)                    \
  do {                                          \
    e = (call);                                 \
    if (e != cudaSuccess) {                     \
      cs_status s_ = cuda_fail(e, what);        \
      plan_free(p);                             \
      return s_;                                \
    }                                           \
  } while (0)
  PLAN_TRY(plan_alloc(p, (void**)&p->d_slot, (size_t)N * sizeof(int32_t)), "cudaMalloc slot");
  PLAN_TRY(cudaMemcpyAsync(p->d_slot, slot.data(), (size_t)N * sizeof(int32_t), cudaMemcpyHostToDevice, st),
           "copy slot");
  // plans up to 2^16 also run whole instances on one SM in cs_omp_batched,
  // with the one-CTA chains: their DFT positions and the shared twiddles
  const bool chain = large && logN <= kMaxLogNMulti;
  std::vector<int32_t> slot_chain;
  if (chain && kind == CS_DFT) {
    slot_chain.assign((size_t)N, -1);
    for (int64_t m = 0; m < M; ++m) slot_chain[(size_t)dif_position(omega_host[m], logN)] = (int32_t)m;
    PLAN_TRY(plan_alloc(p, (void**)&p->d_slot_chain, (size_t)N * sizeof(int32_t)), "cudaMalloc slot");
    PLAN_TRY(cudaMemcpyAsync(p->d_slot_chain, slot_chain.data(), (size_t)N * sizeof(int32_t),
                             cudaMemcpyHostToDevice, st),
             "copy slot");
    PLAN_TRY(chain_twiddles(logN, st, &p->v.ctw64, &p->v.ctw32), "chain twiddles");
  }
  // large plans: Omega grouped by the pass-2 row it comes out of (counting
  // sort), so that the residual sink visits only Omega's positions
  std::vector<int32_t> om_off;
  std::vector<int2> om_ent;
  if (large && M > 0) {
    const int n1 = p->v.n1, n2 = p->v.n2, N1 = 1 << n1;
    auto row_of = [&](int j) { return kind == CS_DFT ? (j & (N1 - 1)) : (j >> n2); };
    om_off.assign((size_t)N1 + 1, 0);
    for (int64_t m = 0; m < M; ++m) ++om_off[(size_t)row_of(omega_host[m]) + 1];
    for (int r = 0; r < N1; ++r) om_off[(size_t)r + 1] += om_off[(size_t)r];
    om_ent.resize((size_t)M);
    std::vector<int32_t> fill(om_off.begin(), om_off.end() - 1);
    for (int64_t m = 0; m < M; ++m) {
      const int j = omega_host[m];
      om_ent[(size_t)fill[(size_t)row_of(j)]++] = make_int2(j, (int)m);
    }
    PLAN_TRY(plan_alloc(p, (void**)&p->d_om_off, om_off.size() * sizeof(int32_t)), "cudaMalloc Omega rows");
    PLAN_TRY(cudaMemcpyAsync(p->d_om_off, om_off.data(), om_off.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             st),
             "copy Omega rows");
    PLAN_TRY(plan_alloc(p, (void**)&p->d_om_ent, om_ent.size() * sizeof(int2)), "cudaMalloc Omega rows");
    PLAN_TRY(cudaMemcpyAsync(p->d_om_ent, om_ent.data(), om_ent.size() * sizeof(int2), cudaMemcpyHostToDevice, st),
             "copy Omega rows");
  }
  // and grouped by the pass-1 column it goes into (j mod N2, both kinds), so
  // that pass 1 of a zero-filled input assembles its columns from Omega's
  // entries alone instead of reading a slot for every position
  std::vector<int32_t> oc_off;
  std::vector<int2> oc_ent;
  if (large && M > 0) {
    const int N2 = 1 << p->v.n2;
    oc_off.assign((size_t)N2 + 1, 0);
    for (int64_t m = 0; m < M; ++m) ++oc_off[(size_t)(omega_host[m] & (N2 - 1)) + 1];
    for (int c = 0; c < N2; ++c) oc_off[(size_t)c + 1] += oc_off[(size_t)c];
    oc_ent.resize((size_t)M);
    std::vector<int32_t> fill(oc_off.begin(), oc_off.end() - 1);
    for (int64_t m = 0; m < M; ++m) {
      const int j = omega_host[m];
      oc_ent[(size_t)fill[(size_t)(j & (N2 - 1))]++] = make_int2(j, (int)m);
    }
    PLAN_TRY(plan_alloc(p, (void**)&p->d_oc_off, oc_off.size() * sizeof(int32_t)), "cudaMalloc Omega columns");
    PLAN_TRY(cudaMemcpyAsync(p->d_oc_off, oc_off.data(), oc_off.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             st),
             "copy Omega columns");
    PLAN_TRY(plan_alloc(p, (void**)&p->d_oc_ent, oc_ent.size() * sizeof(int2)), "cudaMalloc Omega columns");
    PLAN_TRY(cudaMemcpyAsync(p->d_oc_ent, oc_ent.data(), oc_ent.size() * sizeof(int2), cudaMemcpyHostToDevice, st),
             "copy Omega columns");
  }
  if (kind == CS_DFT && !large) {
    PLAN_TRY(plan_alloc(p, &p->d_tw64, (size_t)N * sizeof(double2)), "cudaMalloc twiddles");
    if (prec == CS_FP32) PLAN_TRY(plan_alloc(p, &p->d_tw32, (size_t)N * sizeof(float2)), "cudaMalloc twiddles");
  }
  if (kind == CS_DFT && large) {
    const size_t nt = ((size_t)1 << p->v.n1) + ((size_t)1 << p->v.n2) + ((size_t)1 << p->v.wsh) +
                      ((size_t)N >> p->v.wsh);
    PLAN_TRY(plan_alloc(p, &p->d_lt64, nt * sizeof(double2)), "cudaMalloc four-step tables");
    if (prec == CS_FP32) PLAN_TRY(plan_alloc(p, &p->d_lt32, nt * sizeof(float2)), "cudaMalloc four-step tables");
  }
  const int cfmt = p->v.cfmt;
  const size_t nc = cfmt == CFMT_HALF ? (size_t)N / 2 + 1 : (cfmt == CFMT_INT ? 0 : (size_t)N);
  if (nc) PLAN_TRY(plan_alloc(p, &p->d_c64, nc * wb), "cudaMalloc c");
  if (nc && prec == CS_FP32) PLAN_TRY(plan_alloc(p, &p->d_c32, nc * wb / 2), "cudaMalloc c");
  if (cfmt == CFMT_INT) PLAN_TRY(plan_alloc(p, (void**)&p->d_ci, (size_t)N * sizeof(int)), "cudaMalloc c");
  PLAN_TRY(plan_alloc(p, (void**)&p->d_status, sizeof(int)), "cudaMalloc status");
  PLAN_TRY(cudaMemsetAsync(p->d_status, 0, sizeof(int), st), "clear status");
  p->v.slot = p->d_slot;
  p->v.tw64 = p->d_tw64;
  p->v.tw32 = p->d_tw32;
  p->v.c64 = p->d_c64;
  p->v.c32 = p->d_c32;
  p->v.status = p->d_status;
  p->v.lt64 = p->d_lt64;
  p->v.lt32 = p->d_lt32;
  p->v.ci = p->d_ci;
  p->v.om_off = p->d_om_off;
  p->v.om_ent = p->d_om_ent;
  p->v.oc_off = p->d_oc_off;
  p->v.oc_ent = p->d_oc_ent;
  if (!large) {
    p->v.slot_chain = p->d_slot;
    p->v.ctw64 = p->d_tw64;
    p->v.ctw32 = p->d_tw32;
  } else if (chain) {
    p->v.slot_chain = kind == CS_DFT ? p->d_slot_chain : p->d_slot;
  }
  // c in FP64, full length: into the plan's own buffer (CFMT_FULL) or a
  // scratch vector that is then put into the plan's storage format
  {
    const size_t tb0 = p->table_bytes;
    e = cudaSuccess;
    void* full = cfmt == CFMT_FULL ? p->d_c64 : nullptr;
    void* tmp = nullptr;
    if (!full) PLAN_TRY(plan_alloc(p, &full, (size_t)N * wb), "cudaMalloc plan scratch");
    if (large) PLAN_TRY(plan_alloc(p, &tmp, (size_t)N * wb), "cudaMalloc plan scratch");
    if (!large) {
      if (kind == CS_DFT) e = launch_twiddles(p->v, p->d_tw64, p->d_tw32, st);
      if (e == cudaSuccess) e = launch_kernel_vector(p->v, full, st);
    } else {
      e = large_tables(p->v, p->d_lt64, p->d_lt32, st);
      if (e == cudaSuccess) e = large_kernel_vector(p->v, full, tmp, st);
    }
    if (e == cudaSuccess) {
      if (cfmt == CFMT_FULL) {
        if (p->d_c32) e = launch_round(kind == CS_DFT, p->d_c64, p->d_c32, (int)N, st);
      } else {
        e = launch_compress_c(p->v, full, p->d_c64, p->d_c32, p->d_ci, st);
      }
    }
    void* scratch[] = {cfmt == CFMT_FULL ? nullptr : full, tmp};
    if (ordered)
      for (void* b : scratch)
        if (b) cudaFreeAsync(b, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (!ordered)
      for (void* b : scratch)
        if (b) cudaFree(b);
    p->table_bytes = tb0;  // scratch is not part of the plan
    PLAN_TRY(e, "kernel-vector kernels");
    PLAN_TRY(e2, "plan synchronize");
  }
#undef PLAN_TRY
  *out = p;
  return CS_OK;
}

extern "C" cs_status cs_plan_create(int64_t N, const int32_t* omega_host, int64_t M, int32_t kind, int32_t prec,
                                    void* stream, cs_plan_t* out) {
  return plan_create_impl(N, omega_host, M, kind, prec, 0u, stream, false, out);
}

extern "C" cs_status cs_plan_create_ex(int64_t N, const int32_t* omega_host, int64_t M, int32_t kind, int32_t prec,
                                       uint32_t flags, void* stream, cs_plan_t* out) {
  return plan_create_impl(N, omega_host, M, kind, prec, flags, stream, false, out);
}

extern "C" cs_status cs_plan_memory(cs_plan_t plan, int64_t* table_bytes) {
  if (!plan || !table_bytes) return CS_ERR_INVALID;
  *table_bytes = (int64_t)plan->table_bytes;
  return CS_OK;
}

namespace csf {
// Plans of the request runtime: every buffer stream-ordered on `stream`, so
// that creating and releasing one never synchronises the device.
cs_status plan_create_ordered(int64_t N, const int32_t* omega_host, int64_t M, int32_t kind, int32_t prec,
                              cudaStream_t stream, cs_plan_t* out) {
  return plan_create_impl(N, omega_host, M, kind, prec, 0u, stream, true, out);
}
// Queues the release of a stream-ordered plan's buffers on its stream.
void plan_release_ordered(cs_plan_t plan) { plan_free(plan); }

// Device bytes a plan and one solve of `K` columns on one measurement take
// (plan tables, the largest workspace of the path, inputs and outputs), for
// admission against a memory budget.  algo: 0 OMP, 1 CoSaMP, 2 SP.
size_t solve_footprint(int64_t N, int64_t M, int32_t kind, int32_t prec, int32_t K, int32_t algo) {
  int logN = 0;
  while ((int64_t(1) << logN) < N) ++logN;
  PlanView v{};
  v.N = (int)N;
  v.logN = logN;
  v.M = (int)M;
  v.dft = kind == CS_DFT;
  v.fp32 = prec == CS_FP32;
  v.large = logN > kMaxLogN;
  v.n1 = v.large ? logN / 2 : 0;
  v.n2 = v.large ? logN - logN / 2 : 0;
  v.wsh = v.large ? (logN + 1) / 2 : 0;
  const size_t wb = v.dft ? 16 : 8, eb = elem_bytes(kind, prec);
  size_t b = (size_t)N * 4 + (size_t)N * wb + (v.fp32 ? (size_t)N * wb / 2 : 0) + 256;
  if (v.dft && !v.large) b += (size_t)N * (16 + (v.fp32 ? 8 : 0));
  if (v.dft && v.large)
    b += (((size_t)1 << v.n1) + ((size_t)1 << v.n2) + ((size_t)1 << v.wsh) + ((size_t)N >> v.wsh)) *
         (16 + (v.fp32 ? 8 : 0));
  if (v.large) b += (size_t)N * wb;  // kernel-vector scratch while the plan is built
  if (v.dft && v.large && logN <= kMaxLogNMulti) b += (size_t)N * 4;  // chain-order slot map
  if (v.large) b += ((size_t)1 << v.n1) * 4 + 4 + (size_t)M * 8;      // Omega grouped by pass-2 row
  if (v.large) b += ((size_t)1 << v.n2) * 4 + 4 + (size_t)M * 8;      //   and by pass-1 column
  size_t ws = 0;
  if (algo == 0) ws = v.large ? large_omp_ws(v, K, CS_PATH_HYBRID, 1) : omp_workspace_bytes(v, K, 1);
  else if (v.large) ws = large_pursuit_ws(v, K, algo == 2 ? 0 : 1, 0, 1);
  else ws = pursuit_workspace_bytes(v, K, algo == 2 ? 0 : 1, 1);
  b += ws + (size_t)M * eb + (size_t)K * (wb + 4) + 64;
  return b;
}
}  // namespace csf

extern "C" cs_status cs_plan_destroy(cs_plan_t plan) {
  if (!plan) return CS_ERR_INVALID;
  cudaDeviceSynchronize();
  plan_free(plan);
  return CS_OK;
}

extern "C" cs_status cs_plan_info(cs_plan_t plan, int64_t* N, int64_t* M, int32_t* kind, int32_t* prec,
                                  int32_t* t_switch_default) {
  if (!plan) return CS_ERR_INVALID;
  if (N) *N = plan->v.N;
  if (M) *M = plan->v.M;
  if (kind) *kind = plan->kind;
  if (prec) *prec = plan->prec;
  if (t_switch_default) *t_switch_default = plan->t_switch_default;
  return CS_OK;
}

extern "C" cs_status cs_plan_status(cs_plan_t plan, int32_t* device_error, void* stream) {
  if (!plan || !device_error) return CS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  CS_CUDA(cudaMemcpyAsync(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
  CS_CUDA(cudaStreamSynchronize(st), "status synchronize");
  CS_CUDA(cudaMemsetAsync(plan->d_status, 0, sizeof(int), st), "clear status");
  *device_error = h;
  return CS_OK;
}

extern "C" cs_status cs_plan_kernel(cs_plan_t plan, void* c_dev, int32_t prec, void* stream) {
  if (!plan || !c_dev) return CS_ERR_INVALID;
  if (prec != CS_FP64 && prec != CS_FP32) return CS_ERR_INVALID;
  const size_t n = (size_t)plan->v.N;
  if (plan->v.cfmt != CFMT_FULL) {
    CS_CUDA(launch_expand_c(plan->v, c_dev, prec == CS_FP32, (cudaStream_t)stream), "expand c");
    return CS_OK;
  }
  if (prec == CS_FP64) {
    CS_CUDA(cudaMemcpyAsync(c_dev, plan->d_c64, n * elem_bytes(plan->kind, CS_FP64), cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream),
            "copy c");
    return CS_OK;
  }
  if (plan->d_c32) {
    CS_CUDA(cudaMemcpyAsync(c_dev, plan->d_c32, n * elem_bytes(plan->kind, CS_FP32), cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream),
            "copy c");
    return CS_OK;
  }
  // FP64 plan asked for FP32 c: round the FP64 vector
  CS_CUDA(launch_round(plan->v.dft, plan->d_c64, c_dev, plan->v.N, (cudaStream_t)stream), "round c");
  return CS_OK;
}

extern "C" cs_status cs_correlate(cs_plan_t plan, const void* r_dev, int64_t batch, void* h_dev, int32_t* argmax_dev,
                                  void* stream) {
  if (!plan || batch < 0) return CS_ERR_INVALID;
  if (batch > 0 && plan->v.M > 0 && !r_dev) return CS_ERR_INVALID;
  if (batch == 0 || (!h_dev && !argmax_dev)) return CS_OK;
  if (plan->v.large) {
    if (batch > kMaxLargeBatch) return CS_ERR_UNSUPPORTED;
    const cs_status r = ensure_ws(plan, large_correlate_ws(plan->v, batch), (cudaStream_t)stream);
    if (r != CS_OK) return r;
    CS_CUDA(large_correlate(plan->v, r_dev, batch, h_dev, argmax_dev, plan->ws, (cudaStream_t)stream),
            "correlate");
    return CS_OK;
  }
  CS_CUDA(launch_correlate(plan->v, r_dev, batch, h_dev, argmax_dev, (cudaStream_t)stream), "correlate");
  return CS_OK;
}

extern "C" cs_status cs_correlate_fast(cs_plan_t plan, const void* h0_dev, const int32_t* supp_dev,
                                       const void* x_dev, int32_t s, int64_t batch, void* h_dev, int32_t* argmax_dev,
                                       void* stream) {
  if (!plan || batch < 0 || s < 0 || s > plan->v.N) return CS_ERR_INVALID;
  if (batch > 0 && !h0_dev) return CS_ERR_INVALID;
  if (batch > 0 && s > 0 && (!supp_dev || !x_dev)) return CS_ERR_INVALID;
  if (s > (plan->v.large ? kMaxKLarge : kMaxK)) return CS_ERR_UNSUPPORTED;
  if (batch == 0 || (!h_dev && !argmax_dev)) return CS_OK;
  if (plan->v.large) {
    if (batch > kMaxLargeBatch) return CS_ERR_UNSUPPORTED;
    const cs_status r = ensure_ws(plan, large_fast_ws(plan->v, batch), (cudaStream_t)stream);
    if (r != CS_OK) return r;
    CS_CUDA(large_correlate_fast(plan->v, h0_dev, supp_dev, x_dev, s, batch, h_dev, argmax_dev, plan->ws,
                                 (cudaStream_t)stream),
            "correlate_fast");
    return CS_OK;
  }
  CS_CUDA(launch_correlate_fast(plan->v, h0_dev, supp_dev, x_dev, s, batch, h_dev, argmax_dev, (cudaStream_t)stream),
          "correlate_fast");
  return CS_OK;
}

extern "C" cs_status cs_omp(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K, const cs_halt* halt,
                            void* x_dev, int32_t* supp_dev, int32_t* iters_dev, double* resnorm_dev, void* stream) {
  if (!plan || batch < 0 || K < 0) return CS_ERR_INVALID;
  if (K > plan->v.M) return CS_ERR_INVALID;
  if (K > (plan->v.large ? kMaxKLarge : kMaxK)) return CS_ERR_UNSUPPORTED;
  cs_halt h = {1e-6, CS_PATH_HYBRID, -1, 0};
  if (halt) h = *halt;
  if (!(h.rel_tol >= 0.0) || !std::isfinite(h.rel_tol)) return CS_ERR_INVALID;
  if (h.path != CS_PATH_FAST && h.path != CS_PATH_CONV && h.path != CS_PATH_HYBRID) return CS_ERR_INVALID;
  if (batch == 0) return CS_OK;
  if (K > 0 && !supp_dev) return CS_ERR_INVALID;
  if (plan->v.M > 0 && !y_dev) return CS_ERR_INVALID;
  const int t_switch = h.t_switch >= 0 ? h.t_switch : plan_switch(plan);
  cudaStream_t st = (cudaStream_t)stream;

  int err = 0, grid = 0;
  // a few instances: one cluster of CTAs per instance (same results as the
  // persistent kernel, spread over more SMs)
  const bool cluster = !plan->v.large && batch <= kClusterMaxBatch && K <= kClusterMaxK &&
                       omp_cluster_smem(plan->v, K, h.path) <= (size_t)200 * 1024;
  if (plan->v.large) {
    if (batch > kMaxLargeBatch) return CS_ERR_UNSUPPORTED;
    const cs_status r = ensure_ws(plan, large_omp_ws(plan->v, K, h.path, batch), st);
    if (r != CS_OK) return r;
  } else if (cluster) {
    const cs_status r = ensure_ws(plan, omp_cluster_workspace_bytes(plan->v, K, batch), st);
    if (r != CS_OK) return r;
  } else {
    grid = omp_grid(plan->v, K, h.path, batch, &err);
    if (err) return cuda_fail((cudaError_t)err, "omp configuration");
    const cs_status r = ensure_ws(plan, omp_workspace_bytes(plan->v, K, grid), st);
    if (r != CS_OK) return r;
  }
  OmpLaunch a;
  a.y = y_dev;
  a.batch = batch;
  a.K = K;
  a.rel_tol = h.rel_tol;
  a.path = h.path;
  a.t_switch = t_switch;
  a.x_out = x_dev;
  a.supp_out = supp_dev;
  a.iters_out = iters_dev;
  a.res_out = resnorm_dev;
  if (plan->v.large) CS_CUDA(large_omp(plan->v, a, plan->ws, st), "omp kernels");
  else if (cluster) CS_CUDA(launch_omp_cluster(plan->v, a, plan->ws, st), "omp cluster kernel");
  else CS_CUDA(launch_omp(plan->v, a, plan->ws, grid, st), "omp kernel");
  return CS_OK;
}

extern "C" cs_status cs_omp_batched(const cs_plan_t* plans, int64_t count, const void* const* y_dev,
                                    const int32_t* K, const cs_halt* halt, void* const* x_dev,
                                    int32_t* const* supp_dev, int32_t* iters_dev, double* resnorm_dev,
                                    void* stream) {
  if (count < 0 || count > ((int64_t)1 << 30)) return CS_ERR_INVALID;
  cs_halt h = {1e-6, CS_PATH_HYBRID, -1, 0};
  if (halt) h = *halt;
  if (!(h.rel_tol >= 0.0) || !std::isfinite(h.rel_tol)) return CS_ERR_INVALID;
  if (h.path != CS_PATH_FAST && h.path != CS_PATH_CONV && h.path != CS_PATH_HYBRID) return CS_ERR_INVALID;
  if (count == 0) return CS_OK;
  if (!plans || !y_dev || !K || !supp_dev) return CS_ERR_INVALID;
  int dev = 0;
  cudaGetDevice(&dev);
  // one launch per element type (kind, precision) and residence (instances
  // held in shared memory, N <= 8192, or in global memory, N <= 2^16); larger
  // N: the large-plan path of cs_omp, one instance at a time
  std::vector<MultiItem> group[8];
  struct Solo {
    cs_plan_s* p;
    const void* y;
    void* x;
    int* supp;
    int K, t_switch, idx;
  };
  std::vector<Solo> solo;
  for (int64_t b = 0; b < count; ++b) {
    const cs_plan_s* p = plans[b];
    if (!p) return CS_ERR_INVALID;
    if (p->device != dev) {
      set_last_error("cs_omp_batched: every plan must live on the current device");
      return CS_ERR_INVALID;
    }
    const int k = K[b];
    if (k < 0 || k > p->v.M) return CS_ERR_INVALID;
    if (p->v.M > 0 && !y_dev[b]) return CS_ERR_INVALID;
    if (k > 0 && (!supp_dev[b] || (x_dev && !x_dev[b]))) return CS_ERR_INVALID;
    if (p->v.logN > kMaxLogNMulti) {
      if (k > kMaxKLarge) {
        set_last_error("cs_omp_batched: K above 4096 (N > 2^16)");
        return CS_ERR_UNSUPPORTED;
      }
      solo.push_back({plans[b], y_dev[b], x_dev ? x_dev[b] : nullptr, supp_dev[b], k,
                      h.t_switch >= 0 ? h.t_switch : plan_switch(p), (int)b});
      continue;
    }
    if (k > kMaxK) {
      set_last_error("cs_omp_batched: K above 1024 (N <= 2^16)");
      return CS_ERR_UNSUPPORTED;
    }
    if (p->v.large && p->v.cfmt != CFMT_FULL) {
      set_last_error("cs_omp_batched: plans with 8192 < N <= 2^16 need the full storage of c");
      return CS_ERR_UNSUPPORTED;
    }
    MultiItem it;
    it.P = &p->v;
    it.y = y_dev[b];
    it.x = x_dev ? x_dev[b] : nullptr;
    it.supp = supp_dev[b];
    it.K = k;
    const BatchShape shp = batch_shape(dev, batch_group(p->v));
    it.t_switch = h.t_switch >= 0 ? h.t_switch
                  : shp.t_switch >= 0 ? shp.t_switch
                  : (p->v.large ? multi_switch_big(p->v.logN) : plan_switch(p));
    it.idx = (int)b;
    it.cost = multi_cost(p->v, k, it.t_switch, h.path);
    group[batch_group(p->v)].push_back(it);
  }
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (auto& g : group) {
    if (g.empty()) continue;
    if (omp_multi_smem(g.data(), (int64_t)g.size(), h.path) > (size_t)optin) {
      set_last_error("cs_omp_batched: N and K of one element type need more shared memory than a CTA has");
      return CS_ERR_UNSUPPORTED;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  // Jobs: the persistent launches, most work first, on streams 0..7, and the
  // large-plan instances on streams 8..11 chosen by plan (instances of one
  // plan share its workspace, so they stay in order on one stream).  With
  // more than one job, each stream is forked from `stream` and joined back
  // into it, so that the CTAs of later launches fill the SMs an earlier one
  // leaves idle in its tail.
  std::vector<int> order;
  std::vector<double> work(8, 0.0);
  for (int gi = 0; gi < 8; ++gi) {
    for (const MultiItem& it : group[gi]) work[gi] += it.cost;
    if (!group[gi].empty()) order.push_back(gi);
  }
  std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return work[u] > work[v]; });
  struct Job {
    int stream, group, solo;
  };
  std::vector<Job> jobs;
  for (size_t k = 0; k < order.size(); ++k) jobs.push_back({(int)k, order[k], -1});
  for (size_t i = 0; i < solo.size(); ++i)
    jobs.push_back({8 + (int)(((uintptr_t)solo[i].p >> 4) % 4), -1, (int)i});
  auto run = [&](const Job& j, cudaStream_t s) -> cs_status {
    if (j.group >= 0) {
      std::vector<MultiItem>& g = group[j.group];
      const cudaError_t e = launch_omp_multi(g.data(), (int64_t)g.size(), h.rel_tol, h.path,
                                             batch_shape(dev, j.group).ctas_per_sm, iters_dev,
                                             resnorm_dev, plans[0]->v.status, s);
      return e == cudaSuccess ? CS_OK : cuda_fail(e, "omp_batched kernel");
    }
    const Solo& so = solo[(size_t)j.solo];
    const cs_status r = ensure_ws(so.p, large_omp_ws(so.p->v, so.K, h.path, 1), s);
    if (r != CS_OK) return r;
    OmpLaunch a;
    a.y = so.y;
    a.batch = 1;
    a.K = so.K;
    a.rel_tol = h.rel_tol;
    a.path = h.path;
    a.t_switch = so.t_switch;
    a.x_out = so.x;
    a.supp_out = so.supp;
    a.iters_out = iters_dev ? iters_dev + so.idx : nullptr;
    a.res_out = resnorm_dev ? resnorm_dev + so.idx : nullptr;
    const cudaError_t e = large_omp(so.p->v, a, so.p->ws, s);
    return e == cudaSuccess ? CS_OK : cuda_fail(e, "omp_batched large-plan kernels");
  };
  if (jobs.size() == 1) return run(jobs[0], st);
  cudaEvent_t fork = nullptr;
  CS_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "omp_batched event");
  cs_status r = CS_OK;
  cudaError_t e = cudaEventRecord(fork, st);
  std::map<int, cudaStream_t> aux;
  for (const Job& j : jobs) {
    if (e != cudaSuccess || aux.count(j.stream)) continue;
    cudaStream_t s = nullptr;
    e = fork_stream(dev, j.stream, &s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fork, 0);
    if (e == cudaSuccess) aux[j.stream] = s;
  }
  for (const Job& j : jobs) {
    if (e != cudaSuccess || r != CS_OK) break;
    r = run(j, aux[j.stream]);
  }
  // join every forked stream back, also after a failure: nothing queued on
  // it may outlive the caller's stream
  for (const auto& kv : aux) {
    cudaEvent_t done = nullptr;
    cudaError_t e2 = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    if (e2 == cudaSuccess) e2 = cudaEventRecord(done, kv.second);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, done, 0);
    if (done) cudaEventDestroy(done);
    if (e == cudaSuccess) e = e2;
  }
  cudaEventDestroy(fork);
  if (r != CS_OK) return r;
  CS_CUDA(e, "omp_batched streams");
  return CS_OK;
}

// Measures the launch shapes of an uneven batch (the autotuner of
// cs_omp_batched): for each launch group present (element type and
// residence), the resident CTAs per SM and then the switch point, each
// candidate timed on the group's own instances (one warm-up, best of two).
extern "C" cs_status cs_omp_batched_tune(const cs_plan_t* plans, int64_t count, const void* const* y_dev,
                                         const int32_t* K, double rel_tol, int32_t* group_out, int32_t* ctas_out,
                                         int32_t* tswitch_out, float* ms_out, int32_t cap, int32_t* n_out,
                                         void* stream) {
  using namespace csf;
  if (n_out) *n_out = 0;
  if (count < 0 || !(rel_tol >= 0.0) || !std::isfinite(rel_tol) || cap < 0) return CS_ERR_INVALID;
  int dev = 0;
  cudaGetDevice(&dev);
  if (count == 0) {  // forget the shapes stored for this device
    for (int gi = 0; gi < 8; ++gi) set_batch_shape(dev, gi, BatchShape{});
    return CS_OK;
  }
  if (!plans || !y_dev || !K) return CS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<size_t> off((size_t)count, 0);
  size_t tot = 0;
  for (int64_t b = 0; b < count; ++b) {
    const cs_plan_s* p = plans[b];
    if (!p || p->device != dev) return CS_ERR_INVALID;
    if (K[b] < 0 || K[b] > p->v.M || (p->v.M > 0 && !y_dev[b])) return CS_ERR_INVALID;
    if (p->v.logN <= kMaxLogNMulti && (K[b] > kMaxK || (p->v.large && p->v.cfmt != CFMT_FULL)))
      return CS_ERR_UNSUPPORTED;
    if (p->v.logN > kMaxLogNMulti && K[b] > kMaxKLarge) return CS_ERR_UNSUPPORTED;
    off[(size_t)b] = tot;
    tot += a16((size_t)K[b] * 16) + a16((size_t)K[b] * 4);
  }
  const size_t o_it = tot, o_rn = a16(o_it + (size_t)count * 4), total = a16(o_rn + (size_t)count * 8) + 16;
  char* tmp = nullptr;
  CS_CUDA(cudaMallocAsync((void**)&tmp, total, st), "cudaMallocAsync tune outputs");
  std::vector<MultiItem> group[8];
  std::map<const PlanView*, int> dflt;  // each plan's default switch point
  for (int64_t b = 0; b < count; ++b) {
    const cs_plan_s* p = plans[b];
    if (p->v.logN > kMaxLogNMulti) continue;
    MultiItem it;
    it.P = &p->v;
    it.y = y_dev[b];
    it.x = tmp + off[(size_t)b];
    it.supp = (int*)(tmp + off[(size_t)b] + a16((size_t)K[b] * 16));
    it.K = K[b];
    it.t_switch = p->v.large ? multi_switch_big(p->v.logN) : plan_switch(p);
    it.idx = (int)b;
    it.cost = 0.0;
    group[batch_group(p->v)].push_back(it);
    dflt[&p->v] = it.t_switch;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cs_status r = CS_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = CS_ERR_CUDA;
  BatchShape prev[8];  // what later calls would have used before this tuning
  for (int gi = 0; gi < 8; ++gi) prev[gi] = batch_shape(dev, gi);
  int nrec = 0;
  for (int gi = 0; gi < 8 && r == CS_OK; ++gi) {
    std::vector<MultiItem>& g = group[gi];
    if (g.empty()) continue;
    int err = 0;
    const int occ = omp_multi_occupancy(g.data(), (int64_t)g.size(), CS_PATH_HYBRID, &err);
    if (err || occ < 1) {
      r = CS_ERR_CUDA;
      break;
    }
    // one candidate: every instance at switch point ts (< 0: its default)
    auto time_it = [&](int ctas, int ts) -> float {
      for (MultiItem& it : g) {
        it.t_switch = ts >= 0 ? ts : dflt[it.P];
        it.cost = multi_cost(*it.P, it.K, it.t_switch, CS_PATH_HYBRID);
      }
      float best = -1.f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaError_t e = cudaEventRecord(e0, st);
        if (e == cudaSuccess)
          e = launch_omp_multi(g.data(), (int64_t)g.size(), rel_tol, CS_PATH_HYBRID, ctas, (int*)(tmp + o_it),
                               (double*)(tmp + o_rn), plans[0]->v.status, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          cuda_fail(e, "omp_batched_tune");
          return -1.f;
        }
        if (rep > 0 && (best < 0.f || ms < best)) best = ms;
      }
      return best;
    };
    BatchShape shp;
    float best = time_it(0, -1);
    if (best < 0.f) { r = CS_ERR_CUDA; break; }
    for (int c = 1; c < occ; ++c) {  // fewer resident CTAs per SM
      const float ms = time_it(c, -1);
      if (ms < 0.f) { r = CS_ERR_CUDA; break; }
      if (ms < 0.98f * best) { best = ms; shp.ctas_per_sm = c; }
    }
    if (r != CS_OK) break;
    const bool big = gi & 1;
    const int cands_big[] = {16, 64, 128}, cands_small[] = {32, 128};
    const int* cands = big ? cands_big : cands_small;
    const int nc = big ? 3 : 2;
    for (int i = 0; i < nc; ++i) {
      const float ms = time_it(shp.ctas_per_sm, cands[i]);
      if (ms < 0.f) { r = CS_ERR_CUDA; break; }
      if (ms < 0.98f * best) { best = ms; shp.t_switch = cands[i]; }
    }
    if (r != CS_OK) break;
    set_batch_shape(dev, gi, shp);
    if (nrec < cap) {
      if (group_out) group_out[nrec] = gi;
      if (ctas_out) ctas_out[nrec] = shp.ctas_per_sm;
      if (tswitch_out) tswitch_out[nrec] = shp.t_switch;
      if (ms_out) ms_out[nrec] = best;
    }
    ++nrec;
  }
  // The groups' launches run side by side in a cs_omp_batched call and share
  // the SMs and L2, so the shapes measured per group are kept only if the
  // whole call is faster with them than with the shapes it had before (and
  // than with the tuned switch points alone).
  if (r == CS_OK && nrec > 0) {
    std::vector<void*> xs((size_t)count), ss((size_t)count);
    for (int64_t b = 0; b < count; ++b) {
      xs[(size_t)b] = tmp + off[(size_t)b];
      ss[(size_t)b] = tmp + off[(size_t)b] + a16((size_t)K[b] * 16);
    }
    const cs_halt hh = {rel_tol, CS_PATH_HYBRID, -1, 0};
    auto full_call = [&]() -> float {
      float best = -1.f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaError_t e = cudaEventRecord(e0, st);
        if (e != cudaSuccess) return -1.f;
        if (cs_omp_batched(plans, count, y_dev, K, &hh, xs.data(), (int32_t* const*)ss.data(), (int*)(tmp + o_it),
                           (double*)(tmp + o_rn), st) != CS_OK)
          return -1.f;
        e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return -1.f;
        if (rep > 0 && (best < 0.f || ms < best)) best = ms;
      }
      return best;
    };
    BatchShape tuned[8], only_ts[8];
    for (int gi = 0; gi < 8; ++gi) {
      tuned[gi] = batch_shape(dev, gi);
      only_ts[gi] = tuned[gi];
      only_ts[gi].ctas_per_sm = prev[gi].ctas_per_sm;
    }
    auto install = [&](const BatchShape* v) { for (int gi = 0; gi < 8; ++gi) set_batch_shape(dev, gi, v[gi]); };
    const float t_tuned = full_call();
    install(only_ts);
    const float t_ts = full_call();
    install(prev);
    const float t_prev = full_call();
    if (t_tuned < 0.f || t_ts < 0.f || t_prev < 0.f) {
      r = CS_ERR_CUDA;
    } else if (t_tuned < 0.98f * t_prev && t_tuned <= t_ts) {
      install(tuned);
    } else if (t_ts < 0.98f * t_prev) {
      install(only_ts);
    }
    // the records report what is stored
    for (int i = 0; i < nrec && i < cap; ++i) {
      const BatchShape v = batch_shape(dev, group_out ? group_out[i] : 0);
      if (group_out && ctas_out) ctas_out[i] = v.ctas_per_sm;
      if (group_out && tswitch_out) tswitch_out[i] = v.t_switch;
    }
  }
  if (n_out) *n_out = nrec;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  const cudaError_t ef = cudaFreeAsync(tmp, st);
  if (r != CS_OK) return r;
  CS_CUDA(ef, "cudaFreeAsync tune outputs");
  return CS_OK;
}

static cs_status pursuit_call(int algo, cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K,
                              const cs_halt* halt, void* x_dev, int32_t* supp_dev, int32_t* iters_dev,
                              double* resnorm_dev, void* stream) {
  if (!plan || batch < 0 || K < 1) return CS_ERR_INVALID;
  if ((algo == 0 ? 2 : 3) * (int64_t)K > plan->v.M) return CS_ERR_INVALID;
  if (K > (plan->v.large ? kMaxPursuitKLarge : kMaxPursuitK)) return CS_ERR_UNSUPPORTED;
  if (plan->v.large && batch > kMaxLargeBatch) return CS_ERR_UNSUPPORTED;
  cs_halt h = {1e-6, CS_PATH_HYBRID, -1, 0};
  if (halt) h = *halt;
  if (!(h.rel_tol >= 0.0) || !std::isfinite(h.rel_tol)) return CS_ERR_INVALID;
  if (h.path != CS_PATH_FAST && h.path != CS_PATH_CONV && h.path != CS_PATH_HYBRID) return CS_ERR_INVALID;
  if (batch == 0) return CS_OK;
  if (!supp_dev || !y_dev) return CS_ERR_INVALID;
  const int t_switch = h.t_switch >= 0 ? h.t_switch : plan_switch(plan);
  const int fast = h.path == CS_PATH_FAST || (h.path == CS_PATH_HYBRID && K <= t_switch);
  cudaStream_t st = (cudaStream_t)stream;
  int err = 0, grid = 0;
  if (plan->v.large) {
    const cs_status r = ensure_ws(plan, large_pursuit_ws(plan->v, K, algo, fast, batch), st);
    if (r != CS_OK) return r;
  } else {
    grid = pursuit_grid(plan->v, K, algo, fast, batch, &err);
    if (err) return cuda_fail((cudaError_t)err, "pursuit configuration");
    const cs_status r = ensure_ws(plan, pursuit_workspace_bytes(plan->v, K, algo, grid), st);
    if (r != CS_OK) return r;
  }
  PursuitLaunch a;
  a.y = y_dev;
  a.batch = batch;
  a.K = K;
  a.algo = algo;
  a.max_iter = h.max_iter > 0 ? h.max_iter : (algo == 0 ? K : 50);
  a.fast = fast;
  a.rel_tol = h.rel_tol;
  a.x_out = x_dev;
  a.supp_out = supp_dev;
  a.iters_out = iters_dev;
  a.res_out = resnorm_dev;
  if (plan->v.large) CS_CUDA(large_pursuit(plan->v, a, plan->ws, st), "pursuit kernels");
  else CS_CUDA(launch_pursuit(plan->v, a, plan->ws, grid, st), "pursuit kernel");
  return CS_OK;
}

extern "C" cs_status cs_sp(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K, const cs_halt* halt,
                           void* x_dev, int32_t* supp_dev, int32_t* iters_dev, double* resnorm_dev, void* stream) {
  return pursuit_call(0, plan, y_dev, batch, K, halt, x_dev, supp_dev, iters_dev, resnorm_dev, stream);
}

extern "C" cs_status cs_cosamp(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K, const cs_halt* halt,
                               void* x_dev, int32_t* supp_dev, int32_t* iters_dev, double* resnorm_dev,
                               void* stream) {
  return pursuit_call(1, plan, y_dev, batch, K, halt, x_dev, supp_dev, iters_dev, resnorm_dev, stream);
}

// Switch-point tuning (Sec. IV: the paper picks the switch from its flop
// model; here the crossover is measured).  Runs cs_omp on the caller's batch
// with the hybrid path at a ladder of switch points and keeps the fastest.
extern "C" cs_status cs_plan_tune(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K, double rel_tol,
                                  int32_t* t_best, int32_t* cand_out, float* ms_out, int32_t cap, int32_t* n_out,
                                  void* stream) {
  if (!plan || !t_best || batch < 1 || K < 1 || K > plan->v.M || cap < 0) return CS_ERR_INVALID;
  if ((cap > 0 && (!cand_out || !ms_out)) || !(rel_tol >= 0.0) || !std::isfinite(rel_tol)) return CS_ERR_INVALID;
  if (plan->v.M > 0 && !y_dev) return CS_ERR_INVALID;
  if (K > kMaxK) return CS_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  // ladder: 1 (transforms from t = 2 on), the flop-model point, then roughly
  // geometric steps up to K (kernel sums throughout)
  std::vector<int> cand = {1, plan->t_switch_default};
  for (int t = 8; t < K; t = t < 16 ? t + 4 : t + t / 2) cand.push_back(t);
  cand.push_back(K);
  std::vector<int> ladder;
  for (int t : cand) {
    const int u = t < 1 ? 1 : (t > K ? K : t);
    bool seen = false;
    for (int v : ladder) seen = seen || v == u;
    if (!seen) ladder.push_back(u);
  }
  for (size_t i = 1; i < ladder.size(); ++i)
    for (size_t j = i; j > 0 && ladder[j - 1] > ladder[j]; --j) std::swap(ladder[j - 1], ladder[j]);

  const size_t wb = elem_bytes(plan->kind, CS_FP64);
  void* x = nullptr;
  int32_t* supp = nullptr;
  cs_status rc = CS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<float> ms(ladder.size(), 0.0f);
  do {
    cudaError_t e;
    if ((e = cudaMallocAsync(&x, (size_t)batch * K * wb, st)) != cudaSuccess) { rc = cuda_fail(e, "tune alloc"); break; }
    if ((e = cudaMallocAsync((void**)&supp, (size_t)batch * K * sizeof(int32_t), st)) != cudaSuccess) {
      rc = cuda_fail(e, "tune alloc");
      break;
    }
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
      rc = cuda_fail(e, "tune events");
      break;
    }
    // rounds over the whole ladder (one warm-up round, then the best of
    // five per candidate), so that a slow drift of the clocks or of the
    // memory state during the sweep weighs on every candidate alike
    for (int rep = 0; rep < 6 && rc == CS_OK; ++rep) {
      for (size_t i = 0; i < ladder.size() && rc == CS_OK; ++i) {
        const cs_halt h = {rel_tol, CS_PATH_HYBRID, ladder[i], 0};
        if ((e = cudaEventRecord(e0, st)) != cudaSuccess) { rc = cuda_fail(e, "tune record"); break; }
        rc = cs_omp(plan, y_dev, batch, K, &h, x, supp, nullptr, nullptr, stream);
        if (rc != CS_OK) break;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
          rc = cuda_fail(e, "tune timing");
          break;
        }
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep == 1 || (rep > 1 && t < ms[i])) ms[i] = t;
      }
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (x) cudaFreeAsync(x, st);
  if (supp) cudaFreeAsync(supp, st);
  if (rc != CS_OK) return rc;
  CS_CUDA(cudaStreamSynchronize(st), "tune synchronize");
  size_t bi = 0;
  for (size_t i = 1; i < ladder.size(); ++i)
    if (ms[i] < ms[bi]) bi = i;
  plan->t_switch_tuned = ladder[bi];
  *t_best = ladder[bi];
  const int n = (int)ladder.size() < cap ? (int)ladder.size() : cap;
  for (int i = 0; i < n; ++i) {
    cand_out[i] = ladder[i];
    ms_out[i] = ms[i];
  }
  if (n_out) *n_out = (int)ladder.size();
  return CS_OK;
}

extern "C" cs_status cs_plan_switch(cs_plan_t plan, int32_t* t_switch) {
  if (!plan || !t_switch) return CS_ERR_INVALID;
  *t_switch = plan_switch(plan);
  return CS_OK;
}

extern "C" cs_status cs_fma_probe(int32_t iters, float* sink_dev, double* flops, void* stream) {
  using namespace csf;
  if (iters < 1 || !flops) return CS_ERR_INVALID;
  double f = 0.0;
  CS_CUDA(launch_fma_probe(iters, sink_dev, (cudaStream_t)stream, &f), "fma probe");
  *flops = f;
  return CS_OK;
}
