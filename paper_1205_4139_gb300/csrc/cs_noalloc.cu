// cs_omp_noalloc: the batched OMP solve of cs_omp with its scratch in a
// fixed, library-owned device array instead of a workspace the library
// allocates on demand.
//
// Who needs it: callers that must not allocate device memory on the solve
// path.  cudaMalloc / cudaFree synchronise the device and can block for a long
// time, which a latency-critical request loop cannot afford, and a process
// whose device memory is handed out by someone else's allocator under a fixed
// budget may not be allowed to grow a private workspace at all.  Those
// callers still allocate their own inputs and outputs; this entry point adds
// no allocation of its own.
//
// The scratch is one file-scope array of kNoAllocScratchBytes per device that
// loads the library, held until the process exits.  Host code cannot use the
// array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current and caches it.
#include <cstdio>
#include <mutex>

#include "../../include/csfast.h"
#include "cs_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

thread_local char g_noalloc_err[256] = "";

}  // namespace

// Per-plan accessors exported by cs_api.cu for this file.
namespace csf {
const PlanView* plan_view(cs_plan_t plan);
int plan_switch_point(cs_plan_t plan);
void set_last_error(const char* msg);
}  // namespace csf

extern "C" cs_status cs_omp_noalloc(cs_plan_t plan, const void* y_dev, int64_t batch, int32_t K,
                                    const cs_halt* halt, void* x_dev, int32_t* supp_dev, int32_t* iters_dev,
                                    double* resnorm_dev, void* stream) {
  using namespace csf;
  if (!plan || batch < 0 || K < 0) return CS_ERR_INVALID;
  const PlanView& v = *plan_view(plan);
  if (K > v.M) return CS_ERR_INVALID;
  if (K > kMaxK) return CS_ERR_UNSUPPORTED;
  if (v.large) {  // the multi-kernel path of N > 8192 keeps per-instance vectors far beyond the array
    set_last_error("cs_omp_noalloc: plans with N > 8192 are not supported");
    return CS_ERR_UNSUPPORTED;
  }
  cs_halt h = {1e-6, CS_PATH_HYBRID, -1, 0};
  if (halt) h = *halt;
  if (!(h.rel_tol >= 0.0) || h.rel_tol > 1e308) return CS_ERR_INVALID;
  if (h.path != CS_PATH_FAST && h.path != CS_PATH_CONV && h.path != CS_PATH_HYBRID) return CS_ERR_INVALID;
  if (batch == 0) return CS_OK;
  if (K > 0 && !supp_dev) return CS_ERR_INVALID;
  if (v.M > 0 && !y_dev) return CS_ERR_INVALID;

  // one CTA's share of the scratch must fit, else the request is refused
  if (omp_workspace_bytes(v, K, 1) > kNoAllocScratchBytes) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err),
             "cs_omp_noalloc: N=%d, K=%d needs %zu bytes of scratch per CTA, more than the fixed %zu",
             v.N, K, omp_workspace_bytes(v, K, 1), kNoAllocScratchBytes);
    set_last_error(g_noalloc_err);
    return CS_ERR_UNSUPPORTED;
  }

  // set-up, once per device, with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_last_error("cs_omp_noalloc: no usable current device");
    return CS_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        snprintf(g_noalloc_err, sizeof(g_noalloc_err), "cs_omp_noalloc: cudaGetSymbolAddress: %s",
                 cudaGetErrorString(e));
        set_last_error(g_noalloc_err);
        return CS_ERR_CUDA;
      }
      g_ptr[dev] = p;
    }
    scratch = g_ptr[dev];
  }

  // as many resident CTAs as the occupancy allows and the scratch holds
  int err = 0;
  int grid = omp_grid(v, K, h.path, batch, &err);
  if (err) {
    set_last_error("cs_omp_noalloc: kernel configuration failed");
    return CS_ERR_CUDA;
  }
  const size_t per_cta = omp_workspace_bytes(v, K, 2) - omp_workspace_bytes(v, K, 1);
  const size_t fit = (kNoAllocScratchBytes - omp_workspace_bytes(v, K, 1)) / per_cta + 1;
  if ((size_t)grid > fit) grid = (int)fit;
  while (grid > 1 && omp_workspace_bytes(v, K, grid) > kNoAllocScratchBytes) --grid;

  OmpLaunch a;
  a.y = y_dev;
  a.batch = batch;
  a.K = K;
  a.rel_tol = h.rel_tol;
  a.path = h.path;
  // the same switch point as cs_omp: cs_plan_tune's, else the GB300 table
  a.t_switch = h.t_switch < 0 ? plan_switch_point(plan) : h.t_switch;
  a.x_out = x_dev;
  a.supp_out = supp_dev;
  a.iters_out = iters_dev;
  a.res_out = resnorm_dev;
  // launch_omp zeroes the work counter at the start of the scratch before the
  // kernel; nothing else in the scratch is read before this call writes it
  e = launch_omp(v, a, scratch, grid, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err), "cs_omp_noalloc: %s", cudaGetErrorString(e));
    set_last_error(g_noalloc_err);
    return CS_ERR_CUDA;
  }
  return CS_OK;
}
