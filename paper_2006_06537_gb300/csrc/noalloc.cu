// Allocation-free variant of the H-matrix product (fifa_matvec_static).
//
// Some callers cannot allocate device memory on their own: a plug-in whose
// host framework owns every byte of device memory and forbids direct
// allocation, a process whose memory is fully reserved by a pooling allocator
// (so a raw cudaMalloc would fail), or a latency-critical loop that must not
// enter the allocator because cudaMalloc may synchronize the device.  For them
// this entry point keeps its scratch in a file-scope device array instead of
// the context arena, and calls no allocation routine at all.
//
// The array is FIFA_STATIC_SCRATCH_DOUBLES doubles (8 MiB); every GPU that
// loads the library holds it until the process exits.  All calls share it, so
// calls that overlap on the GPU (different streams, different contexts) race
// on it and must be ordered by the caller.  Every entry a call reads is first
// written by that same call (leaf partial projections, then their per-node
// sums), so stale contents from a previous call are never used and nothing
// needs clearing.
#include <cuda.h>  // types of the two driver entry points looked up at run time (no link to the driver)
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fifa.h"
#include "fifa_api_internal.h"
#include "fifa_launch.h"

#define FIFA_STATIC_SCRATCH_DOUBLES (1 << 20)
#define FIFA_STATIC_MAX_DEVICES 64

static __device__ __align__(256) double g_matvec_scratch[FIFA_STATIC_SCRATCH_DOUBLES];

// Device address of g_matvec_scratch per device, looked up with that device
// current and kept together with the unique id of the context it belongs to:
// a device reset (or any re-creation of the context) makes the next call look
// the address up again instead of using a stale one.  In host code the symbol
// itself is only a host-side stand-in.
static double* g_scratch_addr[FIFA_STATIC_MAX_DEVICES];
static unsigned long long g_scratch_ctx[FIFA_STATIC_MAX_DEVICES];
static std::mutex g_scratch_mu;

// Unique id of the calling thread's current context, 0 if unknown.
static unsigned long long current_context_id() {
  typedef CUresult (*get_current_t)(CUcontext*);
  typedef CUresult (*get_id_t)(CUcontext, unsigned long long*);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {  // called with g_scratch_mu held
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, nullptr) == cudaSuccess)
      get_current = (get_current_t)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, nullptr) == cudaSuccess)
      get_id = (get_id_t)f;
    cudaGetLastError();
    looked_up = true;
  }
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

static cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  const unsigned long long id = current_context_id();
  if (!g_scratch_addr[dev] || id == 0 || id != g_scratch_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_matvec_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (double*)p;
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

extern "C" fifa_status fifa_matvec_static(fifa_ctx* ctx, const fifa_hmat* A, const double* in_dev, double* out_dev,
                                          int nrhs) {
  if (!ctx || !A || !in_dev || !out_dev || in_dev == out_dev || nrhs < 1 || nrhs > SWEEP_RHS_MAX)
    return FIFA_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device || dev < 0 || dev >= FIFA_STATIC_MAX_DEVICES)
    return FIFA_ERR_INVALID_ARG;
  const Plan* P = A->plan;
  const int cap = A->host.cap;
  const size_t part = (size_t)P->nleaf * (P->L > 0 ? P->L : 1) * cap * SWEEP_RHS_MAX;
  const size_t proj = (size_t)(P->nnodes > 0 ? P->nnodes : 1) * 2 * cap * SWEEP_RHS_MAX;
  if (part + proj > FIFA_STATIC_SCRATCH_DOUBLES) return FIFA_ERR_UNSUPPORTED;
  double* base = nullptr;
  cudaError_t e = scratch_address(dev, &base);
  if (e != cudaSuccess) {
    ctx->last_cuda = e;
    return FIFA_ERR_CUDA;
  }
  e = launch_matvec(A->dev, P->nleaf, P->L, in_dev, nrhs, base, base + part, out_dev, ctx->stream);
  if (e != cudaSuccess) {
    ctx->last_cuda = e;
    return FIFA_ERR_CUDA;
  }
  return FIFA_OK;
}
