// Allocation-free upscaling entry point.
//
// stomsfem_upscale needs device scratch for the per-warp banded factors;
// normally the caller allocates it.  Some callers cannot allocate device
// memory at the point where they upscale: code that runs inside another
// framework's memory pool or a plugin that must not grow the process's
// device footprint, real-time loops where cudaMalloc's implicit
// synchronisation is not allowed, or host programs that only receive device
// pointers.  This file gives them one more entry point whose scratch is a
// fixed file-scope device array, so the call itself allocates nothing.
//
// The array lives in this translation unit's own module: under CUDA's
// default lazy module loading a device reserves it when this entry point is
// first used there, and keeps it until the process exits.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace stomsfem {

// 64 MiB: about 150 unit slots for H/h = 32 with oversampling up to 4 in
// FP32 (one block of the launch is the minimum it needs: 8 slots with the
// two-units-per-warp FP32 kernel, 4 in FP64).
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_upscale_scratch[kStaticScratchBytes];

static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {nullptr};
static unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // context id the address belongs to

// Device address of the array on the current device (the symbol's name is
// only a host-side handle), looked up once per device and context: the
// cache is keyed on the current context's unique id, so after a device
// reset (a new primary context, the module loaded again) the address is
// looked up afresh instead of reusing the old context's.
static int scratch_address(void** out) {
  int dev = 0;
  STOMSFEM_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(STOMSFEM_EINVAL, "device ordinal %d beyond %d", dev, kMaxDevices);
  STOMSFEM_TRY_CUDA(cudaFree(nullptr));  // makes the device's primary context current
  // the two driver calls are fetched through the runtime, so the library
  // does not link the driver library itself (it loads without a GPU)
  static CUresult (*get_current)(CUcontext*) = nullptr;
  static CUresult (*get_id)(CUcontext, unsigned long long*) = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!get_current || !get_id) {
      cudaDriverEntryPointQueryResult q1, q2;
      void *f1 = nullptr, *f2 = nullptr;
      if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
          cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
          q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
        return set_error(STOMSFEM_ECUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId unavailable");
      get_current = reinterpret_cast<CUresult (*)(CUcontext*)>(f1);
      get_id = reinterpret_cast<CUresult (*)(CUcontext, unsigned long long*)>(f2);
    }
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return set_error(STOMSFEM_ECUDA, "no current CUDA context for the static scratch");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != id) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_upscale_scratch);
    if (e != cudaSuccess || !p)
      return set_error(STOMSFEM_ECUDA, "cudaGetSymbolAddress(static scratch): %s",
                       cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = id;
  }
  *out = g_scratch_addr[dev];
  return STOMSFEM_OK;
}

}  // namespace stomsfem

using namespace stomsfem;

extern "C" size_t stomsfem_upscale_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" int stomsfem_upscale_noalloc(const stomsfem_grid* grid, const double* a,
                                        const int8_t* oversample, int32_t max_oversample,
                                        int32_t S, int32_t precision, int32_t refine_iters,
                                        double* Ke, double* be, double* phi,
                                        int32_t* unit_status, stomsfem_stream_t stream) {
  size_t slot = 0;
  int rc = stomsfem_upscale_workspace_size(grid, oversample ? max_oversample : 0, precision, &slot,
                                           nullptr);
  if (rc != STOMSFEM_OK) return rc;
  // the upscaling launch needs at least the slots of one block
  const int need = upscale_slots_per_block(grid, oversample ? max_oversample : 0, precision);
  if (slot * need > kStaticScratchBytes)
    return set_error(STOMSFEM_EINVAL,
                     "patch too large for the static scratch: %d slots of %zu bytes exceed %zu bytes "
                     "(reduce rho + 2*max_oversample or use stomsfem_upscale with a workspace)",
                     need, slot, kStaticScratchBytes);
  void* ws = nullptr;
  rc = scratch_address(&ws);
  if (rc != STOMSFEM_OK) return rc;
  return stomsfem_upscale(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be,
                          phi, unit_status, ws, kStaticScratchBytes, stream);
}
