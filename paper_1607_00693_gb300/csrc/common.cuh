// Shared host/device helpers of the StoMsFEM CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "stomsfem.h"

namespace stomsfem {

// Records a one-line error message for the calling host thread and returns code.
int set_error(int code, const char* fmt, ...);
int check_cuda(cudaError_t e, const char* what);
int device_sm_count();

#define STOMSFEM_TRY_CUDA(expr)                                  \
  do {                                                           \
    int _rc = ::stomsfem::check_cuda((expr), #expr);             \
    if (_rc != STOMSFEM_OK) return _rc;                          \
  } while (0)

// Full-warp sum (every lane receives the total).
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int wrap_inc(int c, int R) { return (c + 1 == R) ? 0 : c + 1; }

}  // namespace stomsfem
