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

// Internal: FP64 upscaling of a device-side list of units (no oversampling).
int upscale_list_fp64(const stomsfem_grid* grid, const double* a, int32_t S, const int32_t* unit_list,
                      const int32_t* unit_count, double* Ke, double* be, void* workspace,
                      size_t workspace_bytes, cudaStream_t st);
size_t upscale_slot_bytes_fp64(const stomsfem_grid* grid);
// Workspace of upscale_list_fp64 that keeps every SM at its resident units
// (16 slots per SM: four blocks of two warps, two units per warp).
size_t upscale_list_workspace_fp64(const stomsfem_grid* grid);
// Scratch slots (units in flight) of one block of the upscaling launch for a
// grid, oversampling limit and precision with the default engine: the least
// workspace stomsfem_upscale accepts, in slots (8 in the FP32 forms, two
// units per warp; 4 in FP64).
int upscale_slots_per_block(const stomsfem_grid* grid, int32_t max_oversample, int precision);
// stomsfem_upscale (Galerkin, no phi/status) with the plan's launch
// choices: at most blocks_per_sm resident CTAs per SM (0: as many as fit),
// split_fp32 = 0 runs the FP32 form as one launch, engine picks the FP32
// forms' factorisation (STOMSFEM_ENGINE_*), order the unit order
// (STOMSFEM_ORDER_*).
int upscale_tuned(const stomsfem_grid* grid, const double* a, const int8_t* oversample, int32_t max_oversample,
                  int32_t S, int32_t precision, int32_t refine_iters, double* Ke, double* be, void* workspace,
                  size_t workspace_bytes, cudaStream_t st, int blocks_per_sm, int split_fp32, int engine,
                  int order);
// The factorisation engine (STOMSFEM_ENGINE_*) a request resolves to for a
// grid, oversampling limit and precision.
int upscale_engine_of(const stomsfem_grid* grid, int32_t max_oversample, int precision, int requested);
// Whether engine (not AUTO) can serve a grid, oversampling limit and
// precision: BLOCKED always, WIDE in the FP32 forms, the tensor-core
// engines in the FP32 forms with 4 <= nf/nc and a half bandwidth <= 40.
bool upscale_engine_ok(const stomsfem_grid* grid, int32_t max_oversample, int precision, int engine);

// Petrov-Galerkin upscaling with the oscillatory boundary data of the cell
// problems (the Petrov-Galerkin half of stomsfem_upscale_bc).
int upscale_pg_oscillatory(const stomsfem_grid* grid, const double* a, const int8_t* oversample,
                           int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters, double* Ke,
                           double* be, double* phi, int32_t* unit_status, void* workspace, size_t workspace_bytes,
                           stomsfem_stream_t stream);

// Fine-grid Q1 FEM by multigrid-preconditioned CG (fine_mg.cu): grids whose
// element count halves down to at most 16, workspace bytes for S samples,
// and the solve (synchronises the stream).
bool fine_mg_supported(int nf);
size_t fine_mg_workspace_bytes(int nf, int S);
int fine_mg_solve(int nf, double f, const double* a, int S, double* u, void* workspace, size_t workspace_bytes,
                  double rtol, int max_iters, cudaStream_t st, double* res, int* iters);

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
