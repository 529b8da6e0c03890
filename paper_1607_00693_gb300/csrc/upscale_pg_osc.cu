// Petrov-Galerkin local upscaling with the oscillatory boundary data of the
// cell problems (Sec. 5.3; Eq. stiffness_local_petrov): the second half of
// stomsfem_upscale_bc, a translation unit of its own.
#include "upscale_impl.cuh"

namespace stomsfem {

int upscale_pg_oscillatory(const stomsfem_grid* grid, const double* a, const int8_t* oversample,
                           int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters, double* Ke,
                           double* be, double* phi, int32_t* unit_status, void* workspace, size_t workspace_bytes,
                           stomsfem_stream_t stream) {
  return upscale_run<true, true>(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, phi,
                                 unit_status, workspace, workspace_bytes, stream);
}

}  // namespace stomsfem
