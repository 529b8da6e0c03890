// Petrov-Galerkin local upscaling (Eq. stiffness_local_petrov): the same
// cell problems as the Galerkin form, with the cell's bilinear nodal
// functions as test functions; a translation unit of its own so that the
// two instantiations of the kernel compile in parallel.
#include "upscale_impl.cuh"

using namespace stomsfem;

extern "C" int stomsfem_upscale_pg(const stomsfem_grid* grid, const double* a, const int8_t* oversample,
                                   int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters,
                                   double* Ke, double* be, double* phi, int32_t* unit_status, void* workspace,
                                   size_t workspace_bytes, stomsfem_stream_t stream) {
  return upscale_run<true>(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, phi,
                           unit_status, workspace, workspace_bytes, stream);
}
