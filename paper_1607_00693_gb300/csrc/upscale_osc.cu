// Local upscaling with the oscillatory boundary data of the cell problems
// (the MsFEM option of the short-correlation example, Sec. 5.3): Galerkin
// here, Petrov-Galerkin in upscale_pg_osc.cu (translation units of their
// own, compiled in parallel); bilinear data go to stomsfem_upscale and
// stomsfem_upscale_pg.
#include "upscale_impl.cuh"

using namespace stomsfem;

extern "C" int stomsfem_upscale_bc(const stomsfem_grid* grid, int32_t pg, int32_t bc, const double* a,
                                   const int8_t* oversample, int32_t max_oversample, int32_t S, int32_t precision,
                                   int32_t refine_iters, double* Ke, double* be, double* phi, int32_t* unit_status,
                                   void* workspace, size_t workspace_bytes, stomsfem_stream_t stream) {
  if (pg != 0 && pg != 1) return set_error(STOMSFEM_EINVAL, "pg must be 0 or 1");
  if (bc != STOMSFEM_BC_BILINEAR && bc != STOMSFEM_BC_OSCILLATORY) return set_error(STOMSFEM_EINVAL, "bad bc %d", bc);
  if (bc == STOMSFEM_BC_BILINEAR)
    return pg ? stomsfem_upscale_pg(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, phi,
                                    unit_status, workspace, workspace_bytes, stream)
              : stomsfem_upscale(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, phi,
                                 unit_status, workspace, workspace_bytes, stream);
  if (pg)
    return upscale_pg_oscillatory(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, phi,
                                  unit_status, workspace, workspace_bytes, stream);
  return upscale_run<false, true>(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, phi,
                                  unit_status, workspace, workspace_bytes, stream);
}
