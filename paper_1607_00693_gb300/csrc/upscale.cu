// Galerkin local upscaling (Eq. stiffness_local): the C entry points, and
// the FP64 list mode used by the fallbacks of the surrogate and of the
// random interpolation.  The kernel and its host runner are in
// upscale_impl.cuh.
#include "upscale_impl.cuh"

using namespace stomsfem;

extern "C" int stomsfem_upscale_workspace_size(const stomsfem_grid* grid, int32_t max_oversample,
                                               int32_t precision, size_t* slot_bytes,
                                               size_t* recommended_bytes) {
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (max_oversample < 0 || precision < 0 || precision > 2)
    return set_error(STOMSFEM_EINVAL, "bad max_oversample/precision");
  int nmax, bmax;
  patch_limits(grid, max_oversample, &nmax, &bmax);
  size_t sb, lb;
  slot_layout(nmax, bmax, precision, &sb, &lb);
  if (slot_bytes) *slot_bytes = sb;
  if (recommended_bytes) {
    const int sms = device_sm_count();
    *recommended_bytes = sb * (size_t)(sms > 0 ? sms : 152) * 32 + cell_list_bytes(grid);
  }
  return STOMSFEM_OK;
}

extern "C" int stomsfem_upscale(const stomsfem_grid* grid, const double* a,
                                const int8_t* oversample, int32_t max_oversample, int32_t S,
                                int32_t precision, int32_t refine_iters, double* Ke, double* be,
                                double* phi, int32_t* unit_status, void* workspace,
                                size_t workspace_bytes, stomsfem_stream_t stream) {
  return upscale_run<false>(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, phi,
                            unit_status, workspace, workspace_bytes, stream);
}

extern "C" int stomsfem_upscale_engine(const stomsfem_grid* grid, const double* a, const int8_t* oversample,
                                       int32_t max_oversample, int32_t S, int32_t precision, int32_t refine_iters,
                                       int32_t engine, int32_t order, double* Ke, double* be, double* phi,
                                       int32_t* unit_status, void* workspace, size_t workspace_bytes,
                                       stomsfem_stream_t stream) {
  if (engine < STOMSFEM_ENGINE_AUTO || engine > STOMSFEM_ENGINE_WIDE)
    return set_error(STOMSFEM_EINVAL, "unknown engine %d", engine);
  if (order != STOMSFEM_ORDER_CELL && order != STOMSFEM_ORDER_PATCH)
    return set_error(STOMSFEM_EINVAL, "unknown unit order %d", order);
  int rc = validate_grid(grid);
  if (rc) return rc;
  if (precision < 0 || precision > 2) return set_error(STOMSFEM_EINVAL, "bad precision %d", precision);
  if (engine != STOMSFEM_ENGINE_AUTO) {
    int nmax, bmax;
    patch_limits(grid, oversample ? max_oversample : 0, &nmax, &bmax);
    if (!upscale_engine_eligible(engine, precision, grid->nf / grid->nc, bmax))
      return set_error(STOMSFEM_EINVAL,
                       "engine %d is not offered here (FP64: BLOCKED only; tensor-core engines: 4 <= nf/nc and a "
                       "half bandwidth <= 40)", engine);
  }
  UpscaleTuning t;
  t.engine = engine;
  t.order = order;
  return upscale_run<false>(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, phi,
                            unit_status, workspace, workspace_bytes, stream, t);
}

namespace stomsfem {

// FP64 upscaling of the units listed on the device (list and count device
// pointers; the count is read by the kernel), no oversampling; used by the
// surrogate's fallback.  Launches one grid sized to the resident warps.
int upscale_list_fp64(const stomsfem_grid* grid, const double* a, int32_t S, const int32_t* unit_list,
                      const int32_t* unit_count, double* Ke, double* be, void* workspace,
                      size_t workspace_bytes, cudaStream_t st) {
  int rc = validate_grid(grid);
  if (rc) return rc;
  int nmax, bmax;
  patch_limits(grid, 0, &nmax, &bmax);
  if (bmax > kMaxBand) return set_error(STOMSFEM_EINVAL, "bandwidth %d > %d", bmax, kMaxBand);
  size_t sb, lb;
  slot_layout(nmax, bmax, STOMSFEM_FP64, &sb, &lb);
  // two units per warp, as the plain FP64 upscaler (the list's cells have no
  // oversampling: one patch shape)
  constexpr int kSlotsPerBlock = upscale_warps(true, 16) * 2;
  const long long slots = (long long)(workspace_bytes / sb);
  if (slots < kSlotsPerBlock) return set_error(STOMSFEM_ENOMEM, "fallback workspace too small");
  UpscaleArgs A;
  A.a = a;
  A.oversample = nullptr;
  A.nf = grid->nf;
  A.nc = grid->nc;
  A.rho = grid->nf / grid->nc;
  A.max_o = 0;
  A.S = S;
  A.f = grid->f;
  A.fq = grid->f / (4.0 * (double)grid->nf * (double)grid->nf);
  A.fH2 = grid->f / ((double)grid->nc * (double)grid->nc);
  A.refine = 0;
  A.Ke = Ke;
  A.be = be;
  A.phi = nullptr;
  A.status = nullptr;
  A.ws = static_cast<unsigned char*>(workspace);
  A.slot_bytes = sb;
  A.l_bytes = lb;
  A.bmax = bmax;
  A.nmax = nmax;
  A.units = (long long)S * grid->nc * grid->nc;
  A.unit_list = unit_list;
  A.unit_count = unit_count;
  A.cell_list = nullptr;
  A.cell_count = nullptr;
  A.blocks_per_sm_cap = 0;
  A.order = 0;
  return launch_rpl<double, double, 16>(A, slots / kSlotsPerBlock, st);
}

int upscale_slots_per_block(const stomsfem_grid* grid, int32_t max_oversample, int precision) {
  int nmax, bmax;
  patch_limits(grid, max_oversample, &nmax, &bmax);
  const int G = upscale_engine_lanes(upscale_engine(kEngineAuto, precision, grid->nf / grid->nc, bmax));
  return upscale_warps(precision == STOMSFEM_FP64, G) * (32 / G);
}

int upscale_engine_of(const stomsfem_grid* grid, int32_t max_oversample, int precision, int requested) {
  int nmax, bmax;
  patch_limits(grid, max_oversample, &nmax, &bmax);
  return upscale_engine(requested, precision, grid->nf / grid->nc, bmax);
}

bool upscale_engine_ok(const stomsfem_grid* grid, int32_t max_oversample, int precision, int engine) {
  int nmax, bmax;
  patch_limits(grid, max_oversample, &nmax, &bmax);
  return upscale_engine_eligible(engine, precision, grid->nf / grid->nc, bmax);
}

size_t upscale_slot_bytes_fp64(const stomsfem_grid* grid) {
  int nmax, bmax;
  patch_limits(grid, 0, &nmax, &bmax);
  size_t sb, lb;
  slot_layout(nmax, bmax, STOMSFEM_FP64, &sb, &lb);
  return sb;
}

size_t upscale_list_workspace_fp64(const stomsfem_grid* grid) {
  return upscale_slot_bytes_fp64(grid) * (size_t)(device_sm_count() > 0 ? device_sm_count() : 152) * 16;
}

// stomsfem_upscale with launch choices (the plan's autotuner).
int upscale_tuned(const stomsfem_grid* grid, const double* a, const int8_t* oversample, int32_t max_oversample,
                  int32_t S, int32_t precision, int32_t refine_iters, double* Ke, double* be, void* workspace,
                  size_t workspace_bytes, cudaStream_t st, int blocks_per_sm, int split_fp32, int engine,
                  int order) {
  UpscaleTuning t;
  t.blocks_per_sm = blocks_per_sm;
  t.split_fp32 = split_fp32;
  t.engine = engine;
  t.order = order;
  return upscale_run<false>(grid, a, oversample, max_oversample, S, precision, refine_iters, Ke, be, nullptr,
                            nullptr, workspace, workspace_bytes, reinterpret_cast<stomsfem_stream_t>(st), t);
}

}  // namespace stomsfem
