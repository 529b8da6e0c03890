// The WIDE factorisation engine of the FP32 forms (Galerkin, no
// oscillatory data): the FMA banded Cholesky of band_block.cuh with one unit
// per warp and column blocks of 16, instantiated in a translation unit of
// its own so that it compiles beside the others.
#include "upscale_impl.cuh"

namespace stomsfem {

int launch_wide(bool fp64_acc, int mode, const UpscaleArgs& A, long long max_blocks, cudaStream_t st) {
  if (fp64_acc) {
    if (mode != kModeAll) return set_error(STOMSFEM_EINVAL, "FP32 + refinement runs one launch mode");
    return launch_rpl<float, double, 32, kModeAll, false, false>(A, max_blocks, st);
  }
  if (mode == kModeFwd) return launch_rpl<float, float, 32, kModeFwd, false, false>(A, max_blocks, st);
  if (mode == kModeRest) return launch_rpl<float, float, 32, kModeRest, false, false>(A, max_blocks, st);
  return launch_rpl<float, float, 32, kModeAll, false, false>(A, max_blocks, st);
}

}  // namespace stomsfem
