// Coefficient sampling a(x, xi) at fine-element centroids (Sec. 2.1.3).
//
// The bumps are Gaussians on a tensor lattice, so
//   z(x, y) = sum_bx gx_bx(x) * U_bx(y),   U_bx(y) = sum_by xi[by][bx] gy_by(y),
// with gx_bx(x) = exp(-(x - cx_bx)^2 / w^2) (and gy likewise): a block
// handles one sample and a strip of kRows element rows; U for the strip is
// built in shared memory, each thread keeps gx of its column in registers
// and sweeps the strip, so the work per element is nbx FMAs plus the
// final exponential.
#include "common.cuh"

namespace stomsfem {

constexpr int kRows = 32;      // element rows per block
constexpr int kMaxBumps = 64;  // per lattice side held in registers
constexpr int kCoefThreads = 128;

template <int NBX>
__global__ void __launch_bounds__(kCoefThreads)
sample_coef_kernel(int nf, int kind, int nbx, int nby, double w, double scale, double clog,
                   double gain, const double* __restrict__ xi, double* __restrict__ a) {
  __shared__ double U[kMaxBumps][kRows];
  const int s = blockIdx.y;
  const int ey0 = blockIdx.x * kRows;
  const int rows = min(kRows, nf - ey0);
  const double h = 1.0 / nf;
  const double iw2 = 1.0 / (w * w);
  const double* xs = xi + (size_t)s * nbx * nby;
  for (int q = threadIdx.x; q < nbx * rows; q += blockDim.x) {
    const int bx = q / rows, r = q % rows;
    const double y = (ey0 + r + 0.5) * h;
    double acc = 0.0;
    for (int by = 0; by < nby; ++by) {
      const double dy = y - (by + 0.5) / nby;
      acc += xs[by * nbx + bx] * exp(-dy * dy * iw2);
    }
    U[bx][r] = acc;
  }
  __syncthreads();
  for (int ex = threadIdx.x; ex < nf; ex += blockDim.x) {
    const double x = (ex + 0.5) * h;
    double gx[NBX];
#pragma unroll
    for (int bx = 0; bx < NBX; ++bx) {
      const double dx = x - (bx + 0.5) / nbx;
      gx[bx] = bx < nbx ? exp(-dx * dx * iw2) : 0.0;
    }
    for (int r = 0; r < rows; ++r) {
      double z = 0.0;
#pragma unroll
      for (int bx = 0; bx < NBX; ++bx)
        if (bx < nbx) z += gx[bx] * U[bx][r];
      double v;
      if (kind == STOMSFEM_FIELD_EXP)
        v = exp(scale * z);
      else
        v = exp(clog / (1.0 + exp(-gain * z)));
      a[((size_t)s * nf + ey0 + r) * nf + ex] = v;
    }
  }
}

}  // namespace stomsfem

using namespace stomsfem;

extern "C" int stomsfem_sample_coef(const stomsfem_grid* grid, const stomsfem_field* field,
                                    const double* xi, int32_t S, double* a,
                                    stomsfem_stream_t stream) {
  if (!grid || !field) return set_error(STOMSFEM_EINVAL, "grid/field is NULL");
  if (grid->nf <= 0 || S < 0) return set_error(STOMSFEM_EINVAL, "bad nf or S");
  if (field->kind != STOMSFEM_FIELD_EXP && field->kind != STOMSFEM_FIELD_EXP_SIGMOID)
    return set_error(STOMSFEM_EINVAL, "unknown field kind %d", field->kind);
  if (field->nbx <= 0 || field->nby <= 0 || field->nbx > kMaxBumps || field->nby > 4096)
    return set_error(STOMSFEM_EINVAL, "bump lattice %dx%d outside 1..%d x 1..4096", field->nbx,
                     field->nby, kMaxBumps);
  if (!(field->width > 0.0)) return set_error(STOMSFEM_EINVAL, "width must be > 0");
  if (S == 0) return STOMSFEM_OK;
  if (!xi || !a) return set_error(STOMSFEM_EINVAL, "xi and a must be device pointers");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nbx = field->nbx;
  const size_t K = (size_t)field->nbx * field->nby;
  // the sample index runs over gridDim.y (at most 65535 per launch)
  for (int s0 = 0; s0 < S; s0 += 65535) {
    const int Sc = S - s0 < 65535 ? S - s0 : 65535;
    dim3 grd((grid->nf + kRows - 1) / kRows, Sc);
    const double* xs = xi + (size_t)s0 * K;
    double* as = a + (size_t)s0 * grid->nf * grid->nf;
#define LAUNCH(N)                                                                              \
  sample_coef_kernel<N><<<grd, kCoefThreads, 0, st>>>(grid->nf, field->kind, nbx, field->nby,  \
                                                      field->width, field->scale,              \
                                                      field->contrast_log, field->gain, xs, as)
    if (nbx <= 4) LAUNCH(4);
    else if (nbx <= 8) LAUNCH(8);
    else if (nbx <= 16) LAUNCH(16);
    else if (nbx <= 32) LAUNCH(32);
    else LAUNCH(64);
#undef LAUNCH
    STOMSFEM_TRY_CUDA(cudaGetLastError());
  }
  return STOMSFEM_OK;
}
