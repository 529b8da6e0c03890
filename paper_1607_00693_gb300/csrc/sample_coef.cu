// Coefficient sampling a(x, xi) at fine-element centroids (Sec. 2.1.3).
//
// The bumps are Gaussians on a tensor lattice, so
//   z(x, y) = sum_bx gx_bx(x) * U_bx(y),   U_bx(y) = sum_by xi[by][bx] gy_by(y),
// with gx_bx(x) = exp(-(x - cx_bx)^2 / w^2) (and gy likewise).  A block
// handles one sample and a strip of R element rows: gy of the strip and then
// U are built once in shared memory, each thread keeps gx of its column in
// registers and sweeps the strip, so the work per element is nbx FMAs plus
// the final exponential (the table-driven FP64 exp of fexp.cuh); the strip
// height R amortises the nbx exponentials of gx over R elements.
#include "common.cuh"
#include "fexp.cuh"

namespace stomsfem {

constexpr int kMaxBumps = 64;  // per lattice side
constexpr int kCoefThreads = 128;
constexpr size_t kCoefSmem = 48 * 1024;

__host__ __device__ inline int coef_rows(int nbx, int nby) {
  int R = 128;
  while (R > 8 && (size_t)(64 + (size_t)(nbx + nby) * R) * sizeof(double) > kCoefSmem) R >>= 1;
  return R;
}

template <int NBX>
__global__ void __launch_bounds__(kCoefThreads)
sample_coef_kernel(int nf, int kind, int nbx, int nby, int R, double w, double scale, double clog,
                   double gain, const double* __restrict__ xi, double* __restrict__ a) {
  extern __shared__ double csm[];
  double* tab = csm;                     // [64] 2^(j/64)
  double* gy = csm + 64;                 // [nby][R]
  double* U = gy + (size_t)nby * R;      // [nbx][R]
  const int s = blockIdx.y;
  const int ey0 = blockIdx.x * R;
  const int rows = min(R, nf - ey0);
  const double h = 1.0 / nf;
  const double iw2 = 1.0 / (w * w);
  const double* xs = xi + (size_t)s * nbx * nby;
  exp_table_fill(tab);
  __syncthreads();
  for (int q = threadIdx.x; q < nby * rows; q += blockDim.x) {
    const int by = q / rows, r = q % rows;
    const double dy = (ey0 + r + 0.5) * h - (by + 0.5) / nby;
    gy[by * R + r] = fexp(-dy * dy * iw2, tab);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nbx * rows; q += blockDim.x) {
    const int bx = q / rows, r = q % rows;
    double acc = 0.0;
    for (int by = 0; by < nby; ++by) acc = fma(__ldg(xs + by * nbx + bx), gy[by * R + r], acc);
    U[bx * R + r] = acc;
  }
  __syncthreads();
  for (int ex = threadIdx.x; ex < nf; ex += blockDim.x) {
    const double x = (ex + 0.5) * h;
    double gx[NBX];
#pragma unroll
    for (int bx = 0; bx < NBX; ++bx) {
      const double dx = x - (bx + 0.5) / nbx;
      gx[bx] = bx < nbx ? fexp(-dx * dx * iw2, tab) : 0.0;
    }
    double* arow = a + ((size_t)s * nf + ey0) * nf + ex;
    for (int r = 0; r < rows; ++r) {
      double z = 0.0;
#pragma unroll
      for (int bx = 0; bx < NBX; ++bx)
        if (bx < nbx) z = fma(gx[bx], U[bx * R + r], z);
      double v;
      if (kind == STOMSFEM_FIELD_EXP)
        v = fexp(scale * z, tab);
      else if (kind == STOMSFEM_FIELD_AFFINE)
        v = fma(scale, z, gain);
      else
        v = fexp(clog / (1.0 + fexp(-gain * z, tab)), tab);
      arow[(size_t)r * nf] = v;
    }
  }
}

// The same sum in FP32 arithmetic (expf, FP32 bump tables and sums; the
// stored values are FP64): for the FP32 upscaling form, whose cell matrices
// are FP32 anyway.  Relative error of a about |scale z| times a few 1e-7.
template <int NBX>
__global__ void __launch_bounds__(kCoefThreads)
sample_coef_f32_kernel(int nf, int kind, int nbx, int nby, int R, float w, float scale, float clog,
                       float gain, const double* __restrict__ xi, double* __restrict__ a) {
  extern __shared__ float fsm[];
  float* gy = fsm;                      // [nby][R]
  float* U = gy + (size_t)nby * R;      // [nbx][R]
  const int s = blockIdx.y;
  const int ey0 = blockIdx.x * R;
  const int rows = min(R, nf - ey0);
  const float h = 1.0f / (float)nf;
  const float iw2 = 1.0f / (w * w);
  const double* xs = xi + (size_t)s * nbx * nby;
  for (int q = threadIdx.x; q < nby * rows; q += blockDim.x) {
    const int by = q / rows, r = q % rows;
    const float dy = ((float)(ey0 + r) + 0.5f) * h - ((float)by + 0.5f) / (float)nby;
    gy[by * R + r] = expf(-dy * dy * iw2);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nbx * rows; q += blockDim.x) {
    const int bx = q / rows, r = q % rows;
    float acc = 0.f;
    for (int by = 0; by < nby; ++by) acc = fmaf((float)__ldg(xs + by * nbx + bx), gy[by * R + r], acc);
    U[bx * R + r] = acc;
  }
  __syncthreads();
  for (int ex = threadIdx.x; ex < nf; ex += blockDim.x) {
    const float x = ((float)ex + 0.5f) * h;
    float gx[NBX];
#pragma unroll
    for (int bx = 0; bx < NBX; ++bx) {
      const float dx = x - ((float)bx + 0.5f) / (float)nbx;
      gx[bx] = bx < nbx ? expf(-dx * dx * iw2) : 0.f;
    }
    double* arow = a + ((size_t)s * nf + ey0) * nf + ex;
    for (int r = 0; r < rows; ++r) {
      float z = 0.f;
#pragma unroll
      for (int bx = 0; bx < NBX; ++bx)
        if (bx < nbx) z = fmaf(gx[bx], U[bx * R + r], z);
      const float v = kind == STOMSFEM_FIELD_EXP      ? expf(scale * z)
                      : kind == STOMSFEM_FIELD_AFFINE ? fmaf(scale, z, gain)
                                                      : expf(clog / (1.0f + expf(-gain * z)));
      arow[(size_t)r * nf] = (double)v;
    }
  }
}

}  // namespace stomsfem

using namespace stomsfem;

static int sample_coef_impl(const stomsfem_grid* grid, const stomsfem_field* field, const double* xi,
                            int32_t S, int32_t precision, double* a, stomsfem_stream_t stream) {
  if (!grid || !field) return set_error(STOMSFEM_EINVAL, "grid/field is NULL");
  if (grid->nf <= 0 || S < 0) return set_error(STOMSFEM_EINVAL, "bad nf or S");
  if (precision != STOMSFEM_FP64 && precision != STOMSFEM_FP32)
    return set_error(STOMSFEM_EINVAL, "sampling precision must be STOMSFEM_FP64 or STOMSFEM_FP32");
  if (field->kind != STOMSFEM_FIELD_EXP && field->kind != STOMSFEM_FIELD_EXP_SIGMOID &&
      field->kind != STOMSFEM_FIELD_AFFINE)
    return set_error(STOMSFEM_EINVAL, "unknown field kind %d", field->kind);
  if (field->nbx <= 0 || field->nby <= 0 || field->nbx > kMaxBumps || field->nby > kMaxBumps)
    return set_error(STOMSFEM_EINVAL, "bump lattice %dx%d outside 1..%d per side", field->nbx,
                     field->nby, kMaxBumps);
  if (!(field->width > 0.0)) return set_error(STOMSFEM_EINVAL, "width must be > 0");
  if (S == 0) return STOMSFEM_OK;
  if (!xi || !a) return set_error(STOMSFEM_EINVAL, "xi and a must be device pointers");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nbx = field->nbx;
  const int R = coef_rows(field->nbx, field->nby);
  const size_t smem = precision == STOMSFEM_FP64
                          ? (64 + (size_t)(field->nbx + field->nby) * R) * sizeof(double)
                          : (size_t)(field->nbx + field->nby) * R * sizeof(float);
  const size_t K = (size_t)field->nbx * field->nby;
  // the sample index runs over gridDim.y (at most 65535 per launch)
  for (int s0 = 0; s0 < S; s0 += 65535) {
    const int Sc = S - s0 < 65535 ? S - s0 : 65535;
    dim3 grd((grid->nf + R - 1) / R, Sc);
    const double* xs = xi + (size_t)s0 * K;
    double* as = a + (size_t)s0 * grid->nf * grid->nf;
#define LAUNCH(N)                                                                                        \
  do {                                                                                                   \
    if (precision == STOMSFEM_FP64)                                                                      \
      sample_coef_kernel<N><<<grd, kCoefThreads, smem, st>>>(grid->nf, field->kind, nbx, field->nby, R,  \
                                                             field->width, field->scale,                 \
                                                             field->contrast_log, field->gain, xs, as);  \
    else                                                                                                 \
      sample_coef_f32_kernel<N><<<grd, kCoefThreads, smem, st>>>(                                        \
          grid->nf, field->kind, nbx, field->nby, R, (float)field->width, (float)field->scale,            \
          (float)field->contrast_log, (float)field->gain, xs, as);                                       \
  } while (0)
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

extern "C" int stomsfem_sample_coef(const stomsfem_grid* grid, const stomsfem_field* field,
                                    const double* xi, int32_t S, double* a,
                                    stomsfem_stream_t stream) {
  return sample_coef_impl(grid, field, xi, S, STOMSFEM_FP64, a, stream);
}

extern "C" int stomsfem_sample_coef_precision(const stomsfem_grid* grid, const stomsfem_field* field,
                                              const double* xi, int32_t S, int32_t precision, double* a,
                                              stomsfem_stream_t stream) {
  return sample_coef_impl(grid, field, xi, S, precision, a, stream);
}
