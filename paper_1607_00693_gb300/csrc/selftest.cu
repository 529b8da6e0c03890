// Failure-path self test of the bounded device waits used by the
// tensor-core kernels: a CTA initialises an mbarrier that nothing ever
// arrives at and waits on it with a short iteration limit; the wait gives up,
// the kernel records the timeout in a status word and returns normally, so
// the context stays usable.
#include "common.cuh"
#include "fexp.cuh"
#include "tc_gemm.cuh"

namespace stomsfem {

__global__ void wait_timeout_kernel(int32_t* status, uint32_t iters) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  __syncthreads();
  const bool ok = tc::mbar_wait_bounded(&mbar, 0, iters);
  if (threadIdx.x == 0) *status = ok ? STOMSFEM_OK : STOMSFEM_ETIMEOUT;
}

__global__ void exp_selftest_kernel(const double* __restrict__ t, int n, double* __restrict__ out) {
  __shared__ double tab[64];
  exp_table_fill(tab);
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = fexp(t[i], tab);
}

// Peak FMA rate probe: every thread runs 8 independent FMA chains (no
// memory traffic but one store per thread at the end).
template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(T* out, T s, int iters) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x * 1e-3 + i);
  const T c = (T)1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], s, c);
  }
  T t = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += a[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

template <typename T>
static int fma_rate(int iters, float* tflops) {
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  const int blocks = sms * 8, threads = 256;
  T* d = nullptr;
  STOMSFEM_TRY_CUDA(cudaMalloc(&d, sizeof(T) * (size_t)blocks * threads));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = check_cuda(cudaEventCreate(&e0), "event");
  if (!rc) rc = check_cuda(cudaEventCreate(&e1), "event");
  float best = 1e30f;
  for (int r = 0; r < 4 && !rc; ++r) {  // the first run warms up (clocks, module)
    cudaEventRecord(e0);
    fma_rate_kernel<T><<<blocks, threads>>>(d, (T)0.999, iters);
    cudaEventRecord(e1);
    rc = check_cuda(cudaEventSynchronize(e1), "fma probe");
    float ms = 0.f;
    if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    if (!rc && r > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d);
  if (rc) return rc;
  *tflops = (float)(2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12);
  return STOMSFEM_OK;
}

// mma.sync throughput probe: every warp runs 8 independent accumulator
// chains of m16n8k8 TF32 (kind 0) or m16n8k16 BF16 (kind 1) products.
template <int KIND>
__global__ void __launch_bounds__(256) mma_rate_kernel(float* out, uint32_t seed, int iters) {
  float d[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) d[i][j] = (float)(threadIdx.x + 4 * i + j) * 1e-3f;
  const uint32_t mask = KIND == 0 ? 0x3f7fe000u : 0x3f7f3f7fu;  // finite TF32 / BF16x2 operands
  const uint32_t a0 = (seed ^ threadIdx.x) & mask, a1 = (a0 * 3u) & mask, a2 = (a0 * 5u) & mask,
                 a3 = (a0 * 7u) & mask, b0 = (a0 * 11u) & mask, b1 = (a0 * 13u) & mask;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if constexpr (KIND == 0)
        asm volatile(
            "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[i][0]), "+f"(d[i][1]), "+f"(d[i][2]), "+f"(d[i][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
      else
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[i][0]), "+f"(d[i][1]), "+f"(d[i][2]), "+f"(d[i][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) t += d[i][j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

template <int KIND>
static int mma_rate(int iters, float* tflops) {
  const int sms = device_sm_count() > 0 ? device_sm_count() : 152;
  const int blocks = sms * 8, threads = 256;
  float* dout = nullptr;
  STOMSFEM_TRY_CUDA(cudaMalloc(&dout, sizeof(float) * (size_t)blocks * threads));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = check_cuda(cudaEventCreate(&e0), "event");
  if (!rc) rc = check_cuda(cudaEventCreate(&e1), "event");
  float best = 1e30f;
  for (int r = 0; r < 4 && !rc; ++r) {
    cudaEventRecord(e0);
    mma_rate_kernel<KIND><<<blocks, threads>>>(dout, 12345u, iters);
    cudaEventRecord(e1);
    rc = check_cuda(cudaEventSynchronize(e1), "mma probe");
    float ms = 0.f;
    if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    if (!rc && r > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(dout);
  if (rc) return rc;
  const double k = KIND == 0 ? 8.0 : 16.0;
  const double warps = (double)blocks * threads / 32.0;
  *tflops = (float)(2.0 * 16.0 * 8.0 * k * 8.0 * iters * warps / (best * 1e-3) / 1e12);
  return STOMSFEM_OK;
}

}  // namespace stomsfem

using namespace stomsfem;

extern "C" int stomsfem_selftest_mma_rate(int32_t kind, float* tflops_host) {
  if (!tflops_host || (kind != 0 && kind != 1)) return set_error(STOMSFEM_EINVAL, "kind 0 (TF32) or 1 (BF16)");
  return kind == 0 ? mma_rate<0>(2048, tflops_host) : mma_rate<1>(1024, tflops_host);
}

extern "C" int stomsfem_selftest_fma_rate(int32_t precision, float* tflops_host) {
  if (!tflops_host || (precision != STOMSFEM_FP64 && precision != STOMSFEM_FP32))
    return set_error(STOMSFEM_EINVAL, "precision must be STOMSFEM_FP64 or STOMSFEM_FP32, tflops non-NULL");
  return precision == STOMSFEM_FP32 ? fma_rate<float>(16384, tflops_host) : fma_rate<double>(512, tflops_host);
}

extern "C" int stomsfem_selftest_exp(const double* t, int32_t n, double* out, stomsfem_stream_t stream) {
  if (n < 0) return set_error(STOMSFEM_EINVAL, "n < 0");
  if (n == 0) return STOMSFEM_OK;
  if (!t || !out) return set_error(STOMSFEM_EINVAL, "NULL device pointer");
  const int blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  exp_selftest_kernel<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(t, n, out);
  STOMSFEM_TRY_CUDA(cudaGetLastError());
  return STOMSFEM_OK;
}

extern "C" int stomsfem_selftest_wait_timeout(int32_t iters, int32_t* status_host) {
  if (iters < 1 || iters > (1 << 20) || !status_host) return set_error(STOMSFEM_EINVAL, "bad arguments");
  int32_t* d = nullptr;
  STOMSFEM_TRY_CUDA(cudaMalloc(&d, sizeof(int32_t)));
  int rc = check_cuda(cudaMemset(d, 0xFF, sizeof(int32_t)), "memset");
  if (rc == STOMSFEM_OK) {
    wait_timeout_kernel<<<1, 32>>>(d, (uint32_t)iters);
    rc = check_cuda(cudaGetLastError(), "launch");
  }
  if (rc == STOMSFEM_OK) rc = check_cuda(cudaMemcpy(status_host, d, sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
  cudaFree(d);
  return rc;
}
