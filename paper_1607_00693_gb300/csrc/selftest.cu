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

}  // namespace stomsfem

using namespace stomsfem;

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
