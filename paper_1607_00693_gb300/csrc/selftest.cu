// Failure-path self test of the bounded device waits used by the
// tensor-core kernels: a CTA initialises an mbarrier that nothing ever
// arrives at and waits on it with a short iteration limit; the wait gives up,
// the kernel records the timeout in a status word and returns normally, so
// the context stays usable.
#include "common.cuh"
#include "tc_gemm.cuh"

namespace stomsfem {

__global__ void wait_timeout_kernel(int32_t* status, uint32_t iters) {
  __shared__ uint64_t mbar;
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  __syncthreads();
  const bool ok = tc::mbar_wait_bounded(&mbar, 0, iters);
  if (threadIdx.x == 0) *status = ok ? STOMSFEM_OK : STOMSFEM_ETIMEOUT;
}

}  // namespace stomsfem

using namespace stomsfem;

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
