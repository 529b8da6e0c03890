// Library-wide host utilities: version, per-thread error messages.
#include <cstdarg>
#include <cstdio>

#include "common.cuh"

namespace stomsfem {

static thread_local char g_err[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return STOMSFEM_OK;
  return set_error(STOMSFEM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

}  // namespace stomsfem

extern "C" const char* stomsfem_version(void) { return "stomsfem-gb300 0.9 (sm_103a)"; }
extern "C" const char* stomsfem_last_error(void) { return stomsfem::g_err; }
