// Per-thread error text of libnsort.
#include <cuda_runtime.h>

#include <string>

#include "nsort.h"
#include "nsort_internal.h"

namespace nsort {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }
const char *last_error_cstr() { return g_last_error.c_str(); }

}  // namespace nsort

using namespace nsort;

// The first word of every scratch buffer is the device status of the call
// that last used it.
extern "C" int nsort_device_status(const void *d_tmp, void *stream) {
  if (!d_tmp) return NSORT_EINVAL;
  int status = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&status, d_tmp, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_last_error(std::string("nsort_device_status: ") + cudaGetErrorString(cudaGetLastError()));
    return NSORT_ECUDA;
  }
  return status;
}
