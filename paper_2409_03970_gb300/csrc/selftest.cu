// Self-test of the bounded waits: waits, with the library's own wait
// helpers, on an mbarrier and on a completion counter that nothing will
// ever signal, so that both give up and the kernel reports NSORT_ETIMEOUT in
// the status word of a scratch buffer instead of hanging.  No fault, no
// trap: the kernel returns normally and the context stays usable.
#include <cuda_runtime.h>

#include <string>

#include "nsort.h"
#include "nsort_internal.h"
#include "tma_device.cuh"

namespace nsort {

__global__ void selftest_wait_kernel(int *status, unsigned long long *ctr, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);   // one arrival expected; nobody arrives
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool got = mbar_wait(&bar, 0, limit_ns);
    const bool counted = wait_at_least(ctr, 1, status, limit_ns);   // *ctr stays 0
    if (!got || !counted) atomicExch(status, (int)NSORT_ETIMEOUT);
    // the barrier's phase never completed: release it by arriving, so the
    // CTA leaves no pending phase behind
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&bar)) : "memory");
  }
}

}  // namespace nsort

using namespace nsort;

extern "C" int nsort_selftest_wait(void *d_tmp, size_t tmp_bytes, uint32_t limit_us,
                                   void *stream) {
  if (!d_tmp || tmp_bytes < 512 || (reinterpret_cast<uintptr_t>(d_tmp) & 255)) return NSORT_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int *status = static_cast<int *>(d_tmp);
  unsigned long long *ctr =
      reinterpret_cast<unsigned long long *>(static_cast<char *>(d_tmp) + 256);
  if (cudaMemsetAsync(d_tmp, 0, 512, st) != cudaSuccess) {
    set_last_error(std::string("nsort_selftest_wait: ") + cudaGetErrorString(cudaGetLastError()));
    return NSORT_ECUDA;
  }
  selftest_wait_kernel<<<1, 32, 0, st>>>(status, ctr, (uint64_t)limit_us * 1000ull);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("nsort_selftest_wait: ") + cudaGetErrorString(e));
    return NSORT_ECUDA;
  }
  return NSORT_OK;
}
