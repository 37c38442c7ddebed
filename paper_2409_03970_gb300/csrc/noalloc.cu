// nsort_keys_noalloc: the plain key sort for callers that cannot allocate
// device memory.
//
// Some callers have no way to provide the scratch buffer nsort_keys wants:
// their device memory belongs entirely to someone else's allocator (a
// framework's caching pool, a fixed arena sized at start-up), or they run on
// a path where a cudaMalloc is not allowed because it may block or
// synchronise the device.  This entry point takes no scratch argument.  Its
// scratch is a fixed array in this file, in device global memory, which
// exists on every GPU that loads the library until the process exits.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, the first
// time the entry point runs on it.  The address is kept for the life of the
// process: it does not survive cudaDeviceReset (or any other end of the
// device's primary context), after which these entry points must not be
// called again in the process.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "nsort.h"
#include "nsort_internal.h"

namespace nsort {

namespace {

// Scratch of a plain key sort of NSORT_NOALLOC_MAX_KEYS keys, laid out as
// nsort_keys lays out its scratch: the device status word, one ping-pong
// copy of the keys, one int64 merge-path splitter per merge tile (sized for
// merge tiles of 256 keys or more) and every 64th key of a pass's output;
// each part rounded up to 256 bytes (about 4.1 MiB in all).
constexpr size_t kStatusBytes = 256;
constexpr size_t kKeysBytes = size_t(NSORT_NOALLOC_MAX_KEYS) * 4;
constexpr size_t kSplitBytes = ((NSORT_NOALLOC_MAX_KEYS / 256 + 2) * 8 + 255) / 256 * 256;
constexpr size_t kSampleBytes = ((NSORT_NOALLOC_MAX_KEYS / 64 + 2) * 4 + 255) / 256 * 256;
constexpr size_t kScratchBytes = kStatusBytes + kKeysBytes + kSplitBytes + kSampleBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once.
int scratch_for_current_device(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_last_error(std::string("nsort_keys_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return NSORT_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_last_error("nsort_keys_noalloc: device ordinal out of range");
    return NSORT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      set_last_error(std::string("nsort_keys_noalloc: cudaGetSymbolAddress: ") +
                     cudaGetErrorString(e));
      return NSORT_ECUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return NSORT_OK;
}

}  // namespace

}  // namespace nsort

using namespace nsort;

extern "C" int nsort_keys_noalloc(const void *d_keys_in, void *d_keys_out, uint64_t n,
                                  int dtype, void *stream) {
  if (dtype != NSORT_U32 && dtype != NSORT_I32 && dtype != NSORT_F32) return NSORT_EINVAL;
  if (n == 0) return NSORT_OK;
  if (n > NSORT_NOALLOC_MAX_KEYS) {
    set_last_error("nsort_keys_noalloc: n exceeds the maximum of NSORT_NOALLOC_MAX_KEYS (2^20) "
                   "keys; use nsort_keys with a caller-provided scratch buffer");
    return NSORT_ENOMEM;
  }
  if (!d_keys_in || !d_keys_out) return NSORT_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_keys_in) | reinterpret_cast<uintptr_t>(d_keys_out)) & 3)
    return NSORT_EINVAL;
  if (make_plan(NSORT_KIND_KEYS, n).total > kScratchBytes) {
    set_last_error("nsort_keys_noalloc: internal scratch size mismatch");
    return NSORT_ENOMEM;
  }
  void *scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != NSORT_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The status word (the array's first bytes) starts every call at
  // NSORT_OK, also for sorts without merge passes, which never write it:
  // nsort_keys_noalloc_status then always reports this call.  Nothing else
  // in the scratch has to start at zero: the tile sort writes the whole key
  // buffer and every pass writes its splitters before reading them.
  if (cudaMemsetAsync(scratch, 0, sizeof(int), st) != cudaSuccess) {
    set_last_error(std::string("nsort_keys_noalloc: cudaMemsetAsync: ") +
                   cudaGetErrorString(cudaGetLastError()));
    return NSORT_ECUDA;
  }
  return sort_keys_impl(static_cast<const uint32_t *>(d_keys_in),
                        static_cast<uint32_t *>(d_keys_out), (int64_t)n, dtype, scratch, st);
}

extern "C" int nsort_keys_noalloc_status(void *stream) {
  void *scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != NSORT_OK) return rc;
  int status = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&status, scratch, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_last_error(std::string("nsort_keys_noalloc_status: ") +
                   cudaGetErrorString(cudaGetLastError()));
    return NSORT_ECUDA;
  }
  return status;
}
