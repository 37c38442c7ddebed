// Splitters of a sharded sort: where the sorted parts of P workers split
// the output (paper Sec. 2.1, last paragraph: the parts sorted by the
// threads are merged in parallel after a load-balanced partition; Sec. 3.2
// calls the partition points "segmentation points").  Here a worker is a
// shard of one array; on one GPU all shards lie in one buffer, and across
// GPUs each rank counts on its own shard (nsort_count_le) and the counts
// are summed by the caller's collective.
//
// The output order is the stable merge of the shards: ascending order key,
// equal keys by shard (lower first), then by position.  For an output
// position d, the d-th output's key v* is the smallest order key v with
//     sum over shards of |{x : key(x) <= v}|  >  d,
// found by bisection on the key space (32 or 64 rounds).  Shard r then
// gives all its keys below v*, plus as many keys equal to v* as are left
// after the lower shards' equal keys.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "nsort.h"
#include "nsort_internal.h"
#include "sort_device.cuh"

namespace nsort {

namespace {

__device__ __forceinline__ int64_t warp_sum(int64_t v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

__device__ __forceinline__ int64_t warp_exclusive_sum(int64_t v, int lane) {
  int64_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += u;
  }
  return inc - v;
}

// First index in [lo, hi) of the sorted run `base` whose order key exceeds
// v (= the number of keys <= v, given that the first lo are <= v and those
// from hi on are not).
template <typename K, int DT>
__device__ __forceinline__ int64_t upper_bound_key(const K *base, int64_t lo, int64_t hi, K v) {
  while (lo < hi) {
    const int64_t m = (lo + hi) >> 1;
    if (to_key(__ldg(base + m), DT) <= v) lo = m + 1;
    else hi = m;
  }
  return lo;
}

// One warp per target output position; lane r < P owns shard r.  Each
// round halves the key interval [lo, hi] that holds v*; every lane keeps
// the counts of its keys below lo (cl) and at most hi (ch), which bound the
// next search.
template <typename K, int DT>
__global__ void shard_corank_kernel(const K *__restrict__ keys, const int64_t *__restrict__ off,
                                    int P, const int64_t *__restrict__ targets, int T,
                                    int64_t *__restrict__ out) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= T) return;                       // whole warps leave together
  const bool mine = lane < P;
  const int64_t s0 = mine ? off[lane] : 0;
  const int64_t len = mine ? off[lane + 1] - s0 : 0;
  const K *base = keys + s0;
  const int64_t total = warp_sum(len);
  int64_t d = targets[w];
  d = d < 0 ? 0 : (d > total ? total : d);
  int64_t c = len;
  if (d < total) {
    K lo = 0, hi = ~K(0);
    int64_t cl = 0, ch = len;
    while (lo < hi) {                       // the same bounds in every lane
      const K mid = lo + ((hi - lo) >> 1);
      const int64_t le = upper_bound_key<K, DT>(base, cl, ch, mid);
      if (warp_sum(le) > d) {
        hi = mid;
        ch = le;
      } else {
        lo = mid + 1;
        cl = le;
      }
    }
    const int64_t eq = ch - cl;             // keys equal to v* = lo
    const int64_t rem = d - warp_sum(cl);   // outputs at v*: 0 <= rem < sum of eq
    int64_t take = rem - warp_exclusive_sum(eq, lane);
    take = take < 0 ? 0 : (take > eq ? eq : take);
    c = cl + take;
  }
  if (mine) out[w * P + lane] = c;
}

// le[i] = number of keys of the sorted array whose order key is <= bounds[i].
template <typename K, int DT>
__global__ void count_le_kernel(const K *__restrict__ keys, int64_t n, const K *__restrict__ bounds,
                                int64_t m, int64_t *__restrict__ le) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  le[i] = upper_bound_key<K, DT>(keys, 0, n, __ldg(bounds + i));
}

int cuda_status(const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return NSORT_OK;
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return NSORT_ECUDA;
}

bool valid_dtype(int dt) { return dt >= NSORT_U32 && dt <= NSORT_F64; }
bool wide_dtype(int dt) { return dt >= NSORT_U64; }

}  // namespace

}  // namespace nsort

using namespace nsort;

extern "C" int nsort_shard_coranks(const void *d_keys, const int64_t *d_shard_off, int nshards,
                                   const int64_t *d_targets, int ntargets, int dtype,
                                   int64_t *d_coranks, void *stream) {
  if (!valid_dtype(dtype) || nshards < 1 || nshards > 32 || ntargets < 0) return NSORT_EINVAL;
  if (ntargets == 0) return NSORT_OK;
  if (!d_keys || !d_shard_off || !d_targets || !d_coranks) return NSORT_EINVAL;
  const uintptr_t align = wide_dtype(dtype) ? 7 : 3;
  if (reinterpret_cast<uintptr_t>(d_keys) & align) return NSORT_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned threads = 256;
  const unsigned blocks = (unsigned)(((int64_t)ntargets * 32 + threads - 1) / threads);
#define NSORT_CR(K, DT)                                                                      \
  shard_corank_kernel<K, DT><<<blocks, threads, 0, st>>>(static_cast<const K *>(d_keys),     \
                                                         d_shard_off, nshards, d_targets,    \
                                                         ntargets, d_coranks)
  switch (dtype) {
    case NSORT_U32: NSORT_CR(uint32_t, DT_U32); break;
    case NSORT_I32: NSORT_CR(uint32_t, DT_I32); break;
    case NSORT_F32: NSORT_CR(uint32_t, DT_F32); break;
    case NSORT_U64: NSORT_CR(uint64_t, DT_U64); break;
    case NSORT_I64: NSORT_CR(uint64_t, DT_I64); break;
    default: NSORT_CR(uint64_t, DT_F64); break;
  }
#undef NSORT_CR
  return cuda_status("shard_corank_kernel");
}

extern "C" int nsort_count_le(const void *d_sorted, uint64_t n, int dtype, const void *d_bounds,
                              uint64_t m, int64_t *d_le, void *stream) {
  if (!valid_dtype(dtype) || n > MAX_KEYS) return NSORT_EINVAL;
  if (m == 0) return NSORT_OK;
  if ((n > 0 && !d_sorted) || !d_bounds || !d_le) return NSORT_EINVAL;
  const uintptr_t align = wide_dtype(dtype) ? 7 : 3;
  if ((reinterpret_cast<uintptr_t>(d_sorted) | reinterpret_cast<uintptr_t>(d_bounds)) & align)
    return NSORT_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned threads = 256;
  const unsigned blocks = (unsigned)((m + threads - 1) / threads);
#define NSORT_CL(K, DT)                                                                       \
  count_le_kernel<K, DT><<<blocks, threads, 0, st>>>(static_cast<const K *>(d_sorted),        \
                                                     (int64_t)n, static_cast<const K *>(d_bounds), \
                                                     (int64_t)m, d_le)
  switch (dtype) {
    case NSORT_U32: NSORT_CL(uint32_t, DT_U32); break;
    case NSORT_I32: NSORT_CL(uint32_t, DT_I32); break;
    case NSORT_F32: NSORT_CL(uint32_t, DT_F32); break;
    case NSORT_U64: NSORT_CL(uint64_t, DT_U64); break;
    case NSORT_I64: NSORT_CL(uint64_t, DT_I64); break;
    default: NSORT_CL(uint64_t, DT_F64); break;
  }
#undef NSORT_CL
  return cuda_status("count_le_kernel");
}
