// Network and keys-per-thread ablation of the block sort (C ABI in
// include/nsort_ablation.h): Table 1's networks (bitonic, odd-even, best)
// as the column sort, with 4, 8, 16 or 32 keys per thread (Table 2's R).
// The kernels reuse the production column sort, warp merge and block merge
// code (sort_device.cuh), so only the network and the width change.
#include <cuda_runtime.h>

#include <string>

#include "nsort.h"
#include "nsort_ablation.h"
#include "nsort_internal.h"
#include "sort_device.cuh"

namespace nsort {
namespace {

constexpr int ABL_NT = 512;   // threads per CTA, as in the production tile sort

template <int FAMILY>
struct NetColumns {
  template <typename K, int W>
  __device__ __forceinline__ static void sort(K (&r)[W]) { column_sort_net<FAMILY, W>(r); }
};

__device__ __forceinline__ bool is_aligned16(const void *p) {
  return !(reinterpret_cast<uintptr_t>(p) & 15);
}

// Thread-contiguous load of keys [e0, e0 + W); keys past n read as the
// largest key, which sorts behind every real key and is never stored.
template <int W>
__device__ __forceinline__ void load_contig(const uint32_t *in, int64_t n, int64_t e0,
                                            uint32_t (&r)[W]) {
  if (e0 + W <= n && is_aligned16(in + e0)) {
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
      const uint4 v = reinterpret_cast<const uint4 *>(in + e0)[q];
      r[4 * q + 0] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k) r[k] = e0 + k < n ? in[e0 + k] : 0xFFFFFFFFu;
  }
}

template <int W>
__device__ __forceinline__ void store_contig(uint32_t *out, int64_t n, int64_t e0,
                                             const uint32_t (&r)[W]) {
  if (e0 + W <= n && is_aligned16(out + e0)) {
#pragma unroll
    for (int q = 0; q < W / 4; ++q)
      reinterpret_cast<uint4 *>(out + e0)[q] =
          make_uint4(r[4 * q + 0], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (e0 + k < n) out[e0 + k] = r[k];
  }
}

// One thread per group of W keys: the column sort alone.
template <int FAMILY, int W>
__global__ void __launch_bounds__(256) network_kernel(const uint32_t *in, uint32_t *out,
                                                      int64_t groups) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= groups) return;
  uint32_t r[W];
#pragma unroll
  for (int k = 0; k < W; ++k) r[k] = in[g * W + k];
  column_sort_net<FAMILY, W>(r);
#pragma unroll
  for (int k = 0; k < W; ++k) out[g * W + k] = r[k];
}

// The in-register sort: thread t of the grid sorts keys [IPT t, IPT t + IPT)
// with the network, then `levels` levels of the warp's flip merger make
// sorted runs of IPT * 2^levels.  Every lane takes part in the shuffles,
// including lanes wholly past n (they hold only padding).
template <int FAMILY, int IPT>
__global__ void __launch_bounds__(ABL_NT) warp_runs_kernel(const uint32_t *in, uint32_t *out,
                                                           int64_t n, int levels) {
  const int64_t e0 = ((int64_t)blockIdx.x * ABL_NT + threadIdx.x) * IPT;
  uint32_t r[IPT];
  load_contig<IPT>(in, n, e0, r);
  column_sort_net<FAMILY, IPT>(r);
  warp_merge<IPT>(r, threadIdx.x & 31, levels);
  store_contig<IPT>(out, n, e0, r);
}

// The block sort of one tile of ABL_NT * IPT keys, as the production tile
// sort does it (coalesced 16-byte loads in any assignment, the column sort,
// the warp merge, the shared-memory merges), with the network of FAMILY.
template <int FAMILY, int IPT>
__global__ void __launch_bounds__(ABL_NT) block_runs_kernel(const uint32_t *in, uint32_t *out,
                                                            int64_t n) {
  constexpr int TILE = ABL_NT * IPT;
  extern __shared__ __align__(16) unsigned char abl_smem[];   // block_smem_len<u32>(ABL_NT, IPT) words
  uint32_t *s = reinterpret_cast<uint32_t *>(abl_smem);
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  const int count = (int)(n - base < TILE ? n - base : TILE);
  uint32_t r[IPT];
  if (count == TILE && is_aligned16(in + base)) {
    const uint4 *p = reinterpret_cast<const uint4 *>(in + base);
#pragma unroll
    for (int q = 0; q < IPT / 4; ++q) {
      const uint4 v = p[tid + ABL_NT * q];
      r[4 * q + 0] = v.x;
      r[4 * q + 1] = v.y;
      r[4 * q + 2] = v.z;
      r[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < IPT / 4; ++q) {
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int e = 4 * (tid + ABL_NT * q) + w;
        r[4 * q + w] = e < count ? in[base + e] : 0xFFFFFFFFu;
      }
    }
  }
  sort_tile_in_block<ABL_NT, IPT, NetColumns<FAMILY>>(r, s);
  store_contig<IPT>(out + base, count, (int64_t)tid * IPT, r);
}

// ---- merger ablation (Sec. 2.4, Table 3) ----------------------------------
// Three ways to merge every two adjacent sorted runs of L keys into one
// sorted run of 2L, all with IPT keys per thread.

// Hybrid (the production warp merge): lane l holds keys [IPT l, IPT l + IPT)
// of its warp's chunk; one level of the flip merger with cross-lane stages
// while the compare distance is at least IPT, then the in-thread tail.
// Valid for IPT <= L <= 16 IPT.
template <int IPT>
__device__ __forceinline__ void hybrid_merge(uint32_t (&r)[IPT], int lane, int log2_span) {
  switch (log2_span) {   // span = 2L / IPT lanes
    case 1: warp_merge_level<1>(r, lane); break;
    case 2: warp_merge_level<2>(r, lane); break;
    case 3: warp_merge_level<3>(r, lane); break;
    case 4: warp_merge_level<4>(r, lane); break;
    default: warp_merge_level<5>(r, lane); break;
  }
}

// All-shuffle ("vectorized") merge: lane l holds keys 32 k + l (k < IPT)
// of its warp's chunk, so every compare distance below 32 is a shuffle and
// only distances of 32 and more stay inside a thread.  The flip stage
// compares key i with key i ^ (2L - 1); the half-cleaners compare key i
// with key i ^ d for d = L/2 .. 1; the smaller index keeps the minimum.
// Valid for 1 <= L <= 16 IPT.
template <int LOG2L, int IPT>
__device__ __forceinline__ void shuffle_merge_level(uint32_t (&r)[IPT], int lane) {
  constexpr int L = 1 << LOG2L;
  if constexpr (2 * L <= 32) {
    const bool lower = !(lane & L);
#pragma unroll
    for (int k = 0; k < IPT; ++k) r[k] = keep(lower, r[k], shfl_x(r[k], 2 * L - 1));
  } else {
    // partner of (register k, lane l) is (k ^ KM, l ^ 31); k with bit L/32
    // clear holds the smaller index
    constexpr int KM = 2 * L / 32 - 1;
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
      if (k & (L / 32)) continue;
      const int kp = k ^ KM;
      const uint32_t for_k = shfl_x(r[kp], 31);
      const uint32_t for_kp = shfl_x(r[k], 31);
      r[k] = kmin(r[k], for_k);
      r[kp] = kmax(r[kp], for_kp);
    }
  }
#pragma unroll
  for (int d = L / 2; d >= 1; d >>= 1) {
    if (d >= 32) {
#pragma unroll
      for (int k = 0; k < IPT; ++k)
        if (!(k & (d / 32))) ce(r[k], r[k + d / 32]);
    } else {
      const bool lo = !(lane & d);
#pragma unroll
      for (int k = 0; k < IPT; ++k) r[k] = keep(lo, r[k], shfl_x(r[k], d));
    }
  }
}

template <int IPT>
__device__ __forceinline__ void shuffle_merge(uint32_t (&r)[IPT], int lane, int log2_l) {
  switch (log2_l) {
    case 0: shuffle_merge_level<0>(r, lane); break;
    case 1: shuffle_merge_level<1>(r, lane); break;
    case 2: shuffle_merge_level<2>(r, lane); break;
    case 3: shuffle_merge_level<3>(r, lane); break;
    case 4: shuffle_merge_level<4>(r, lane); break;
    case 5: shuffle_merge_level<5>(r, lane); break;
    case 6: if constexpr (IPT >= 4) shuffle_merge_level<6>(r, lane); break;
    case 7: if constexpr (IPT >= 8) shuffle_merge_level<7>(r, lane); break;
    case 8: if constexpr (IPT >= 16) shuffle_merge_level<8>(r, lane); break;
    default: if constexpr (IPT >= 32) shuffle_merge_level<9>(r, lane); break;
  }
}

enum { MERGE_HYBRID = 0, MERGE_SHUFFLE = 1, MERGE_SERIAL = 2 };

template <int IPT>
__global__ void __launch_bounds__(ABL_NT) hybrid_merge_kernel(const uint32_t *in, uint32_t *out,
                                                              int64_t n, int log2_span) {
  const int64_t e0 = ((int64_t)blockIdx.x * ABL_NT + threadIdx.x) * IPT;
  uint32_t r[IPT];
  load_contig<IPT>(in, n, e0, r);
  hybrid_merge<IPT>(r, threadIdx.x & 31, log2_span);
  store_contig<IPT>(out, n, e0, r);
}

template <int IPT>
__global__ void __launch_bounds__(ABL_NT) shuffle_merge_kernel(const uint32_t *in, uint32_t *out,
                                                               int64_t n, int log2_l) {
  const int lane = threadIdx.x & 31;
  const int64_t chunk = ((int64_t)blockIdx.x * ABL_NT + (threadIdx.x & ~31)) * IPT;
  uint32_t r[IPT];
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const int64_t e = chunk + 32 * k + lane;
    r[k] = e < n ? in[e] : 0xFFFFFFFFu;
  }
  shuffle_merge<IPT>(r, lane, log2_l);
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const int64_t e = chunk + 32 * k + lane;
    if (e < n) out[e] = r[k];
  }
}

// Serial merge path: the tile of ABL_NT * IPT keys is staged in shared
// memory; thread t finds where its IPT outputs [IPT t, IPT t + IPT) start in
// its pair of runs by a merge-path search and merges them serially.  Valid
// for IPT / 2 <= L <= ABL_NT * IPT / 2.
template <int IPT>
__global__ void __launch_bounds__(ABL_NT) serial_merge_kernel(const uint32_t *in, uint32_t *out,
                                                              int64_t n, int run) {
  constexpr int TILE = ABL_NT * IPT;
  extern __shared__ __align__(16) unsigned char abl_smem[];   // block_smem_len<u32>(ABL_NT, IPT) words
  uint32_t *s = reinterpret_cast<uint32_t *>(abl_smem);
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  const int count = (int)(n - base < TILE ? n - base : TILE);
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const int e = tid + ABL_NT * k;
    s[pidx<uint32_t>(e)] = e < count ? in[base + e] : 0xFFFFFFFFu;
  }
  __syncthreads();
  const int e0 = tid * IPT;
  const int g0 = e0 & ~(2 * run - 1);
  const int diag = e0 - g0;
  const int ai = merge_path_smem(s, g0, run, g0 + run, run, diag);
  uint32_t r[IPT];
  int unused[IPT];
  serial_merge<IPT, false>(s, g0 + ai, g0 + run, g0 + run + diag - ai, g0 + 2 * run, r, unused);
  store_contig<IPT>(out + base, count, (int64_t)e0, r);
}

template <int IPT>
constexpr size_t block_smem_bytes() {
  return sizeof(uint32_t) * (size_t)block_smem_len<uint32_t>(ABL_NT, IPT);
}

int launch_error(const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return NSORT_OK;
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return NSORT_ECUDA;
}

template <int FAMILY, int W>
int apply_w(const uint32_t *in, uint32_t *out, int64_t groups, cudaStream_t st) {
  const unsigned grid = (unsigned)((groups + 255) / 256);
  network_kernel<FAMILY, W><<<grid, 256, 0, st>>>(in, out, groups);
  return launch_error("nsort_network_apply");
}

template <int FAMILY>
int apply_f(const uint32_t *in, uint32_t *out, int64_t groups, int w, cudaStream_t st) {
  switch (w) {
    case 4: return apply_w<FAMILY, 4>(in, out, groups, st);
    case 8: return apply_w<FAMILY, 8>(in, out, groups, st);
    case 16: return apply_w<FAMILY, 16>(in, out, groups, st);
    default: return apply_w<FAMILY, 32>(in, out, groups, st);
  }
}

template <int FAMILY, int IPT>
int runs_fi(const uint32_t *in, uint32_t *out, int64_t n, int levels, bool block,
            cudaStream_t st) {
  const int64_t tile = (int64_t)ABL_NT * IPT;
  const unsigned grid = (unsigned)((n + tile - 1) / tile);
  if (block) {
    constexpr size_t smem = block_smem_bytes<IPT>();
    if (cudaFuncSetAttribute(block_runs_kernel<FAMILY, IPT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return launch_error("cudaFuncSetAttribute");
    block_runs_kernel<FAMILY, IPT><<<grid, ABL_NT, smem, st>>>(in, out, n);
  } else {
    warp_runs_kernel<FAMILY, IPT><<<grid, ABL_NT, 0, st>>>(in, out, n, levels);
  }
  return launch_error("nsort_runs");
}

template <int FAMILY>
int runs_f(const uint32_t *in, uint32_t *out, int64_t n, int ipt, int levels, bool block,
           cudaStream_t st) {
  switch (ipt) {
    case 4: return runs_fi<FAMILY, 4>(in, out, n, levels, block, st);
    case 8: return runs_fi<FAMILY, 8>(in, out, n, levels, block, st);
    case 16: return runs_fi<FAMILY, 16>(in, out, n, levels, block, st);
    default: return runs_fi<FAMILY, 32>(in, out, n, levels, block, st);
  }
}

template <int IPT>
int merge_i(const uint32_t *in, uint32_t *out, int64_t n, int method, int log2_l,
            cudaStream_t st) {
  const int64_t tile = (int64_t)ABL_NT * IPT;
  const unsigned grid = (unsigned)((n + tile - 1) / tile);
  if (method == MERGE_HYBRID) {
    int log2_ipt = 0;
    while ((1 << log2_ipt) < IPT) ++log2_ipt;
    hybrid_merge_kernel<IPT><<<grid, ABL_NT, 0, st>>>(in, out, n, log2_l + 1 - log2_ipt);
  } else if (method == MERGE_SHUFFLE) {
    shuffle_merge_kernel<IPT><<<grid, ABL_NT, 0, st>>>(in, out, n, log2_l);
  } else {
    constexpr size_t smem = block_smem_bytes<IPT>();
    if (cudaFuncSetAttribute(serial_merge_kernel<IPT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return launch_error("cudaFuncSetAttribute");
    serial_merge_kernel<IPT><<<grid, ABL_NT, smem, st>>>(in, out, n, 1 << log2_l);
  }
  return launch_error("nsort_merge_runs");
}

bool valid_width(int w) { return w == 4 || w == 8 || w == 16 || w == 32; }
bool valid_family(int f) { return f == NET_BITONIC || f == NET_ODDEVEN || f == NET_BEST; }

}  // namespace
}  // namespace nsort

using namespace nsort;

extern "C" int nsort_network(int family, int width, int32_t *lo, int32_t *hi, int cap) {
  if (!valid_family(family) || !valid_width(width)) return -1;
  const CmpList l = make_network(family, width);
  for (int c = 0; c < l.n && c < cap; ++c) {
    if (lo) lo[c] = l.lo[c];
    if (hi) hi[c] = l.hi[c];
  }
  return l.n;
}

extern "C" int nsort_network_apply(const uint32_t *d_in, uint32_t *d_out, uint64_t groups,
                                   int family, int width, void *stream) {
  if (!valid_family(family) || !valid_width(width) || groups > (uint64_t(1) << 32))
    return NSORT_EINVAL;
  if (groups == 0) return NSORT_OK;
  if (!d_in || !d_out) return NSORT_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t g = (int64_t)groups;
  switch (family) {
    case NET_BITONIC: return apply_f<NET_BITONIC>(d_in, d_out, g, width, st);
    case NET_ODDEVEN: return apply_f<NET_ODDEVEN>(d_in, d_out, g, width, st);
    default: return apply_f<NET_BEST>(d_in, d_out, g, width, st);
  }
}

extern "C" int nsort_runs(const uint32_t *d_in, uint32_t *d_out, uint64_t n, int family, int ipt,
                          uint64_t run, void *stream) {
  if (!valid_family(family) || !valid_width(ipt) || n > MAX_KEYS) return NSORT_EINVAL;
  int levels = -1;
  for (int l = 0; l <= 5; ++l)
    if (run == (uint64_t)ipt << l) levels = l;
  const bool block = run == (uint64_t)ABL_NT * ipt;
  if (levels < 0 && !block) return NSORT_EINVAL;
  if (n == 0) return NSORT_OK;
  if (!d_in || !d_out) return NSORT_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nn = (int64_t)n;
  switch (family) {
    case NET_BITONIC: return runs_f<NET_BITONIC>(d_in, d_out, nn, ipt, levels, block, st);
    case NET_ODDEVEN: return runs_f<NET_ODDEVEN>(d_in, d_out, nn, ipt, levels, block, st);
    default: return runs_f<NET_BEST>(d_in, d_out, nn, ipt, levels, block, st);
  }
}

extern "C" int nsort_merge_runs(const uint32_t *d_in, uint32_t *d_out, uint64_t n, uint64_t run,
                                int method, int ipt, void *stream) {
  if (!valid_width(ipt) || n > MAX_KEYS || run == 0 || (run & (run - 1))) return NSORT_EINVAL;
  const uint64_t u = (uint64_t)ipt;
  bool ok = false;
  if (method == MERGE_HYBRID) ok = run >= u && run <= 16 * u;
  else if (method == MERGE_SHUFFLE) ok = run <= 16 * u;
  else if (method == MERGE_SERIAL) ok = 2 * run >= u && run <= (uint64_t)ABL_NT * u / 2;
  if (!ok) return NSORT_EINVAL;
  if (n == 0) return NSORT_OK;
  if (!d_in || !d_out) return NSORT_EINVAL;
  int log2_l = 0;
  while ((uint64_t(1) << log2_l) < run) ++log2_l;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nn = (int64_t)n;
  switch (ipt) {
    case 4: return merge_i<4>(d_in, d_out, nn, method, log2_l, st);
    case 8: return merge_i<8>(d_in, d_out, nn, method, log2_l, st);
    case 16: return merge_i<16>(d_in, d_out, nn, method, log2_l, st);
    default: return merge_i<32>(d_in, d_out, nn, method, log2_l, st);
  }
}
