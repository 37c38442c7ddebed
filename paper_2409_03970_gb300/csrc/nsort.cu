// nsort: plain and pair sorts (C ABI in include/nsort.h).
//
// A sort of n keys is
//   1 tile-sort launch   — each CTA sorts one tile in registers and shared
//                          memory: column sort, warp merge, block merges
//                          (paper Sec. 2.1-2.4, the "in-register sort" and
//                          "vectorized merge" levels);
//   P merge passes       — each pass merges adjacent sorted runs pairwise;
//                          a partition kernel finds every CTA's merge-path
//                          splitter ("segmentation points", Sec. 3.2), then
//                          each CTA stages its slices in shared memory and
//                          every thread runs a serial merge of its share
//                          (the "multi-thread parallel merge", Sec. 2.1).
// Buffers ping-pong between the output and the caller's scratch so that the
// last pass lands in the output.  The order-preserving key map is applied
// when the tile sort loads the input and undone when the last pass stores.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstring>
#include <string>

#include "nsort.h"
#include "nsort_internal.h"
#include "sort_device.cuh"

namespace nsort {

// ---------------------------------------------------------------- kernels

// Sorts one tile of NT*16 elements that is already in registers (16 per
// thread, any assignment) and leaves it sorted in s (padded layout).
template <int NT, typename K>
__device__ __forceinline__ void sort_tile_in_block(K (&r)[16], K *s) {
  constexpr int TILE = NT * 16;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  column_sort16(r);
  warp_merge512(r, lane);
  const int ew = warp * 512 + lane * 16;
#pragma unroll
  for (int k = 0; k < 16; ++k) s[pidx<K>(ew + k)] = r[k];
  int unused[16];
#pragma unroll 1
  for (int run = 512; run < TILE; run <<= 1) {
    __syncthreads();
    const int e0 = tid * 16;
    const int g0 = e0 & ~(2 * run - 1);
    const int diag = e0 - g0;
    const int ai = merge_path_smem(s, g0, run, g0 + run, run, diag);
    serial_merge<16, false>(s, g0 + ai, g0 + run, g0 + run + diag - ai, g0 + 2 * run,
                            TILE - 1, r, unused);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) s[pidx<K>(e0 + k)] = r[k];
  }
  __syncthreads();
}

// Stores `count` sorted keys from s (padded layout) to out, mapping each
// key back to its bit pattern with dt_out (DT_U32 = leave as is).
template <int NT, int VT>
__device__ __forceinline__ void store_keys(const uint32_t *s, uint32_t *out, int count,
                                           int dt_out) {
  constexpr int TILE = NT * VT;
  const int tid = threadIdx.x;
  if (count == TILE && !(reinterpret_cast<uintptr_t>(out) & 15)) {
#pragma unroll
    for (int j = 0; j < VT / 4; ++j) {
      const int c = tid + NT * j;
      const int e = 4 * c;
      uint4 v;
      v.x = from_key(s[pidx<uint32_t>(e)], dt_out);
      v.y = from_key(s[pidx<uint32_t>(e + 1)], dt_out);
      v.z = from_key(s[pidx<uint32_t>(e + 2)], dt_out);
      v.w = from_key(s[pidx<uint32_t>(e + 3)], dt_out);
      reinterpret_cast<uint4 *>(out)[c] = v;
    }
  } else {
#pragma unroll
    for (int j = 0; j < VT; ++j) {
      const int e = tid + NT * j;
      if (e < count) out[e] = from_key(s[pidx<uint32_t>(e)], dt_out);
    }
  }
}

// Tile sort, keys only.  Tile t covers [t*TILE, min((t+1)*TILE, n)); a short
// last tile is padded with the largest key, which sorts behind every real
// key and is never stored.  in may equal out (each CTA reads its whole tile
// before the first barrier and writes it after the last).
template <int NT>
__global__ void __launch_bounds__(NT) tile_sort_keys_kernel(const uint32_t *in, uint32_t *out,
                                                            int64_t n, int dt, int dt_out) {
  constexpr int TILE = NT * 16;
  __shared__ uint32_t s[padded_len<uint32_t>(TILE)];
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  const int count = (int)(n - base < TILE ? n - base : TILE);
  uint32_t r[16];
  if (count == TILE && !(reinterpret_cast<uintptr_t>(in + base) & 15)) {
    const uint4 *p = reinterpret_cast<const uint4 *>(in + base);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 v = p[tid + NT * j];
      r[4 * j + 0] = to_key(v.x, dt);
      r[4 * j + 1] = to_key(v.y, dt);
      r[4 * j + 2] = to_key(v.z, dt);
      r[4 * j + 3] = to_key(v.w, dt);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int e = 4 * (tid + NT * j) + w;
        r[4 * j + w] = e < count ? to_key(in[base + e], dt) : 0xFFFFFFFFu;
      }
    }
  }
  sort_tile_in_block<NT>(r, s);
  store_keys<NT, 16>(s, out + base, count, dt_out);
}

// Tile sort, key/value pairs.  The networks sort 64-bit composites
// (key << 32 | position in tile); positions make every composite distinct,
// so the network's result is the stable order.  Values are staged in shared
// memory and gathered by position at the end.
template <int NT>
__global__ void __launch_bounds__(NT) tile_sort_pairs_kernel(const uint32_t *kin,
                                                             const uint32_t *vin,
                                                             uint32_t *kout, uint32_t *vout,
                                                             int64_t n, int dt, int dt_out) {
  constexpr int TILE = NT * 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t *s = reinterpret_cast<uint64_t *>(smem_raw);
  uint32_t *sv = reinterpret_cast<uint32_t *>(s + padded_len<uint64_t>(TILE));
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  const int count = (int)(n - base < TILE ? n - base : TILE);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int e = tid + NT * j;
    if (e < count) sv[pidx<uint32_t>(e)] = vin[base + e];
  }
  uint64_t r[16];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int e = 4 * (tid + NT * j) + w;
      r[4 * j + w] = e < count ? ((uint64_t)to_key(kin[base + e], dt) << 32) | (uint32_t)e
                               : ~0ull;
    }
  }
  sort_tile_in_block<NT>(r, s);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int e = tid + NT * j;
    if (e < count) {
      const uint64_t c = s[pidx<uint64_t>(e)];
      kout[base + e] = from_key((uint32_t)(c >> 32), dt_out);
      vout[base + e] = sv[pidx<uint32_t>((int)(c & 0xFFFFu))];
    }
  }
}

// Which slices of the two input runs one merge CTA consumes.
struct PassTile {
  int64_t out0;      // first output element of the tile
  int64_t pair0;     // first element of the run pair (A then B)
  int64_t la;        // length of run A
  int64_t a_beg;     // slice of A: [a_beg, a_beg + na)
  int64_t b_beg;     // slice of B: [b_beg, b_beg + nb)
  int na, nb, count;
};

__device__ __forceinline__ PassTile pass_tile(int64_t n, int64_t run, int tile,
                                              const int64_t *split) {
  PassTile g;
  g.out0 = (int64_t)blockIdx.x * tile;
  const int64_t out1 = g.out0 + tile < n ? g.out0 + tile : n;
  g.pair0 = g.out0 & ~(2 * run - 1);
  g.la = n - g.pair0 < run ? n - g.pair0 : run;
  const int64_t rest = n - g.pair0 - run;
  const int64_t lb = rest <= 0 ? 0 : (rest < run ? rest : run);
  const int64_t pair_end = g.pair0 + g.la + lb;
  const int64_t a_end = out1 == pair_end ? g.la : split[blockIdx.x + 1];
  g.a_beg = split[blockIdx.x];
  g.b_beg = (g.out0 - g.pair0) - g.a_beg;
  const int64_t b_end = (out1 - g.pair0) - a_end;
  g.na = (int)(a_end - g.a_beg);
  g.nb = (int)(b_end - g.b_beg);
  g.count = g.na + g.nb;
  return g;
}

// Merge-path splitters of one pass: for every output tile, how many
// elements of its pair's A run precede the tile (stable: A wins ties).
__global__ void partition_kernel(const uint32_t *__restrict__ src, int64_t n, int64_t run,
                                 int tile, int64_t num_tiles, int64_t *__restrict__ split) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= num_tiles) return;
  const int64_t out0 = t * tile;
  const int64_t pair0 = out0 & ~(2 * run - 1);
  const int64_t la = n - pair0 < run ? n - pair0 : run;
  const int64_t rest = n - pair0 - run;
  const int64_t lb = rest <= 0 ? 0 : (rest < run ? rest : run);
  split[t] = merge_path_global(src + pair0, la, src + pair0 + la, lb, out0 - pair0);
}

// One merge pass over keys: CTA b produces output tile b.
template <int NT, int VT>
__global__ void __launch_bounds__(NT) merge_keys_kernel(const uint32_t *__restrict__ src,
                                                        uint32_t *__restrict__ dst, int64_t n,
                                                        int64_t run,
                                                        const int64_t *__restrict__ split,
                                                        int dt_out) {
  constexpr int TILE = NT * VT;
  __shared__ uint32_t s[padded_len<uint32_t>(TILE)];
  const int tid = threadIdx.x;
  const PassTile g = pass_tile(n, run, TILE, split);
  const uint32_t *A = src + g.pair0 + g.a_beg;
  const uint32_t *B = src + g.pair0 + g.la + g.b_beg;
  uint32_t t[VT];
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    const int i = tid + NT * j;
    t[j] = i < g.na ? A[i] : (i < g.count ? B[i - g.na] : 0u);
  }
#pragma unroll
  for (int j = 0; j < VT; ++j) s[pidx<uint32_t>(tid + NT * j)] = t[j];
  __syncthreads();
  const int diag = tid * VT < g.count ? tid * VT : g.count;
  const int ai = merge_path_smem(s, 0, g.na, g.na, g.nb, diag);
  uint32_t o[VT];
  int unused[VT];
  serial_merge<VT, false>(s, ai, g.na, g.na + diag - ai, g.count, TILE - 1, o, unused);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < VT; ++k) s[pidx<uint32_t>(tid * VT + k)] = o[k];
  __syncthreads();
  store_keys<NT, VT>(s, dst + g.out0, g.count, dt_out);
}

// One merge pass over key/value pairs (stable).
template <int NT, int VT>
__global__ void __launch_bounds__(NT) merge_pairs_kernel(const uint32_t *__restrict__ ksrc,
                                                         const uint32_t *__restrict__ vsrc,
                                                         uint32_t *__restrict__ kdst,
                                                         uint32_t *__restrict__ vdst,
                                                         int64_t n, int64_t run,
                                                         const int64_t *__restrict__ split,
                                                         int dt_out) {
  constexpr int TILE = NT * VT;
  __shared__ uint32_t sk[padded_len<uint32_t>(TILE)];
  __shared__ uint32_t sv[padded_len<uint32_t>(TILE)];
  const int tid = threadIdx.x;
  const PassTile g = pass_tile(n, run, TILE, split);
  const int64_t a_off = g.pair0 + g.a_beg;
  const int64_t b_off = g.pair0 + g.la + g.b_beg;
  uint32_t tk[VT], tv[VT];
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    const int i = tid + NT * j;
    const int64_t at = i < g.na ? a_off + i : b_off + (i - g.na);
    const bool ok = i < g.count;
    tk[j] = ok ? ksrc[at] : 0u;
    tv[j] = ok ? vsrc[at] : 0u;
  }
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    sk[pidx<uint32_t>(tid + NT * j)] = tk[j];
    sv[pidx<uint32_t>(tid + NT * j)] = tv[j];
  }
  __syncthreads();
  const int diag = tid * VT < g.count ? tid * VT : g.count;
  const int ai = merge_path_smem(sk, 0, g.na, g.na, g.nb, diag);
  uint32_t o[VT];
  int from[VT];
  serial_merge<VT, true>(sk, ai, g.na, g.na + diag - ai, g.count, TILE - 1, o, from);
#pragma unroll
  for (int k = 0; k < VT; ++k) tv[k] = sv[pidx<uint32_t>(from[k] < TILE ? from[k] : TILE - 1)];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < VT; ++k) {
    sk[pidx<uint32_t>(tid * VT + k)] = o[k];
    sv[pidx<uint32_t>(tid * VT + k)] = tv[k];
  }
  __syncthreads();
  store_keys<NT, VT>(sk, kdst + g.out0, g.count, dt_out);
  store_keys<NT, VT>(sv, vdst + g.out0, g.count, DT_U32);
}

// ------------------------------------------------------------- host side

namespace {

constexpr int KEYS_SORT_NT = 512;   // tile sort: 512 threads x 16 keys = 8192
constexpr int PAIRS_SORT_NT = 256;  //            256 threads x 16 pairs = 4096
constexpr int MERGE_NT = 256;       // merge pass: 256 threads x 16 = 4096 outputs
constexpr int MERGE_VT = 16;
constexpr int PMERGE_NT = 256;
constexpr int PMERGE_VT = 16;

constexpr int KEYS_SORT_TILE = KEYS_SORT_NT * 16;
constexpr int PAIRS_SORT_TILE = PAIRS_SORT_NT * 16;
constexpr int MERGE_TILE = MERGE_NT * MERGE_VT;
constexpr int PMERGE_TILE = PMERGE_NT * PMERGE_VT;

constexpr size_t PAIRS_SORT_SMEM =
    sizeof(uint64_t) * padded_len<uint64_t>(PAIRS_SORT_TILE) +
    sizeof(uint32_t) * padded_len<uint32_t>(PAIRS_SORT_TILE);

}  // namespace

Plan make_plan(int kind, uint64_t n) {
  Plan p;
  const bool pairs = kind == NSORT_KIND_PAIRS;
  p.n = (int64_t)n;
  p.sort_tile = pairs ? PAIRS_SORT_TILE : KEYS_SORT_TILE;
  p.merge_tile = pairs ? PMERGE_TILE : MERGE_TILE;
  const int64_t runs = (p.n + p.sort_tile - 1) / p.sort_tile;
  p.merge_passes = 0;
  while ((int64_t(1) << p.merge_passes) < runs) ++p.merge_passes;
  p.num_merge_tiles = (p.n + p.merge_tile - 1) / p.merge_tile;
  const size_t kb = align_up((size_t)n * 4, 256);
  p.keys_off = 0;
  p.vals_off = kb;
  p.split_off = pairs ? 2 * kb : kb;
  p.total = p.merge_passes == 0
                ? 0
                : p.split_off + align_up((size_t)(p.num_merge_tiles + 1) * sizeof(int64_t), 256);
  return p;
}

static int launch_status(const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return NSORT_OK;
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return NSORT_ECUDA;
}

static int ensure_pairs_smem_attr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return launch_status("cudaGetDevice");
  static std::atomic<uint64_t> done_mask{0};
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done_mask.load() & bit)) return NSORT_OK;
  if (cudaFuncSetAttribute(tile_sort_pairs_kernel<PAIRS_SORT_NT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)PAIRS_SORT_SMEM) != cudaSuccess)
    return launch_status("cudaFuncSetAttribute");
  done_mask.fetch_or(bit);
  return NSORT_OK;
}

int sort_keys_impl(const uint32_t *in, uint32_t *out, int64_t n, int dt, void *tmp,
                   cudaStream_t st) {
  const Plan p = make_plan(NSORT_KIND_KEYS, (uint64_t)n);
  uint32_t *bufs[2] = {out, reinterpret_cast<uint32_t *>(static_cast<char *>(tmp) + p.keys_off)};
  int64_t *split = p.merge_passes
                       ? reinterpret_cast<int64_t *>(static_cast<char *>(tmp) + p.split_off)
                       : nullptr;
  int cur = p.merge_passes % 2;  // the last pass must land in bufs[0] == out
  const int64_t tiles = (n + p.sort_tile - 1) / p.sort_tile;
  {
    TraceScope tr(TK_TILE_SORT_KEYS, st);
    tile_sort_keys_kernel<KEYS_SORT_NT><<<(unsigned)tiles, KEYS_SORT_NT, 0, st>>>(
        in, bufs[cur], n, dt, p.merge_passes == 0 ? dt : DT_U32);
  }
  int rc = launch_status("tile_sort_keys");
  for (int pass = 0; rc == NSORT_OK && pass < p.merge_passes; ++pass) {
    const int64_t run = (int64_t)p.sort_tile << pass;
    const unsigned pblocks = (unsigned)((p.num_merge_tiles + 255) / 256);
    {
      TraceScope tr(TK_PARTITION, st);
      partition_kernel<<<pblocks, 256, 0, st>>>(bufs[cur], n, run, p.merge_tile,
                                                p.num_merge_tiles, split);
    }
    {
      TraceScope tr(TK_MERGE_KEYS, st);
      merge_keys_kernel<MERGE_NT, MERGE_VT><<<(unsigned)p.num_merge_tiles, MERGE_NT, 0, st>>>(
          bufs[cur], bufs[cur ^ 1], n, run, split, pass == p.merge_passes - 1 ? dt : DT_U32);
    }
    rc = launch_status("merge_keys");
    cur ^= 1;
  }
  return rc;
}

int sort_pairs_impl(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                    int64_t n, int dt, void *tmp, cudaStream_t st) {
  int rc = ensure_pairs_smem_attr();
  if (rc != NSORT_OK) return rc;
  const Plan p = make_plan(NSORT_KIND_PAIRS, (uint64_t)n);
  char *t = static_cast<char *>(tmp);
  uint32_t *kb[2] = {kout, reinterpret_cast<uint32_t *>(t + p.keys_off)};
  uint32_t *vb[2] = {vout, reinterpret_cast<uint32_t *>(t + p.vals_off)};
  int64_t *split = p.merge_passes ? reinterpret_cast<int64_t *>(t + p.split_off) : nullptr;
  int cur = p.merge_passes % 2;
  const int64_t tiles = (n + p.sort_tile - 1) / p.sort_tile;
  {
    TraceScope tr(TK_TILE_SORT_PAIRS, st);
    tile_sort_pairs_kernel<PAIRS_SORT_NT><<<(unsigned)tiles, PAIRS_SORT_NT, PAIRS_SORT_SMEM, st>>>(
        kin, vin, kb[cur], vb[cur], n, dt, p.merge_passes == 0 ? dt : DT_U32);
  }
  rc = launch_status("tile_sort_pairs");
  for (int pass = 0; rc == NSORT_OK && pass < p.merge_passes; ++pass) {
    const int64_t run = (int64_t)p.sort_tile << pass;
    const unsigned pblocks = (unsigned)((p.num_merge_tiles + 255) / 256);
    {
      TraceScope tr(TK_PARTITION, st);
      partition_kernel<<<pblocks, 256, 0, st>>>(kb[cur], n, run, p.merge_tile,
                                                p.num_merge_tiles, split);
    }
    {
      TraceScope tr(TK_MERGE_PAIRS, st);
      merge_pairs_kernel<PMERGE_NT, PMERGE_VT><<<(unsigned)p.num_merge_tiles, PMERGE_NT, 0, st>>>(
          kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n, run, split,
          pass == p.merge_passes - 1 ? dt : DT_U32);
    }
    rc = launch_status("merge_pairs");
    cur ^= 1;
  }
  return rc;
}

}  // namespace nsort

// ---------------------------------------------------------------- C ABI

using namespace nsort;

extern "C" size_t nsort_temp_bytes(int kind, uint64_t n, uint64_t nseg, int dtype) {
  (void)dtype;
  if (kind == NSORT_KIND_KEYS || kind == NSORT_KIND_PAIRS) return make_plan(kind, n).total;
  return segmented_temp_bytes(kind, n, nseg);
}

extern "C" int nsort_plan(int kind, uint64_t n, int *passes, int *sort_tile, int *merge_tile) {
  if (kind != NSORT_KIND_KEYS && kind != NSORT_KIND_PAIRS) return NSORT_EINVAL;
  if (n > MAX_KEYS) return NSORT_EINVAL;
  const Plan p = make_plan(kind, n);
  if (passes) *passes = 1 + p.merge_passes;
  if (sort_tile) *sort_tile = p.sort_tile;
  if (merge_tile) *merge_tile = p.merge_tile;
  return NSORT_OK;
}

static int check_common(const void *a, const void *b, uint64_t n, int dtype, void *tmp,
                        size_t tmp_bytes, int kind) {
  if (dtype != NSORT_U32 && dtype != NSORT_I32 && dtype != NSORT_F32) return NSORT_EINVAL;
  if (n > MAX_KEYS) return NSORT_EINVAL;
  if (n == 0) return NSORT_OK;
  if (!a || !b) return NSORT_EINVAL;
  if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 3) return NSORT_EINVAL;
  const Plan p = make_plan(kind, n);
  if (p.total > 0) {
    if (!tmp || tmp_bytes < p.total) return NSORT_ENOMEM;
    if (reinterpret_cast<uintptr_t>(tmp) & 255) return NSORT_EINVAL;
  }
  return NSORT_OK;
}

extern "C" int nsort_keys(const void *d_keys_in, void *d_keys_out, uint64_t n, int dtype,
                          void *d_tmp, size_t tmp_bytes, void *stream) {
  const int rc = check_common(d_keys_in, d_keys_out, n, dtype, d_tmp, tmp_bytes,
                              NSORT_KIND_KEYS);
  if (rc != NSORT_OK || n == 0) return rc;
  return sort_keys_impl(static_cast<const uint32_t *>(d_keys_in),
                        static_cast<uint32_t *>(d_keys_out), (int64_t)n, dtype, d_tmp,
                        static_cast<cudaStream_t>(stream));
}

extern "C" int nsort_pairs(const void *d_keys_in, const uint32_t *d_vals_in, void *d_keys_out,
                           uint32_t *d_vals_out, uint64_t n, int dtype, void *d_tmp,
                           size_t tmp_bytes, void *stream) {
  int rc = check_common(d_keys_in, d_keys_out, n, dtype, d_tmp, tmp_bytes, NSORT_KIND_PAIRS);
  if (rc != NSORT_OK || n == 0) return rc;
  if (!d_vals_in || !d_vals_out) return NSORT_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_vals_in) | reinterpret_cast<uintptr_t>(d_vals_out)) & 3)
    return NSORT_EINVAL;
  return sort_pairs_impl(static_cast<const uint32_t *>(d_keys_in), d_vals_in,
                         static_cast<uint32_t *>(d_keys_out), d_vals_out, (int64_t)n, dtype,
                         d_tmp, static_cast<cudaStream_t>(stream));
}

extern "C" const char *nsort_status_string(int status) {
  switch (status) {
    case NSORT_OK: return "ok";
    case NSORT_EINVAL: return "invalid argument";
    case NSORT_ENOMEM: return "scratch buffer too small or memory budget exceeded";
    case NSORT_ECUDA: return "CUDA error";
    case NSORT_EBUSY: return "busy";
    case NSORT_ETIMEOUT: return "timed out";
    case NSORT_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
  }
}

extern "C" const char *nsort_last_error(void) { return last_error_cstr(); }
