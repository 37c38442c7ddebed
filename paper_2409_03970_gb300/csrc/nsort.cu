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
#include <cstdlib>
#include <cstring>
#include <string>

#include "nsort.h"
#include "nsort_testing.h"
#include "nsort_internal.h"
#include "sort_device.cuh"
#include "tma_device.cuh"

namespace nsort {

// ---------------------------------------------------------------- kernels

// Thread t stores its VT consecutive outputs o[] at out[t*VT ...], mapped
// back to bit patterns by DT_OUT.  Full, 16-byte aligned tiles use 128-bit
// stores straight from registers; others store element by element.  K is
// the key word (32 or 64 bits).
template <int VT, int DT_OUT, typename K>
__device__ __forceinline__ void store_run(const K (&o)[VT], K *tile_out, int count, bool full) {
  constexpr int EPV = 16 / sizeof(K);   // keys per 128-bit store
  const int e0 = threadIdx.x * VT;
  K *out = tile_out + e0;
  if (full) {
#pragma unroll
    for (int q = 0; q < VT / EPV; ++q) {
      uint4 v;
      if constexpr (EPV == 4) {
        v.x = from_key(o[4 * q + 0], DT_OUT);
        v.y = from_key(o[4 * q + 1], DT_OUT);
        v.z = from_key(o[4 * q + 2], DT_OUT);
        v.w = from_key(o[4 * q + 3], DT_OUT);
      } else {
        const uint64_t lo = from_key(o[2 * q + 0], DT_OUT);
        const uint64_t hi = from_key(o[2 * q + 1], DT_OUT);
        v.x = (uint32_t)lo;
        v.y = (uint32_t)(lo >> 32);
        v.z = (uint32_t)hi;
        v.w = (uint32_t)(hi >> 32);
      }
      reinterpret_cast<uint4 *>(out)[q] = v;
    }
  } else {
#pragma unroll
    for (int k = 0; k < VT; ++k)
      if (e0 + k < count) out[k] = from_key(o[k], DT_OUT);
  }
}

__device__ __forceinline__ bool aligned16(const void *p) {
  return !(reinterpret_cast<uintptr_t>(p) & 15);
}

// Tile sort, keys only.  Tile b covers [b*TILE, min((b+1)*TILE, n)); a short
// last tile is padded with the largest key, which sorts behind every real
// key and is never stored.  DT is the key type (its order-preserving map is
// applied on load); FINAL maps the keys back on store (the tile sort is the
// whole sort when n fits one tile).  in may equal out: each CTA reads its
// whole tile before its first barrier and writes it after its last.
// Every SAMPLE-th output key of a sort stage (tile sort or merge pass) is
// also written to a sample array; the next pass's partition searches the
// samples first (section "sampled partition" below).
constexpr int SAMPLE = 64;

// Column sort of the keys tile sort: the fewest-comparator network of the
// thread's width (Table 1): Green's 60 comparators for 16 keys, two of them
// and an odd-even merge (185) for 32.
struct BestColumns {
  template <typename K, int W>
  __device__ __forceinline__ static void sort(K (&r)[W]) { column_sort_net<NET_BEST, W>(r); }
};

template <int NT, int IPT, int DT, bool FINAL>
__global__ void __launch_bounds__(NT) tile_sort_keys_kernel(const uint32_t *in, uint32_t *out,
                                                            int64_t n, uint32_t *samp) {
  constexpr int TILE = NT * IPT;
  extern __shared__ __align__(16) unsigned char tile_smem[];   // block_smem_len<u32>(NT, IPT) words
  uint32_t *s = reinterpret_cast<uint32_t *>(tile_smem);
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  const int count = (int)(n - base < TILE ? n - base : TILE);
  const bool full = count == TILE && aligned16(in + base) && aligned16(out + base);
  uint32_t r[IPT];
  if (full) {
    const uint4 *p = reinterpret_cast<const uint4 *>(in + base);
#pragma unroll
    for (int j = 0; j < IPT / 4; ++j) {
      const uint4 v = p[tid + NT * j];
      r[4 * j + 0] = to_key(v.x, DT);
      r[4 * j + 1] = to_key(v.y, DT);
      r[4 * j + 2] = to_key(v.z, DT);
      r[4 * j + 3] = to_key(v.w, DT);
    }
  } else {
#pragma unroll
    for (int j = 0; j < IPT / 4; ++j) {
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int e = 4 * (tid + NT * j) + w;
        r[4 * j + w] = e < count ? to_key(in[base + e], DT) : 0xFFFFFFFFu;
      }
    }
  }
  sort_tile_in_block<NT, IPT, BestColumns>(r, s);
  store_run<IPT, FINAL ? DT : DT_U32>(r, out + base, count, full);
  static_assert(SAMPLE % IPT == 0, "a sample starts a thread's run");
  if (!FINAL && samp && !(tid & (SAMPLE / IPT - 1)) && tid * IPT < count)
    store_keep_in_l2(samp + (base + tid * IPT) / SAMPLE, r[0]);
}

// Tile sort, key/value pairs.  The networks sort 64-bit composites
// (key << 32 | position in tile); positions make every composite distinct,
// so the network's result is the stable order.  32-bit values (V) are
// staged in shared memory and gathered by position at the end; 64-bit ones
// are gathered by position from global memory, all of them before the
// first store (in == out is allowed).
template <int NT, int DT, bool FINAL, typename V = uint32_t>
__global__ void __launch_bounds__(NT, 2) tile_sort_pairs_kernel(const uint32_t *kin,
                                                             const V *vin, uint32_t *kout,
                                                             V *vout, int64_t n, uint32_t *samp) {
  constexpr int TILE = NT * 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t *s = reinterpret_cast<uint64_t *>(smem_raw);
  [[maybe_unused]] uint32_t *sv =
      reinterpret_cast<uint32_t *>(s + merge_smem_len<uint64_t>(NT * 16, 16));
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  const int count = (int)(n - base < TILE ? n - base : TILE);
  if constexpr (sizeof(V) == 4) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int e = tid + NT * j;
      if (e < count) sv[pidx<uint32_t>(e)] = vin[base + e];
    }
  }
  uint64_t r[16];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int e = 4 * (tid + NT * j) + w;
      r[4 * j + w] = e < count ? ((uint64_t)to_key(kin[base + e], DT) << 32) | (uint32_t)e
                               : ~0ull;
    }
  }
  sort_tile_in_block<NT, 16, Green16Columns, uint64_t, false>(r, s);
  // every thread passed a barrier after the values were staged
  const bool full = count == TILE && aligned16(kout + base) && aligned16(vout + base);
  uint32_t ko[16];
  if constexpr (sizeof(V) == 4) {
    V vo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      ko[k] = (uint32_t)(r[k] >> 32);
      vo[k] = sv[pidx<uint32_t>((int)(r[k] & 0xFFFFu) & (TILE - 1))];
    }
    store_run<16, FINAL ? DT : DT_U32>(ko, kout + base, count, full);
    store_run<16, DT_U32>(vo, vout + base, count, full);
  } else {
    // keys first (every key was read before the block merges' barriers),
    // then the payloads by position, all read before any is written
    int pos[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      ko[k] = (uint32_t)(r[k] >> 32);
      pos[k] = (int)(r[k] & 0xFFFFu) & (TILE - 1);
    }
    store_run<16, FINAL ? DT : DT_U32>(ko, kout + base, count, full);
    V vo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) vo[k] = tid * 16 + k < count ? vin[base + pos[k]] : V(0);
    __syncthreads();
    store_run<16, DT_U32>(vo, vout + base, count, full);
  }
  if (!FINAL && samp && !(tid & (SAMPLE / 16 - 1)) && tid * 16 < count)
    store_keep_in_l2(samp + (base + tid * 16) / SAMPLE, ko[0]);
}

// Tile sort, 64-bit keys (u64 / i64 / f64): the keys tile sort on 64-bit
// words, NT * 16 keys per tile, the same networks and merges.  Every
// SAMPLE-th output key goes to the sample array as for 32-bit keys.
template <int NT, int DT, bool FINAL>
__global__ void __launch_bounds__(NT) tile_sort_keys64_kernel(const uint64_t *in, uint64_t *out,
                                                              int64_t n, uint64_t *samp) {
  constexpr int TILE = NT * 16;
  extern __shared__ __align__(16) unsigned char tile64_smem[];   // block_smem_len<u64>(NT, 16)
  uint64_t *s = reinterpret_cast<uint64_t *>(tile64_smem);
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * TILE;
  const int count = (int)(n - base < TILE ? n - base : TILE);
  const bool full = count == TILE && aligned16(in + base) && aligned16(out + base);
  uint64_t r[16];
  if (full) {
    const uint4 *p = reinterpret_cast<const uint4 *>(in + base);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint4 v = p[tid + NT * j];
      r[2 * j + 0] = to_key(((uint64_t)v.y << 32) | v.x, DT);
      r[2 * j + 1] = to_key(((uint64_t)v.w << 32) | v.z, DT);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const int e = 2 * (tid + NT * j) + w;
        r[2 * j + w] = e < count ? to_key(in[base + e], DT) : ~0ull;
      }
    }
  }
  sort_tile_in_block<NT, 16, Green16Columns>(r, s);
  store_run<16, FINAL ? DT : DT_U64>(r, out + base, count, full);
  if (!FINAL && samp && !(tid & (SAMPLE / 16 - 1)) && tid * 16 < count)
    store_keep_in_l2(samp + (base + tid * 16) / SAMPLE, r[0]);
}

// Clamps a tile's A co-ranks so that both slices stay inside their runs and
// add up to the tile: a0 in [max(0, d0 - lb), min(d0, la)] and a1 in
// [max(a0, d1 - lb), min(la, a0 + d1 - d0)].  For sorted runs the splitters
// already satisfy this; the clamps only matter when the runs are not what
// the splitters were computed from (another kernel writing the buffers
// during the sort), and then keep every index of the merge in range.
__device__ __forceinline__ void clamp_coranks(int64_t la, int64_t lb, int64_t d0, int64_t d1,
                                              int64_t &a0, int64_t &a1) {
  const int64_t lo0 = d0 - lb > 0 ? d0 - lb : 0, hi0 = d0 < la ? d0 : la;
  a0 = a0 < lo0 ? lo0 : (a0 > hi0 ? hi0 : a0);
  int64_t lo1 = d1 - lb > a0 ? d1 - lb : a0;
  int64_t hi1 = a0 + (d1 - d0) < la ? a0 + (d1 - d0) : la;
  a1 = a1 < lo1 ? lo1 : (a1 > hi1 ? hi1 : a1);
}

// Which slices of the two input runs one merge CTA consumes.
struct PassTile {
  int64_t out0;      // first output element of the tile
  int64_t a_off;     // global index of the first element of the A slice
  int64_t b_off;     // global index of the first element of the B slice
  int na, nb, count;
};

__device__ __forceinline__ PassTile pass_tile(int64_t n, int64_t run, int tile,
                                              const int64_t *split) {
  PassTile g;
  g.out0 = (int64_t)blockIdx.x * tile;
  const int64_t out1 = g.out0 + tile < n ? g.out0 + tile : n;
  const int64_t pair0 = g.out0 & ~(2 * run - 1);
  const int64_t la = n - pair0 < run ? n - pair0 : run;
  const int64_t rest = n - pair0 - run;
  const int64_t lb = rest <= 0 ? 0 : (rest < run ? rest : run);
  const int64_t pair_end = pair0 + la + lb;
  int64_t a_end = out1 == pair_end ? la : split[blockIdx.x + 1];
  int64_t a_beg = split[blockIdx.x];
  clamp_coranks(la, lb, g.out0 - pair0, out1 - pair0, a_beg, a_end);
  const int64_t b_beg = (g.out0 - pair0) - a_beg;
  const int64_t b_end = (out1 - pair0) - a_end;
  g.a_off = pair0 + a_beg;
  g.b_off = pair0 + la + b_beg;
  g.na = (int)(a_end - a_beg);
  g.nb = (int)(b_end - b_beg);
  g.count = g.na + g.nb;
  return g;
}

// Merge-path splitters of one pass, one thread per output tile: how many
// elements of its pair's A run precede the tile (stable: A wins ties).
template <typename K>
__global__ void partition_kernel(const K *__restrict__ src, int64_t n, int64_t run, int tile,
                                 int64_t num_tiles, int64_t *__restrict__ split) {
  pdl_wait();      // the previous kernel of the stream has finished writing
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= num_tiles) return;
  const int64_t out0 = t * tile;
  const int64_t pair0 = out0 & ~(2 * run - 1);
  const int64_t la = n - pair0 < run ? n - pair0 : run;
  const int64_t rest = n - pair0 - run;
  const int64_t lb = rest <= 0 ? 0 : (rest < run ? rest : run);
  split[t] = merge_path_global(src + pair0, la, src + pair0 + la, lb, out0 - pair0);
}

// Stages the merge inputs of one tile, A slice then B slice, into
// s[0, count) (padded layout).  Element i = tid + NT*j of the tile comes
// from A[i] or B[i - na]; all loads are issued before the shared stores.
template <int NT, int VT, typename T>
__device__ __forceinline__ void stage_slices(T *s, const T *__restrict__ src, int64_t a_off,
                                             int64_t b_off, int na, int count) {
  static_assert(NT % 32 == 0, "NT must be a multiple of the warp size");
  const int tid = threadIdx.x;
  const T *pa = src + a_off + tid;
  const T *pb = src + b_off + (tid - na);
  T t[VT];
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    const int i = tid + NT * j;
    T v = 0;
    if (i < na) v = __ldg(pa + NT * j);
    else if (i < count) v = __ldg(pb + NT * j);
    t[j] = v;
  }
  const int sbase = pidx<T>(tid);
#pragma unroll
  for (int j = 0; j < VT; ++j) s[sbase + j * (NT + (NT >> Pad<T>::SHIFT))] = t[j];
}

// One merge pass over keys: CTA b produces output tile b.  DT_OUT maps the
// keys back to bit patterns (last pass only).
template <int NT, int VT, int DT_OUT, typename K = uint32_t>
__global__ void __launch_bounds__(NT, sizeof(K) == 4 ? 6 : 3) merge_keys_kernel(const K *__restrict__ src,
                                                           K *__restrict__ dst, int64_t n,
                                                           int64_t run,
                                                           const int64_t *__restrict__ split) {
  pdl_wait();      // the previous kernel of the stream has finished writing
  constexpr int TILE = NT * VT;
  __shared__ K s[merge_smem_len<K>(TILE, VT)];
  const int tid = threadIdx.x;
  const PassTile g = pass_tile(n, run, TILE, split);
  stage_slices<NT, VT>(s, src, g.a_off, g.b_off, g.na, g.count);
  __syncthreads();
  const int diag = tid * VT < g.count ? tid * VT : g.count;
  const int ai = merge_path_smem(s, 0, g.na, g.na, g.nb, diag);
  K o[VT];
  int unused[VT];
  serial_merge<VT, false>(s, ai, g.na, g.na + diag - ai, g.count, o, unused);
  K *out = dst + g.out0;
  store_run<VT, DT_OUT>(o, out, g.count, g.count == TILE && aligned16(out));
}

// One merge pass over key/value pairs (stable).
template <int NT, int VT, int DT_OUT>
__global__ void __launch_bounds__(NT, 3) merge_pairs_kernel(const uint32_t *__restrict__ ksrc,
                                                            const uint32_t *__restrict__ vsrc,
                                                            uint32_t *__restrict__ kdst,
                                                            uint32_t *__restrict__ vdst,
                                                            int64_t n, int64_t run,
                                                            const int64_t *__restrict__ split) {
  pdl_wait();      // the previous kernel of the stream has finished writing
  constexpr int TILE = NT * VT;
  __shared__ uint32_t sk[merge_smem_len<uint32_t>(TILE, VT)];
  __shared__ uint32_t sv[merge_smem_len<uint32_t>(TILE, VT)];
  const int tid = threadIdx.x;
  const PassTile g = pass_tile(n, run, TILE, split);
  stage_slices<NT, VT>(sk, ksrc, g.a_off, g.b_off, g.na, g.count);
  stage_slices<NT, VT>(sv, vsrc, g.a_off, g.b_off, g.na, g.count);
  __syncthreads();
  const int diag = tid * VT < g.count ? tid * VT : g.count;
  const int ai = merge_path_smem(sk, 0, g.na, g.na, g.nb, diag);
  uint32_t o[VT], ov[VT];
  int from[VT];
  serial_merge<VT, true>(sk, ai, g.na, g.na + diag - ai, g.count, o, from);
#pragma unroll
  for (int k = 0; k < VT; ++k) ov[k] = sv[pidx<uint32_t>(from[k])];
  uint32_t *ko = kdst + g.out0;
  uint32_t *vo = vdst + g.out0;
  const bool full = g.count == TILE && aligned16(ko) && aligned16(vo);
  store_run<VT, DT_OUT>(o, ko, g.count, full);
  store_run<VT, DT_U32>(ov, vo, g.count, full);
}

// ---- persistent merge pass with bulk copies (TMA) ------------------------
//
// Tiles are laid out per run pair: pair p (A = run 2p, B = run 2p+1) owns
// tiles_per_pair = ceil(2*run / TILE) consecutive tiles, so no tile spans
// two pairs and TILE need not be a power of two.  TILE = NT * VT with VT
// odd: thread t starts its merge near element VT*t/2 of each run, which
// spreads a warp's shared-memory reads over the banks without padding (so
// the slices can be staged by plain 1-D bulk copies).

struct PairTile {
  int64_t out0;    // first output of the tile
  int64_t a_off;   // global index of the A slice
  int64_t b_off;   // global index of the B slice
  int na, nb, count;
  int flags;       // DescTiles only: bit 0 input in buf[1], bit 1 last level of its segment
};

// Where tile t of a merge pass lies: the first element of its pair of runs
// (run A, then run B, back to back), the two run lengths, and the tile's
// index within the pair.
struct PairSpan {
  int64_t pair0, la, lb, j;
};

// The runs of one pass of a sort: n elements in runs of `run` (the last ones
// shorter); pair p owns tpp = ceil(2 run / tile) consecutive tiles.  Keys
// are order keys in and out (the kernel's DT_OUT maps them back).
struct UniformRuns {
  static constexpr bool kMaps = false;
  static constexpr bool kDesc = false;
  static constexpr bool kAnyStart = false;   // pairs start at multiples of 2 run
  int64_t n, run, tpp;
  int dt_in = DT_U32, dt_out = DT_U32;   // unused
  __device__ __forceinline__ PairSpan span(int64_t t) const {
    PairSpan s;
    const int64_t pair = t / tpp;
    s.j = t - pair * tpp;
    s.pair0 = pair * 2 * run;
    s.la = n - s.pair0 < run ? n - s.pair0 : run;
    const int64_t rest = n - s.pair0 - run;
    s.lb = rest <= 0 ? 0 : (rest < run ? rest : run);
    return s;
  }
};

// Runs of any lengths, back to back (the merge of sorted shards): pair p
// is runs 2p and 2p+1 (B empty for an odd last run) and owns the tiles
// [first_tile[p], first_tile[p+1]).  Passed by value as a kernel argument.
// The keys arrive as bit patterns of dtype dt_in (DT_U32 / DT_U64: order
// keys already) and leave mapped back to dt_out, chosen at run time: a
// merge of shards runs a few passes, so one kernel serves every dtype.
constexpr int MAX_TABLE_PAIRS = 32;
struct TableRuns {
  static constexpr bool kMaps = true;
  static constexpr bool kDesc = false;
  static constexpr bool kAnyStart = true;    // runs start anywhere
  int dt_in, dt_out;
  int npairs;
  int64_t first_tile[MAX_TABLE_PAIRS + 1];
  int64_t pair0[MAX_TABLE_PAIRS];
  int64_t la[MAX_TABLE_PAIRS];
  int64_t lb[MAX_TABLE_PAIRS];
  __device__ __forceinline__ PairSpan span(int64_t t) const {
    int lo = 0, hi = npairs - 1;   // the last pair p with first_tile[p] <= t (skips empty pairs)
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (first_tile[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    PairSpan s;
    s.pair0 = pair0[lo];
    s.la = la[lo];
    s.lb = lb[lo];
    s.j = t - first_tile[lo];
    return s;
  }
};

// Merge tiles listed one by one in device memory (the merge levels of a
// segmented batch): desc[t] is tile t's complete geometry, written by the
// level's partition kernel, and *count the number of tiles.  Each tile
// reads buf1 if flags bit 0 is set, else buf0, and writes the other buffer
// (segments alternate buffers by the parity of their number of levels, so
// that each one's last level lands in the output); tiles of a segment's
// last level (flags bit 1) map their keys back to dt.
template <typename K>
struct DescTiles {
  static constexpr bool kMaps = false;
  static constexpr bool kDesc = true;
  static constexpr bool kAnyStart = true;    // segments start anywhere
  const PairTile *desc;
  const unsigned long long *count;
  K *buf0, *buf1;
  uint32_t *vbuf0, *vbuf1;
  int dt;
  int dt_in = DT_U32, dt_out = DT_U32;   // unused: kMaps is false
};

// Geometry of tile t from its start splitter s0 and the next tile's s1
// (s1 is ignored when the tile ends its pair).
template <class GEOM>
__device__ __forceinline__ PairTile pair_tile_from(int64_t t, const GEOM &geom, int tile,
                                                   int64_t s0, int64_t s1) {
  PairTile g;
  const PairSpan sp = geom.span(t);
  const int64_t pair0 = sp.pair0, la = sp.la, lb = sp.lb;
  const int64_t pend = pair0 + la + lb;
  g.out0 = pair0 + sp.j * tile;
  const int64_t out1 = g.out0 + tile < pend ? g.out0 + tile : pend;
  int64_t a0 = s0;
  int64_t a1 = out1 == pend ? la : s1;
  clamp_coranks(la, lb, g.out0 - pair0, out1 - pair0, a0, a1);
  g.a_off = pair0 + a0;
  g.b_off = pair0 + la + (g.out0 - pair0 - a0);
  g.na = (int)(a1 - a0);
  g.count = (int)(out1 - g.out0);
  g.nb = g.count - g.na;
  g.flags = 0;
  return g;
}

// Splitter of tile v of the pair-aligned tiling (what the partition kernels
// write to split[v]), found by a group of W lanes of one warp.
template <int W, typename K, class GEOM>
__device__ __forceinline__ int64_t tile_corank_group(const K *src, const GEOM &geom, int tile,
                                                     int64_t v, int glane, unsigned gmask) {
  const PairSpan sp = geom.span(v);
  return merge_path_global_group<W>(src + sp.pair0, sp.la, src + sp.pair0 + sp.la, sp.lb,
                                    sp.j * tile, glane, gmask);
}

// Splitters for the pair-aligned tiling, one thread per tile, by a full
// merge-path search.  The keys are compared as order keys: a geometry that
// maps (the first pass over bit patterns) maps every key it loads.
template <typename K, class GEOM>
__global__ void partition_pairs_kernel(const K *__restrict__ src, const GEOM geom, int tile,
                                       int64_t num_tiles, int64_t *__restrict__ split) {
  pdl_wait();      // the previous kernel of the stream has finished writing
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= num_tiles) return;
  const PairSpan sp = geom.span(t);
  const int dt = GEOM::kMaps ? geom.dt_in : DT_U32;
  const K *A = src + sp.pair0;
  const K *B = A + sp.la;
  const int64_t d = sp.j * tile;
  int64_t lo = d - sp.lb > 0 ? d - sp.lb : 0;
  int64_t hi = d < sp.la ? d : sp.la;
  while (lo < hi) {   // A's share of the first d outputs (A first on ties)
    const int64_t mid = (lo + hi) >> 1;
    if (to_key(__ldg(A + mid), dt) <= to_key(__ldg(B + (d - 1 - mid)), dt)) lo = mid + 1;
    else hi = mid;
  }
  split[t] = lo;
}

// Sampled partition for the pair-aligned tiling.  SA / SB are the samples
// A[64q] / B[64r] written by the previous stage.  A merge-path search on the
// samples at diagonal floor(d/64) gives qs; the true co-rank i* then lies in
// [64(qs-1)+1, 64(qs+2)]: A[64(qs-1)] has at most 64(qs-1) + 64(floor(d/64)
// - qs) < d elements before it in the merge, and A[64(qs+2)] at least
// 64(qs+2) + 64(floor(d/64) - qs - 1) + 1 > d.  The full arrays are then
// searched in that window only, the merge-path conditions are checked at
// the result, and a full search is done if they fail, so the splitter is
// exact whatever the samples say.
template <typename K>
__global__ void partition_sampled_kernel(const K *__restrict__ src, const K *__restrict__ samp,
                                         int64_t n, int64_t run, int64_t tpp, int tile,
                                         int64_t num_tiles, int64_t *__restrict__ split) {
  pdl_wait();      // the previous kernel of the stream has finished writing
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= num_tiles) return;
  const int64_t pair = t / tpp;
  const int64_t j = t - pair * tpp;
  const int64_t pair0 = pair * 2 * run;
  const int64_t la = n - pair0 < run ? n - pair0 : run;
  const int64_t rest = n - pair0 - run;
  const int64_t lb = rest <= 0 ? 0 : (rest < run ? rest : run);
  const int64_t d = j * tile;
  const K *A = src + pair0;
  const K *B = A + la;
  const int64_t lo = d - lb > 0 ? d - lb : 0;
  const int64_t hi = d < la ? d : la;
  const int64_t qs = merge_path_global(samp + pair0 / SAMPLE, (la + SAMPLE - 1) / SAMPLE,
                                       samp + (pair0 + la) / SAMPLE, (lb + SAMPLE - 1) / SAMPLE,
                                       d / SAMPLE);
  int64_t w0 = SAMPLE * (qs - 1) + 1, w1 = SAMPLE * (qs + 2);
  w0 = w0 > lo ? w0 : lo;
  w1 = w1 < hi ? w1 : hi;
  int64_t i = w0 <= w1 ? w0 : lo, e = w0 <= w1 ? w1 : hi;
  while (i < e) {
    const int64_t mid = (i + e) >> 1;
    if (__ldg(A + mid) <= __ldg(B + (d - 1 - mid))) i = mid + 1;
    else e = mid;
  }
  const bool ok = i >= lo && i <= hi &&
                  (i == 0 || d - i >= lb || __ldg(A + i - 1) <= __ldg(B + (d - i))) &&
                  (i >= la || d - i == 0 || __ldg(B + (d - i - 1)) < __ldg(A + i));
  split[t] = ok ? i : merge_path_global(A, la, B, lb, d);
}

// Where a tile's slices sit in its shared-memory buffer.  The A window
// starts at the 16-byte boundary below a_off, so A[i] is at sh_a + i; the B
// window starts at the first 16-byte boundary at least SENT elements after
// A's end, leaving room for the largest-key sentinels of the unchecked
// serial merge.  EPV keys of type K fill 16 bytes.
constexpr int SENT = 32;
struct SmemSlices {
  int sh_a, base_b, sh_b;
};
template <typename K>
__device__ __forceinline__ SmemSlices smem_slices(const PairTile &g) {
  constexpr int EPV = 16 / sizeof(K);
  SmemSlices l;
  l.sh_a = (int)(g.a_off & (EPV - 1));
  l.base_b = (l.sh_a + g.na + SENT + EPV - 1) & ~(EPV - 1);
  l.sh_b = (int)(g.b_off & (EPV - 1));
  return l;
}

// Issues the bulk copies of tile g into buf (and, for pairs, of the values
// into vbuf at the same offsets); lane 0 of warp 0, into buffers no thread
// is reading.  Each slice's window is rounded out to 16-byte boundaries, so
// up to EPV - 1 elements past a slice land in the gap behind it
// (overwritten by sentinels, or never read by the bounds-checked merge);
// windows are clipped at n_al = n rounded down to a multiple of EPV, past
// which the warps load the at most EPV - 1 remaining elements themselves.
// Values (pairs, 32-bit keys only) are 32-bit words at the keys' offsets.
template <typename K, typename V = uint32_t>
__device__ __forceinline__ void issue_tile(const K *__restrict__ src, const V *__restrict__ vsrc,
                                           int64_t n_al, const PairTile &g, K *buf, V *vbuf,
                                           uint64_t *bar) {
  constexpr int64_t EPV = 16 / sizeof(K);
  const SmemSlices l = smem_slices<K>(g);
  const int64_t aw0 = g.a_off & ~(EPV - 1);
  int64_t aw1 = (g.a_off + g.na + EPV - 1) & ~(EPV - 1);
  const int64_t bw0 = g.b_off & ~(EPV - 1);
  int64_t bw1 = (g.b_off + g.nb + EPV - 1) & ~(EPV - 1);
  aw1 = aw1 < n_al ? aw1 : n_al;
  bw1 = bw1 < n_al ? bw1 : n_al;
  const uint32_t bytes_a =
      (g.na > 0 && aw1 > aw0) ? (uint32_t)((aw1 - aw0) * (int64_t)sizeof(K)) : 0u;
  const uint32_t bytes_b =
      (g.nb > 0 && bw1 > bw0) ? (uint32_t)((bw1 - bw0) * (int64_t)sizeof(K)) : 0u;
  // values sit at the keys' element offsets, so a window holds as many
  // values as keys (16-byte aligned as long as a value is not narrower
  // than a key, which the merge kernel checks for pairs)
  const uint32_t vbytes_a = vsrc ? (uint32_t)((uint64_t)bytes_a * sizeof(V) / sizeof(K)) : 0u;
  const uint32_t vbytes_b = vsrc ? (uint32_t)((uint64_t)bytes_b * sizeof(V) / sizeof(K)) : 0u;
  mbar_arrive_expect_tx(bar, bytes_a + bytes_b + vbytes_a + vbytes_b);
  if (bytes_a) bulk_load(buf, src + aw0, bytes_a, bar);
  if (bytes_b) bulk_load(buf + l.base_b, src + bw0, bytes_b, bar);
  if (vsrc) {
    if (vbytes_a) bulk_load(vbuf, vsrc + aw0, vbytes_a, bar);
    if (vbytes_b) bulk_load(vbuf + l.base_b, vsrc + bw0, vbytes_b, bar);
  }
}

// Persistent merge pass with bulk copies, keys (PAIRS = false) or stable
// key/value pairs (PAIRS = true).  Per tile, one CTA-wide barrier: after it,
// every thread is done with the previous tile, so lane 0 of warp 0 can reuse
// that buffer for the next tile's copies while the CTA merges this one.
// Keys: every warp writes the largest-key sentinels it will read itself and
// merges without bounds checks (equal keys are equal bits).  Pairs: the
// merge keeps its bounds checks (a real largest key must win over a
// sentinel to stay stable), records where each output came from and
// gathers the values from shared memory.  Each warp's outputs are
// contiguous (32 * VT), so each warp stages and bulk-stores its own part
// with warp-level synchronisation only.  Lane 0 of warp 0 loads the
// splitters of the tile after next one iteration early.  K is the key word:
// 32-bit keys (keys or pairs) or 64-bit keys (keys only).
// SELF: a self-partitioned pass (split unused), launched only when no CTA has
// more than two tiles.  Warp 0 then finds the splitters itself, which saves
// the separate partition launch and its chain of dependent loads on passes
// too small to hide them: the first tile's start and end (lanes 0-15 and
// 16-31 at once, 16-ary searches) before its copies are issued, then the
// second tile's while those copies land.
// GEOM: where each tile's runs lie (UniformRuns for the passes of a sort,
// TableRuns for merging runs of any lengths; the latter also maps keys from
// bit patterns on arrival and back on the way out, by its run-time dtypes,
// in place of DT_OUT).
// V: the payload word of pairs (32- or 64-bit).
template <int NT, int VT, int DT_OUT, bool PAIRS, typename K = uint32_t, bool SELF = false,
          class GEOM = UniformRuns, typename V = uint32_t>
__global__ void __launch_bounds__(NT, PAIRS ? 3 : 4) merge_tma_kernel(
    const K *__restrict__ src, const V *__restrict__ vsrc, K *__restrict__ dst,
    V *__restrict__ vdst, int64_t n, const GEOM geom, int64_t num_tiles_arg,
    const int64_t *__restrict__ split, int *status, K *samp, int reverse) {
  pdl_wait();      // the previous kernel of the stream has finished writing
  int64_t num_tiles = num_tiles_arg;
  if constexpr (GEOM::kDesc) num_tiles = (int64_t)*geom.count;
  constexpr int TILE = NT * VT;
  constexpr int WOUT = 32 * VT;                       // outputs per warp
  // staging stride per warp: runs of any start (kAnyStart) can start a
  // warp's outputs anywhere, so their staging is shifted to the output's
  // 16-byte phase
  constexpr int WSTRIDE = WOUT + (GEOM::kAnyStart ? 16 / (int)sizeof(K) : 0);
  constexpr int EPV = 16 / sizeof(K);                 // keys per 16 bytes
  // A window + gap, B window + gap, rounding slack
  constexpr int IN_LEN = (TILE + 2 * SENT + 16) & ~3;
  static_assert(SENT >= (PAIRS ? VT + 2 : VT + 1), "the gap behind each run covers a merge's overrun");
  static_assert(SENT == 32, "one sentinel per lane and slice");
  static_assert(WOUT % 4 == 0, "warp output slices must be 16-byte multiples");
  static_assert(WOUT <= 32 * SAMPLE, "one sample per lane and warp slice");
  static_assert(!PAIRS || sizeof(K) == 4, "pairs carry 32-bit keys");
  static_assert(!PAIRS || sizeof(V) >= sizeof(K), "value windows stay 16-byte aligned");
  // dynamic shared memory: keys [in 0][in 1] | values [in 0][in 1] | keys out | values out
  extern __shared__ __align__(128) unsigned char tma_smem[];
  K(*in_buf)[IN_LEN] = reinterpret_cast<K(*)[IN_LEN]>(tma_smem);
  V(*vin_buf)[IN_LEN] = reinterpret_cast<V(*)[IN_LEN]>(tma_smem + (PAIRS ? 2 * IN_LEN * sizeof(K) : 0));
  K *out_buf = reinterpret_cast<K *>(tma_smem + (PAIRS ? 2 * IN_LEN * (sizeof(K) + sizeof(V))
                                                        : 2 * IN_LEN * sizeof(K)));
  V *vout_buf = reinterpret_cast<V *>(out_buf + (NT / 32) * WSTRIDE);
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ PairTile desc[2];   // geometry of the tile in each buffer, written by thread 0
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int64_t n_al = n & ~int64_t(EPV - 1);
  const int64_t G = gridDim.x;
  int64_t t = blockIdx.x;
  // the arrays a tile reads and writes (per tile for DescTiles)
  auto ksrc_of = [&](const PairTile &g) -> const K * {
    if constexpr (GEOM::kDesc) return (g.flags & 1) ? geom.buf1 : geom.buf0;
    else return src;
  };
  auto vsrc_of = [&](const PairTile &g) -> const V * {
    if constexpr (GEOM::kDesc) return (g.flags & 1) ? geom.vbuf1 : geom.vbuf0;
    else return vsrc;
  };
  auto kdst_of = [&](const PairTile &g) -> K * {
    if constexpr (GEOM::kDesc) return (g.flags & 1) ? geom.buf0 : geom.buf1;
    else return dst;
  };
  auto vdst_of = [&](const PairTile &g) -> V * {
    if constexpr (GEOM::kDesc) return (g.flags & 1) ? geom.vbuf0 : geom.vbuf1;
    else return vdst;
  };
  // loop index i -> tile: ascending, or descending when `reverse` (passes
  // alternate direction so that each pass starts where the previous one
  // ended, on data still in L2)
  auto tile_of = [&](int64_t i) { return reverse ? num_tiles - 1 - i : i; };
  int64_t pf0 = 0, pf1 = 0;   // thread 0: splitters of loop index t + G
  [[maybe_unused]] PairTile pfd{};   // thread 0, DescTiles: the descriptor of loop index t + G
  [[maybe_unused]] int64_t own0 = 0, own1 = 0;   // SELF: the first tile's splitters (warp 0)
  // Self-partitioned: warp 0 finds the start splitter of tile u (lanes 0-15)
  // and of the next tile, u's end (lanes 16-31).
  [[maybe_unused]] auto self_split = [&](int64_t i, int64_t &s0, int64_t &s1) {
    if constexpr (!GEOM::kDesc) {   // (descriptor lists carry their splitters)
      const int64_t v = tile_of(i) + (lane >> 4);
      const unsigned gmask = 0xFFFFu << (lane & 16);
      int64_t c = 0;
      if (v < num_tiles) c = tile_corank_group<16>(src, geom, TILE, v, lane & 15, gmask);
      s1 = __shfl_sync(0xffffffffu, c, 16);
      s0 = c;
    }
  };
  if constexpr (SELF) {
    if (warp == 0 && t < num_tiles) self_split(t, own0, own1);
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    if (t < num_tiles) {
      const int64_t u = tile_of(t);
      if constexpr (GEOM::kDesc)
        desc[0] = geom.desc[u];
      else if constexpr (SELF)
        desc[0] = pair_tile_from(u, geom, TILE, own0, own1);
      else
        desc[0] = pair_tile_from(u, geom, TILE, split[u], u + 1 < num_tiles ? split[u + 1] : 0);
      issue_tile(ksrc_of(desc[0]), PAIRS ? vsrc_of(desc[0]) : nullptr, n_al, desc[0], in_buf[0],
                 vin_buf[0], &bar[0]);
    }
    if constexpr (GEOM::kDesc) {
      if (t + G < num_tiles) pfd = geom.desc[tile_of(t + G)];
    } else if constexpr (!SELF) {
      if (t + G < num_tiles) {
        const int64_t u = tile_of(t + G);
        pf0 = split[u];
        pf1 = u + 1 < num_tiles ? split[u + 1] : 0;
      }
    }
  }
  if constexpr (SELF) {
    if (warp == 0 && t + G < num_tiles) self_split(t + G, pf0, pf1);
  }
  __syncthreads();
  bool ok = true;
  K *wout = out_buf + warp * WSTRIDE;
  V *wvout = vout_buf + warp * WSTRIDE;
  for (int it = 0; t < num_tiles; ++it, t += G) {
    const int b = it & 1;
    const int64_t tn = t + G;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const bool got = mbar_wait(&bar[b], parity);
    if (!__syncthreads_and(got)) {
      // a copy did not arrive in time: wait (bounded) for the copies still
      // in flight into this CTA's shared memory, report, and stop
      if (tid == 0) mbar_wait(&bar[b], parity);
      ok = false;
      break;
    }
    // every thread is past the previous tile: its buffer and descriptor are free
    if (tid == 0 && tn < num_tiles) {
      if constexpr (GEOM::kDesc) desc[b ^ 1] = pfd;
      else desc[b ^ 1] = pair_tile_from(tile_of(tn), geom, TILE, pf0, pf1);
      issue_tile(ksrc_of(desc[b ^ 1]), PAIRS ? vsrc_of(desc[b ^ 1]) : nullptr, n_al, desc[b ^ 1],
                 in_buf[b ^ 1], vin_buf[b ^ 1], &bar[b ^ 1]);
      if constexpr (GEOM::kDesc) {
        if (tn + G < num_tiles) pfd = geom.desc[tile_of(tn + G)];
      } else if constexpr (!SELF) {   // (a self-partitioned pass has at most two tiles per CTA)
        const int64_t tp = tn + G;
        if (tp < num_tiles) {
          const int64_t u = tile_of(tp);
          pf0 = split[u];
          pf1 = u + 1 < num_tiles ? split[u + 1] : 0;
        }
      }
    }
    const PairTile g = desc[b];
    const K *tsrc = ksrc_of(g);
    const V *tvsrc = vsrc_of(g);
    K *tdst = kdst_of(g);
    V *tvdst = vdst_of(g);
    const SmemSlices l = smem_slices<K>(g);
    K *s = in_buf[b];
    V *sv = vin_buf[b];
    const int a0 = l.sh_a, b0 = l.base_b + l.sh_b;
    if constexpr (GEOM::kMaps) {
      if (geom.dt_in != DT_U32 && geom.dt_in != DT_U64) {   // the same in every thread
        // bit patterns in: map the bulk-copied part of both slices to order
        // keys in place, all threads, before any warp reads them
        const int64_t ca = n_al - g.a_off, cb = n_al - g.b_off;
        const int na_cp = ca <= 0 ? 0 : (ca < g.na ? (int)ca : g.na);
        const int nb_cp = cb <= 0 ? 0 : (cb < g.nb ? (int)cb : g.nb);
        for (int i = tid; i < na_cp; i += NT) s[a0 + i] = to_key(s[a0 + i], geom.dt_in);
        for (int i = tid; i < nb_cp; i += NT) s[b0 + i] = to_key(s[b0 + i], geom.dt_in);
        __syncthreads();
      }
    }
    // this warp's own array-end elements (and sentinels, for keys); the same
    // values in every warp
    if (g.a_off + g.na > n_al || g.b_off + g.nb > n_al) {
      if (lane < EPV - 1) {
        const int64_t i = (g.a_off > n_al ? g.a_off : n_al) + lane;
        if (i < g.a_off + g.na) {
          s[a0 + (int)(i - g.a_off)] = to_key(__ldg(tsrc + i), GEOM::kMaps ? geom.dt_in : DT_U32);
          if (PAIRS) sv[a0 + (int)(i - g.a_off)] = __ldg(tvsrc + i);
        }
      } else if (lane < 2 * (EPV - 1)) {
        const int64_t i = (g.b_off > n_al ? g.b_off : n_al) + (lane - (EPV - 1));
        if (i < g.b_off + g.nb) {
          s[b0 + (int)(i - g.b_off)] = to_key(__ldg(tsrc + i), GEOM::kMaps ? geom.dt_in : DT_U32);
          if (PAIRS) sv[b0 + (int)(i - g.b_off)] = __ldg(tvsrc + i);
        }
      }
    }
    if (!PAIRS) {
      s[a0 + g.na + lane] = ~K(0);
      s[b0 + g.nb + lane] = ~K(0);
    }
    fence_proxy_async_smem();   // ordered before later bulk copies into this buffer
    __syncwarp();
    const int diag = tid * VT < g.count ? tid * VT : g.count;
    const int ai = merge_path_plain(s, a0, g.na, b0, g.nb, diag);
    K o[VT];
    int from[VT];
    if (PAIRS) serial_merge_plain<VT, true>(s, a0 + ai, a0 + g.na, b0 + diag - ai, b0 + g.nb, o, from);
    else serial_merge_sentinel<VT>(s, a0 + ai, b0 + diag - ai, o);
    V ov[VT];
    if (PAIRS) {
#pragma unroll
      for (int k = 0; k < VT; ++k) ov[k] = sv[from[k]];
    }
    // this warp's slice of the output: stage, then one bulk store per array
    const int w0 = warp * WOUT;
    const int wcount = g.count - w0 < WOUT ? g.count - w0 : WOUT;
    const int64_t gb = g.out0 + w0;                  // the warp's first output
    // sh: gb's offset past a 16-byte boundary, 0 for the uniform runs of a sort
    const int sh = GEOM::kAnyStart ? (int)(gb & (EPV - 1)) : 0;
    K *ws = wout + sh;
    V *wvs = wvout + sh;
    if (lane == 0) bulk_wait_read_all();   // the warp's previous stores have left its slices
    __syncwarp();
    int dt_out = DT_OUT;   // a constant unless GEOM maps at run time
    if constexpr (GEOM::kMaps) dt_out = geom.dt_out;
    if constexpr (GEOM::kDesc) dt_out = (g.flags & 2) ? geom.dt : (sizeof(K) == 8 ? DT_U64 : DT_U32);
    if (g.count == TILE) {
#pragma unroll
      for (int k = 0; k < VT; ++k) {
        ws[lane * VT + k] = from_key(o[k], dt_out);
        if (PAIRS) wvs[lane * VT + k] = ov[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < VT; ++k) {
        if (tid * VT + k < g.count) {
          ws[lane * VT + k] = from_key(o[k], dt_out);
          if (PAIRS) wvs[lane * VT + k] = ov[k];
        }
      }
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (samp && wcount > 0) {   // every SAMPLE-th output key, for the next partition
      const int e = (int)((SAMPLE - (gb & (SAMPLE - 1))) & (SAMPLE - 1)) + SAMPLE * lane;
      if (e < wcount) store_keep_in_l2(samp + (gb + e) / SAMPLE, ws[e]);
    }
    if (wcount > 0) {
      // head: plain stores up to the first 16-byte boundary (none when sh =
      // 0); body: one bulk store per array (smem and global addresses both
      // 16-byte aligned, since ws and dst + gb share their phase); tail:
      // plain stores of the last EPV - 1 or fewer
      const int hd = (EPV - sh) & (EPV - 1);
      const int head = hd < wcount ? hd : wcount;
      const int body = (wcount - head) & ~(EPV - 1);
      const int tail = wcount - head - body;
      if (lane == 0 && body) {
        bulk_store(tdst + gb + head, ws + head, (uint32_t)body * (uint32_t)sizeof(K));
        if (PAIRS) bulk_store(tvdst + gb + head, wvs + head, (uint32_t)body * (uint32_t)sizeof(V));
        bulk_commit();
      }
      if (lane < head) {
        tdst[gb + lane] = ws[lane];
        if (PAIRS) tvdst[gb + lane] = wvs[lane];
      }
      if (lane < tail) {
        tdst[gb + head + body + lane] = ws[head + body + lane];
        if (PAIRS) tvdst[gb + head + body + lane] = wvs[head + body + lane];
      }
    }
  }
  if (lane == 0) bulk_wait_all();
  if (tid == 0 && !ok) atomicExch(status, (int)NSORT_ETIMEOUT);
}

// ---- four-way merge passes ----------------------------------------------
//
// A four-way pass merges each group of four consecutive runs of `run` keys
// into one run of 4 run keys with one read and one write of the array: the
// two merge levels of the group (runs 0+1 and 2+3, then the two results)
// run back to back on each tile, the first one in shared memory.  This
// halves the passes over HBM of the merge phase.
//
// Tiles are cut at samples.  The pass's input samples (the key at every
// SAMPLE-th position, written by the previous stage) of a group, merged in
// stable (key, position) order, give every M4_M-th merged sample b as a tile
// boundary.  Its co-rank c_r(b) in run r is the number of run-r keys that
// precede it in the stable order of the group: keys <= key(b) for runs
// before b's own run, keys < key(b) for runs after it, and b's own index in
// its run.  If q_r samples of run r precede b, c_r(b) lies in
// [SAMPLE q_r - SAMPLE + 1, SAMPLE q_r], so between two boundaries M4_M
// samples apart the four runs give at most SAMPLE M4_M + 4 (SAMPLE - 1)
// keys: a tile's size is bounded without an exact multiway selection.

constexpr int M4_NT = 128;
constexpr int M4_VT = 35;                 // level-two outputs per thread: two chains
constexpr int M4_H = (M4_VT + 1) / 2;     // outputs of the first chain
constexpr int M4_M = 64;                  // merged samples per tile
constexpr int M4_TMAX = SAMPLE * M4_M + 4 * (SAMPLE - 1);   // largest tile (4348)
constexpr int M4_C1 = ((M4_TMAX + M4_NT - 1) / M4_NT) | 1;  // most level-one outputs per chain
constexpr int M4_SENT = 40;               // largest keys behind each slice and level-one run
constexpr int M4_IN_LEN = (M4_TMAX + 4 * (M4_SENT + 8) + 15) & ~15;   // one input buffer
constexpr int M4_MID_LEN = (M4_TMAX + 2 * M4_SENT + 8 + 15) & ~15;    // level-one output
constexpr int M4_WOUT = 32 * M4_VT;       // outputs per warp
constexpr int M4_WSTRIDE = M4_WOUT + 4;   // per-warp staging, shifted to the 16-byte phase
constexpr size_t M4_SMEM =
    sizeof(uint32_t) * (2 * M4_IN_LEN + M4_MID_LEN + (M4_NT / 32) * M4_WSTRIDE);
static_assert(M4_NT * M4_VT >= M4_TMAX, "level two covers the largest tile");
static_assert(M4_SENT >= M4_C1 + 1 && M4_SENT >= M4_H + 1,
              "the gap behind each run covers a chain's overrun");
static_assert(M4_WOUT <= 32 * SAMPLE, "one sample per lane and warp slice");
static_assert(M4_WOUT % 4 == 0, "warp output slices stay 16-byte multiples");
constexpr int M4_CTAS = 3;                // resident CTAs per SM (shared memory bound)

// The partition of a four-way pass runs in two kernels of CTAs that each take
// SMG_CHUNK consecutive outputs of a merge of two sample runs: one warp finds
// the chunk's first co-rank and another its last (32-ary searches), the CTA
// stages both windows in shared memory and merges (or searches) there.
constexpr int SMG_NT = 256;
constexpr int SMG_CHUNK = 4096;
constexpr int SMG_PER = SMG_CHUNK / SMG_NT;   // outputs per thread, level one
constexpr int SMB_NT = 512;                   // level two: one warp per boundary at a time

// Level one: the samples of runs 2p and 2p+1 (sample s is the key at
// position SAMPLE s; rs samples per full run, ns in all) merged stably into
// records (key << 32 | s), at the pair's own sample indices.  A chunk is
// min(SMG_CHUNK, 2 rs) outputs, so no chunk crosses a pair.
__global__ void __launch_bounds__(SMG_NT) sample_merge_kernel(const uint32_t *__restrict__ samp,
                                                              int64_t ns, int64_t rs,
                                                              uint64_t *__restrict__ rec) {
  pdl_wait();
  __shared__ uint32_t sk[SMG_CHUNK];   // the A window, then the B window
  __shared__ int64_t cr[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t unit = 2 * rs;
  const int64_t C = unit < SMG_CHUNK ? unit : SMG_CHUNK;
  const int64_t c0 = (int64_t)blockIdx.x * C;
  if (c0 >= ns) return;
  const int64_t p0 = c0 - c0 % unit;
  const int64_t la = ns - p0 < rs ? ns - p0 : rs;
  const int64_t rest = ns - p0 - rs;
  const int64_t lb = rest <= 0 ? 0 : (rest < rs ? rest : rs);
  const uint32_t *A = samp + p0;
  const uint32_t *B = A + la;
  const int64_t d0 = c0 - p0;
  const int64_t d1 = d0 + C < la + lb ? d0 + C : la + lb;
  if (warp < 2)   // run 2p first on ties
    cr[warp] = merge_path_global_group<32>(A, la, B, lb, warp ? d1 : d0, lane, 0xffffffffu);
  __syncthreads();
  const int64_t a0 = cr[0], b0 = d0 - a0;
  const int na = (int)(cr[1] - a0), nb = (int)(d1 - cr[1] - b0);
  for (int i = tid; i < na; i += SMG_NT) sk[i] = __ldg(A + a0 + i);
  for (int i = tid; i < nb; i += SMG_NT) sk[na + i] = __ldg(B + b0 + i);
  __syncthreads();
  const int cnt = na + nb;
  const int o = tid * SMG_PER;
  if (o >= cnt) return;
  int ia = merge_path_plain(sk, 0, na, na, nb, o);
  int ib = o - ia;
#pragma unroll 4
  for (int k = 0; k < SMG_PER && o + k < cnt; ++k) {
    const bool ta = ia < na && (ib >= nb || sk[ia] <= sk[na + ib]);
    uint64_t r;
    if (ta) {
      r = ((uint64_t)sk[ia] << 32) | (uint64_t)(p0 + a0 + ia);
      ++ia;
    } else {
      r = ((uint64_t)sk[na + ib] << 32) | (uint64_t)(p0 + la + b0 + ib);
      ++ib;
    }
    rec[c0 + o + k] = r;
  }
}

// Level two and the tile boundaries of a four-way pass.  Group g's records
// are X (the level-one merge of runs 0 and 1) and then Y (runs 2 and 3); a
// chunk is min(SMG_CHUNK, 4 rs) consecutive ranks of the merge of X and Y.
// Interior boundary j of the group is the sample of merged rank j M4_M.  For
// each one in its chunk a warp finds X's share x of the ranks below it (a
// merge-path search of the staged windows), takes the boundary b = the
// smaller of X[x] and Y[m - x], and reads from the first record of X and of
// Y not before b how many samples of each run precede b (a record names its
// run and its index there).  Then lanes 8r to 8r+7 count the keys of run r
// before b among the at most SAMPLE - 1 keys where its co-rank can lie.
// Writes c_r of every boundary record (tpg + 1 a group: the group's start,
// its interior boundaries, and its end repeated up to tpg).
__global__ void __launch_bounds__(SMB_NT) merge4_bounds_kernel(const uint32_t *__restrict__ src,
                                                               const uint64_t *__restrict__ rec,
                                                               int64_t n, int64_t run, int64_t tpg,
                                                               int64_t *__restrict__ bnd) {
  pdl_wait();
  __shared__ uint64_t sr[SMG_CHUNK + 2];   // X window (+1 record), then Y window (+1)
  __shared__ int64_t cr[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lrun = 63 - __clzll((unsigned long long)run);   // run is a power of two
  const int64_t unit = 4 * (run / SAMPLE);
  const int64_t C = unit < SMG_CHUNK ? unit : SMG_CHUNK;
  const int64_t c0 = (int64_t)blockIdx.x * C;
  const int64_t g = c0 >> (lrun - 4);   // unit = run / 16
  const int64_t G0 = g << (lrun + 2);
  auto len_of = [&](int q) {
    const int64_t s = n - G0 - q * run;
    return s <= 0 ? int64_t(0) : (s < run ? s : run);
  };
  auto samples_of = [&](int q) { return (len_of(q) + SAMPLE - 1) / SAMPLE; };
  const int64_t nx = samples_of(0) + samples_of(1), ny = samples_of(2) + samples_of(3);
  const int64_t cnt = nx + ny;
  const int64_t tiles_g = (cnt + M4_M - 1) / M4_M;
  const int64_t d0 = c0 - g * unit;
  if (d0 >= cnt) return;   // past the samples of a partial last group
  const int64_t d1 = d0 + C < cnt ? d0 + C : cnt;
  int64_t *grec = bnd + 4 * g * (tpg + 1);
  if (d0 == 0 && tid < 4) grec[tid] = 0;   // the group's start
  if (d1 == cnt)                           // its end, in every record from tiles_g on
    for (int64_t i = tiles_g * 4 + tid; i < (tpg + 1) * 4; i += SMB_NT) grec[i] = len_of((int)(i & 3));
  // interior boundaries with ranks in [d0, d1) (a chunk can start on one)
  const int64_t jf = d0 == 0 ? 1 : (d0 + M4_M - 1) / M4_M;
  const int64_t jl = (d1 - 1) / M4_M;
  if (jf > jl) return;
  const uint64_t *X = rec + G0 / SAMPLE;
  const uint64_t *Y = X + nx;
  if (warp < 2)   // records are distinct
    cr[warp] = merge_path_global_group<32>(X, nx, Y, ny, warp ? d1 : d0, lane, 0xffffffffu);
  __syncthreads();
  const int64_t a0 = cr[0], b0 = d0 - a0;
  const int wa = (int)(cr[1] - a0), wb = (int)(d1 - cr[1] - b0);   // the chunk's windows
  const int na = wa + (cr[1] < nx ? 1 : 0);                        // and one record more
  const int nb = wb + (d1 - cr[1] < ny ? 1 : 0);
  for (int i = tid; i < na; i += SMB_NT) sr[i] = __ldg(X + a0 + i);
  for (int i = tid; i < nb; i += SMB_NT) sr[na + i] = __ldg(Y + b0 + i);
  __syncthreads();
  const int r = lane >> 3, sub = lane & 7;
  const int64_t len_r = len_of(r);
  const uint32_t *R = src + G0 + r * run;
  for (int64_t j = jf + warp; j <= jl; j += SMB_NT / 32) {
    const int64_t m = j * M4_M;
    const int xl = merge_path_plain(sr, 0, wa, na, wb, (int)(m - d0));
    const int64_t x = a0 + xl, y = m - x;
    const bool hx = x < nx, hy = y < ny;
    const uint64_t xr = hx ? sr[xl] : 0ull;
    const uint64_t yr = hy ? sr[na + (int)(y - b0)] : 0ull;
    const uint64_t bs = (hx && (!hy || xr < yr)) ? xr : yr;   // the boundary sample
    const uint32_t vb = (uint32_t)(bs >> 32);
    const int64_t ib = (int64_t)(uint32_t)bs * SAMPLE - G0;   // its position in the group
    const int rb = (int)(ib >> lrun);
    int64_t c;
    if (r == rb) {
      c = ib - rb * run;
    } else {
      // samples of run r before b: from the first record of r's side not before b
      const bool has = r < 2 ? hx : hy;
      const uint64_t nr = r < 2 ? xr : yr;
      const int64_t side = r < 2 ? x : y;
      int64_t q = (len_r + SAMPLE - 1) / SAMPLE;
      if (has) {
        const int64_t pn = (int64_t)(uint32_t)nr * SAMPLE - G0;
        const int rn = (int)(pn >> lrun);
        const int64_t in = (pn - ((int64_t)rn << lrun)) / SAMPLE;
        q = rn == r ? in : side - in;
      }
      int64_t wlo = SAMPLE * q - (SAMPLE - 1);
      int64_t whi = SAMPLE * q;
      wlo = wlo > 0 ? wlo : 0;
      whi = whi < len_r ? whi : len_r;
      int before = 0;   // keys of the window before b (a prefix: the run is sorted)
#pragma unroll
      for (int i = 0; i < SAMPLE / 8; ++i) {
        const int64_t k = wlo + sub + 8 * i;
        if (k < whi) {
          const uint32_t v = __ldg(R + k);
          before += (r < rb ? v <= vb : v < vb) ? 1 : 0;
        }
      }
      before += __shfl_xor_sync(0xffffffffu, before, 1);
      before += __shfl_xor_sync(0xffffffffu, before, 2);
      before += __shfl_xor_sync(0xffffffffu, before, 4);
      c = wlo + before;
    }
    if (sub == 0) grec[4 * j + r] = c;
  }
}

// One serial merge in shared memory, advanced one output at a time (the
// (lo, hi) formulation of serial_merge_sentinel: the run with the smaller
// head, its head, and the other run's head).  Two of these per thread give
// the scheduler two independent chains of loads.
struct MergeChain {
  uint32_t hlo, hhi;
  int ilo, ihi;
  __device__ __forceinline__ void init(const uint32_t *s, int a, int b) {
    const uint32_t ka = s[a], kb = s[b];
    const bool t0 = ka <= kb;
    hlo = t0 ? ka : kb;
    hhi = t0 ? kb : ka;
    ilo = t0 ? a : b;
    ihi = t0 ? b : a;
  }
  __device__ __forceinline__ void step(const uint32_t *s) {
    const int i = ilo + 1;
    const uint32_t kn = s[i];
    const bool p = kn <= hhi;
    hlo = p ? kn : hhi;
    ilo = p ? i : ihi;
    hhi = p ? hhi : kn;
    ihi = p ? ihi : i;
  }
};

// Two merge-path searches in shared memory at once: A's share of the first
// d0 outputs of merging s[a0, a0 + na) with s[b0, b0 + nb) into r0, and of
// the first d1 outputs of merging s[c0, c0 + nc) with s[e0, e0 + ne) into r1.
// Branch-free, so that the two chains of loads overlap: a search that has
// finished keeps probing its answer, whose two loads stay inside the buffer
// (at most A's first element past its end, at least one element before B).
__device__ __forceinline__ void merge_path_pair(const uint32_t *s, int a0, int na, int b0, int nb,
                                                int d0, int c0, int nc, int e0, int ne, int d1,
                                                int &r0, int &r1) {
  int lo0 = d0 - nb > 0 ? d0 - nb : 0, hi0 = d0 < na ? d0 : na;
  int lo1 = d1 - ne > 0 ? d1 - ne : 0, hi1 = d1 < nc ? d1 : nc;
  while (lo0 < hi0 || lo1 < hi1) {
    const int m0 = (lo0 + hi0) >> 1, m1 = (lo1 + hi1) >> 1;
    const bool p0 = s[a0 + m0] <= s[b0 + d0 - 1 - m0];
    const bool p1 = s[c0 + m1] <= s[e0 + d1 - 1 - m1];
    const bool g0 = lo0 < hi0, g1 = lo1 < hi1;
    lo0 = g0 && p0 ? m0 + 1 : lo0;
    hi0 = g0 && !p0 ? m0 : hi0;
    lo1 = g1 && p1 ? m1 + 1 : lo1;
    hi1 = g1 && !p1 ? m1 : hi1;
  }
  r0 = lo0;
  r1 = lo1;
}

// A four-way tile: slice r of run r of its group starts at global index
// off[r] and holds len[r] keys; in the input buffer its copy window starts
// at base[r] (16-byte aligned) and its first key sits at sidx[r].
struct Tile4 {
  int64_t out0;
  int64_t off[4];
  int len[4];
  int base[4];
  int sidx[4];
  int count;
};

// Tile u's geometry from its boundary co-ranks c[0..3] (its start) and
// c[4..7] (its end).  A tile whose co-ranks leave their runs or go
// backwards, or that holds more than M4_TMAX keys (none of which occurs for
// sorted runs and complete boundary records), is made empty and reported in
// *status, so that no copy or store leaves the array.
__device__ __forceinline__ Tile4 tile4_from(int64_t u, int64_t n, int64_t run, int64_t tpg,
                                            const int64_t (&c)[8], int *status) {
  Tile4 g;
  const int64_t G0 = (u / tpg) * 4 * run;
  int64_t out0 = G0, count = 0;
  bool ok = true;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t rest = n - G0 - r * run;
    const int64_t len = rest <= 0 ? 0 : (rest < run ? rest : run);
    const int64_t l = c[4 + r] - c[r];
    ok = ok && l >= 0 && c[r] >= 0 && c[4 + r] <= len;
    out0 += c[r];
    count += l;
  }
  ok = ok && count <= M4_TMAX;
  if (!ok) atomicCAS(status, 0, (int)NSORT_EINVAL);
  g.out0 = out0;
  g.count = ok ? (int)count : 0;
  int base = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    g.off[r] = G0 + r * run + c[r];
    g.len[r] = ok ? (int)(c[4 + r] - c[r]) : 0;
    g.base[r] = base;
    g.sidx[r] = base + (int)(g.off[r] & 3);
    base = (g.sidx[r] + g.len[r] + M4_SENT + 3) & ~3;
  }
  return g;
}

__device__ __forceinline__ void issue_tile4(const uint32_t *__restrict__ src, int64_t n_al,
                                            const Tile4 &g, uint32_t *buf, uint64_t *bar) {
  uint32_t bytes[4];
  int64_t w0[4];
  uint32_t total = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    w0[r] = g.off[r] & ~int64_t(3);
    int64_t w1 = (g.off[r] + g.len[r] + 3) & ~int64_t(3);
    w1 = w1 < n_al ? w1 : n_al;
    bytes[r] = (g.len[r] > 0 && w1 > w0[r]) ? (uint32_t)((w1 - w0[r]) * 4) : 0u;
    total += bytes[r];
  }
  mbar_arrive_expect_tx(bar, total);
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (bytes[r]) bulk_load(buf + g.base[r], src + w0[r], bytes[r], bar);
}

// The four-way pass.  Persistent CTAs, double-buffered bulk copies of each
// tile's four slices as in merge_tma_kernel; per tile: level one (every
// thread merges an odd number of outputs of slices 0+1 and as many of
// slices 2+3, as two interleaved chains, into the shared level-one
// buffer), one CTA barrier, level two (M4_VT outputs per thread as two
// interleaved chains), then per-warp staging and bulk stores as in
// merge_tma_kernel.  Keys are order keys in; DT_OUT maps them back on the
// last pass.  samp: the samples of the output (nullptr on the last pass).
template <int DT_OUT>
__global__ void __launch_bounds__(M4_NT, M4_CTAS) merge4_tma_kernel(
    const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, int64_t n, int64_t run,
    int64_t tpg, int64_t num_tiles, const int64_t *__restrict__ bnd, int *status, uint32_t *samp,
    int reverse) {
  pdl_wait();
  extern __shared__ __align__(128) unsigned char m4_smem[];
  uint32_t(*in_buf)[M4_IN_LEN] = reinterpret_cast<uint32_t(*)[M4_IN_LEN]>(m4_smem);
  uint32_t *mid = reinterpret_cast<uint32_t *>(m4_smem) + 2 * M4_IN_LEN;
  uint32_t *out_buf = mid + M4_MID_LEN;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ Tile4 desc[2];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int64_t n_al = n & ~int64_t(3);
  const int64_t G = gridDim.x;
  int64_t t = blockIdx.x;
  auto tile_of = [&](int64_t i) { return reverse ? num_tiles - 1 - i : i; };
  // boundary record of tile u: the group's records, then the tile's index in it
  auto rec_of = [&](int64_t u) { return (u / tpg) * (tpg + 1) + (u % tpg); };
  int64_t pf[8];   // thread 0: the co-ranks of loop index t + G
  auto load_pf = [&](int64_t u) {
    const int64_t *p = bnd + 4 * rec_of(u);
#pragma unroll
    for (int i = 0; i < 8; ++i) pf[i] = __ldg(p + i);
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    if (t < num_tiles) {
      const int64_t u = tile_of(t);
      load_pf(u);
      desc[0] = tile4_from(u, n, run, tpg, pf, status);
      issue_tile4(src, n_al, desc[0], in_buf[0], &bar[0]);
    }
    if (t + G < num_tiles) load_pf(tile_of(t + G));
  }
  __syncthreads();
  bool ok = true;
  uint32_t *wout = out_buf + warp * M4_WSTRIDE;
  for (int it = 0; t < num_tiles; ++it, t += G) {
    const int b = it & 1;
    const int64_t tn = t + G;
    const uint32_t parity = (uint32_t)((it >> 1) & 1);
    const bool got = mbar_wait(&bar[b], parity);
    if (!__syncthreads_and(got)) {
      // a copy did not arrive in time: wait (bounded) for the copies still
      // in flight into this CTA's shared memory, report, and stop
      if (tid == 0) mbar_wait(&bar[b], parity);
      ok = false;
      break;
    }
    // every thread is past the previous tile: its buffer and descriptor are free
    if (tid == 0 && tn < num_tiles) {
      desc[b ^ 1] = tile4_from(tile_of(tn), n, run, tpg, pf, status);
      issue_tile4(src, n_al, desc[b ^ 1], in_buf[b ^ 1], &bar[b ^ 1]);
      if (tn + G < num_tiles) load_pf(tile_of(tn + G));
    }
    const Tile4 &g = desc[b];   // read in place: the merges index its slices at run time
    uint32_t *s = in_buf[b];
    // every warp: the keys past n_al that the copies left out, then the
    // largest-key sentinels behind each slice (the same values in every warp)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (g.off[r] + g.len[r] > n_al && lane < 3) {
        const int64_t i = (g.off[r] > n_al ? g.off[r] : n_al) + lane;
        if (i < g.off[r] + g.len[r]) s[g.sidx[r] + (int)(i - g.off[r])] = __ldg(src + i);
      }
      for (int i = lane; i < M4_SENT; i += 32) s[g.sidx[r] + g.len[r] + i] = ~0u;
    }
    fence_proxy_async_smem();   // ordered before later bulk copies into this buffer
    __syncwarp();
    // level one: X = slices 0+1 into mid[0, lx), Y = slices 2+3 into
    // mid[yb, yb + ly); every thread takes cx outputs of X and cy of Y and
    // runs the two merges side by side
    const int lx = g.len[0] + g.len[1], ly = g.len[2] + g.len[3];
    const int yb = (lx + M4_SENT + 3) & ~3;
    {
      // odd counts: the threads' start positions then fall in different banks
      const int cx = ((lx + M4_NT - 1) / M4_NT) | 1, cy = ((ly + M4_NT - 1) / M4_NT) | 1;
      const int dx = tid * cx < lx ? tid * cx : lx, dy = tid * cy < ly ? tid * cy : ly;
      int ax, ay;
      merge_path_pair(s, g.sidx[0], g.len[0], g.sidx[1], g.len[1], dx, g.sidx[2], g.len[2],
                      g.sidx[3], g.len[3], dy, ax, ay);
      MergeChain X, Y;
      X.init(s, g.sidx[0] + ax, g.sidx[1] + dx - ax);
      Y.init(s, g.sidx[2] + ay, g.sidx[3] + dy - ay);
      const int ex = lx - dx, ey = ly - dy;   // outputs this thread may store
      uint32_t *wx = mid + dx, *wy = mid + yb + dy;
      const int cm = cx > cy ? cx : cy;
      // both chains step every time (past its count a chain only walks into
      // largest-key sentinels); only the stores are predicated
#pragma unroll
      for (int k = 0; k < M4_C1; ++k) {
        if (k >= cm) break;
        if (k < cx && k < ex) wx[k] = X.hlo;
        if (k < cy && k < ey) wy[k] = Y.hlo;
        X.step(s);
        Y.step(s);
      }
    }
    for (int i = tid; i < M4_SENT; i += M4_NT) {
      mid[lx + i] = ~0u;
      mid[yb + ly + i] = ~0u;
    }
    __syncthreads();
    // level two: X and Y into this thread's M4_VT outputs, as two chains
    // (outputs 0 .. M4_H - 1 and M4_H .. M4_VT - 1)
    uint32_t o[M4_VT];
    {
      const int d0 = tid * M4_VT < g.count ? tid * M4_VT : g.count;
      const int d1 = tid * M4_VT + M4_H < g.count ? tid * M4_VT + M4_H : g.count;
      int a2, b2;
      merge_path_pair(mid, 0, lx, yb, ly, d0, 0, lx, yb, ly, d1, a2, b2);
      MergeChain A, B;
      A.init(mid, a2, yb + d0 - a2);
      B.init(mid, b2, yb + d1 - b2);
#pragma unroll
      for (int k = 0; k < M4_H; ++k) {
        o[k] = A.hlo;
        A.step(mid);
        if (k < M4_VT - M4_H) {
          o[M4_H + k] = B.hlo;
          B.step(mid);
        }
      }
    }
    // this warp's slice of the output: stage, then one bulk store
    const int w0 = warp * M4_WOUT;
    const int wcount = g.count - w0 < 0 ? 0 : (g.count - w0 < M4_WOUT ? g.count - w0 : M4_WOUT);
    const int64_t gb = g.out0 + w0;
    const int sh = (int)(gb & 3);
    uint32_t *ws = wout + sh;
    if (lane == 0) bulk_wait_read_all();   // the warp's previous stores have left its slice
    __syncwarp();
    if (g.count - w0 >= M4_WOUT) {
#pragma unroll
      for (int k = 0; k < M4_VT; ++k) ws[lane * M4_VT + k] = from_key(o[k], DT_OUT);
    } else {
#pragma unroll
      for (int k = 0; k < M4_VT; ++k)
        if (tid * M4_VT + k < g.count) ws[lane * M4_VT + k] = from_key(o[k], DT_OUT);
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (samp && wcount > 0) {   // every SAMPLE-th output key, for the next pass
      const int e = (int)((SAMPLE - (gb & (SAMPLE - 1))) & (SAMPLE - 1)) + SAMPLE * lane;
      if (e < wcount) store_keep_in_l2(samp + (gb + e) / SAMPLE, ws[e]);
    }
    if (wcount > 0) {
      const int hd = (4 - sh) & 3;
      const int head = hd < wcount ? hd : wcount;
      const int body = (wcount - head) & ~3;
      const int tail = wcount - head - body;
      if (lane == 0 && body) {
        bulk_store(dst + gb + head, ws + head, (uint32_t)body * 4u);
        bulk_commit();
      }
      if (lane < head) dst[gb + lane] = ws[lane];
      if (lane < tail) dst[gb + head + body + lane] = ws[head + body + lane];
    }
  }
  if (lane == 0) bulk_wait_all();
  if (tid == 0 && !ok) atomicExch(status, (int)NSORT_ETIMEOUT);
}

// ------------------------------------------------------------- host side

namespace {

constexpr int KEYS_SORT_NT = 512;   // tile sort: 512 threads x 32 keys = 16384
constexpr int KEYS_SORT_IPT = 32;
constexpr int PAIRS_SORT_NT = 512;  //            512 threads x 16 pairs = 8192
constexpr int MERGE_NT = 256;       // merge pass: 256 threads x 16 = 4096 outputs
constexpr int MERGE_VT = 16;
constexpr int PMERGE_NT = 256;
constexpr int PMERGE_VT = 16;

constexpr int TMA_MERGE_NT = 128;   // persistent merge pass: 128 threads x 31 = 3968 outputs
constexpr int TMA_MERGE_VT = 31;
constexpr int TMA_MERGE_TILE = TMA_MERGE_NT * TMA_MERGE_VT;

constexpr int TMA_PMERGE_NT = 128;  // pairs: 128 threads x 15 = 1920 outputs
constexpr int TMA_PMERGE_VT = 15;
constexpr int TMA_PMERGE_TILE = TMA_PMERGE_NT * TMA_PMERGE_VT;

// 64-bit keys: tiles of 256 x 16 keys; merge tiles of 128 x 15 outputs (the
// pairs geometry: the same bytes per element); staged-load fallback 256 x 16
constexpr int KEYS64_SORT_NT = 256;
constexpr int TMA_K64_NT = 128;
constexpr int TMA_K64_VT = 15;
constexpr int TMA_K64_TILE = TMA_K64_NT * TMA_K64_VT;
constexpr int MERGE64_NT = 256;
constexpr int MERGE64_VT = 16;

// dynamic shared memory of merge_tma_kernel: input buffers (two per array)
// and output staging (one per array); key words of kbytes bytes, 32-bit values
constexpr size_t tma_merge_smem(int tile, bool pairs, size_t kbytes = 4, size_t vbytes = 4) {
  return (kbytes + (pairs ? vbytes : 0)) * (2 * ((tile + 2 * 32 + 16) & ~3) + tile);
}
constexpr size_t TMA_MERGE_SMEM = tma_merge_smem(TMA_MERGE_TILE, false);
constexpr size_t TMA_PMERGE_SMEM = tma_merge_smem(TMA_PMERGE_TILE, true);
constexpr size_t TMA_PMERGE64_SMEM = tma_merge_smem(TMA_PMERGE_TILE, true, 4, 8);   // 64-bit payloads
constexpr size_t TMA_K64_SMEM = tma_merge_smem(TMA_K64_TILE, false, 8);
constexpr int KEYS64_SORT_TILE = KEYS64_SORT_NT * 16;
constexpr size_t KEYS64_SORT_SMEM =
    sizeof(uint64_t) * block_smem_len<uint64_t>(KEYS64_SORT_NT, 16);
constexpr int MERGE64_TILE = MERGE64_NT * MERGE64_VT;

constexpr int KEYS_SORT_TILE = KEYS_SORT_NT * KEYS_SORT_IPT;
constexpr size_t KEYS_SORT_SMEM =
    sizeof(uint32_t) * block_smem_len<uint32_t>(KEYS_SORT_NT, KEYS_SORT_IPT);
constexpr int PAIRS_SORT_TILE = PAIRS_SORT_NT * 16;
constexpr int MERGE_TILE = MERGE_NT * MERGE_VT;
constexpr int PMERGE_TILE = PMERGE_NT * PMERGE_VT;

constexpr size_t PAIRS_SORT_SMEM =
    sizeof(uint64_t) * merge_smem_len<uint64_t>(PAIRS_SORT_TILE, 16) +
    sizeof(uint32_t) * padded_len<uint32_t>(PAIRS_SORT_TILE);
// 64-bit payloads are gathered from global memory: no value staging
constexpr size_t PAIRS64_SORT_SMEM = sizeof(uint64_t) * merge_smem_len<uint64_t>(PAIRS_SORT_TILE, 16);

template <typename V>
constexpr size_t pairs_sort_smem() { return sizeof(V) == 4 ? PAIRS_SORT_SMEM : PAIRS64_SORT_SMEM; }

}  // namespace

int64_t pair_tiles(int64_t n, int64_t run, int tile, int64_t *tpp_out) {
  const int64_t tpp = (2 * run + tile - 1) / tile;
  const int64_t full = n / (2 * run);
  const int64_t rem = n - full * 2 * run;
  if (tpp_out) *tpp_out = tpp;
  return full * tpp + (rem + tile - 1) / tile;
}

// ---- four-way passes (host) ----------------------------------------------

// Smallest sort (32-bit keys) whose merge phase takes four-way passes; below
// it every pass is two-way.  Changed only by the test hook.
static std::atomic<uint64_t> g_four_way_min{~uint64_t(0)};

static bool use_four_way(int64_t n, int merge_passes) {
  return merge_passes >= 2 && (uint64_t)n >= g_four_way_min.load();
}

// Tiles of a four-way pass over n keys in runs of `run`: tpg per full group
// of four runs, and those of the last, partial group.
static int64_t merge4_tiles(int64_t n, int64_t run, int64_t *tpg_out, int64_t *groups_out) {
  const int64_t tpg = (4 * (run / SAMPLE) + M4_M - 1) / M4_M;
  const int64_t full = n / (4 * run);
  int64_t tiles = full * tpg;
  const int64_t g0 = full * 4 * run;
  if (g0 < n) {
    int64_t cnt = 0;
    for (int q = 0; q < 4; ++q) {
      const int64_t s = n - g0 - q * run;
      const int64_t len = s <= 0 ? 0 : (s < run ? s : run);
      cnt += (len + SAMPLE - 1) / SAMPLE;
    }
    tiles += (cnt + M4_M - 1) / M4_M;
  }
  if (tpg_out) *tpg_out = tpg;
  if (groups_out) *groups_out = (n + 4 * run - 1) / (4 * run);
  return tiles;
}

// Boundary records of the four-way passes of a plan (the most any pass
// needs: the first four-way pass has the shortest runs).
static int64_t merge4_records(int64_t n, int64_t run0) {
  int64_t tpg = 0, groups = 0;
  merge4_tiles(n, run0, &tpg, &groups);
  return groups * (tpg + 1);
}

Plan make_plan(int kind, uint64_t n, int dtype) {
  Plan p;
  const bool pairs = kind == NSORT_KIND_PAIRS || kind == NSORT_KIND_PAIRS64;
  const size_t vw = kind == NSORT_KIND_PAIRS64 ? 8 : 4;   // bytes per payload word
  const bool wide = !pairs && dtype >= NSORT_U64;   // 64-bit keys
  const size_t kw = wide ? 8 : 4;                   // bytes per key word
  p.n = (int64_t)n;
  p.sort_tile = pairs ? PAIRS_SORT_TILE : (wide ? KEYS64_SORT_TILE : KEYS_SORT_TILE);
  // the bulk-copy pass's tile; the staged-load fallback uses (P)MERGE_TILE
  p.merge_tile = pairs ? TMA_PMERGE_TILE : (wide ? TMA_K64_TILE : TMA_MERGE_TILE);
  const int fallback_tile = pairs ? PMERGE_TILE : (wide ? MERGE64_TILE : MERGE_TILE);
  const int64_t runs = (p.n + p.sort_tile - 1) / p.sort_tile;
  p.merge_passes = 0;
  while ((int64_t(1) << p.merge_passes) < runs) ++p.merge_passes;
  // 32-bit keys: two merge levels per pass over HBM on large arrays, and a
  // two-way pass first when the number of levels is odd
  const bool four = kind == NSORT_KIND_KEYS && !wide && use_four_way(p.n, p.merge_passes);
  p.merge4_passes = four ? p.merge_passes / 2 : 0;
  p.merge2_passes = p.merge_passes - 2 * p.merge4_passes;
  p.num_merge_tiles = (p.n + fallback_tile - 1) / fallback_tile;
  // splitters: enough for the power-of-two tiling and for the pair-aligned
  // tiling of every pass
  int64_t max_tiles = p.num_merge_tiles;
  for (int pass = 0; pass < p.merge_passes; ++pass) {
    const int64_t t = pair_tiles(p.n, (int64_t)p.sort_tile << pass, p.merge_tile, nullptr);
    if (t > max_tiles) max_tiles = t;
  }
  const size_t kb = align_up((size_t)n * kw, 256);
  const size_t vb = align_up((size_t)n * vw, 256);
  p.status_off = 0;
  p.keys_off = 256;
  p.vals_off = p.keys_off + kb;
  p.split_off = pairs ? p.vals_off + vb : p.keys_off + kb;
  p.samp_off = p.split_off + align_up((size_t)(max_tiles + 1) * sizeof(int64_t), 256);
  p.rec_off = p.samp_off + align_up((size_t)(n / SAMPLE + 2) * kw, 256);
  p.bnd_off = p.rec_off;
  if (four) {
    const int64_t run0 = (int64_t)p.sort_tile << p.merge2_passes;   // the first four-way pass's runs
    p.bnd_off = p.rec_off + align_up((size_t)(n / SAMPLE + 2) * sizeof(uint64_t), 256);
    p.total = p.bnd_off + align_up((size_t)merge4_records(p.n, run0) * 4 * sizeof(int64_t), 256);
  } else {
    p.total = p.merge_passes == 0 ? 0 : p.rec_off;
  }
  return p;
}

// Launches a kernel with programmatic stream serialisation: the launch is
// processed while the previous kernel of the stream still runs and its CTAs
// start as soon as that kernel completes, which hides the launch latency
// between the dependent kernels of a sort (about 20% of a 2^20-key sort, 1%
// at 2^28).  Every kernel so launched calls pdl_wait() before it reads or
// writes anything the previous kernels touch.  NSORT_NO_PDL=1 in the
// environment selects plain launches.
static bool pdl_enabled() {
  static const bool on = [] {
    const char *e = getenv("NSORT_NO_PDL");
    return !(e && e[0] == '1');
  }();
  return on;
}

template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                       cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

static int launch_status(const char *what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return NSORT_OK;
  set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return NSORT_ECUDA;
}

// ---- template dispatch (key type and "last pass" are compile-time) -------

template <int DT, bool FIN>
static void keys_sort_smem_attr() {
  cudaFuncSetAttribute(tile_sort_keys_kernel<KEYS_SORT_NT, KEYS_SORT_IPT, DT, FIN>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KEYS_SORT_SMEM);
}

static void launch_tile_sort_keys(const uint32_t *in, uint32_t *out, int64_t n, int dt,
                                  bool final_pass, unsigned grid, uint32_t *samp, cudaStream_t st) {
  static std::atomic<uint64_t> done_mask{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (!bit || !(done_mask.load() & bit)) {   // opt in to the dynamic shared memory, once per device
    keys_sort_smem_attr<DT_U32, false>();
    keys_sort_smem_attr<DT_U32, true>();
    keys_sort_smem_attr<DT_I32, false>();
    keys_sort_smem_attr<DT_I32, true>();
    keys_sort_smem_attr<DT_F32, false>();
    keys_sort_smem_attr<DT_F32, true>();
    done_mask.fetch_or(bit);
  }
#define NSORT_TSK(DT, FIN)                                                        \
  tile_sort_keys_kernel<KEYS_SORT_NT, KEYS_SORT_IPT, DT, FIN>                             \
      <<<grid, KEYS_SORT_NT, KEYS_SORT_SMEM, st>>>(                                       \
      in, out, n, samp)
  if (dt == DT_U32) { if (final_pass) NSORT_TSK(DT_U32, true); else NSORT_TSK(DT_U32, false); }
  else if (dt == DT_I32) { if (final_pass) NSORT_TSK(DT_I32, true); else NSORT_TSK(DT_I32, false); }
  else { if (final_pass) NSORT_TSK(DT_F32, true); else NSORT_TSK(DT_F32, false); }
#undef NSORT_TSK
}

// A whole sort in one CTA of NT threads x 16 keys (a tile of 16 NT keys).
template <int NT>
static void small_sort_nt(const uint32_t *in, uint32_t *out, int64_t n, int dt, cudaStream_t st) {
  constexpr size_t smem = sizeof(uint32_t) * block_smem_len<uint32_t>(NT, 16);
  static_assert(smem <= 48 * 1024, "fits the default dynamic shared memory");
  if (dt == DT_U32) tile_sort_keys_kernel<NT, 16, DT_U32, true><<<1, NT, smem, st>>>(in, out, n, nullptr);
  else if (dt == DT_I32) tile_sort_keys_kernel<NT, 16, DT_I32, true><<<1, NT, smem, st>>>(in, out, n, nullptr);
  else tile_sort_keys_kernel<NT, 16, DT_F32, true><<<1, NT, smem, st>>>(in, out, n, nullptr);
}

// A sort that fits one tile of a smaller configuration takes the smallest
// of 512, 2048 and 8192 keys (32, 128 or 512 threads x 16 keys) that holds
// n, so that a short array does not pay for a full 16384-key tile.  Returns
// false when n needs the full tile.
static bool launch_small_sort(const uint32_t *in, uint32_t *out, int64_t n, int dt,
                              cudaStream_t st) {
  if (n <= 512) small_sort_nt<32>(in, out, n, dt, st);
  else if (n <= 2048) small_sort_nt<128>(in, out, n, dt, st);
  else if (n <= 8192) small_sort_nt<512>(in, out, n, dt, st);
  else return false;
  return true;
}

static void launch_merge_keys(const uint32_t *src, uint32_t *dst, int64_t n, int64_t run,
                              const int64_t *split, int dt_out, unsigned grid, cudaStream_t st) {
#define NSORT_MK(DT) \
  merge_keys_kernel<MERGE_NT, MERGE_VT, DT><<<grid, MERGE_NT, 0, st>>>(src, dst, n, run, split)
  if (dt_out == DT_U32) NSORT_MK(DT_U32);
  else if (dt_out == DT_I32) NSORT_MK(DT_I32);
  else NSORT_MK(DT_F32);
#undef NSORT_MK
}

template <int DT, bool FIN, typename V>
static cudaError_t pairs_smem_attr() {
  return cudaFuncSetAttribute(tile_sort_pairs_kernel<PAIRS_SORT_NT, DT, FIN, V>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)pairs_sort_smem<V>());
}

template <typename V>
static int ensure_pairs_smem_attr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return launch_status("cudaGetDevice");
  static std::atomic<uint64_t> done_mask{0};
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done_mask.load() & bit)) return NSORT_OK;
  cudaError_t e = pairs_smem_attr<DT_U32, false, V>();
  if (e == cudaSuccess) e = pairs_smem_attr<DT_U32, true, V>();
  if (e == cudaSuccess) e = pairs_smem_attr<DT_I32, false, V>();
  if (e == cudaSuccess) e = pairs_smem_attr<DT_I32, true, V>();
  if (e == cudaSuccess) e = pairs_smem_attr<DT_F32, false, V>();
  if (e == cudaSuccess) e = pairs_smem_attr<DT_F32, true, V>();
  if (e != cudaSuccess) return launch_status("cudaFuncSetAttribute");
  done_mask.fetch_or(bit);
  return NSORT_OK;
}

template <typename V>
static void launch_tile_sort_pairs(const uint32_t *kin, const V *vin, uint32_t *kout, V *vout,
                                   int64_t n, int dt, bool final_pass, unsigned grid,
                                   uint32_t *samp, cudaStream_t st) {
#define NSORT_TSP(DT, FIN)                                                                  \
  tile_sort_pairs_kernel<PAIRS_SORT_NT, DT, FIN, V><<<grid, PAIRS_SORT_NT, pairs_sort_smem<V>(), \
                                                      st>>>(kin, vin, kout, vout, n, samp)
  if (dt == DT_U32) { if (final_pass) NSORT_TSP(DT_U32, true); else NSORT_TSP(DT_U32, false); }
  else if (dt == DT_I32) { if (final_pass) NSORT_TSP(DT_I32, true); else NSORT_TSP(DT_I32, false); }
  else { if (final_pass) NSORT_TSP(DT_F32, true); else NSORT_TSP(DT_F32, false); }
#undef NSORT_TSP
}

static void launch_merge_pairs(const uint32_t *ks, const uint32_t *vs, uint32_t *kd, uint32_t *vd,
                               int64_t n, int64_t run, const int64_t *split, int dt_out,
                               unsigned grid, cudaStream_t st) {
#define NSORT_MP(DT) \
  merge_pairs_kernel<PMERGE_NT, PMERGE_VT, DT><<<grid, PMERGE_NT, 0, st>>>(ks, vs, kd, vd, n, run, split)
  if (dt_out == DT_U32) NSORT_MP(DT_U32);
  else if (dt_out == DT_I32) NSORT_MP(DT_I32);
  else NSORT_MP(DT_F32);
#undef NSORT_MP
}

static void launch_partition(const uint32_t *src, int64_t n, int64_t run, const Plan &p,
                             int tile, int64_t *split, cudaStream_t st) {
  const unsigned blocks = (unsigned)((p.num_merge_tiles + 255) / 256);
  partition_kernel<<<blocks, 256, 0, st>>>(src, n, run, tile, p.num_merge_tiles, split);
}

template <int NT, int VT, bool PAIRS, typename V = uint32_t>
static void tma_merge_attrs(size_t smem) {
  using U = UniformRuns;
  const void *fns[6] = {(const void *)merge_tma_kernel<NT, VT, DT_U32, PAIRS, uint32_t, false, U, V>,
                        (const void *)merge_tma_kernel<NT, VT, DT_I32, PAIRS, uint32_t, false, U, V>,
                        (const void *)merge_tma_kernel<NT, VT, DT_F32, PAIRS, uint32_t, false, U, V>,
                        (const void *)merge_tma_kernel<NT, VT, DT_U32, PAIRS, uint32_t, true, U, V>,
                        (const void *)merge_tma_kernel<NT, VT, DT_I32, PAIRS, uint32_t, true, U, V>,
                        (const void *)merge_tma_kernel<NT, VT, DT_F32, PAIRS, uint32_t, true, U, V>};
  for (const void *f : fns) {   // opt in to the dynamic shared memory; prefer it over L1
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
}

// Persistent merge pass: SMs x resident CTAs, found once per device and
// kind (0 keys, 1 pairs, 2 64-bit keys, 3 pairs with 64-bit payloads).
static int tma_merge_grid(int64_t tiles, int kind) {
  static std::atomic<int> cached[4][64];
  int dev = 0;
  cudaGetDevice(&dev);
  int g = dev < 64 ? cached[kind][dev].load() : 0;
  if (g == 0) {
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (kind == 2) {
      const void *fns[6] = {
          (const void *)merge_tma_kernel<TMA_K64_NT, TMA_K64_VT, DT_U64, false, uint64_t>,
          (const void *)merge_tma_kernel<TMA_K64_NT, TMA_K64_VT, DT_I64, false, uint64_t>,
          (const void *)merge_tma_kernel<TMA_K64_NT, TMA_K64_VT, DT_F64, false, uint64_t>,
          (const void *)merge_tma_kernel<TMA_K64_NT, TMA_K64_VT, DT_U64, false, uint64_t, true>,
          (const void *)merge_tma_kernel<TMA_K64_NT, TMA_K64_VT, DT_I64, false, uint64_t, true>,
          (const void *)merge_tma_kernel<TMA_K64_NT, TMA_K64_VT, DT_F64, false, uint64_t, true>};
      for (const void *f : fns) {
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_K64_SMEM);
        cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      }
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &occ, merge_tma_kernel<TMA_K64_NT, TMA_K64_VT, DT_U64, false, uint64_t>, TMA_K64_NT,
          TMA_K64_SMEM);
    } else if (kind == 3) {
      tma_merge_attrs<TMA_PMERGE_NT, TMA_PMERGE_VT, true, uint64_t>(TMA_PMERGE64_SMEM);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &occ, merge_tma_kernel<TMA_PMERGE_NT, TMA_PMERGE_VT, DT_U32, true, uint32_t, false,
                                 UniformRuns, uint64_t>,
          TMA_PMERGE_NT, TMA_PMERGE64_SMEM);
    } else if (kind == 1) {
      tma_merge_attrs<TMA_PMERGE_NT, TMA_PMERGE_VT, true>(TMA_PMERGE_SMEM);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &occ, merge_tma_kernel<TMA_PMERGE_NT, TMA_PMERGE_VT, DT_U32, true>, TMA_PMERGE_NT,
          TMA_PMERGE_SMEM);
    } else {
      tma_merge_attrs<TMA_MERGE_NT, TMA_MERGE_VT, false>(TMA_MERGE_SMEM);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &occ, merge_tma_kernel<TMA_MERGE_NT, TMA_MERGE_VT, DT_U32, false>, TMA_MERGE_NT,
          TMA_MERGE_SMEM);
    }
    g = (sms > 0 ? sms : 1) * (occ > 0 ? occ : 1);
    if (dev < 64) cached[kind][dev].store(g);
  }
  return (int)(tiles < g ? tiles : g);
}

// One bulk-copy merge pass (keys when vsrc is null, else stable pairs with
// payload word V).
// samp_in: samples of src (from the previous stage); samp_out: where this
// pass writes the samples of dst (nullptr for the last pass).
template <typename V = uint32_t>
static void launch_merge_tma(const uint32_t *src, const V *vsrc, uint32_t *dst, V *vdst,
                             int64_t n, int64_t run, int64_t *split, int *status, int dt_out,
                             const uint32_t *samp_in, uint32_t *samp_out, int reverse,
                             cudaStream_t st) {
  constexpr bool V64 = sizeof(V) == 8;
  const bool pairs = vsrc != nullptr;
  const int tile = pairs ? TMA_PMERGE_TILE : TMA_MERGE_TILE;
  int64_t tpp = 0;
  const int64_t tiles = pair_tiles(n, run, tile, &tpp);
  const unsigned grid = (unsigned)tma_merge_grid(tiles, pairs ? (V64 ? 3 : 1) : 0);
  const UniformRuns geom{n, run, tpp};
  if (tiles > 2 * (int64_t)grid) {
    TraceScope tr(TK_PARTITION, st);
    launch_pdl(partition_sampled_kernel<uint32_t>, (unsigned)((tiles + 255) / 256), 256, 0, st,
               src, samp_in, n, run, tpp, tile, tiles, split);
  } else {
    split = nullptr;   // at most two tiles per CTA: each finds its own splitters
  }
  TraceScope tr(pairs ? TK_MERGE_PAIRS : TK_MERGE_KEYS, st);
#define NSORT_MT1(NT, VT, DT, P, SMEM, SELF)                                                  \
  launch_pdl(merge_tma_kernel<NT, VT, DT, P, uint32_t, SELF, UniformRuns, V>, grid, NT, SMEM, st, \
             src, vsrc, dst, vdst, n, geom, tiles, split, status, samp_out, reverse)
#define NSORT_MT(NT, VT, DT, P, SMEM)                                                        \
  do {                                                                                       \
    if (split) NSORT_MT1(NT, VT, DT, P, SMEM, false);                                       \
    else NSORT_MT1(NT, VT, DT, P, SMEM, true);                                              \
  } while (0)
  if constexpr (V64) {   // pairs with 64-bit payloads
    if (dt_out == DT_U32) NSORT_MT(TMA_PMERGE_NT, TMA_PMERGE_VT, DT_U32, true, TMA_PMERGE64_SMEM);
    else if (dt_out == DT_I32) NSORT_MT(TMA_PMERGE_NT, TMA_PMERGE_VT, DT_I32, true, TMA_PMERGE64_SMEM);
    else NSORT_MT(TMA_PMERGE_NT, TMA_PMERGE_VT, DT_F32, true, TMA_PMERGE64_SMEM);
  } else if (!pairs) {
    if (dt_out == DT_U32) NSORT_MT(TMA_MERGE_NT, TMA_MERGE_VT, DT_U32, false, TMA_MERGE_SMEM);
    else if (dt_out == DT_I32) NSORT_MT(TMA_MERGE_NT, TMA_MERGE_VT, DT_I32, false, TMA_MERGE_SMEM);
    else NSORT_MT(TMA_MERGE_NT, TMA_MERGE_VT, DT_F32, false, TMA_MERGE_SMEM);
  } else {
    if (dt_out == DT_U32) NSORT_MT(TMA_PMERGE_NT, TMA_PMERGE_VT, DT_U32, true, TMA_PMERGE_SMEM);
    else if (dt_out == DT_I32) NSORT_MT(TMA_PMERGE_NT, TMA_PMERGE_VT, DT_I32, true, TMA_PMERGE_SMEM);
    else NSORT_MT(TMA_PMERGE_NT, TMA_PMERGE_VT, DT_F32, true, TMA_PMERGE_SMEM);
  }
#undef NSORT_MT
#undef NSORT_MT1
}

template <int DT>
static void merge4_attr() {
  cudaFuncSetAttribute(merge4_tma_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)M4_SMEM);
  cudaFuncSetAttribute(merge4_tma_kernel<DT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

// SMs x resident CTAs of the four-way kernel, found once per device.
static int merge4_grid(int64_t tiles) {
  static std::atomic<int> cached[64];
  int dev = 0;
  cudaGetDevice(&dev);
  int g = dev < 64 ? cached[dev].load() : 0;
  if (g == 0) {
    merge4_attr<DT_U32>();
    merge4_attr<DT_I32>();
    merge4_attr<DT_F32>();
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, merge4_tma_kernel<DT_U32>, M4_NT, M4_SMEM);
    g = (sms > 0 ? sms : 1) * (occ > 0 ? occ : 1);
    if (dev < 64) cached[dev].store(g);
  }
  return (int)(tiles < g ? tiles : g);
}

// One four-way pass: the level-one merge of the input samples, the tile
// boundaries, then the merge.  samp holds the input's samples and receives
// the output's (unless samp_out is null: the last pass).
static void launch_merge4(const uint32_t *src, uint32_t *dst, int64_t n, int64_t run,
                          const uint32_t *samp, uint64_t *rec, int64_t *bnd, int *status,
                          int dt_out, uint32_t *samp_out, int reverse, cudaStream_t st) {
  const int64_t ns = (n + SAMPLE - 1) / SAMPLE;
  int64_t tpg = 0, groups = 0;
  const int64_t tiles = merge4_tiles(n, run, &tpg, &groups);
  const unsigned grid = (unsigned)merge4_grid(tiles);
  const int64_t rs = run / SAMPLE;
  {
    TraceScope tr(TK_SAMPLE_MERGE, st);
    const int64_t c1 = 2 * rs < SMG_CHUNK ? 2 * rs : SMG_CHUNK;
    launch_pdl(sample_merge_kernel, (unsigned)((ns + c1 - 1) / c1), SMG_NT, 0, st, samp, ns, rs,
               rec);
  }
  {
    TraceScope tr(TK_MERGE4_BOUNDS, st);
    const int64_t c2 = 4 * rs < SMG_CHUNK ? 4 * rs : SMG_CHUNK;
    launch_pdl(merge4_bounds_kernel, (unsigned)(groups * (4 * rs / c2)), SMB_NT, 0, st, src,
               (const uint64_t *)rec, n, run, tpg, bnd);
  }
  TraceScope tr(TK_MERGE4_KEYS, st);
#define NSORT_M4(DT)                                                                         \
  launch_pdl(merge4_tma_kernel<DT>, grid, M4_NT, M4_SMEM, st, src, dst, n, run, tpg, tiles, \
             (const int64_t *)bnd, status, samp_out, reverse)
  if (dt_out == DT_U32) NSORT_M4(DT_U32);
  else if (dt_out == DT_I32) NSORT_M4(DT_I32);
  else NSORT_M4(DT_F32);
#undef NSORT_M4
}

// ---- 64-bit keys -------------------------------------------------------------

static void launch_tile_sort_keys64(const uint64_t *in, uint64_t *out, int64_t n, int dt,
                                    bool final_pass, unsigned grid, uint64_t *samp,
                                    cudaStream_t st) {
  static_assert(KEYS64_SORT_SMEM <= 48 * 1024, "fits the default dynamic shared memory");
#define NSORT_TSK64(DT, FIN)                                                            \
  tile_sort_keys64_kernel<KEYS64_SORT_NT, DT, FIN><<<grid, KEYS64_SORT_NT, KEYS64_SORT_SMEM, \
                                                     st>>>(in, out, n, samp)
  if (dt == DT_U64) { if (final_pass) NSORT_TSK64(DT_U64, true); else NSORT_TSK64(DT_U64, false); }
  else if (dt == DT_I64) { if (final_pass) NSORT_TSK64(DT_I64, true); else NSORT_TSK64(DT_I64, false); }
  else { if (final_pass) NSORT_TSK64(DT_F64, true); else NSORT_TSK64(DT_F64, false); }
#undef NSORT_TSK64
}

// One bulk-copy merge pass over 64-bit keys (sampled partition, then the
// persistent merge), as launch_merge_tma does for 32-bit keys.
static void launch_merge_tma64(const uint64_t *src, uint64_t *dst, int64_t n, int64_t run,
                               int64_t *split, int *status, int dt_out, const uint64_t *samp_in,
                               uint64_t *samp_out, int reverse, cudaStream_t st) {
  int64_t tpp = 0;
  const int64_t tiles = pair_tiles(n, run, TMA_K64_TILE, &tpp);
  const unsigned grid = (unsigned)tma_merge_grid(tiles, 2);
  const UniformRuns geom{n, run, tpp};
  if (tiles > 2 * (int64_t)grid) {
    TraceScope tr(TK_PARTITION, st);
    launch_pdl(partition_sampled_kernel<uint64_t>, (unsigned)((tiles + 255) / 256), 256, 0, st,
               src, samp_in, n, run, tpp, TMA_K64_TILE, tiles, split);
  } else {
    split = nullptr;   // at most two tiles per CTA: each finds its own splitters
  }
  TraceScope tr(TK_MERGE_KEYS64, st);
  const uint32_t *no_vals = nullptr;
  uint32_t *no_vals_out = nullptr;
#define NSORT_MT64S(DT, SELF)                                                                \
  launch_pdl(merge_tma_kernel<TMA_K64_NT, TMA_K64_VT, DT, false, uint64_t, SELF>, grid,       \
             TMA_K64_NT, TMA_K64_SMEM, st, src, no_vals, dst, no_vals_out, n, geom, tiles, \
             split, status, samp_out, reverse)
#define NSORT_MT64(DT)                                                                       \
  do {                                                                                       \
    if (split) NSORT_MT64S(DT, false);                                                       \
    else NSORT_MT64S(DT, true);                                                              \
  } while (0)
  if (dt_out == DT_U64) NSORT_MT64(DT_U64);
  else if (dt_out == DT_I64) NSORT_MT64(DT_I64);
  else NSORT_MT64(DT_F64);
#undef NSORT_MT64
#undef NSORT_MT64S
}

// Staged-load merge pass over 64-bit keys, for output buffers that are not
// 16-byte aligned.
static void launch_merge_staged64(const uint64_t *src, uint64_t *dst, int64_t n, int64_t run,
                                  int64_t *split, int dt_out, int64_t tiles, cudaStream_t st) {
  {
    TraceScope tr(TK_PARTITION, st);
    partition_kernel<<<(unsigned)((tiles + 255) / 256), 256, 0, st>>>(src, n, run, MERGE64_TILE,
                                                                     tiles, split);
  }
  TraceScope tr(TK_MERGE_KEYS64, st);
#define NSORT_MK64(DT)                                                                   \
  merge_keys_kernel<MERGE64_NT, MERGE64_VT, DT, uint64_t><<<(unsigned)tiles, MERGE64_NT, 0, \
                                                           st>>>(src, dst, n, run, split)
  if (dt_out == DT_U64) NSORT_MK64(DT_U64);
  else if (dt_out == DT_I64) NSORT_MK64(DT_I64);
  else NSORT_MK64(DT_F64);
#undef NSORT_MK64
}

int sort_keys64_impl(const uint64_t *in, uint64_t *out, int64_t n, int dt, void *tmp,
                     cudaStream_t st) {
  const Plan p = make_plan(NSORT_KIND_KEYS, (uint64_t)n, dt);
  char *t = static_cast<char *>(tmp);
  uint64_t *bufs[2] = {out, p.merge_passes ? reinterpret_cast<uint64_t *>(t + p.keys_off) : nullptr};
  int64_t *split = p.merge_passes ? reinterpret_cast<int64_t *>(t + p.split_off) : nullptr;
  int *status = p.merge_passes ? reinterpret_cast<int *>(t + p.status_off) : nullptr;
  uint64_t *samp = p.merge_passes ? reinterpret_cast<uint64_t *>(t + p.samp_off) : nullptr;
  if (status && cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
    return launch_status("cudaMemsetAsync");
  const bool tma = !(reinterpret_cast<uintptr_t>(out) & 15);
  int cur = p.merge_passes % 2;   // the last pass must land in bufs[0] == out
  const int64_t tiles = (n + p.sort_tile - 1) / p.sort_tile;
  {
    TraceScope tr(TK_TILE_SORT_KEYS64, st);
    launch_tile_sort_keys64(in, bufs[cur], n, dt, p.merge_passes == 0, (unsigned)tiles,
                            tma ? samp : nullptr, st);
  }
  int rc = launch_status("tile_sort_keys64");
  for (int pass = 0; rc == NSORT_OK && pass < p.merge_passes; ++pass) {
    const int64_t run = (int64_t)p.sort_tile << pass;
    const bool last = pass == p.merge_passes - 1;
    const int dt_out = last ? dt : DT_U64;
    if (tma)
      launch_merge_tma64(bufs[cur], bufs[cur ^ 1], n, run, split, status, dt_out, samp,
                         last ? nullptr : samp, (pass & 1) == 0, st);
    else
      launch_merge_staged64(bufs[cur], bufs[cur ^ 1], n, run, split, dt_out, p.num_merge_tiles,
                            st);
    rc = launch_status("merge_keys64");
    cur ^= 1;
  }
  return rc;
}

// ---- the sorts ------------------------------------------------------------

int sort_keys_impl(const uint32_t *in, uint32_t *out, int64_t n, int dt, void *tmp,
                   cudaStream_t st) {
  const Plan p = make_plan(NSORT_KIND_KEYS, (uint64_t)n);
  char *t = static_cast<char *>(tmp);
  uint32_t *bufs[2] = {out, p.merge_passes ? reinterpret_cast<uint32_t *>(t + p.keys_off) : nullptr};
  int64_t *split = p.merge_passes ? reinterpret_cast<int64_t *>(t + p.split_off) : nullptr;
  int *status = p.merge_passes ? reinterpret_cast<int *>(t + p.status_off) : nullptr;
  uint32_t *samp = p.merge_passes ? reinterpret_cast<uint32_t *>(t + p.samp_off) : nullptr;
  if (status && cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
    return launch_status("cudaMemsetAsync");
  // the bulk-copy merge pass needs 16-byte aligned ping-pong buffers (the
  // scratch always is); otherwise the staged-load pass is used
  const bool tma = !(reinterpret_cast<uintptr_t>(out) & 15);
  // the plan's passes: two-way ones (one level each) first, then four-way
  // ones (two levels each); the staged-load fallback merges one level a pass
  const int n2 = tma ? p.merge2_passes : p.merge_passes;
  const int n4 = tma ? p.merge4_passes : 0;
  const int npass = n2 + n4;
  int cur = npass % 2;  // the last pass must land in bufs[0] == out
  const int64_t tiles = (n + p.sort_tile - 1) / p.sort_tile;
  {
    TraceScope tr(TK_TILE_SORT_KEYS, st);
    if (p.merge_passes > 0 || !launch_small_sort(in, bufs[cur], n, dt, st))
      launch_tile_sort_keys(in, bufs[cur], n, dt, p.merge_passes == 0, (unsigned)tiles,
                            tma ? samp : nullptr, st);
  }
  int rc = launch_status("tile_sort_keys");
  int64_t run = p.sort_tile;
  for (int pass = 0; rc == NSORT_OK && pass < npass; ++pass) {
    const bool last = pass == npass - 1;
    const int dt_out = last ? dt : DT_U32;
    if (pass >= n2) {   // (passes alternate direction as below)
      launch_merge4(bufs[cur], bufs[cur ^ 1], n, run, samp,
                    reinterpret_cast<uint64_t *>(t + p.rec_off),
                    reinterpret_cast<int64_t *>(t + p.bnd_off), status, dt_out,
                    last ? nullptr : samp, (pass & 1) == 0, st);
      rc = launch_status("merge4_keys");
      run *= 4;
      cur ^= 1;
      continue;
    }
    if (tma) {
      // the partition reads the samples of this pass's input before the
      // merge overwrites them with the samples of its output
      // the tile sort writes low to high; passes then alternate direction
      launch_merge_tma<uint32_t>(bufs[cur], nullptr, bufs[cur ^ 1], nullptr, n, run, split,
                                 status, dt_out, samp, last ? nullptr : samp,
                                 (pass & 1) == 0, st);
    } else {
      {
        TraceScope tr(TK_PARTITION, st);
        launch_partition(bufs[cur], n, run, p, MERGE_TILE, split, st);
      }
      TraceScope tr(TK_MERGE_KEYS, st);
      launch_merge_keys(bufs[cur], bufs[cur ^ 1], n, run, split, dt_out,
                        (unsigned)p.num_merge_tiles, st);
    }
    rc = launch_status("merge_keys");
    run *= 2;
    cur ^= 1;
  }
  return rc;
}

// Stable pairs with payload word V.  64-bit payloads take no staged-load
// fallback: their outputs must be 16-byte aligned (the C ABI checks).
template <typename V>
static int sort_pairs_typed(const uint32_t *kin, const V *vin, uint32_t *kout, V *vout, int64_t n,
                            int dt, void *tmp, cudaStream_t st) {
  constexpr bool V64 = sizeof(V) == 8;
  int rc = ensure_pairs_smem_attr<V>();
  if (rc != NSORT_OK) return rc;
  const Plan p = make_plan(V64 ? NSORT_KIND_PAIRS64 : NSORT_KIND_PAIRS, (uint64_t)n);
  char *t = static_cast<char *>(tmp);
  uint32_t *kb[2] = {kout, p.merge_passes ? reinterpret_cast<uint32_t *>(t + p.keys_off) : nullptr};
  V *vb[2] = {vout, p.merge_passes ? reinterpret_cast<V *>(t + p.vals_off) : nullptr};
  int64_t *split = p.merge_passes ? reinterpret_cast<int64_t *>(t + p.split_off) : nullptr;
  int *status = p.merge_passes ? reinterpret_cast<int *>(t + p.status_off) : nullptr;
  uint32_t *samp = p.merge_passes ? reinterpret_cast<uint32_t *>(t + p.samp_off) : nullptr;
  if (status && cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
    return launch_status("cudaMemsetAsync");
  // the bulk-copy merge pass needs 16-byte aligned ping-pong buffers
  const bool tma = !((reinterpret_cast<uintptr_t>(kout) | reinterpret_cast<uintptr_t>(vout)) & 15);
  int cur = p.merge_passes % 2;
  const int64_t tiles = (n + p.sort_tile - 1) / p.sort_tile;
  {
    TraceScope tr(TK_TILE_SORT_PAIRS, st);
    launch_tile_sort_pairs<V>(kin, vin, kb[cur], vb[cur], n, dt, p.merge_passes == 0,
                              (unsigned)tiles, tma ? samp : nullptr, st);
  }
  rc = launch_status("tile_sort_pairs");
  for (int pass = 0; rc == NSORT_OK && pass < p.merge_passes; ++pass) {
    const int64_t run = (int64_t)p.sort_tile << pass;
    const int dt_out = pass == p.merge_passes - 1 ? dt : DT_U32;
    if (tma) {
      launch_merge_tma<V>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n, run, split, status,
                          dt_out, samp, pass == p.merge_passes - 1 ? nullptr : samp,
                          (pass & 1) == 0, st);
    } else if constexpr (!V64) {
      {
        TraceScope tr(TK_PARTITION, st);
        launch_partition(kb[cur], n, run, p, PMERGE_TILE, split, st);
      }
      TraceScope tr(TK_MERGE_PAIRS, st);
      launch_merge_pairs(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n, run, split, dt_out,
                         (unsigned)p.num_merge_tiles, st);
    } else {
      set_last_error("nsort_pairs64: outputs must be 16-byte aligned");
      return NSORT_EINVAL;
    }
    rc = launch_status("merge_pairs");
    cur ^= 1;
  }
  return rc;
}

int sort_pairs_impl(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                    int64_t n, int dt, void *tmp, cudaStream_t st) {
  return sort_pairs_typed<uint32_t>(kin, vin, kout, vout, n, dt, tmp, st);
}

int sort_pairs64_impl(const uint32_t *kin, const uint64_t *vin, uint32_t *kout, uint64_t *vout,
                      int64_t n, int dt, void *tmp, cudaStream_t st) {
  return sort_pairs_typed<uint64_t>(kin, vin, kout, vout, n, dt, tmp, st);
}

// ---- merging sorted runs of any lengths (the local merge of a sharded sort)
//
// A tree of two-way passes: pass 1 merges runs (0,1), (2,3), ...; each pass
// halves the number of runs (an odd last run is copied through as a merge
// with an empty partner).  Every pass is the persistent bulk-copy merge
// kernel with a table of the pass's run pairs (TableRuns); ties take the
// earlier run, so the merge is stable by run, then by position.  The first
// pass maps the bit patterns to order keys as they arrive and the last one
// maps them back.  Buffers ping-pong between the output and the scratch so
// that the last pass lands in the output.

size_t merge_runs_temp_bytes(bool pairs, uint64_t n, uint64_t nruns, int dtype) {
  if (nruns < 2) return 0;
  const bool wide = !pairs && dtype >= NSORT_U64;
  const size_t kw = wide ? 8 : 4;
  const int tile = pairs ? TMA_PMERGE_TILE : (wide ? TMA_K64_TILE : TMA_MERGE_TILE);
  const size_t tiles = (size_t)(n / (uint64_t)tile) + (size_t)nruns + 2;
  size_t total = 256;                                        // status word
  total += align_up((size_t)n * kw, 256);                    // ping-pong keys
  if (pairs) total += align_up((size_t)n * 4, 256);          // ping-pong values
  total += align_up(tiles * sizeof(int64_t), 256);           // splitters
  return total;
}

// Fills the run-pair table of one pass over runs with boundaries off[0..nr]
// and returns its number of tiles.
static int64_t fill_run_table(const int64_t *off, int nr, int tile, int dt_in, int dt_out,
                              TableRuns &tab) {
  tab.dt_in = dt_in;
  tab.dt_out = dt_out;
  tab.npairs = (nr + 1) / 2;
  int64_t tiles = 0;
  for (int p = 0; p < tab.npairs; ++p) {
    const int64_t a = off[2 * p];
    const int64_t m = off[2 * p + 1 < nr ? 2 * p + 1 : nr];
    const int64_t e = off[2 * p + 2 < nr ? 2 * p + 2 : nr];
    tab.pair0[p] = a;
    tab.la[p] = m - a;
    tab.lb[p] = e - m;
    tab.first_tile[p] = tiles;
    tiles += (e - a + tile - 1) / tile;
  }
  tab.first_tile[tab.npairs] = tiles;
  return tiles;
}

// Opts kernel fn (one per GEOM, K, PAIRS) in to its dynamic shared memory,
// once per device.
template <class GEOM, typename K, bool PAIRS>
static void table_merge_attrs(const void *fn, size_t smem) {
  static std::atomic<uint64_t> done_mask{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done_mask.load() & bit)) return;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  done_mask.fetch_or(bit);
}

// One pass over a table of run pairs: the partition (one splitter per tile,
// a full merge-path search each), then the persistent merge.
template <typename K, bool PAIRS>
static void launch_table_pass(const K *src, const uint32_t *vsrc, K *dst, uint32_t *vdst,
                              int64_t n, const TableRuns &tab, int64_t tiles, int64_t *split,
                              int *status, cudaStream_t st) {
  constexpr bool WIDE = sizeof(K) == 8;
  constexpr int NT = PAIRS ? TMA_PMERGE_NT : (WIDE ? TMA_K64_NT : TMA_MERGE_NT);
  constexpr int VT = PAIRS ? TMA_PMERGE_VT : (WIDE ? TMA_K64_VT : TMA_MERGE_VT);
  constexpr int TILE = NT * VT;
  // the uniform-run kernel's shared memory plus the shifted staging: 16
  // bytes per warp and output array
  constexpr size_t SMEM = (PAIRS ? TMA_PMERGE_SMEM : (WIDE ? TMA_K64_SMEM : TMA_MERGE_SMEM)) +
                          (size_t)(NT / 32) * 16 * (PAIRS ? 2 : 1);
  constexpr int DT0 = WIDE ? DT_U64 : DT_U32;   // unused: TableRuns maps at run time
  auto kernel = merge_tma_kernel<NT, VT, DT0, PAIRS, K, false, TableRuns>;
  table_merge_attrs<TableRuns, K, PAIRS>((const void *)kernel, SMEM);
  const unsigned grid = (unsigned)tma_merge_grid(tiles, PAIRS ? 1 : (WIDE ? 2 : 0));
  {
    TraceScope tr(TK_PARTITION, st);
    launch_pdl(partition_pairs_kernel<K, TableRuns>, (unsigned)((tiles + 255) / 256), 256, 0, st,
               src, tab, TILE, tiles, split);
  }
  TraceScope tr(PAIRS ? TK_MERGE_PAIRS : (WIDE ? TK_MERGE_KEYS64 : TK_MERGE_KEYS), st);
  K *no_samples = nullptr;
  launch_pdl(kernel, grid, NT, SMEM, st, src, vsrc, dst, vdst, n, tab, tiles,
             (const int64_t *)split, status, no_samples, 0);
}

template <typename K, bool PAIRS>
static int merge_runs_typed(const K *kin, const uint32_t *vin, K *kout, uint32_t *vout,
                            const int64_t *off, int nruns, int dt, void *tmp, cudaStream_t st) {
  constexpr bool WIDE = sizeof(K) == 8;
  constexpr int TILE = PAIRS ? TMA_PMERGE_TILE : (WIDE ? TMA_K64_TILE : TMA_MERGE_TILE);
  const int64_t n = off[nruns];
  int passes = 0;
  while ((1 << passes) < nruns) ++passes;
  if (passes == 0) {   // one run: already sorted
    if (n > 0 && kout != kin &&
        cudaMemcpyAsync(kout, kin, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return launch_status("cudaMemcpyAsync");
    if (PAIRS && n > 0 && vout != vin &&
        cudaMemcpyAsync(vout, vin, (size_t)n * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return launch_status("cudaMemcpyAsync");
    return NSORT_OK;
  }
  char *t = static_cast<char *>(tmp);
  int *status = reinterpret_cast<int *>(t);
  K *ktmp = reinterpret_cast<K *>(t + 256);
  const size_t kb = align_up((size_t)n * sizeof(K), 256);
  uint32_t *vtmp = PAIRS ? reinterpret_cast<uint32_t *>(t + 256 + kb) : nullptr;
  int64_t *split = reinterpret_cast<int64_t *>(t + 256 + kb + (PAIRS ? align_up((size_t)n * 4, 256) : 0));
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess)
    return launch_status("cudaMemsetAsync");
  int64_t cur_off[2 * MAX_TABLE_PAIRS + 1];
  int nr = nruns;
  for (int r = 0; r <= nr; ++r) cur_off[r] = off[r];
  const K *src = kin;
  const uint32_t *vsrc = vin;
  const int order = WIDE ? DT_U64 : DT_U32;   // order keys between passes
  int rc = NSORT_OK;
  for (int pass = 0; rc == NSORT_OK && pass < passes; ++pass) {
    const bool last = pass == passes - 1;
    const bool to_out = ((passes - 1 - pass) & 1) == 0;
    K *dst = to_out ? kout : ktmp;
    uint32_t *vdst = PAIRS ? (to_out ? vout : vtmp) : nullptr;
    TableRuns tab;
    const int64_t tiles = fill_run_table(cur_off, nr, TILE, pass == 0 ? dt : order,
                                         last ? dt : order, tab);
    if (tiles > 0)
      launch_table_pass<K, PAIRS>(src, vsrc, dst, vdst, n, tab, tiles, split, status, st);
    rc = launch_status("merge_shards");
    // the merged pairs are the next pass's runs
    int m = 0;
    for (int r = 0; r < nr; r += 2) cur_off[m++] = cur_off[r];
    cur_off[m] = cur_off[nr];
    nr = m;
    src = dst;
    vsrc = vdst;
  }
  return rc;
}

// ---- the merge levels of a segmented batch ------------------------------
//
// Level k merges, in every large segment with at least k merge levels, the
// runs of tile * 2^(k-1) keys pairwise (the level-0 runs are the segment's
// tile sorts).  Three launches per level: one thread per segment reserves
// its merge tiles and lists them as (segment, tile in the segment); one
// thread per listed tile computes the tile's geometry from its two
// merge-path splitters and writes it as a descriptor; the persistent
// bulk-copy merge kernel then runs over the descriptors (DescTiles).

int seg_merge_tile(bool pairs) { return pairs ? TMA_PMERGE_TILE : TMA_MERGE_TILE; }
size_t seg_tile_desc_bytes() { return sizeof(PairTile); }

__device__ __forceinline__ int ceil_log2_i64(int64_t x) {
  int p = 0;
  while ((int64_t(1) << p) < x) ++p;
  return p;
}

// Grid-stride over the segments; nothing to do (and an immediate return)
// when the offsets were malformed or no segment has k levels.
__global__ void seg_describe_kernel(const int64_t *__restrict__ off, int64_t nseg,
                                    int64_t min_len, int tile, int k, int mt,
                                    const int *status, const int *max_level,
                                    unsigned long long *count, int64_t *__restrict__ tile_seg) {
  pdl_wait();      // the previous kernel of the stream has finished writing
  if (*status != NSORT_OK || *max_level < k) return;
  const int64_t run = (int64_t)tile << (k - 1);
  const int64_t tpp = (2 * run + mt - 1) / mt;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nseg;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t L = off[s + 1] - off[s];
    if (L <= min_len || ceil_log2_i64((L + tile - 1) / tile) < k) continue;
    const int64_t full = L / (2 * run);
    const int64_t tiles = full * tpp + (L - full * 2 * run + mt - 1) / mt;
    const int64_t base = (int64_t)atomicAdd(count, (unsigned long long)tiles);
    for (int64_t j = 0; j < tiles; ++j) tile_seg[base + j] = (s << 32) | j;
  }
}

// Descriptor of merge tile (segment, tile in segment) = e of level k.
template <typename K>
__device__ __forceinline__ void seg_partition_tile(const int64_t *__restrict__ off, int tile,
                                                   int k, int mt, int64_t e, const K *buf0,
                                                   const K *buf1, PairTile *out) {
  const int64_t sid = e >> 32, j = e & 0xFFFFFFFFll;
  const int64_t o = off[sid];
  const int64_t L = off[sid + 1] - o;
  const int P = ceil_log2_i64((L + tile - 1) / tile);
  const int64_t run = (int64_t)tile << (k - 1);
  const int64_t tpp = (2 * run + mt - 1) / mt;
  const int64_t pair = j / tpp, jj = j - pair * tpp;
  const int64_t pair0 = pair * 2 * run;
  const int64_t la = L - pair0 < run ? L - pair0 : run;
  const int64_t rest = L - pair0 - run;
  const int64_t lb = rest <= 0 ? 0 : (rest < run ? rest : run);
  const int64_t d0 = jj * mt;
  const int64_t d1 = d0 + mt < la + lb ? d0 + mt : la + lb;
  const int in1 = (P - (k - 1)) & 1;   // level k-1 of this segment is in buf1
  const K *A = (in1 ? buf1 : buf0) + o + pair0;
  const K *B = A + la;
  int64_t a0 = merge_path_global(A, la, B, lb, d0);
  int64_t a1 = d1 == la + lb ? la : merge_path_global(A, la, B, lb, d1);
  clamp_coranks(la, lb, d0, d1, a0, a1);
  PairTile g;
  g.out0 = o + pair0 + d0;
  g.a_off = o + pair0 + a0;
  g.b_off = o + pair0 + la + (d0 - a0);
  g.na = (int)(a1 - a0);
  g.count = (int)(d1 - d0);
  g.nb = g.count - g.na;
  g.flags = in1 | (k == P ? 2 : 0);
  *out = g;
}

template <typename K>
__global__ void seg_partition_kernel(const int64_t *__restrict__ off, int tile, int k, int mt,
                                     const unsigned long long *count,
                                     const int64_t *__restrict__ tile_seg,
                                     const K *buf0, const K *buf1, PairTile *__restrict__ desc) {
  pdl_wait();      // the previous kernel of the stream has finished writing
  const int64_t ntiles = (int64_t)*count;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles;
       t += (int64_t)gridDim.x * blockDim.x)
    seg_partition_tile(off, tile, k, mt, tile_seg[t], buf0, buf1, desc + t);
}

template <bool PAIRS>
static void launch_seg_level_merge(const SegLevelArgs &a, cudaStream_t st) {
  using K = uint32_t;
  constexpr int NT = PAIRS ? TMA_PMERGE_NT : TMA_MERGE_NT;
  constexpr int VT = PAIRS ? TMA_PMERGE_VT : TMA_MERGE_VT;
  constexpr size_t SMEM = (PAIRS ? TMA_PMERGE_SMEM : TMA_MERGE_SMEM) +
                          (size_t)(NT / 32) * 16 * (PAIRS ? 2 : 1);   // shifted staging
  auto kernel = merge_tma_kernel<NT, VT, DT_U32, PAIRS, K, false, DescTiles<K>>;
  table_merge_attrs<DescTiles<K>, K, PAIRS>((const void *)kernel, SMEM);
  const unsigned grid = (unsigned)tma_merge_grid(a.max_tiles, PAIRS ? 1 : 0);
  DescTiles<K> geom;
  geom.desc = static_cast<const PairTile *>(a.desc);
  geom.count = a.count;
  geom.buf0 = a.kout;
  geom.buf1 = a.ktmp;
  geom.vbuf0 = a.vout;
  geom.vbuf1 = a.vtmp;
  geom.dt = a.dt;
  TraceScope tr(TK_SEG_MERGE, st);
  const int64_t *no_split = nullptr;
  K *no_samples = nullptr;
  launch_pdl(kernel, grid, NT, SMEM, st, (const K *)a.kout, (const uint32_t *)a.vout, a.ktmp,
             a.vtmp, a.n, geom, (int64_t)0, no_split, a.status, no_samples, 0);
}

int launch_segmented_level(const SegLevelArgs &a, cudaStream_t st) {
  const bool pairs = a.vout != nullptr;
  const int mt = seg_merge_tile(pairs);
  {
    TraceScope tr(TK_SEG_BIN, st);
    const int64_t blocks = (a.nseg + 255) / 256;
    launch_pdl(seg_describe_kernel, (unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st, a.off,
               a.nseg, a.min_len, a.tile, a.k, mt, (const int *)a.status, a.max_level, a.count,
               a.tile_seg);
  }
  {
    TraceScope tr(TK_PARTITION, st);
    const int64_t blocks = (a.max_tiles + 255) / 256;
    launch_pdl(seg_partition_kernel<uint32_t>, (unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st,
               a.off, a.tile, a.k, mt, (const unsigned long long *)a.count,
               (const int64_t *)a.tile_seg, (const uint32_t *)a.kout, (const uint32_t *)a.ktmp,
               static_cast<PairTile *>(a.desc));
  }
  if (pairs) launch_seg_level_merge<true>(a, st);
  else launch_seg_level_merge<false>(a, st);
  return launch_status("segmented merge level");
}

int merge_runs_impl(const void *kin, const uint32_t *vin, void *kout, uint32_t *vout,
                    const int64_t *off, int nruns, int dt, void *tmp, cudaStream_t st) {
  if (vin)
    return merge_runs_typed<uint32_t, true>(static_cast<const uint32_t *>(kin), vin,
                                            static_cast<uint32_t *>(kout), vout, off, nruns, dt,
                                            tmp, st);
  if (dt >= NSORT_U64)
    return merge_runs_typed<uint64_t, false>(static_cast<const uint64_t *>(kin), nullptr,
                                             static_cast<uint64_t *>(kout), nullptr, off, nruns,
                                             dt, tmp, st);
  return merge_runs_typed<uint32_t, false>(static_cast<const uint32_t *>(kin), nullptr,
                                           static_cast<uint32_t *>(kout), nullptr, off, nruns, dt,
                                           tmp, st);
}

}  // namespace nsort

// ---------------------------------------------------------------- C ABI

using namespace nsort;

static bool is_wide(int dtype) {
  return dtype == NSORT_U64 || dtype == NSORT_I64 || dtype == NSORT_F64;
}

extern "C" size_t nsort_temp_bytes(int kind, uint64_t n, uint64_t nseg, int dtype) {
  if (kind == NSORT_KIND_KEYS) return make_plan(kind, n, is_wide(dtype) ? dtype : 0).total;
  if (kind == NSORT_KIND_PAIRS || kind == NSORT_KIND_PAIRS64) return make_plan(kind, n).total;
  if (kind == NSORT_KIND_MERGE) return merge_runs_temp_bytes(false, n, nseg, dtype);
  if (kind == NSORT_KIND_MERGE_PAIRS) return merge_runs_temp_bytes(true, n, nseg, dtype);
  return segmented_temp_bytes(kind, n, nseg);
}

extern "C" int nsort_plan_dtype(int kind, uint64_t n, int dtype, int *passes, int *sort_tile,
                                int *merge_tile) {
  if (kind != NSORT_KIND_KEYS && kind != NSORT_KIND_PAIRS) return NSORT_EINVAL;
  if (n > MAX_KEYS) return NSORT_EINVAL;
  if (is_wide(dtype) && kind != NSORT_KIND_KEYS) return NSORT_EINVAL;
  const Plan p = make_plan(kind, n, is_wide(dtype) ? dtype : 0);
  if (passes) *passes = 1 + p.merge2_passes + p.merge4_passes;
  if (sort_tile) *sort_tile = p.sort_tile;
  if (merge_tile) *merge_tile = p.merge_tile;
  return NSORT_OK;
}

extern "C" uint64_t nsort_testing_set_four_way_min(uint64_t min_keys) {
  return g_four_way_min.exchange(min_keys);
}

extern "C" int nsort_merge_grid(int kind, int dtype) {
  if (kind != NSORT_KIND_KEYS && kind != NSORT_KIND_PAIRS) return 0;
  if (is_wide(dtype) && kind != NSORT_KIND_KEYS) return 0;
  const int which = kind == NSORT_KIND_PAIRS ? 1 : (is_wide(dtype) ? 2 : 0);
  const int g = tma_merge_grid(INT64_MAX, which);
  return cudaGetLastError() == cudaSuccess ? g : 0;
}

extern "C" int nsort_plan(int kind, uint64_t n, int *passes, int *sort_tile, int *merge_tile) {
  return nsort_plan_dtype(kind, n, NSORT_U32, passes, sort_tile, merge_tile);
}

static int check_common(const void *a, const void *b, uint64_t n, int dtype, void *tmp,
                        size_t tmp_bytes, int kind) {
  const bool wide = is_wide(dtype);
  if (dtype != NSORT_U32 && dtype != NSORT_I32 && dtype != NSORT_F32 && !wide)
    return NSORT_EINVAL;
  if (wide && kind != NSORT_KIND_KEYS) return NSORT_EINVAL;
  if (n > MAX_KEYS) return NSORT_EINVAL;
  if (n == 0) return NSORT_OK;
  if (!a || !b) return NSORT_EINVAL;
  if ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & (wide ? 7 : 3))
    return NSORT_EINVAL;
  const Plan p = make_plan(kind, n, wide ? dtype : 0);
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
  if (is_wide(dtype))
    return sort_keys64_impl(static_cast<const uint64_t *>(d_keys_in),
                            static_cast<uint64_t *>(d_keys_out), (int64_t)n, dtype, d_tmp,
                            static_cast<cudaStream_t>(stream));
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

extern "C" int nsort_merge_shards(const void *d_keys_in, const uint32_t *d_vals_in,
                                  void *d_keys_out, uint32_t *d_vals_out, const int64_t *h_run_off,
                                  int nruns, int dtype, void *d_tmp, size_t tmp_bytes,
                                  void *stream) {
  const bool pairs = d_vals_in != nullptr || d_vals_out != nullptr;
  const bool wide = is_wide(dtype);
  if (dtype < NSORT_U32 || dtype > NSORT_F64 || (pairs && wide)) return NSORT_EINVAL;
  if (!h_run_off || nruns < 1 || nruns > 2 * MAX_TABLE_PAIRS) return NSORT_EINVAL;
  if (h_run_off[0] != 0) return NSORT_EINVAL;
  for (int r = 0; r < nruns; ++r)
    if (h_run_off[r + 1] < h_run_off[r]) return NSORT_EINVAL;
  const int64_t n = h_run_off[nruns];
  if ((uint64_t)n > MAX_KEYS) return NSORT_EINVAL;
  if (n == 0) return NSORT_OK;
  if (!d_keys_in || !d_keys_out || (pairs && (!d_vals_in || !d_vals_out))) return NSORT_EINVAL;
  const uintptr_t bufs = reinterpret_cast<uintptr_t>(d_keys_in) |
                         reinterpret_cast<uintptr_t>(d_keys_out) |
                         reinterpret_cast<uintptr_t>(d_vals_in) |
                         reinterpret_cast<uintptr_t>(d_vals_out);
  if (bufs & 15) return NSORT_EINVAL;   // the passes stage their slices with bulk copies
  if (nruns > 1) {
    const size_t kw = wide ? 8 : 4;
    const char *ki = static_cast<const char *>(d_keys_in);
    const char *ko = static_cast<const char *>(d_keys_out);
    if (ki < ko + (size_t)n * kw && ko < ki + (size_t)n * kw) return NSORT_EINVAL;
    if (pairs) {
      const char *vi = reinterpret_cast<const char *>(d_vals_in);
      const char *vo = reinterpret_cast<const char *>(d_vals_out);
      if (vi < vo + (size_t)n * 4 && vo < vi + (size_t)n * 4) return NSORT_EINVAL;
    }
    const size_t need = merge_runs_temp_bytes(pairs, (uint64_t)n, (uint64_t)nruns, dtype);
    if (!d_tmp || tmp_bytes < need) return NSORT_ENOMEM;
    if (reinterpret_cast<uintptr_t>(d_tmp) & 255) return NSORT_EINVAL;
  }
  return merge_runs_impl(d_keys_in, d_vals_in, d_keys_out, d_vals_out, h_run_off, nruns, dtype,
                         d_tmp, static_cast<cudaStream_t>(stream));
}

extern "C" int nsort_pairs64(const void *d_keys_in, const uint64_t *d_vals_in, void *d_keys_out,
                             uint64_t *d_vals_out, uint64_t n, int dtype, void *d_tmp,
                             size_t tmp_bytes, void *stream) {
  int rc = check_common(d_keys_in, d_keys_out, n, dtype, d_tmp, tmp_bytes, NSORT_KIND_PAIRS64);
  if (rc != NSORT_OK || n == 0) return rc;
  if (!d_vals_in || !d_vals_out) return NSORT_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_vals_in) | reinterpret_cast<uintptr_t>(d_vals_out)) & 7)
    return NSORT_EINVAL;
  if ((reinterpret_cast<uintptr_t>(d_keys_out) | reinterpret_cast<uintptr_t>(d_vals_out)) & 15)
    return NSORT_EINVAL;
  return sort_pairs64_impl(static_cast<const uint32_t *>(d_keys_in), d_vals_in,
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
