// nsort_segmented: many independent arrays sorted in one batch.
//
// Segments are binned by length on the device:
//   tiny   L <= W_t          one thread sorts the segment in registers with
//                            the W_t-input network (W_t = 8 or 16);
//   small  L <= 32 * IPT     one warp: column sort of IPT keys per lane and
//                            the warp flip merger (IPT = 8 or 16);
//   medium L <= 16 NT        one CTA: tile sort with the active size rounded
//                            up to a power of two;
//   large  L >  16 NT        tile sorts of the segment's TILE-key tiles
//                            (level 0; keys take 32 per thread, TILE = 32 NT,
//                            pairs 16, TILE = 16 NT), then one merge level per
//                            doubling of the run length.
// A persistent kernel takes the level-0 tiles and the medium, small and tiny
// segments from a queue (one atomic counter):
// [level-0 tiles of all large segments][medium][small batches][tiny batches].
// The merge levels then run as the plain sort's bulk-copy merge passes over
// lists of merge tiles (launch_segmented_level): level k merges, in every
// segment with at least k levels, its runs of TILE * 2^(k-1) keys pairwise.
// Every step is stream-ordered, with no host synchronisation, so a batch can
// be captured into a CUDA graph: the host launches as many levels as the
// longest possible segment could need, and levels past the batch's longest
// segment find no tiles.
//
// The tunables (block size NT, tiny network width W_t, small-bin IPT, CTAs
// per SM) come from nsort_segmented_set_config, fed by the autotuner.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <type_traits>

#include "nsort.h"
#include "nsort_internal.h"
#include "sort_device.cuh"
#include "tma_device.cuh"

namespace nsort {
namespace seg {

constexpr int MAXLV = 40;          // merge levels a segment can need (2^40 keys / 4096)
constexpr int MIN_TILE = 256 * 16; // smallest tile over the configurations

struct Ctrl {
  int status;                          // NSORT_OK, NSORT_EINVAL (offsets), NSORT_ETIMEOUT
  int max_level;
  unsigned long long next_item;        // queue head
  unsigned long long n_tiny, n_small, n_medium;
  unsigned long long bucket_tiles[MAXLV + 1];   // tiles of large segments needing b levels
  unsigned long long bucket_base[MAXLV + 2];    // exclusive prefix of bucket_tiles
  unsigned long long q_medium, q_small, q_tiny, q_total;
  unsigned long long lvl_count[MAXLV + 2];      // merge tiles of level k (launch_segmented_level)
};

struct Params {
  const uint32_t *kin;
  uint32_t *kout;
  const uint32_t *vin;   // nullptr: keys only
  uint32_t *vout;
  uint32_t *ktmp;
  uint32_t *vtmp;
  const int64_t *off;
  int64_t nseg;
  int64_t n;
  Ctrl *ctrl;
  int *tiny_list;
  int *small_list;
  int *medium_list;
  int64_t *slot_base;    // large segment -> first slot of its tiles
  int *owner;            // slot -> large segment
  int dt;
  int tile;              // keys per level-0 tile: NT * 32 (keys) or NT * 16 (pairs)
  int mt;                // longest medium segment: NT * 16
  int nt;
  int tiny_w;            // 8 or 16
  int small_ipt;         // 8 or 16
};

__device__ __forceinline__ int ceil_log2(int64_t x) {
  int p = 0;
  while ((int64_t(1) << p) < x) ++p;
  return p;
}

// ---- set-up kernels ----------------------------------------------------------

__global__ void seg_classify_kernel(Params p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.nseg) return;
  const int64_t o0 = p.off[s], o1 = p.off[s + 1];
  const bool bad = o0 < 0 || o1 < o0 || o1 > p.n || (s == 0 && o0 != 0) ||
                   (s == p.nseg - 1 && o1 != p.n);
  if (bad) {
    atomicExch(&p.ctrl->status, (int)NSORT_EINVAL);
    return;
  }
  const int64_t L = o1 - o0;
  Ctrl *c = p.ctrl;
  if (L == 0) return;
  if (L <= p.tiny_w) {
    p.tiny_list[atomicAdd(&c->n_tiny, 1ull)] = (int)s;
  } else if (L <= 32 * p.small_ipt) {
    p.small_list[atomicAdd(&c->n_small, 1ull)] = (int)s;
  } else if (L <= p.mt) {
    p.medium_list[atomicAdd(&c->n_medium, 1ull)] = (int)s;
  } else {
    const int64_t T = (L + p.tile - 1) / p.tile;
    p.slot_base[s] = (int64_t)atomicAdd(&c->bucket_tiles[ceil_log2(T)], (unsigned long long)T);
  }
}

// Lays out the work queue (one thread).
__global__ void seg_plan_kernel(Params p) {
  Ctrl *c = p.ctrl;
  if (c->status != NSORT_OK) {
    c->q_total = 0;
    return;
  }
  unsigned long long base = 0;
  int maxlv = 0;
  for (int b = 0; b <= MAXLV; ++b) {
    c->bucket_base[b] = base;
    base += c->bucket_tiles[b];
    if (c->bucket_tiles[b]) maxlv = b;
  }
  c->bucket_base[MAXLV + 1] = base;
  c->q_medium = base;
  c->q_small = c->q_medium + c->n_medium;
  const unsigned long long warps = p.nt / 32;
  c->q_tiny = c->q_small + (c->n_small + warps - 1) / warps;
  c->q_total = c->q_tiny + (c->n_tiny + p.nt - 1) / p.nt;
  c->max_level = maxlv;
}

// One warp per segment: gives each large segment its global slot range and
// records the owner of every slot.
__global__ void seg_owner_kernel(Params p) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= p.nseg || p.ctrl->status != NSORT_OK) return;
  const int64_t L = p.off[w + 1] - p.off[w];
  if (L <= p.mt) return;
  const int64_t T = (L + p.tile - 1) / p.tile;
  const int64_t g = (int64_t)p.ctrl->bucket_base[ceil_log2(T)] + p.slot_base[w];
  __syncwarp();
  if (lane == 0) p.slot_base[w] = g;
  for (int64_t i = lane; i < T; i += 32) p.owner[g + i] = (int)w;
}

// ---- the persistent kernel ------------------------------------------------




template <typename K>
__device__ __forceinline__ K make_elem(uint32_t key, int pos) {
  if (sizeof(K) == 8) return (K)(((uint64_t)key << 32) | (uint32_t)pos);
  return (K)key;
}
template <typename K>
__device__ __forceinline__ uint32_t elem_key(K e) {
  return sizeof(K) == 8 ? (uint32_t)((uint64_t)e >> 32) : (uint32_t)e;
}
template <typename K>
__device__ __forceinline__ int elem_pos(K e) {
  return (int)((uint64_t)e & 0xFFFFu);
}

// Tile sort with an active size m (a power of two, 512 <= m <= NT*16): only
// the first m/16 threads hold data; all threads take part in the barriers.
// On return thread t (< m/16) holds sorted elements [16t, 16t + 16).
template <int NT, typename K>
__device__ __forceinline__ void sort_tile_dyn(K (&r)[16], K *s, int m) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int e0 = tid * 16;
  if (e0 < m) {   // whole warps: m is a multiple of 512
    column_sort16(r);
    warp_merge<16>(r, lane);
  }
  if (m == 512) return;
  if (e0 < m) {
#pragma unroll
    for (int k = 0; k < 16; ++k) s[pidx<K>(e0 + k)] = r[k];
  }
  int unused[16];
#pragma unroll 1
  for (int run = 512; run < m; run <<= 1) {
    __syncthreads();
    if (e0 < m) {
      const int g0 = e0 & ~(2 * run - 1);
      const int diag = e0 - g0;
      const int ai = merge_path_smem(s, g0, run, g0 + run, run, diag);
      serial_merge<16, false>(s, g0 + ai, g0 + run, g0 + run + diag - ai, g0 + 2 * run, r, unused);
    }
    if (2 * run < m) {
      __syncthreads();
      if (e0 < m) {
#pragma unroll
        for (int k = 0; k < 16; ++k) s[pidx<K>(e0 + k)] = r[k];
      }
    }
  }
}

// Sorts `count` elements of a segment starting at kin[base] with one CTA and
// active size m; stores them (mapped back when `final_map`) at kdst[base].
template <int NT, bool PAIRS>
__device__ void block_sort_range(const Params &p, void *smem, int64_t base, int count, int m,
                                 uint32_t *kdst, uint32_t *vdst, bool final_map) {
  using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
  K *s = static_cast<K *>(smem);
  const int tid = threadIdx.x;
  const int e0 = tid * 16;
  K r[16];
  if (e0 < m) {
    const int act = m / 16;     // active threads; loads are striped over them
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int e = tid + act * j;
      r[j] = e < count ? make_elem<K>(to_key(p.kin[base + e], p.dt), e) : (K)~(K)0;
    }
  }
  sort_tile_dyn<NT>(r, s, m);
  uint32_t vo[16];
  if (PAIRS && e0 < m) {
#pragma unroll
    for (int k = 0; k < 16; ++k) vo[k] = e0 + k < count ? p.vin[base + elem_pos(r[k])] : 0u;
  }
  const int dto = final_map ? p.dt : (int)DT_U32;
  // thread t holds sorted elements [16t, 16t + 16): staged in shared memory
  // (padded; keys, then values for pairs) so that the global stores are
  // coalesced whatever the segment's alignment
  uint32_t *sk = reinterpret_cast<uint32_t *>(smem);
  uint32_t *sv = sk + padded_len<uint32_t>(m);
  __syncthreads();   // s is no longer read; every value gathered (vdst may alias vin)
  if (e0 < m) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (e0 + k < count) {
        sk[pidx<uint32_t>(e0 + k)] = from_key(elem_key(r[k]), dto);
        if (PAIRS) sv[pidx<uint32_t>(e0 + k)] = vo[k];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < count; e += NT) {
    kdst[base + e] = sk[pidx<uint32_t>(e)];
    if (PAIRS) vdst[base + e] = sv[pidx<uint32_t>(e)];
  }
}

struct Best32Columns {
  template <typename K>
  __device__ __forceinline__ static void sort(K (&r)[32]) { column_sort_net<NET_BEST, 32>(r); }
};

// Level-0 tile of a large keys-only segment: `count` keys at kin[base],
// sorted with 32 keys per thread by the keys tile sort's code (the best
// 32-input network, the warp merge, gapped block merges); stored (mapped
// back when `final_map`) at kdst[base].
template <int NT>
__device__ void tile_sort32_range(const Params &p, void *smem, int64_t base, int count,
                                  uint32_t *kdst, bool final_map) {
  uint32_t *s = static_cast<uint32_t *>(smem);
  const int tid = threadIdx.x;
  uint32_t r[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int e = tid + NT * j;
    r[j] = e < count ? to_key(p.kin[base + e], p.dt) : 0xFFFFFFFFu;
  }
  sort_tile_in_block<NT, 32, Best32Columns, uint32_t, true>(r, s);
  const int dto = final_map ? p.dt : (int)DT_U32;
  // thread t holds tile elements [32t, 32t + 32): staged in shared memory
  // (padded, conflict-free both ways) so that the global stores are
  // coalesced whatever the segment's alignment
  const int e0 = tid * 32;
  __syncthreads();   // every thread is done reading s in the last merge level
#pragma unroll
  for (int k = 0; k < 32; ++k) s[pidx<uint32_t>(e0 + k)] = r[k];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int e = tid + NT * j;
    if (e < count) kdst[base + e] = from_key(s[pidx<uint32_t>(e)], dto);
  }
}

// One warp sorts one segment of at most 32*IPT elements.
template <int IPT, bool PAIRS>
__device__ void warp_sort_segment(const Params &p, int64_t sid) {
  using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
  const int lane = threadIdx.x & 31;
  const int64_t off = p.off[sid];
  const int L = (int)(p.off[sid + 1] - off);
  K r[IPT];
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const int e = lane + 32 * k;
    r[k] = e < L ? make_elem<K>(to_key(p.kin[off + e], p.dt), e) : (K)~(K)0;
  }
  column_sort(r);
  warp_merge<IPT>(r, lane);
  uint32_t vo[IPT];
  const int e0 = lane * IPT;
  if (PAIRS) {
#pragma unroll
    for (int k = 0; k < IPT; ++k) vo[k] = e0 + k < L ? p.vin[off + elem_pos(r[k])] : 0u;
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    if (e0 + k < L) {
      p.kout[off + e0 + k] = from_key(elem_key(r[k]), p.dt);
      if (PAIRS) p.vout[off + e0 + k] = vo[k];
    }
  }
}

// One thread sorts one segment of at most W elements.
template <int W, bool PAIRS>
__device__ void thread_sort_segment(const Params &p, int64_t sid) {
  using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
  const int64_t off = p.off[sid];
  const int L = (int)(p.off[sid + 1] - off);
  K r[W];
#pragma unroll
  for (int k = 0; k < W; ++k)
    r[k] = k < L ? make_elem<K>(to_key(p.kin[off + k], p.dt), k) : (K)~(K)0;
  column_sort(r);
  uint32_t vo[W];
  if (PAIRS) {
#pragma unroll
    for (int k = 0; k < W; ++k) vo[k] = k < L ? p.vin[off + elem_pos(r[k])] : 0u;
  }
#pragma unroll
  for (int k = 0; k < W; ++k) {
    if (k < L) {
      p.kout[off + k] = from_key(elem_key(r[k]), p.dt);
      if (PAIRS) p.vout[off + k] = vo[k];
    }
  }
}

template <int NT, bool PAIRS>
__global__ void __launch_bounds__(NT, PAIRS ? 1 : 2) seg_sort_kernel(Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long item_sh;
  // The queue's bin boundaries live in shared memory and are read per item:
  // held in registers for the whole loop they would cost the tile sorts
  // (at 2 CTAs of 512 threads, 64 registers a thread) registers they need.
  __shared__ unsigned long long q_sh[4];   // medium, small, tiny, total
  const int tid = threadIdx.x;
  Ctrl *c = p.ctrl;
  if (tid == 0) {
    q_sh[0] = c->q_medium;
    q_sh[1] = c->q_small;
    q_sh[2] = c->q_tiny;
    q_sh[3] = c->q_total;
  }
  for (;;) {
    if (tid == 0) item_sh = atomicAdd(&c->next_item, 1ull);
    __syncthreads();
    const unsigned long long item = item_sh;
    const unsigned long long q_medium = q_sh[0], q_small = q_sh[1], q_tiny = q_sh[2],
                             q_total = q_sh[3];
    __syncthreads();
    if (item >= q_total) break;
    if (item < q_medium) {
      // level 0: tile sort of one tile of a large segment (the whole sort,
      // key map included, when the segment fits one tile)
      const int sid = p.owner[item];
      const int64_t t = (int64_t)item - p.slot_base[sid];
      const int64_t off = p.off[sid];
      const int64_t L = p.off[sid + 1] - off;
      const int P = ceil_log2((L + p.tile - 1) / p.tile);
      const int64_t b0 = t * p.tile;
      const int count = (int)(L - b0 < p.tile ? L - b0 : p.tile);
      uint32_t *kd = (P & 1) ? p.ktmp : p.kout;
      uint32_t *vd = (P & 1) ? p.vtmp : p.vout;
      if (PAIRS) block_sort_range<NT, PAIRS>(p, smem_raw, off + b0, count, NT * 16, kd, vd, P == 0);
      else tile_sort32_range<NT>(p, smem_raw, off + b0, count, kd, P == 0);
    } else if (item < q_small) {
      const int sid = p.medium_list[item - q_medium];
      const int64_t off = p.off[sid];
      const int L = (int)(p.off[sid + 1] - off);
      int m = 512;
      while (m < L) m <<= 1;
      block_sort_range<NT, PAIRS>(p, smem_raw, off, L, m, p.kout, p.vout, true);
    } else if (item < q_tiny) {
      const unsigned long long idx = (item - q_small) * (NT / 32) + (tid >> 5);
      if (idx < c->n_small) {
        const int sid = p.small_list[idx];
        if (p.small_ipt == 8) warp_sort_segment<8, PAIRS>(p, sid);
        else warp_sort_segment<16, PAIRS>(p, sid);
      }
    } else {
      const unsigned long long idx = (item - q_tiny) * NT + tid;
      if (idx < c->n_tiny) {
        const int sid = p.tiny_list[idx];
        if (p.tiny_w == 8) thread_sort_segment<8, PAIRS>(p, sid);
        else thread_sort_segment<16, PAIRS>(p, sid);
      }
    }
  }
}

// ---- host side -------------------------------------------------------------

struct Layout {
  size_t ctrl, keys, vals, tiny, small, medium, slot, owner, tile_seg, desc, total;
  int64_t max_tiles;   // merge tiles one level can have
};

Layout layout(uint64_t n, uint64_t nseg, bool pairs) {
  Layout l{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  l.ctrl = take(sizeof(Ctrl));
  l.keys = take(n * 4);
  l.vals = pairs ? take(n * 4) : 0;
  l.tiny = take(nseg * 4);
  l.small = take(nseg * 4);
  l.medium = take(nseg * 4);
  l.slot = take(nseg * 8);
  l.owner = take((2 * (n / MIN_TILE) + 2) * 4);
  // a segment of L keys has at most L / merge tile + (pairs of runs) + 1
  // merge tiles in a level, and at most L / MIN_TILE / 2 + 1 pairs of runs
  l.max_tiles = (int64_t)(n / (uint64_t)seg_merge_tile(pairs) + n / MIN_TILE + 2 * nseg + 16);
  l.tile_seg = take((size_t)l.max_tiles * 8);
  l.desc = take((size_t)l.max_tiles * seg_tile_desc_bytes());
  l.total = o;
  return l;
}

std::mutex g_cfg_mu;
nsort_seg_config g_cfg = {512, 16, 16, 0};

template <int NT, bool PAIRS>
size_t smem_bytes() {
  using K = typename std::conditional<PAIRS, uint64_t, uint32_t>::type;
  const size_t tile_b = sizeof(K) * merge_smem_len<K>(NT * 16, 16);
  const size_t tile32_b = PAIRS ? 0 : sizeof(uint32_t) * block_smem_len<uint32_t>(NT, 32);
  return tile_b > tile32_b ? tile_b : tile32_b;
}

template <int NT, bool PAIRS>
int launch_sort(const Params &p, int blocks_per_sm, cudaStream_t st) {
  const size_t smem = smem_bytes<NT, PAIRS>();
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaFuncSetAttribute(seg_sort_kernel<NT, PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, seg_sort_kernel<NT, PAIRS>, NT, smem) !=
          cudaSuccess) {
    set_last_error(std::string("nsort_segmented set-up: ") + cudaGetErrorString(cudaGetLastError()));
    return NSORT_ECUDA;
  }
  if (occ < 1) occ = 1;
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
  TraceScope tr(TK_SEG_SORT, st);
  seg_sort_kernel<NT, PAIRS><<<sms * per_sm, NT, smem, st>>>(p);
  return NSORT_OK;
}

}  // namespace seg

size_t segmented_temp_bytes(int kind, uint64_t n, uint64_t nseg) {
  if (kind != NSORT_KIND_SEGMENTED && kind != NSORT_KIND_SEGMENTED_PAIRS) return 0;
  return seg::layout(n, nseg, kind == NSORT_KIND_SEGMENTED_PAIRS).total;
}

}  // namespace nsort

using namespace nsort;

extern "C" int nsort_segmented_set_config(const nsort_seg_config *cfg) {
  if (!cfg) return NSORT_EINVAL;
  if ((cfg->block_threads != 256 && cfg->block_threads != 512) ||
      (cfg->tiny_width != 8 && cfg->tiny_width != 16) ||
      (cfg->small_ipt != 8 && cfg->small_ipt != 16) || cfg->blocks_per_sm < 0)
    return NSORT_EINVAL;
  std::lock_guard<std::mutex> lk(seg::g_cfg_mu);
  seg::g_cfg = *cfg;
  return NSORT_OK;
}

extern "C" int nsort_segmented_get_config(nsort_seg_config *cfg) {
  if (!cfg) return NSORT_EINVAL;
  std::lock_guard<std::mutex> lk(seg::g_cfg_mu);
  *cfg = seg::g_cfg;
  return NSORT_OK;
}

namespace nsort {

int segmented_impl(const void *d_keys_in, void *d_keys_out, const uint32_t *d_vals_in,
                   uint32_t *d_vals_out, const int64_t *d_offsets, uint64_t nseg, uint64_t n,
                   int dtype, void *d_tmp, size_t tmp_bytes, void *stream, uint64_t max_seg_len) {
  if (dtype != NSORT_U32 && dtype != NSORT_I32 && dtype != NSORT_F32) return NSORT_EINVAL;
  if (n > MAX_KEYS || nseg >= (uint64_t(1) << 31)) return NSORT_EINVAL;
  if ((d_vals_in == nullptr) != (d_vals_out == nullptr)) return NSORT_EINVAL;
  if (nseg == 0) return n == 0 ? NSORT_OK : NSORT_EINVAL;
  if (!d_offsets || (n > 0 && (!d_keys_in || !d_keys_out))) return NSORT_EINVAL;
  const uintptr_t al = reinterpret_cast<uintptr_t>(d_keys_in) |
                       reinterpret_cast<uintptr_t>(d_keys_out) |
                       reinterpret_cast<uintptr_t>(d_vals_in) |
                       reinterpret_cast<uintptr_t>(d_vals_out);
  if ((al & 3) || (reinterpret_cast<uintptr_t>(d_offsets) & 7)) return NSORT_EINVAL;
  const bool pairs = d_vals_in != nullptr;
  const seg::Layout l = seg::layout(n, nseg, pairs);
  if (!d_tmp || tmp_bytes < l.total) return NSORT_ENOMEM;
  if (reinterpret_cast<uintptr_t>(d_tmp) & 255) return NSORT_EINVAL;
  nsort_seg_config cfg;
  {
    std::lock_guard<std::mutex> lk(seg::g_cfg_mu);
    cfg = seg::g_cfg;
  }
  char *t = static_cast<char *>(d_tmp);
  seg::Params p;
  p.kin = static_cast<const uint32_t *>(d_keys_in);
  p.kout = static_cast<uint32_t *>(d_keys_out);
  p.vin = d_vals_in;
  p.vout = d_vals_out;
  p.ktmp = reinterpret_cast<uint32_t *>(t + l.keys);
  p.vtmp = pairs ? reinterpret_cast<uint32_t *>(t + l.vals) : nullptr;
  p.off = d_offsets;
  p.nseg = (int64_t)nseg;
  p.n = (int64_t)n;
  p.ctrl = reinterpret_cast<seg::Ctrl *>(t + l.ctrl);
  p.tiny_list = reinterpret_cast<int *>(t + l.tiny);
  p.small_list = reinterpret_cast<int *>(t + l.small);
  p.medium_list = reinterpret_cast<int *>(t + l.medium);
  p.slot_base = reinterpret_cast<int64_t *>(t + l.slot);
  p.owner = reinterpret_cast<int *>(t + l.owner);
  p.dt = dtype;
  p.nt = cfg.block_threads;
  p.mt = cfg.block_threads * 16;
  p.tile = pairs ? p.mt : cfg.block_threads * 32;
  p.tiny_w = cfg.tiny_width;
  p.small_ipt = cfg.small_ipt;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(p.ctrl, 0, sizeof(seg::Ctrl), st) != cudaSuccess) {
    set_last_error(std::string("nsort_segmented: ") + cudaGetErrorString(cudaGetLastError()));
    return NSORT_ECUDA;
  }
  const unsigned cblocks = (unsigned)((nseg + 255) / 256);
  {
    TraceScope tr(TK_SEG_BIN, st);
    seg::seg_classify_kernel<<<cblocks, 256, 0, st>>>(p);
    seg::seg_plan_kernel<<<1, 1, 0, st>>>(p);
    seg::seg_owner_kernel<<<(unsigned)((nseg * 32 + 255) / 256), 256, 0, st>>>(p);
  }
  int rc;
  if (p.nt == 512) rc = pairs ? seg::launch_sort<512, true>(p, cfg.blocks_per_sm, st)
                              : seg::launch_sort<512, false>(p, cfg.blocks_per_sm, st);
  else rc = pairs ? seg::launch_sort<256, true>(p, cfg.blocks_per_sm, st)
                  : seg::launch_sort<256, false>(p, cfg.blocks_per_sm, st);
  if (rc != NSORT_OK) return rc;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("nsort_segmented: ") + cudaGetErrorString(e));
    return NSORT_ECUDA;
  }
  // the merge levels: as many as a segment of max_seg_len keys would need
  // (the host does not know the batch's longest segment; later levels find
  // no tiles)
  const uint64_t longest = max_seg_len < n ? max_seg_len : n;
  const int64_t tiles0 = ((int64_t)longest + p.tile - 1) / p.tile;
  int levels = 0;
  while ((int64_t(1) << levels) < tiles0) ++levels;
  SegLevelArgs a;
  a.off = d_offsets;
  a.nseg = (int64_t)nseg;
  a.n = (int64_t)n;
  a.min_len = p.mt;
  a.tile = p.tile;
  a.dt = dtype;
  a.kout = p.kout;
  a.ktmp = p.ktmp;
  a.vout = pairs ? p.vout : nullptr;
  a.vtmp = pairs ? p.vtmp : nullptr;
  a.status = &p.ctrl->status;
  a.max_level = &p.ctrl->max_level;
  a.tile_seg = reinterpret_cast<int64_t *>(t + l.tile_seg);
  a.desc = t + l.desc;
  a.max_tiles = l.max_tiles;
  for (int k = 1; k <= levels && k <= seg::MAXLV; ++k) {
    a.k = k;
    a.count = &p.ctrl->lvl_count[k];
    rc = launch_segmented_level(a, st);
    if (rc != NSORT_OK) return rc;
  }
  return NSORT_OK;
}

}  // namespace nsort

extern "C" int nsort_segmented(const void *d_keys_in, void *d_keys_out, const uint32_t *d_vals_in,
                               uint32_t *d_vals_out, const int64_t *d_offsets, uint64_t nseg,
                               uint64_t n, int dtype, void *d_tmp, size_t tmp_bytes,
                               void *stream) {
  return segmented_impl(d_keys_in, d_keys_out, d_vals_in, d_vals_out, d_offsets, nseg, n, dtype,
                        d_tmp, tmp_bytes, stream, n);
}

