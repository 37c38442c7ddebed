// Device building blocks of the NEON-MS sort on sm_103a.
//
// The paper's three merge levels (Sec. 2.1, Fig. 1) become thread / warp /
// block / grid levels here:
//   column sort   (Sec. 2.3)  16 or 32 keys in one thread's registers; each
//                             16-key column is sorted by the 60-comparator
//                             16-input network (two columns are then merged
//                             in registers: 185 comparators for 32 keys);
//   row merge     (Sec. 2.4)  the 32 sorted runs of a warp are merged by
//                             flip ("asymmetric") bitonic merging networks:
//                             stages whose comparators span lanes use warp
//                             shuffles (the vectorised part), the stages
//                             inside a thread's run run in registers (the
//                             serial tail of the hybrid merger);
//   vectorised / parallel merge (Sec. 2.1, last paragraph) merge path: each
//                             thread finds its share of a merge by a binary
//                             search on the cross diagonal and runs a
//                             branch-free serial merge of it.
// Keys travel as unsigned integers after an order-preserving map (to_key);
// pair sorts use 64-bit composites (key << 32 | position) in the networks,
// which makes every composite distinct and the result stable.
#pragma once

#include <cstdint>

#include "networks_device.cuh"

namespace nsort {

enum { DT_U32 = 0, DT_I32 = 1, DT_F32 = 2, DT_U64 = 3, DT_I64 = 4, DT_F64 = 5 };

// Order-preserving map of a 32-bit pattern to an unsigned key.
//  u32: identity.  i32: flip the sign bit.  f32: negatives (sign set) are
//  complemented, non-negatives get the sign bit set — IEEE totalOrder.
__device__ __forceinline__ uint32_t to_key(uint32_t b, int dt) {
  uint32_t m = 0u;
  if (dt == DT_I32) m = 0x80000000u;
  if (dt == DT_F32) m = (uint32_t)((int32_t)b >> 31) | 0x80000000u;
  return b ^ m;
}

// Inverse of to_key.
__device__ __forceinline__ uint32_t from_key(uint32_t k, int dt) {
  uint32_t m = 0u;
  if (dt == DT_I32) m = 0x80000000u;
  if (dt == DT_F32) m = (uint32_t)((int32_t)~k >> 31) | 0x80000000u;
  return k ^ m;
}

// The same maps on 64-bit patterns (u64, i64, binary64 totalOrder).
__device__ __forceinline__ uint64_t to_key(uint64_t b, int dt) {
  uint64_t m = 0ull;
  if (dt == DT_I64) m = 0x8000000000000000ull;
  if (dt == DT_F64) m = (uint64_t)((int64_t)b >> 63) | 0x8000000000000000ull;
  return b ^ m;
}

__device__ __forceinline__ uint64_t from_key(uint64_t k, int dt) {
  uint64_t m = 0ull;
  if (dt == DT_I64) m = 0x8000000000000000ull;
  if (dt == DT_F64) m = (uint64_t)((int64_t)~k >> 63) | 0x8000000000000000ull;
  return k ^ m;
}

// Shared-memory index with one pad word per 32 (u32) or per 16 (u64)
// elements: a thread writing 16 consecutive elements and a warp reading
// consecutive elements are both free of bank conflicts.
template <typename K> struct Pad;
template <> struct Pad<uint32_t> { static constexpr int SHIFT = 5; };
template <> struct Pad<uint64_t> { static constexpr int SHIFT = 4; };
template <typename K>
__device__ __forceinline__ int pidx(int e) { return e + (e >> Pad<K>::SHIFT); }
template <typename K>
__host__ __device__ constexpr int padded_len(int tile) { return tile + (tile >> Pad<K>::SHIFT) + 2; }
// Shared-memory length for a tile that serial merges of VT outputs read
// without clamping their indices: they may look up to VT + 1 elements past
// the end of the tile.
template <typename K>
__host__ __device__ constexpr int merge_smem_len(int tile, int vt) {
  return padded_len<K>(tile + vt + 2);
}

// ---- compare-exchange --------------------------------------------------
__device__ __forceinline__ uint32_t kmin(uint32_t a, uint32_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t kmax(uint32_t a, uint32_t b) { return a < b ? b : a; }
__device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t kmax(uint64_t a, uint64_t b) { return a < b ? b : a; }

template <typename K>
__device__ __forceinline__ void ce(K &a, K &b) {
  const K lo = kmin(a, b);
  b = kmax(a, b);
  a = lo;
}

// ---- column sort (Sec. 2.3, Table 1) -------------------------------------
// Runs the network of the given family and width (networks_device.cuh) on
// the thread's W registers.  The comparator list is a compile-time constant
// and the loop is fully unrolled, so every index is a constant.
template <int FAMILY, int W, typename K>
__device__ __forceinline__ void column_sort_net(K (&r)[W]) {
  constexpr CmpList net = make_network(FAMILY, W);
  static_assert(net.n > 0, "no network of this family and width");
#pragma unroll
  for (int c = 0; c < net.n; ++c) ce(r[net.lo[c]], r[net.hi[c]]);
}

// The production column sort: M. W. Green's 60-comparator, depth-10
// network (the "best" 16-input network of Table 1).
template <typename K>
__device__ __forceinline__ void column_sort16(K (&r)[16]) {
  column_sort_net<NET_BEST, 16>(r);
}

// ---- warp-level flip merging network (Sec. 2.4) -------------------------
__device__ __forceinline__ uint32_t shfl_x(uint32_t v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}
__device__ __forceinline__ uint64_t shfl_x(uint64_t v, int m) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
  return ((uint64_t)hi << 32) | lo;
}
template <typename K>
__device__ __forceinline__ K keep(bool lower, K mine, K other) {
  return lower ? kmin(mine, other) : kmax(mine, other);
}

// 8 keys per thread: Batcher's odd-even merge sort, 19 comparators in 6
// layers, which is also the fewest possible for n = 8 (Table 1, n = 8).
template <typename K>
__device__ __forceinline__ void column_sort8(K (&r)[8]) {
  column_sort_net<NET_ODDEVEN, 8>(r);
}

template <typename K>
__device__ __forceinline__ void column_sort(K (&r)[16]) { column_sort16(r); }
template <typename K>
__device__ __forceinline__ void column_sort(K (&r)[8]) { column_sort8(r); }

// In-thread half-cleaners at distances IPT/2, ..., 1: sorts each thread's
// IPT registers once they form a bitonic sequence (the serial tail).
template <int IPT, typename K>
__device__ __forceinline__ void thread_tail(K (&r)[IPT]) {
#pragma unroll
  for (int d = IPT / 2; d >= 1; d >>= 1) {
#pragma unroll
    for (int i = 0; i < IPT; ++i)
      if (!(i & d)) ce(r[i], r[i + d]);
  }
}

// Lane l holds a sorted run of IPT in r[] (warp element IPT*l + k).  One
// level J of the warp merge merges the sorted runs held by groups of
// 2^(J-1) lanes pairwise: a flip stage (element p against element 2m-1-p of
// the 2m-element group: lane l ^ (2^J - 1), register IPT-1-k), half-cleaner
// stages across lanes at lane distances 2^(J-2)..1, then the in-thread
// tail.  In each cross-lane comparator the lower lane keeps the minimum and
// the upper lane the maximum.
template <int J, int IPT, typename K>
__device__ __forceinline__ void warp_merge_level(K (&r)[IPT], int lane) {
  constexpr int span = 1 << J;
  const bool lower = !(lane & (span >> 1));
#pragma unroll
  for (int k = 0; k < IPT / 2; ++k) {
    const K from_hi = shfl_x(r[IPT - 1 - k], span - 1);   // partner's mirror of r[k]
    const K from_lo = shfl_x(r[k], span - 1);             // partner's mirror of r[IPT-1-k]
    r[k] = keep(lower, r[k], from_hi);
    r[IPT - 1 - k] = keep(lower, r[IPT - 1 - k], from_lo);
  }
#pragma unroll
  for (int d = span >> 2; d >= 1; d >>= 1) {
    const bool lo2 = !(lane & d);
#pragma unroll
    for (int k = 0; k < IPT; ++k) r[k] = keep(lo2, r[k], shfl_x(r[k], d));
  }
  thread_tail<IPT>(r);
}

// Transposes a warp's 32 x 32 block of keys through t (32 rows of 33: the
// padding keeps both the row writes and the column reads free of bank
// conflicts): lane l's r[k] becomes lane k's r[l].  Its own inverse.
template <typename K>
__device__ __forceinline__ void warp_transpose32(K (&r)[32], K *t, int lane) {
  __syncwarp();   // every lane is done reading t
#pragma unroll
  for (int k = 0; k < 32; ++k) t[lane * 33 + k] = r[k];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 32; ++k) r[k] = t[k * 33 + lane];
}

// warp_merge_level for 32 keys per thread done on the transposed block:
// after the transpose, element 32 l + k of the warp sits in lane k,
// register l, so a group of 2^J lanes (the run pair this level merges) is
// the 2^J registers [g 2^J, (g+1) 2^J) of every lane.  Instead of the flip
// stage the second run of each pair is reversed (register l and its mirror
// within that half swap between lanes k and 31 - k, one shuffle for every
// two keys), which makes each pair a bitonic sequence; the J half-cleaner
// stages (lane distances 2^(J-1) .. 1 before the transpose) are then
// in-thread compare-exchanges of registers l and l + d, the lower keeping
// the minimum.  A second transpose restores the lane-major runs for the
// in-thread tail (distances 16 .. 1).  Per key and level: J shuffle stages
// (a shuffle and two integer instructions each: the lane decides min or
// max) become half a shuffle and J in-thread stages (one instruction each),
// for four shared-memory accesses.
template <int J, typename K>
__device__ __forceinline__ void warp_merge_level_t(K (&r)[32], int lane, K *t) {
  constexpr int G = 1 << J;    // registers per run pair after the transpose
  constexpr int H = G >> 1;
  warp_transpose32(r, t, lane);
  // reverse the second run of every pair: its registers l and m, mirrors
  // within that half, each take the other's key from lane 31 - lane
  static_assert(H % 2 == 0, "mirror registers pair up");
#pragma unroll
  for (int g = 0; g < 32 / G; ++g) {
#pragma unroll
    for (int i = 0; i < H / 2; ++i) {
      const int l = g * G + H + i, m = g * G + G - 1 - i;
      const K to_l = shfl_x(r[m], 31);
      const K to_m = shfl_x(r[l], 31);
      r[l] = to_l;
      r[m] = to_m;
    }
  }
#pragma unroll
  for (int d = H; d >= 1; d >>= 1) {
#pragma unroll
    for (int l = 0; l < 32; ++l)
      if (!(l & d)) ce(r[l], r[l + d]);
  }
  warp_transpose32(r, t, lane);
  thread_tail<32>(r);
}

// The same for 16 keys per thread (64-bit words: the pairs' composites and
// 64-bit keys), within each half-warp: lane 16h + l's r[k] becomes lane
// 16h + k's r[l], through 256 words of t per half-warp.  An XOR swizzle
// (row l, column k at 16 l + (k ^ l)) instead of padding keeps the row
// writes and the column reads free of bank conflicts in the same space.
template <typename K>
__device__ __forceinline__ void halfwarp_transpose16(K (&r)[16], K *t, int lane) {
  K *b = t + (lane >> 4) * 256;
  const int l = lane & 15;
  __syncwarp();   // every lane is done reading t
#pragma unroll
  for (int k = 0; k < 16; ++k) b[16 * l + (k ^ l)] = r[k];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; ++k) r[k] = b[16 * k + (l ^ k)];
}

// warp_merge_level_t for 16 keys per thread, levels 2-4 (run pairs within
// a half-warp): after the half-warp transpose a run pair is 2^J registers
// of the half-warp's 16 lanes; the second run is reversed (mirror
// registers swap between lanes k and 15 - k) and every half-cleaner is
// in-thread, then the transpose back and the in-thread tail.
template <int J, typename K>
__device__ __forceinline__ void warp_merge_level16_t(K (&r)[16], int lane, K *t) {
  constexpr int G = 1 << J;
  constexpr int H = G >> 1;
  static_assert(J >= 2 && J <= 4, "run pairs within a half-warp");
  halfwarp_transpose16(r, t, lane);
#pragma unroll
  for (int g = 0; g < 16 / G; ++g) {
#pragma unroll
    for (int i = 0; i < H / 2; ++i) {
      const int l = g * G + H + i, m = g * G + G - 1 - i;
      const K to_l = shfl_x(r[m], 15);
      const K to_m = shfl_x(r[l], 15);
      r[l] = to_l;
      r[m] = to_m;
    }
  }
#pragma unroll
  for (int d = H; d >= 1; d >>= 1) {
#pragma unroll
    for (int l = 0; l < 16; ++l)
      if (!(l & d)) ce(r[l], r[l + d]);
  }
  halfwarp_transpose16(r, t, lane);
  thread_tail<16>(r);
}

// Level 5 for 16 keys per thread: the flip stage across the two half-warps
// by shuffles, then the half-cleaners at lane distances 8 .. 1 in-thread on
// the half-warp transposes, then the in-thread tail.
template <typename K>
__device__ __forceinline__ void warp_merge_level16_5t(K (&r)[16], int lane, K *t) {
  const bool lower = !(lane & 16);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const K from_hi = shfl_x(r[15 - k], 31);
    const K from_lo = shfl_x(r[k], 31);
    r[k] = keep(lower, r[k], from_hi);
    r[15 - k] = keep(lower, r[15 - k], from_lo);
  }
  halfwarp_transpose16(r, t, lane);
#pragma unroll
  for (int d = 8; d >= 1; d >>= 1) {
#pragma unroll
    for (int l = 0; l < 16; ++l)
      if (!(l & d)) ce(r[l], r[l + d]);
  }
  halfwarp_transpose16(r, t, lane);
  thread_tail<16>(r);
}

// The five levels merge the warp's 32 runs into one sorted run of 32*IPT.
// With levels < 5 only the first levels levels run: the warp then holds
// sorted runs of IPT * 2^levels.
template <int IPT, typename K>
__device__ __forceinline__ void warp_merge(K (&r)[IPT], int lane, int levels = 5) {
  if (levels >= 1) warp_merge_level<1>(r, lane);
  if (levels >= 2) warp_merge_level<2>(r, lane);
  if (levels >= 3) warp_merge_level<3>(r, lane);
  if (levels >= 4) warp_merge_level<4>(r, lane);
  if (levels >= 5) warp_merge_level<5>(r, lane);
}

// ---- merge path (Sec. 2.1: load-balanced partitioning) -------------------
// Number of elements of A among the first `diag` outputs of the stable
// merge of A[0, na) and B[0, nb) (A wins ties).  Shared-memory runs at
// element offsets a0 / b0 in the padded layout.
template <typename K>
__device__ __forceinline__ int merge_path_smem(const K *s, int a0, int na, int b0, int nb,
                                               int diag) {
  int lo = diag - nb > 0 ? diag - nb : 0;
  int hi = diag < na ? diag : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s[pidx<K>(a0 + mid)] <= s[pidx<K>(b0 + diag - 1 - mid)]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Same search on global memory, one thread (64-bit lengths).
template <typename K>
__device__ __forceinline__ int64_t merge_path_global(const K *A, int64_t na, const K *B, int64_t nb,
                                                     int64_t diag) {
  int64_t lo = diag - nb > 0 ? diag - nb : 0;
  int64_t hi = diag < na ? diag : na;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(A + mid) <= __ldg(B + (diag - 1 - mid))) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Same search on global memory, by a whole warp: each round the 32 lanes
// test 32 evenly spaced candidates at once, which shrinks the interval by a
// factor of about 33 (6 rounds of loads for a 2^27-long run instead of 27
// dependent loads).  All lanes must call it with the same arguments; all get
// the result.
// COHERENT loads bypass L1 (ld.global.cg), for data written earlier in the
// same launch by other CTAs; otherwise the read-only path is used.
template <bool COHERENT>
__device__ __forceinline__ uint32_t load_key(const uint32_t *p) {
  return COHERENT ? __ldcg(p) : __ldg(p);
}

template <bool COHERENT = false>
__device__ __forceinline__ int64_t merge_path_global_warp(const uint32_t *A, int64_t na,
                                                          const uint32_t *B, int64_t nb,
                                                          int64_t diag, int lane) {
  int64_t lo = diag - nb > 0 ? diag - nb : 0;
  int64_t hi = diag < na ? diag : na;
  while (lo < hi) {                                  // answer in [lo, hi]
    const int64_t step = (hi - lo + 32) / 33;        // >= 1
    const int64_t q = lo + (int64_t)(lane + 1) * step - 1;
    bool p = false;                                  // p: A[q] goes before the diagonal
    if (q < hi) p = load_key<COHERENT>(A + q) <= load_key<COHERENT>(B + (diag - 1 - q));
    const int c = __popc(__ballot_sync(0xffffffffu, p));   // true probes form a prefix
    int64_t nhi = hi;
    if (c < 32) {
      const int64_t qc = lo + (int64_t)(c + 1) * step - 1;
      if (qc < hi) nhi = qc;
    }
    lo = lo + (int64_t)c * step;
    hi = nhi;
  }
  return lo;
}

// The same search by a group of W lanes of one warp (W a power of two;
// glane = lane within the group, gmask = the group's lanes), on keys of any
// word size: each round the W lanes test W evenly spaced candidates, which
// shrinks the interval by a factor of about W + 1.  All lanes of the group
// must call it with the same arguments; all get the result.
template <int W, typename K>
__device__ __forceinline__ int64_t merge_path_global_group(const K *A, int64_t na, const K *B,
                                                           int64_t nb, int64_t diag, int glane,
                                                           unsigned gmask) {
  int64_t lo = diag - nb > 0 ? diag - nb : 0;
  int64_t hi = diag < na ? diag : na;
  while (lo < hi) {                                  // answer in [lo, hi]
    const int64_t step = (hi - lo + W) / (W + 1);    // >= 1
    const int64_t q = lo + (int64_t)(glane + 1) * step - 1;
    bool p = false;                                  // p: A[q] goes before the diagonal
    if (q < hi) p = __ldg(A + q) <= __ldg(B + (diag - 1 - q));
    const int c = __popc(__ballot_sync(gmask, p) & gmask);   // true probes form a prefix
    int64_t nhi = hi;
    if (c < W) {
      const int64_t qc = lo + (int64_t)(c + 1) * step - 1;
      if (qc < hi) nhi = qc;
    }
    lo = lo + (int64_t)c * step;
    hi = nhi;
  }
  return lo;
}

// Merge path on unpadded shared memory: A and B are separate contiguous
// runs (the merge pass stages them with bulk copies, which cannot pad).
template <typename K>
__device__ __forceinline__ int merge_path_plain(const K *s, int a0, int na, int b0, int nb,
                                                int diag) {
  int lo = diag - nb > 0 ? diag - nb : 0;
  int hi = diag < na ? diag : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s[a0 + mid] <= s[b0 + diag - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Serial merge on unpadded shared memory (indices into s): VT outputs of the
// stable merge of s[a, a_end) and s[b, b_end) (A first on ties).  Reads at
// most VT + 1 elements past the larger end.  With TRACK, src[k] receives
// the index in s that output k came from.
template <int VT, bool TRACK = false, typename K = uint32_t>
__device__ __forceinline__ void serial_merge_plain(const K *s, int a, int a_end, int b,
                                                   int b_end, K (&out)[VT],
                                                   int (&src)[VT]) {
  K ka = s[a];
  K kb = s[b];
#pragma unroll
  for (int k = 0; k < VT; ++k) {
    const bool take_a = (b >= b_end) || (a < a_end && ka <= kb);
    out[k] = take_a ? ka : kb;
    if (TRACK) src[k] = take_a ? a : b;
    const int nx = (take_a ? a : b) + 1;
    const K kn = s[nx];
    a = take_a ? nx : a;
    b = take_a ? b : nx;
    ka = take_a ? kn : ka;
    kb = take_a ? kb : kn;
  }
}

// Keys-only serial merge without bounds checks: both runs must be followed
// in shared memory by at least VT copies of the largest key (all ones).
// Once a run is exhausted its head reads as the largest key, so the other
// run is taken; when both heads are the largest key, either may be output —
// keys only, so equal keys are the same bits and the outputs are exact.
// The loop keeps the head and index of the run whose head is smaller (lo)
// and of the other run (hi): each output is lo's head; lo's next key is
// compared with hi's head once, and four selects set the new (lo, hi).
// That is one compare and four selects per output, against one compare and
// seven selects and adds when the two runs keep fixed roles.
template <int VT, typename K>
__device__ __forceinline__ void serial_merge_sentinel(const K *s, int a, int b, K (&out)[VT]) {
  K ka = s[a];
  K kb = s[b];
  const bool t0 = ka <= kb;
  K hlo = t0 ? ka : kb, hhi = t0 ? kb : ka;
  int ilo = t0 ? a : b, ihi = t0 ? b : a;
#pragma unroll
  for (int k = 0; k < VT; ++k) {
    out[k] = hlo;
    const int i = ilo + 1;
    const K kn = s[i];
    const bool p = kn <= hhi;
    hlo = p ? kn : hhi;
    ilo = p ? i : ihi;
    hhi = p ? hhi : kn;
    ihi = p ? ihi : i;
  }
}

// ---- serial merge (the serial half of the hybrid merger) ----------------
// Produces VT outputs of the stable merge of s[a, a_end) and s[b, b_end)
// (element indices, padded layout) into out[].  Branch-free: one compare,
// selects and one shared load per output.  A thread whose range runs past
// the end of both runs keeps going (its extra outputs are discarded by the
// caller); it then reads at most VT + 1 elements past the larger end, which
// the buffer must hold (merge_smem_len).  src[k] receives the element index
// each output came from when TRACK is set.
template <int VT, bool TRACK, typename K>
__device__ __forceinline__ void serial_merge(const K *s, int a, int a_end, int b, int b_end,
                                             K (&out)[VT], int (&src)[VT]) {
  K ka = s[pidx<K>(a)];
  K kb = s[pidx<K>(b)];
#pragma unroll
  for (int k = 0; k < VT; ++k) {
    const bool take_a = (b >= b_end) || (a < a_end && ka <= kb);
    out[k] = take_a ? ka : kb;
    if (TRACK) src[k] = take_a ? a : b;
    const K kn = s[pidx<K>((take_a ? a : b) + 1)];
    ka = take_a ? kn : ka;
    kb = take_a ? kb : kn;
    a += take_a;
    b += !take_a;
  }
}

// ---- block sort (Sec. 2.1: in-register sort, then vectorized merges) -----
// The 16-input column sort as a policy of the block sort; other policies
// (other networks, other numbers of keys per thread) are plugged in by the
// network ablation.
struct Green16Columns {
  template <typename K>
  __device__ __forceinline__ static void sort(K (&r)[16]) { column_sort16(r); }
};

// Shared-memory layout of the block merges: the tile's runs of R elements
// lie back to back, each followed by a gap of IPT + 1 largest keys, in the
// padded index space (pidx).  The gaps let the serial merge run without
// bounds checks: once a run is used up its head reads as the largest key, so
// the other run is taken, and a thread's IPT outputs can read at most IPT
// elements past a run's end.  Valid for keys only and for the pairs'
// distinct (key, position) composites: a largest key taken from a gap
// instead of a real one has the same bits, and no composite is all ones.
// The gap is IPT + 1 rounded up to whole pad blocks (32 elements for 32-bit
// keys, 16 for 64-bit ones), so that every run, and every thread's IPT
// outputs, start at a multiple of IPT within a pad block: a thread's outputs
// then sit at consecutive padded indices.
template <typename K>
__host__ __device__ constexpr int block_gap(int ipt) {
  return (ipt + 1 + (1 << Pad<K>::SHIFT) - 1) >> Pad<K>::SHIFT << Pad<K>::SHIFT;
}

// Elements of the block merges' buffer: the tile and one gap per run of the
// first level (runs of 32 IPT), padded.
template <typename K>
__host__ __device__ constexpr int block_smem_len(int nt, int ipt) {
  return padded_len<K>(nt * ipt + (nt / 32) * block_gap<K>(ipt));
}

// Thread t's IPT consecutive outputs [e0, e0 + IPT), part of a run of R
// (a multiple of the warp's 32 IPT outputs), into the gapped layout; the
// warp whose outputs end a run fills that run's gap, a slot or two a lane.
template <int IPT, typename K>
__device__ __forceinline__ void stage_gapped(const K (&r)[IPT], K *s, int e0, int run) {
  constexpr int GAP = block_gap<K>(IPT);
  static_assert(((1 << Pad<K>::SHIFT) % IPT) == 0, "a thread's outputs stay in one pad block");
  const int base = e0 + (e0 / run) * GAP;
  const int pb = pidx<K>(base);   // base's pad block holds all IPT outputs
#pragma unroll
  for (int k = 0; k < IPT; ++k) s[pb + k] = r[k];
  const int lane = threadIdx.x & 31;
  const int wend = e0 + (32 - lane) * IPT;   // end of the warp's outputs (same in every lane)
  if (wend % run == 0) {
    const int gap0 = wend + (wend / run - 1) * GAP;   // first slot behind the run
    for (int j = lane; j < GAP; j += 32) s[pidx<K>(gap0 + j)] = ~K(0);
  }
}

// Unchecked serial merge on the padded layout: VT outputs of the merge of
// the runs at element indices a and b, each followed by at least VT + 1
// largest keys.  The same (lo, hi) formulation as serial_merge_sentinel.
template <int VT, typename K>
__device__ __forceinline__ void serial_merge_gapped(const K *s, int a, int b, K (&out)[VT]) {
  K ka = s[pidx<K>(a)];
  K kb = s[pidx<K>(b)];
  const bool t0 = ka <= kb;
  K hlo = t0 ? ka : kb, hhi = t0 ? kb : ka;
  int ilo = t0 ? a : b, ihi = t0 ? b : a;
#pragma unroll
  for (int k = 0; k < VT; ++k) {
    out[k] = hlo;
    const int i = ilo + 1;
    const K kn = s[pidx<K>(i)];
    const bool p = kn <= hhi;
    hlo = p ? kn : hhi;
    ilo = p ? i : ihi;
    hhi = p ? hhi : kn;
    ihi = p ? ihi : i;
  }
}

// Sorts one tile of NT*IPT elements that is already in registers (IPT per
// thread, any assignment).  On return thread t holds tile elements
// [IPT t, IPT t + IPT) of the sorted tile in r.  The thread's registers are
// sorted by COLS, the warp merge makes runs of 32 IPT, and log2(NT/32)
// shared-memory levels (a merge-path split per thread, then a serial merge
// of IPT outputs) merge those pairwise.  GAPPED: the runs sit in the gapped
// layout and the serial merge runs unchecked (s holds block_smem_len<K>(NT,
// IPT) elements); otherwise they lie back to back and the merge checks its
// bounds (s holds merge_smem_len<K>(NT * IPT, IPT)).  The gapped form is
// faster for keys (1.96 vs 2.09 ms for 2^28 32-bit keys); the pairs' tile
// sort, at 64 registers and two 105 KB CTAs per SM, is faster checked.
template <int NT, int IPT, class COLS, typename K, bool GAPPED = true>
__device__ __forceinline__ void sort_tile_in_block(K (&r)[IPT], K *s) {
  constexpr int TILE = NT * IPT;
  constexpr int GAP = block_gap<K>(IPT);
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  COLS::sort(r);
  if constexpr (IPT == 32 && sizeof(K) == 4) {
    // levels 3-5 transpose through this warp's part of s (32 x 33 keys)
    static_assert(NT * 33 <= block_smem_len<K>(NT, IPT), "transpose buffers fit in s");
    K *t = s + (tid >> 5) * (32 * 33);
    warp_merge_level<1>(r, lane);
    warp_merge_level<2>(r, lane);
    warp_merge_level_t<3>(r, lane, t);
    warp_merge_level_t<4>(r, lane, t);
    warp_merge_level_t<5>(r, lane, t);
    if (TILE == 32 * IPT) return;
    __syncthreads();   // every warp is done with its transpose buffer
  } else if constexpr (IPT == 16 && sizeof(K) == 8 && GAPPED) {
    // 64-bit keys: levels 2-5 use the half-warp transposes, 512 words of s
    // per warp (the pairs' tile sort, at 64 registers, would spill)
    K *t = s + (tid >> 5) * 512;
    warp_merge_level<1>(r, lane);
    warp_merge_level16_t<2>(r, lane, t);
    warp_merge_level16_t<3>(r, lane, t);
    warp_merge_level16_t<4>(r, lane, t);
    warp_merge_level16_5t(r, lane, t);
    if (TILE == 32 * IPT) return;
    __syncthreads();   // every warp is done with its transpose buffer
  } else {
    warp_merge<IPT>(r, lane);
    if (TILE == 32 * IPT) return;
  }
  const int e0 = tid * IPT;
  if (GAPPED) {
    stage_gapped(r, s, e0, 32 * IPT);
  } else {
#pragma unroll
    for (int k = 0; k < IPT; ++k) s[pidx<K>(e0 + k)] = r[k];
  }
  int unused[IPT];
#pragma unroll 1
  for (int run = 32 * IPT; run < TILE; run <<= 1) {
    __syncthreads();
    const int g0 = e0 & ~(2 * run - 1);
    const int diag = e0 - g0;
    if (GAPPED) {
      const int a0 = g0 + (g0 / run) * GAP;   // run 2p and its gap, then run 2p+1
      const int b0 = a0 + run + GAP;
      const int ai = merge_path_smem(s, a0, run, b0, run, diag);
      serial_merge_gapped<IPT>(s, a0 + ai, b0 + diag - ai, r);
    } else {
      const int ai = merge_path_smem(s, g0, run, g0 + run, run, diag);
      serial_merge<IPT, false>(s, g0 + ai, g0 + run, g0 + run + diag - ai, g0 + 2 * run, r,
                               unused);
    }
    if (2 * run < TILE) {
      __syncthreads();
      if (GAPPED) {
        stage_gapped(r, s, e0, 2 * run);
      } else {
#pragma unroll
        for (int k = 0; k < IPT; ++k) s[pidx<K>(e0 + k)] = r[k];
      }
    }
  }
}

}  // namespace nsort
