// Host-side helpers shared by the translation units of libnsort.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

namespace nsort {

// Largest key count a call accepts (keeps every in-kernel index in range).
constexpr uint64_t MAX_KEYS = uint64_t(1) << 40;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Layout of the scratch buffer of a plain sort.
struct Plan {
  int64_t n = 0;
  int sort_tile = 0;         // keys per tile-sort CTA
  int merge_tile = 0;        // outputs per merge CTA
  int merge_passes = 0;      // merge levels: ceil(log2(ceil(n / sort_tile)))
  int merge2_passes = 0;     // passes over HBM that merge one level (pairs of runs)
  int merge4_passes = 0;     // passes that merge two levels (groups of four runs; 32-bit keys)
  int64_t num_merge_tiles = 0;
  size_t status_off = 0;     // device status word (NSORT_OK / NSORT_ETIMEOUT)
  size_t keys_off = 0;       // ping-pong key buffer
  size_t vals_off = 0;       // ping-pong value buffer (pairs)
  size_t split_off = 0;      // int64 merge-path splitters, one per merge tile
  size_t samp_off = 0;       // keys: every 64th key of the last stage's output
  size_t rec_off = 0;        // four-way passes: level-one merged sample records (uint64)
  size_t bnd_off = 0;        // four-way passes: tile boundary co-ranks (4 int64 a record)
  size_t total = 0;          // bytes of scratch (0 when one tile holds everything)
};

// dtype matters only for keys: 64-bit dtypes take 8-byte words.
Plan make_plan(int kind, uint64_t n, int dtype = 0);

int sort_keys_impl(const uint32_t *in, uint32_t *out, int64_t n, int dt, void *tmp,
                   cudaStream_t st);
int sort_keys64_impl(const uint64_t *in, uint64_t *out, int64_t n, int dt, void *tmp,
                     cudaStream_t st);
int sort_pairs_impl(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                    int64_t n, int dt, void *tmp, cudaStream_t st);

size_t segmented_temp_bytes(int kind, uint64_t n, uint64_t nseg);

// One merge level of the large segments of a segmented batch, as bulk-copy
// merge passes over per-tile descriptors (nsort_segmented).  Segments longer
// than min_len were sorted in tiles of `tile` keys (level 0); level k
// merges their runs of tile * 2^(k-1) keys.  Level k-1 of a segment with P
// levels is in ktmp when P - (k-1) is odd, else in kout.
struct SegLevelArgs {
  const int64_t *off;          // nseg + 1 segment offsets (device)
  int64_t nseg, n;
  int64_t min_len;
  int tile, k, dt;
  uint32_t *kout, *ktmp;
  uint32_t *vout, *vtmp;       // both null for keys only
  int *status;                 // device status word (NSORT_OK: offsets are valid)
  const int *max_level;        // device: the most merge levels any segment of the batch needs
  unsigned long long *count;   // device counter of this level's tiles, zero before the call
  int64_t *tile_seg;           // device scratch, max_tiles entries
  void *desc;                  // device scratch, max_tiles descriptors
  int64_t max_tiles;
};
// nsort_segmented for a caller that knows no segment is longer than
// max_seg_len keys (the server's co-batches): only the merge levels such a
// segment needs are launched.
int segmented_impl(const void *d_keys_in, void *d_keys_out, const uint32_t *d_vals_in,
                   uint32_t *d_vals_out, const int64_t *d_offsets, uint64_t nseg, uint64_t n,
                   int dtype, void *d_tmp, size_t tmp_bytes, void *stream, uint64_t max_seg_len);
int seg_merge_tile(bool pairs);
size_t seg_tile_desc_bytes();
int launch_segmented_level(const SegLevelArgs &a, cudaStream_t st);

// Merge of sorted runs of any lengths (nsort_merge_shards).
size_t merge_runs_temp_bytes(bool pairs, uint64_t n, uint64_t nruns, int dtype);
int merge_runs_impl(const void *kin, const uint32_t *vin, void *kout, uint32_t *vout,
                    const int64_t *off, int nruns, int dt, void *tmp, cudaStream_t st);

// Kernel ids of the tracer (order of its name table).
enum TraceKernel {
  TK_TILE_SORT_KEYS = 0, TK_TILE_SORT_PAIRS, TK_PARTITION, TK_MERGE_KEYS, TK_MERGE_PAIRS,
  TK_SEG_BIN, TK_SEG_SORT, TK_SEG_MERGE, TK_SEG_COPY, TK_TILE_SORT_KEYS64, TK_MERGE_KEYS64,
  TK_SAMPLE_MERGE, TK_MERGE4_BOUNDS, TK_MERGE4_KEYS
};

// Brackets one kernel launch with CUDA events on its stream while tracing
// is enabled (nsort_trace_enable); does nothing otherwise.
class TraceScope {
 public:
  TraceScope(int kernel, cudaStream_t st);
  ~TraceScope();
  TraceScope(const TraceScope &) = delete;
  TraceScope &operator=(const TraceScope &) = delete;

 private:
  int kernel_;
  cudaStream_t st_;
  cudaEvent_t start_ = nullptr, stop_ = nullptr;
  bool active_ = false;
};

void set_last_error(const std::string &msg);
const char *last_error_cstr();

}  // namespace nsort
