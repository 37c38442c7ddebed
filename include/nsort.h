/*
 * nsort — C ABI of a GB300 (sm_103a) merge sort for 32-bit keys and
 * key/value pairs, after "A Hybrid Vectorized Merge Sort on ARM NEON"
 * (NEON-MS, arXiv 2409.03970).
 *
 * The method (paper Sec. 2.1, Fig. 1-2): the input of length N is split into
 * tiles; each tile is sorted "in registers" by a column sort with a
 * few-comparator sorting network (Sec. 2.3, Table 1: the 60-comparator
 * 16-input network), then merged by (hybrid) bitonic merging networks
 * (Sec. 2.4), and the sorted tiles are merged globally with load-balanced
 * partitioning, each worker running a serial merge of its own part
 * (Sec. 2.1, last paragraph; Sec. 3.2 "segmentation points").
 *
 * Conventions shared by every entry point:
 *  - Device pointers are plain CUDA device addresses owned by the caller
 *    (allocated with cudaMalloc, torch, ...).  The library allocates no
 *    device memory in nsort_keys / nsort_pairs / nsort_segmented: scratch
 *    comes from the caller's d_tmp of at least nsort_temp_bytes() bytes.
 *  - Keys are 32-bit patterns of type `dtype` (nsort_dtype), or 64-bit
 *    patterns for the 64-bit dtypes (nsort_keys only).  They are
 *    ordered by an order-preserving map to unsigned integers: identity for
 *    NSORT_U32, sign-bit flip for NSORT_I32, and for NSORT_F32 the IEEE
 *    754-2008 totalOrder (-NaN < -Inf < ... < -0 < +0 < ... < +Inf < +NaN,
 *    NaNs by payload).  Output keys are the input bit patterns, reordered;
 *    the map is applied inside the kernels and never visible.  Ascending.
 *    (The paper sorts 32-bit integers only, Sec. 2.2; the signed and float
 *    orders are this library's extension.)
 *  - Results are unique: keys-only output is determined by the multiset of
 *    keys; pair sorts are stable (equal keys keep input order), so the
 *    payload order is determined too.
 *  - in == out is allowed (in-place sort).  d_tmp must not overlap any
 *    input or output.  Pointers need only 4-byte (64-bit keys: 8-byte)
 *    alignment; 16-byte aligned
 *    buffers take the vectorised path.
 *  - The output (and d_tmp) are working space until the call's work on the
 *    stream is complete: other work must not read or write them meanwhile,
 *    and concurrent calls must use disjoint buffers.  (If they do not, the
 *    result is undefined but every kernel still stays inside its buffers:
 *    tile geometry is clamped to the runs whatever the data.)
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) and return after enqueueing.  Return value: an
 *    nsort_status.  Argument errors are detected before any launch;
 *    NSORT_ECUDA reports a launch error (cudaGetLastError), with its text in
 *    nsort_last_error().
 *  - n = 0 is a valid no-op.  n up to 2^40 keys.
 */
#ifndef NSORT_H
#define NSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NSORT_U32 = 0, NSORT_I32 = 1, NSORT_F32 = 2,
    /* 64-bit keys, nsort_keys only: the same maps on 64-bit patterns (sign
     * flip for int64, IEEE totalOrder for binary64); pointers 8-byte aligned */
    NSORT_U64 = 3, NSORT_I64 = 4, NSORT_F64 = 5
} nsort_dtype;

typedef enum {
    NSORT_KIND_KEYS = 0,            /* nsort_keys */
    NSORT_KIND_PAIRS = 1,           /* nsort_pairs */
    NSORT_KIND_SEGMENTED = 2,       /* nsort_segmented, keys only */
    NSORT_KIND_SEGMENTED_PAIRS = 3, /* nsort_segmented with values */
    NSORT_KIND_MERGE = 4,           /* nsort_merge_shards, keys only (nseg = number of runs) */
    NSORT_KIND_MERGE_PAIRS = 5,     /* nsort_merge_shards with values */
    NSORT_KIND_PAIRS64 = 6          /* nsort_pairs64 */
} nsort_kind;

typedef enum {
    NSORT_OK = 0,
    NSORT_EINVAL = 1,     /* bad argument: dtype, kind, pointer, offsets, size */
    NSORT_ENOMEM = 2,     /* d_tmp too small, or a request above the memory budget */
    NSORT_ECUDA = 3,      /* a CUDA call or kernel launch failed */
    NSORT_EBUSY = 4,      /* serving context: queue full */
    NSORT_ETIMEOUT = 5,   /* nsort_wait deadline passed */
    NSORT_ENOTFOUND = 6   /* serving context: unknown ticket */
} nsort_status;

/* Scratch bytes a call of `kind` needs for n keys (and nseg segments, for
 * the segmented kinds; ignored otherwise).  Only the 64-bit dtypes change
 * the size (kind KEYS: 8-byte key copies and samples).
 * Returns 0 for a bad kind.  Source: the auxiliary O(N) buffer of the
 * paper's merge stages (Sec. 3.2, last paragraph): one ping-pong copy of the
 * keys (and values), plus the per-tile merge-path splitters. */
size_t nsort_temp_bytes(int kind, uint64_t n, uint64_t nseg, int dtype);

/* Number of passes over the data for a plain sort of n 32-bit keys (kind
 * KEYS or PAIRS): one tile sort plus ceil(log2(ceil(n / tile))) global merge
 * passes.  Writes the tile sizes through the non-NULL pointers.  Used to
 * compute the algorithmic bytes of a sort (passes x 2 x element bytes x n). */
int nsort_plan(int kind, uint64_t n, int *passes, int *sort_tile, int *merge_tile);

/* nsort_plan for keys of `dtype`: 64-bit dtypes (kind KEYS only) sort
 * 4096-key tiles and merge 1920-key tiles.  NSORT_EINVAL for a bad kind, a
 * 64-bit dtype with kind PAIRS, or n above 2^40. */
int nsort_plan_dtype(int kind, uint64_t n, int dtype, int *passes, int *sort_tile,
                     int *merge_tile);

/* CTAs of the persistent merge pass on the current device for `kind`
 * (KEYS or PAIRS) and `dtype`: SMs x the merge kernel's resident CTAs per
 * SM.  A merge pass of at most twice that many merge tiles finds its
 * merge-path splitters inside the merge kernel; a larger pass launches the
 * partition kernel first (the paper's "segmentation points", Sec. 3.2).
 * Returns 0 for a bad kind or dtype, or when a CUDA query fails. */
int nsort_merge_grid(int kind, int dtype);

/* Sorts n keys ascending (paper Sec. 2.1: "the input sequence of the length
 * N").  d_keys_in / d_keys_out: n 32-bit patterns, contiguous, or n 64-bit
 * patterns for the 64-bit dtypes (8-byte aligned; the paper's register
 * width W depends on the key type, Sec. 2.2: 64-bit keys are this library's
 * wider-key variant of the same sort).  d_tmp:
 * nsort_temp_bytes(NSORT_KIND_KEYS, n, 0, dtype) bytes of device scratch,
 * 256-byte aligned.  Errors: NSORT_EINVAL (NULL or misaligned pointer with
 * n > 0, bad dtype, n too large), NSORT_ENOMEM (tmp_bytes too small),
 * NSORT_ECUDA. */
int nsort_keys(const void *d_keys_in, void *d_keys_out, uint64_t n, int dtype,
               void *d_tmp, size_t tmp_bytes, void *stream);

/* Stable key/value sort: keys as in nsort_keys, each carrying a 32-bit
 * payload (separate arrays, same length).  Equal keys keep their input
 * order.  d_vals_in == d_vals_out is allowed.  Scratch:
 * nsort_temp_bytes(NSORT_KIND_PAIRS, n, 0, dtype).  Errors as nsort_keys. */
int nsort_pairs(const void *d_keys_in, const uint32_t *d_vals_in,
                void *d_keys_out, uint32_t *d_vals_out, uint64_t n, int dtype,
                void *d_tmp, size_t tmp_bytes, void *stream);

/* Stable key/value sort with 64-bit payloads (row ids, pointers, ...):
 * 32-bit keys of dtype U32 / I32 / F32 as in nsort_pairs, each carrying a
 * 64-bit payload that moves with its key.  Equal keys keep their input
 * order.  d_vals_in / d_vals_out: n uint64, 8-byte aligned; d_keys_out
 * and d_vals_out must be 16-byte aligned (the merge passes move them with
 * bulk copies).  In place (in == out) is allowed.  Scratch:
 * nsort_temp_bytes(NSORT_KIND_PAIRS64, n, 0, dtype).  Errors as
 * nsort_pairs, plus NSORT_EINVAL for a misaligned payload or output.
 * Paper: the sort of Sec. 2.1 with a wider payload word (the register
 * width depends on the element type, Sec. 2.2); the payload width is this
 * library's extension. */
int nsort_pairs64(const void *d_keys_in, const uint64_t *d_vals_in, void *d_keys_out,
                  uint64_t *d_vals_out, uint64_t n, int dtype, void *d_tmp, size_t tmp_bytes,
                  void *stream);

/* Segmented sort: nseg independent arrays stored back to back.  d_offsets
 * is a DEVICE array of nseg+1 int64 (CSR form): segment s is
 * [d_offsets[s], d_offsets[s+1]), d_offsets[0] == 0, non-decreasing,
 * d_offsets[nseg] == n (the total key count).  Empty segments are allowed.
 * Each segment is sorted on its own as nsort_keys / nsort_pairs would sort
 * it (stable when values are given; d_vals_in and d_vals_out both NULL for
 * keys only).  The batch runs as three small set-up kernels (binning by
 * length on the device) and one persistent kernel that takes segments from
 * a work queue: one thread per segment of at most `tiny_width` keys, one
 * warp per segment of at most 32 x `small_ipt`, one CTA per segment of at
 * most 16 x block_threads keys, and tile sorts (32 keys per thread for keys
 * only, 16 with values) plus merge levels for longer ones.  Every
 * step is stream-ordered with no host synchronisation, so the call can be
 * captured into a CUDA graph.  Scratch:
 * nsort_temp_bytes(NSORT_KIND_SEGMENTED[_PAIRS], n, nseg, dtype), 256-byte
 * aligned; in-place (in == out) is allowed.  Host-checked errors:
 * NSORT_EINVAL, NSORT_ENOMEM, NSORT_ECUDA.  Malformed offsets are found on
 * the device: the batch is left unsorted and nsort_device_status()
 * reports NSORT_EINVAL.  Source: the paper's sort (Sec. 2.1) applied per
 * segment; the batching is this library's extension. */
int nsort_segmented(const void *d_keys_in, void *d_keys_out,
                    const uint32_t *d_vals_in, uint32_t *d_vals_out,
                    const int64_t *d_offsets, uint64_t nseg, uint64_t n, int dtype,
                    void *d_tmp, size_t tmp_bytes, void *stream);

/* ---- sharded sort: one array split over P workers ----------------------
 * The paper's parallel merge (Sec. 2.1, last paragraph; Sec. 3.2): P
 * workers each sort a part, the output is partitioned evenly at
 * "segmentation points" (how many keys of each part precede each output
 * position), and each worker merges the slices that fall in its share.
 * With one worker per GPU: each GPU sorts its shard (nsort_keys /
 * nsort_pairs), the splitters come from nsort_count_le summed over the
 * GPUs (or, with every shard in one buffer, from nsort_shard_coranks), the
 * slices are exchanged (an all-to-all), and each GPU merges what it
 * received with nsort_merge_shards.  The result is the stable sort of the
 * concatenated shards: ascending key order, equal keys in shard order, then
 * in their order within the shard. */

/* Segmentation points of P sorted shards stored back to back in one device
 * buffer (shard r = keys [d_shard_off[r], d_shard_off[r+1]); d_shard_off is
 * a DEVICE array of nshards+1 int64, non-decreasing, nshards 1..32; each
 * shard sorted ascending in the key order of dtype).  For each of the
 * ntargets output positions d = d_targets[j] (DEVICE int64, clamped to
 * [0, total keys]) of the stable merge of the shards, writes to
 * d_coranks[j * nshards + r] (DEVICE int64) how many of the first d outputs
 * come from shard r; these sum to d.  Exact for any data, ties included
 * (equal keys go to the lower shard first).  One warp per target, bisection
 * on the order-key space (32 rounds, 64 for the 64-bit dtypes).  Errors:
 * NSORT_EINVAL (bad dtype, shard count, NULL or misaligned pointer),
 * NSORT_ECUDA.  Allocates nothing. */
int nsort_shard_coranks(const void *d_keys, const int64_t *d_shard_off, int nshards,
                        const int64_t *d_targets, int ntargets, int dtype,
                        int64_t *d_coranks, void *stream);

/* The per-GPU step of the same splitter search across GPUs: for a sorted
 * array of n keys (key order of dtype) and m bounds given as ORDER keys
 * (d_bounds: uint32, or uint64 for the 64-bit dtypes: the order-preserving
 * map's unsigned keys, 0 = the smallest key of the dtype), writes
 * d_le[i] = the number of keys whose order key is <= d_bounds[i] (DEVICE
 * int64).  A caller bisects each splitter's key on the sum of these counts
 * over the GPUs (one all-reduce per round), as nsort_shard_coranks does in
 * one kernel.  Errors: NSORT_EINVAL, NSORT_ECUDA.  Allocates nothing. */
int nsort_count_le(const void *d_sorted, uint64_t n, int dtype, const void *d_bounds,
                   uint64_t m, int64_t *d_le, void *stream);

/* Merges nruns sorted runs stored back to back into one sorted array: a
 * worker's merge of the slices it received (paper Sec. 2.1, last
 * paragraph).  h_run_off: HOST array of nruns+1 int64, run r =
 * [h_run_off[r], h_run_off[r+1]), h_run_off[0] == 0, non-decreasing,
 * h_run_off[nruns] = n; nruns 1..64; empty runs allowed.  Each run sorted
 * ascending in the key order of dtype (as nsort_keys / nsort_pairs leave
 * it).  Stable: equal keys keep run order, then position.  d_vals_in /
 * d_vals_out: 32-bit payloads moved with their keys, or both NULL (keys
 * only; the 64-bit dtypes are keys only).  All buffers 16-byte aligned;
 * the output must not overlap the input.  Runs in ceil(log2(nruns))
 * two-way merge passes.  Scratch: nsort_temp_bytes(NSORT_KIND_MERGE[_PAIRS],
 * n, nruns, dtype), 256-byte aligned (0 bytes for one run).  Errors:
 * NSORT_EINVAL (offsets, dtype, pointers, alignment, overlap), NSORT_ENOMEM
 * (scratch too small), NSORT_ECUDA.  If a run is not sorted the output is
 * unspecified, but every access stays inside the buffers. */
int nsort_merge_shards(const void *d_keys_in, const uint32_t *d_vals_in, void *d_keys_out,
                       uint32_t *d_vals_out, const int64_t *h_run_off, int nruns, int dtype,
                       void *d_tmp, size_t tmp_bytes, void *stream);

/* Tunables of nsort_segmented, set by the autotuner (process-wide). */
typedef struct {
    int block_threads;   /* 256 or 512: persistent CTA size; one-CTA segments up to
                            16 x block_threads keys, longer ones in tiles of 32 (keys)
                            or 16 (pairs) x block_threads */
    int tiny_width;      /* 8 or 16: network width of the one-thread bin */
    int small_ipt;       /* 8 or 16: keys per lane of the one-warp bin */
    int blocks_per_sm;   /* persistent CTAs per SM; 0 = as many as fit */
} nsort_seg_config;

int nsort_segmented_set_config(const nsort_seg_config *cfg);
int nsort_segmented_get_config(nsort_seg_config *cfg);

/* Allocation-free key sort, for callers that cannot allocate device memory:
 * their device memory is owned by another allocator (a framework's caching
 * pool, a fixed arena sized at start-up) or they run where a cudaMalloc is
 * not allowed because it may block or synchronise the device.  Same result
 * as nsort_keys, but no scratch argument: the scratch is one fixed array in
 * the library's device global memory (about 4.1 MiB), present on every GPU
 * that loads the library until the process exits.  The paper has no
 * counterpart; this is an interface for such callers.
 *  - n up to NSORT_NOALLOC_MAX_KEYS; larger n returns NSORT_ENOMEM with an
 *    explanation in nsort_last_error().  Other errors as nsort_keys.
 *  - Calls nothing that allocates (no cudaMalloc / cudaFree).
 *  - The array used is the one of the CURRENT device; `stream` must belong
 *    to that device.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and keeps it for the
 *    life of the process; make that first call before any stream capture.
 *    The kept address does not survive cudaDeviceReset: do not call these
 *    entry points again in a process that has reset the device.
 *  - All calls on a device share the one array, which keeps whatever the last
 *    call left in it.  Each call clears the status word (below) on its
 *    stream; nothing else in it needs to start at zero.  Calls whose
 *    work overlaps on the GPU race on it: issue them on one stream, or order
 *    them with events. */
#define NSORT_NOALLOC_MAX_KEYS (1u << 20)
int nsort_keys_noalloc(const void *d_keys_in, void *d_keys_out, uint64_t n, int dtype,
                       void *stream);

/* Device status of the last nsort_keys_noalloc on the current device, read
 * in order on `stream` (it synchronises that stream): NSORT_OK, or
 * NSORT_ETIMEOUT when a bounded wait inside a merge pass gave up and that
 * call's output is incomplete (this does not happen in normal operation).
 * It plays the part nsort_device_status plays for calls given a scratch
 * buffer.  NSORT_ECUDA if the read fails.  Allocates nothing. */
int nsort_keys_noalloc_status(void *stream);

/* ---- serving: continuous batching of sort requests --------------------
 * A context owns a scheduler thread, a pool of CUDA streams and a device
 * memory budget.  Requests (device-resident inputs and outputs owned by the
 * caller) are admitted as soon as a stream slot and budget for their scratch
 * are free; small requests are co-batched into one segmented launch;
 * admitted requests overlap on the device, except that requests of 2^22
 * keys or more (each fills the GPU) run one at a time, and while one runs
 * smaller requests are admitted ahead of the next.  Each result is bit-identical to
 * the plain call on the same input.  Paper: none — the serving layer is this
 * library's extension around the Sec. 2.1 sort. */
typedef struct nsort_ctx nsort_ctx;

typedef struct {
    int kind;                 /* NSORT_KIND_KEYS or NSORT_KIND_PAIRS */
    int dtype;                /* nsort_dtype */
    uint64_t n;
    const void *d_keys_in;
    void *d_keys_out;
    const uint32_t *d_vals_in;  /* PAIRS only */
    uint32_t *d_vals_out;       /* PAIRS only */
} nsort_request;

typedef struct {
    double t_submit;   /* seconds on the host monotonic clock */
    double t_admit;    /* scratch reserved, work enqueued */
    double t_done;     /* completion observed by the scheduler */
    int status;        /* nsort_status of the request */
    int batched;       /* 1 when co-batched into a segmented launch */
} nsort_timing;

/* device: CUDA ordinal.  mem_budget_bytes: size of the scratch arena the
 * context allocates once (cudaMalloc) and sub-allocates to admitted
 * requests; a request whose scratch exceeds the whole arena is rejected
 * with NSORT_ENOMEM at submit.  streams: concurrent stream slots (1..64).
 * batch_max_keys: requests of at most this many keys are co-batched (0
 * disables co-batching; streams = 1 and batch_max_keys = 0 is plain FIFO
 * one-at-a-time sorting).  Returns NSORT_OK and *out, or an error. */
int nsort_ctx_create(int device, size_t mem_budget_bytes, int streams,
                     uint64_t batch_max_keys, nsort_ctx **out);
/* Stops admitting, waits for every admitted request, stops the scheduler
 * and frees the arena and the streams.  Requests still waiting for
 * admission complete with status NSORT_EBUSY (cancelled). */
void nsort_ctx_destroy(nsort_ctx *ctx);
/* Enqueues a request (device buffers owned by the caller, which must not be
 * touched until the request is done); never blocks on the device.  *ticket
 * identifies it.  n = 0 completes at once. */
int nsort_submit(nsort_ctx *ctx, const nsort_request *req, uint64_t *ticket);
/* *done = 1 once the request completed (then *timing, if not NULL, is
 * filled); NSORT_ENOTFOUND for an unknown ticket. */
int nsort_poll(nsort_ctx *ctx, uint64_t ticket, int *done, nsort_timing *timing);
/* Blocks until the request completed or timeout_ms passed (NSORT_ETIMEOUT). */
int nsort_wait(nsort_ctx *ctx, uint64_t ticket, uint32_t timeout_ms);

/* ---- tracing ------------------------------------------------------------
 * Per-kernel device time without a profiler.  While enabled, every kernel
 * launch of the library is bracketed by CUDA events recorded on the stream
 * it is launched on.  Do not enable while a stream is being captured into a
 * CUDA graph.  Paper: none (measurement support). */
typedef struct {
    char kernel[32];     /* kernel name, e.g. "merge_keys" */
    uint64_t launches;   /* launches recorded since tracing was enabled */
    double total_ms;     /* sum of their device durations */
} nsort_trace_entry;

/* on != 0 starts recording (dropping earlier records); on == 0 stops. */
int nsort_trace_enable(int on);
/* Waits for the recorded events, writes one entry per kernel name (at most
 * `capacity`; *count = number of names seen) and drops the records. */
int nsort_trace_read(nsort_trace_entry *out, int capacity, int *count);

/* Synchronises `stream` and returns the device-side status word of the last
 * call that used the scratch buffer d_tmp (the first 4 bytes of every
 * scratch layout): NSORT_OK; NSORT_EINVAL (nsort_segmented: malformed
 * offsets); NSORT_ETIMEOUT (a bounded wait inside a kernel gave up — the
 * output of that call is then incomplete; this does not happen in normal
 * operation).  Calls that need no scratch (n within one tile) have no
 * status word. */
int nsort_device_status(const void *d_tmp, void *stream);

/* Human-readable text of an nsort_status. */
const char *nsort_status_string(int status);
/* Text of the last NSORT_ECUDA error on the calling host thread ("" if none). */
const char *nsort_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NSORT_H */
