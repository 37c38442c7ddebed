/*
 * Test hooks of libnsort: the pure host-side policy of the sort server,
 * exposed so that it can be checked on a machine without a GPU.  They make
 * no CUDA call.  Paper: none (serving is this library's extension).
 */
#ifndef NSORT_TESTING_H
#define NSORT_TESTING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Runs the server's admission choice on a waiting queue of `count`
 * requests (arrival order; kind, dtype and size each): which tickets the
 * next free stream slot takes together.  large_min_keys / large_running:
 * the server's size from which requests run one at a time (2^22 keys;
 * UINT64_MAX for none) and whether one such request is running, in which
 * case the first smaller request goes ahead of waiting large ones.  Writes
 * the tickets to out (capacity `count`) and their number to *out_count
 * (0 when nothing may start). */
int nsort_policy_pick_batch(const uint64_t *tickets, const int *kinds, const int *dtypes,
                            const uint64_t *ns, int count, uint64_t batch_max_keys,
                            int max_batch, uint64_t max_batch_keys, uint64_t large_min_keys,
                            int large_running, uint64_t *out, int *out_count);

/* Replays allocations and releases on the server's scratch arena (first
 * fit, 256-byte granules, coalescing).  ops[i] > 0 allocates ops[i] bytes
 * and writes its offset (or -1 when nothing fits) to offsets[i];
 * ops[i] < 0 releases the block of op number -ops[i]-1. */
int nsort_policy_arena_replay(uint64_t capacity, const int64_t *ops, int nops,
                              int64_t *offsets);

/* Runs the library's bounded waits (the mbarrier wait of the merge pass and
 * the completion-counter wait of the segmented sort) on events that never
 * happen, with a limit of limit_us microseconds each, in one small kernel on
 * `stream`.  Both waits give up; the kernel records NSORT_ETIMEOUT in the
 * status word of d_tmp (at least 512 bytes, 256-byte aligned) and returns
 * normally, so nsort_device_status(d_tmp) reports NSORT_ETIMEOUT and the
 * context stays usable.  This is how time-outs are tested without hanging
 * or faulting a GPU.  Paper: none. */
int nsort_selftest_wait(void *d_tmp, size_t tmp_bytes, uint32_t limit_us, void *stream);

/* Sets the smallest key count at which a sort of 32-bit keys merges two
 * levels per pass over the array (four-way passes) and returns the previous
 * setting.  0 selects four-way passes for every sort with at least two
 * merge levels, UINT64_MAX for none.  Plans and nsort_temp_bytes follow the
 * setting, so change it only while no sort runs, and size scratch after the
 * change.  Makes no CUDA call.  Paper: none (a merge pass of this library
 * merges one or two of the paper's merge levels). */
uint64_t nsort_testing_set_four_way_min(uint64_t min_keys);

#ifdef __cplusplus
}
#endif

#endif /* NSORT_TESTING_H */
