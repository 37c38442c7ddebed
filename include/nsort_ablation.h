/*
 * Ablation entry points of libnsort: the column-sort network and the number
 * of keys per thread of the block sort, varied one at a time, so that the
 * paper's Table 1 (comparators per network) and Table 2 (time to produce
 * sorted runs of X elements with R registers) can be measured on the GPU.
 * The production sorts (nsort.h) use the best networks with 32 keys per
 * thread for 32-bit keys (16 for pairs and 64-bit keys); these calls run
 * the same column sort, warp merge and block merge code with another
 * network or another keys-per-thread count.
 *
 * Keys are unsigned 32-bit integers (the paper's 32-bit integer keys,
 * Sec. 2.2), ascending.  Device pointers are caller-owned CUDA device
 * addresses; nothing is allocated.  Calls are asynchronous on `stream` (a
 * cudaStream_t, NULL = legacy default stream) and return an nsort_status
 * (nsort.h): NSORT_EINVAL for a bad argument before any launch,
 * NSORT_ECUDA for a launch error (text in nsort_last_error()).
 */
#ifndef NSORT_ABLATION_H
#define NSORT_ABLATION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Network families of Table 1 (Sec. 2.3). */
typedef enum {
    NSORT_NET_BITONIC = 0,   /* Batcher's bitonic sorter (flip form): 6 / 24 / 80 / 240 */
    NSORT_NET_ODDEVEN = 1,   /* Batcher's odd-even merge sort: 5 / 19 / 63 / 191 */
    NSORT_NET_BEST = 2       /* fewest known: 5 / 19 / 60 (Green) / 185 (2 x Green + merge) */
} nsort_net_family;

/* Host only, no CUDA call.  Writes the comparators of the column-sort
 * network of `family` on `width` wires (4, 8, 16 or 32) to lo[] / hi[]
 * (capacity `cap`; after comparator c, v[lo[c]] <= v[hi[c]]), in the order
 * the device column sort applies them.  These are the very lists the
 * kernels are generated from.  Returns the number of comparators (entries
 * past `cap` are not written), or -1 for an unknown family or width.
 * Source: Table 1 (Sec. 2.3). */
int nsort_network(int family, int width, int32_t *lo, int32_t *hi, int cap);

/* Applies the network of `family` and `width` (4, 8, 16, 32) to each of
 * `groups` consecutive groups of `width` keys: d_out[g*width ...] receives
 * group g of d_in, sorted by the network, one thread per group.  d_in and
 * d_out hold groups*width uint32 each and may be equal.  groups up to 2^32.
 * Source: the column sort of Sec. 2.3. */
int nsort_network_apply(const uint32_t *d_in, uint32_t *d_out, uint64_t groups, int family,
                        int width, void *stream);

/* Sorts every run [k*run, min((k+1)*run, n)) of d_in into d_out (n uint32
 * each; d_in may equal d_out), with `ipt` keys per thread (4, 8, 16, 32,
 * the paper's R, Sec. 2.2) in 512-thread CTAs:
 *   run = ipt * 2^L, L = 0..5   each thread sorts its ipt keys with the
 *                               network of `family` (the column sort), then
 *                               the warp's flip merger runs L levels (Sec.
 *                               2.4): the in-register sort of Table 2;
 *   run = 512 * ipt             the whole block sort: column sort, the five
 *                               warp levels, then the shared-memory merges
 *                               of Sec. 2.1 (the production tile sort with
 *                               ipt = 16 and NSORT_NET_BEST).
 * Any other run is NSORT_EINVAL.  n up to 2^40; a short last run is sorted
 * on its own.  Source: Sec. 2.1-2.4, Table 2. */
int nsort_runs(const uint32_t *d_in, uint32_t *d_out, uint64_t n, int family, int ipt,
               uint64_t run, void *stream);

/* Mergers of Table 3 (Sec. 2.4). */
typedef enum {
    NSORT_MERGE_HYBRID = 0,   /* flip merger, lane-contiguous keys: shuffles while the compare
                                 distance is >= ipt, then the in-thread tail (production) */
    NSORT_MERGE_SHUFFLE = 1,  /* flip merger, lane-strided keys (key 32k + lane in register k):
                                 every distance below 32 is a shuffle ("vectorized") */
    NSORT_MERGE_SERIAL = 2    /* merge path in shared memory, then a serial merge of ipt
                                 outputs per thread */
} nsort_merger;

/* Merges each pair of adjacent sorted runs of d_in, [2k run, (2k+1) run) and
 * [(2k+1) run, (2k+2) run) (clipped to n), into the sorted run
 * [2k run, (2k+2) run) of d_out, with `method` and `ipt` keys per thread
 * (4, 8, 16, 32) in 512-thread CTAs.  run must be a power of two with
 *   NSORT_MERGE_HYBRID    ipt <= run <= 16 ipt
 *   NSORT_MERGE_SHUFFLE   1 <= run <= 16 ipt
 *   NSORT_MERGE_SERIAL    ipt / 2 <= run <= 256 ipt
 * else NSORT_EINVAL.  d_in must be sorted within each run of `run` keys;
 * if it is not, d_out is unspecified (every access still stays inside the
 * n keys of each buffer).  d_in and d_out hold n uint32 each (n up to
 * 2^40) and may be equal.  Source: the
 * hybrid and vectorized bitonic mergers of Sec. 2.4 (Table 3) and the
 * merge-path serial merge of Sec. 2.1. */
int nsort_merge_runs(const uint32_t *d_in, uint32_t *d_out, uint64_t n, uint64_t run,
                     int method, int ipt, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NSORT_ABLATION_H */
