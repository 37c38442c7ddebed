/*
 * CPU oracle for the NEON-MS sort — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke() check and the CPU-baseline leg of the
 * benchmark may load this library.  The product path (libnsort) never calls
 * it and shares no code with it.
 *
 * What it computes is the plain definition of the result that the paper's
 * method reaches faster: the input sequence of length N sorted ascending
 * (paper Sec. 2.1, first paragraph), by a merge-based sort (Sec. 2.1, the
 * merge stages; Sec. 2.4).  Here that is written as the textbook bottom-up
 * merge sort: runs of width 1, 2, 4, ... are merged pairwise, and on equal
 * keys the element from the left run is taken first, so the sort is stable.
 *
 * Keys are 32-bit patterns.  The paper sorts 32-bit integers only (Sec. 2.2);
 * signed and IEEE binary32 keys are ordered by an order-preserving map to
 * unsigned integers (orc_key below), which for binary32 is the IEEE 754-2008
 * totalOrder predicate (Sec. 5.10 of that standard): -NaN < -Inf < ... < -0 <
 * +0 < ... < +Inf < +NaN, NaNs ordered by payload.  Output keys are the input
 * bit patterns, never canonicalised.
 *
 * 64-bit keys (uint64, int64, IEEE binary64) are the wider-key variant of
 * the same sort (the paper's register width W depends on the key type, Sec.
 * 2.2): orc_key64 is the same map on 64-bit patterns (totalOrder for
 * binary64) and orc_sort_keys64 the same bottom-up merge sort.
 *
 * Parity pins for every function here live in tests/test_oracle.py: brute
 * force on tiny inputs against a textbook insertion sort, the IEEE order of a
 * table of special values and of the signed-integer order, invariants
 * (non-decreasing, permutation, stability) and closed forms.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_U32 = 0, ORC_I32 = 1, ORC_F32 = 2 };

/* Order-preserving map from a key's bit pattern to an unsigned integer.
 * u32: identity.  i32: flip the sign bit (two's complement order).
 * f32: negative patterns (sign set) are complemented, so that a larger
 * magnitude maps lower; non-negative patterns get the sign bit set, so that
 * they all map above every negative one.  Returns 0 for an unknown dtype
 * (callers validate dtype first). */
uint32_t orc_key(uint32_t bits, int dtype)
{
    if (dtype == ORC_U32)
        return bits;
    if (dtype == ORC_I32)
        return bits ^ 0x80000000u;
    if (dtype == ORC_F32) {
        if (bits & 0x80000000u)
            return ~bits;
        return bits ^ 0x80000000u;
    }
    return 0;
}

/* Applies orc_key to n patterns (used by the tests to check the map). */
void orc_key_array(const uint32_t *bits, uint32_t *keys, uint64_t n, int dtype)
{
    for (uint64_t i = 0; i < n; i++)
        keys[i] = orc_key(bits[i], dtype);
}

/* Merges the sorted runs src[lo, mid) and src[mid, hi) into dst[lo, hi).
 * On equal keys the left run's element goes first (stable).  vals may be
 * NULL (keys only). */
static void merge_runs(const uint32_t *src_k, const uint32_t *src_v,
                       uint32_t *dst_k, uint32_t *dst_v,
                       uint64_t lo, uint64_t mid, uint64_t hi, int dtype)
{
    uint64_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        if (orc_key(src_k[j], dtype) < orc_key(src_k[i], dtype)) {
            dst_k[o] = src_k[j];
            if (dst_v) dst_v[o] = src_v[j];
            j++;
        } else {
            dst_k[o] = src_k[i];
            if (dst_v) dst_v[o] = src_v[i];
            i++;
        }
        o++;
    }
    while (i < mid) {
        dst_k[o] = src_k[i];
        if (dst_v) dst_v[o] = src_v[i];
        i++;
        o++;
    }
    while (j < hi) {
        dst_k[o] = src_k[j];
        if (dst_v) dst_v[o] = src_v[j];
        j++;
        o++;
    }
}

/* Stable bottom-up merge sort of n keys (and, when vals_in is not NULL, their
 * payloads).  Output buffers may alias the inputs.  Returns 0, -1 on a bad
 * dtype, -2 when scratch memory cannot be allocated. */
static int sort_impl(const uint32_t *keys_in, const uint32_t *vals_in,
                     uint32_t *keys_out, uint32_t *vals_out,
                     uint64_t n, int dtype)
{
    if (dtype != ORC_U32 && dtype != ORC_I32 && dtype != ORC_F32)
        return -1;
    if (n == 0)
        return 0;
    int with_vals = (vals_in != NULL);
    uint32_t *ak = malloc(n * sizeof(uint32_t));
    uint32_t *bk = malloc(n * sizeof(uint32_t));
    uint32_t *av = with_vals ? malloc(n * sizeof(uint32_t)) : NULL;
    uint32_t *bv = with_vals ? malloc(n * sizeof(uint32_t)) : NULL;
    if (!ak || !bk || (with_vals && (!av || !bv))) {
        free(ak); free(bk); free(av); free(bv);
        return -2;
    }
    memcpy(ak, keys_in, n * sizeof(uint32_t));
    if (with_vals)
        memcpy(av, vals_in, n * sizeof(uint32_t));

    for (uint64_t width = 1; width < n; width *= 2) {
        for (uint64_t lo = 0; lo < n; lo += 2 * width) {
            uint64_t mid = lo + width < n ? lo + width : n;
            uint64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            merge_runs(ak, av, bk, bv, lo, mid, hi, dtype);
        }
        uint32_t *t = ak; ak = bk; bk = t;
        t = av; av = bv; bv = t;
    }

    memcpy(keys_out, ak, n * sizeof(uint32_t));
    if (with_vals)
        memcpy(vals_out, av, n * sizeof(uint32_t));
    free(ak); free(bk); free(av); free(bv);
    return 0;
}

/* Keys only: out = the input bit patterns in ascending orc_key order. */
int orc_sort_keys(const uint32_t *keys_in, uint32_t *keys_out, uint64_t n, int dtype)
{
    return sort_impl(keys_in, NULL, keys_out, NULL, n, dtype);
}

/* Key/value pairs, stable: equal keys keep their input order. */
int orc_sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in,
                   uint32_t *keys_out, uint32_t *vals_out, uint64_t n, int dtype)
{
    if (!vals_in || !vals_out)
        return -1;
    return sort_impl(keys_in, vals_in, keys_out, vals_out, n, dtype);
}

/* ---- multi-threaded variant, the CPU baseline's second figure ----------
 * The same sort on `threads` host threads, parallelised the plain way: the
 * array is cut into `threads` chunks that the threads sort on their own
 * (sort_impl), then ceil(log2(threads)) rounds merge neighbouring sorted
 * chunks pairwise (merge_runs, left chunk first on ties), each merge of a
 * round in its own thread.  A stable merge of stably sorted neighbours is
 * the stable sort, so the result equals orc_sort_keys; the tests check that. */
struct par_job {
    const uint32_t *src;
    uint32_t *dst;
    uint64_t lo, mid, hi;
    int dtype, rc;
};

static void *par_sort_chunk(void *arg)
{
    struct par_job *j = arg;
    j->rc = sort_impl(j->src + j->lo, NULL, j->dst + j->lo, NULL, j->hi - j->lo, j->dtype);
    return NULL;
}

static void *par_merge(void *arg)
{
    struct par_job *j = arg;
    merge_runs(j->src, NULL, j->dst, NULL, j->lo, j->mid, j->hi, j->dtype);
    j->rc = 0;
    return NULL;
}

/* Runs fn on every job, one thread each; returns 0, or -4 when a thread
 * cannot be started, or the first job's nonzero rc. */
static int par_run(void *(*fn)(void *), struct par_job *jobs, int count)
{
    pthread_t *tid = malloc((size_t)count * sizeof(pthread_t));
    int started = 0, rc = 0;
    if (!tid)
        return -2;
    for (; started < count; started++)
        if (pthread_create(&tid[started], NULL, fn, &jobs[started]) != 0) {
            rc = -4;
            break;
        }
    for (int i = 0; i < started; i++)
        pthread_join(tid[i], NULL);
    free(tid);
    for (int i = 0; rc == 0 && i < started; i++)
        rc = jobs[i].rc;
    return rc;
}

/* Keys only, on `threads` threads (1..256).  Returns 0, -1 on a bad dtype or
 * thread count, -2 when memory cannot be allocated, -4 when a thread cannot
 * be started. */
int orc_sort_keys_par(const uint32_t *keys_in, uint32_t *keys_out, uint64_t n, int dtype,
                      int threads)
{
    if (dtype != ORC_U32 && dtype != ORC_I32 && dtype != ORC_F32)
        return -1;
    if (threads < 1 || threads > 256)
        return -1;
    if (n == 0)
        return 0;
    uint64_t bound[257];
    for (int i = 0; i <= threads; i++)
        bound[i] = n * (uint64_t)i / (uint64_t)threads;
    uint32_t *a = malloc(n * sizeof(uint32_t));
    uint32_t *b = malloc(n * sizeof(uint32_t));
    struct par_job *jobs = malloc((size_t)threads * sizeof(struct par_job));
    int rc = 0;
    if (!a || !b || !jobs) {
        rc = -2;
        goto out;
    }
    for (int i = 0; i < threads; i++) {
        jobs[i].src = keys_in;
        jobs[i].dst = a;
        jobs[i].lo = bound[i];
        jobs[i].hi = bound[i + 1];
        jobs[i].dtype = dtype;
    }
    rc = par_run(par_sort_chunk, jobs, threads);
    for (int w = 1; rc == 0 && w < threads; w *= 2) {
        int count = 0;
        for (int c = 0; c < threads; c += 2 * w) {
            const int m = c + w < threads ? c + w : threads;
            const int e = c + 2 * w < threads ? c + 2 * w : threads;
            jobs[count].src = a;
            jobs[count].dst = b;
            jobs[count].lo = bound[c];
            jobs[count].mid = bound[m];
            jobs[count].hi = bound[e];
            jobs[count].dtype = dtype;
            count++;
        }
        rc = par_run(par_merge, jobs, count);
        uint32_t *t = a;
        a = b;
        b = t;
    }
    if (rc == 0)
        memcpy(keys_out, a, n * sizeof(uint32_t));
out:
    free(a);
    free(b);
    free(jobs);
    return rc;
}

/* Segmented: each [offsets[s], offsets[s+1]) is sorted on its own; segments
 * never mix.  offsets has nseg+1 entries, offsets[0] == 0, non-decreasing.
 * vals_in / vals_out may both be NULL (keys only).  Returns -3 on malformed
 * offsets. */
int orc_sort_segmented(const uint32_t *keys_in, const uint32_t *vals_in,
                       uint32_t *keys_out, uint32_t *vals_out,
                       const int64_t *offsets, uint64_t nseg, int dtype)
{
    if (offsets[0] != 0)
        return -3;
    for (uint64_t s = 0; s < nseg; s++)
        if (offsets[s + 1] < offsets[s])
            return -3;
    if ((vals_in == NULL) != (vals_out == NULL))
        return -1;
    for (uint64_t s = 0; s < nseg; s++) {
        uint64_t lo = (uint64_t)offsets[s], len = (uint64_t)(offsets[s + 1] - offsets[s]);
        int rc = sort_impl(keys_in + lo, vals_in ? vals_in + lo : NULL,
                           keys_out + lo, vals_out ? vals_out + lo : NULL, len, dtype);
        if (rc != 0)
            return rc;
    }
    return 0;
}

/* ---- 64-bit keys ------------------------------------------------------ */

enum { ORC_U64 = 3, ORC_I64 = 4, ORC_F64 = 5 };

/* The order-preserving map on 64-bit patterns, with the rules of orc_key:
 * u64 identity; i64 sign bit flipped; f64 negatives complemented and
 * non-negatives given the sign bit (IEEE totalOrder for binary64). */
uint64_t orc_key64(uint64_t bits, int dtype)
{
    const uint64_t sign = (uint64_t)1 << 63;
    if (dtype == ORC_U64)
        return bits;
    if (dtype == ORC_I64)
        return bits ^ sign;
    if (dtype == ORC_F64) {
        if (bits & sign)
            return ~bits;
        return bits ^ sign;
    }
    return 0;
}

void orc_key64_array(const uint64_t *bits, uint64_t *keys, uint64_t n, int dtype)
{
    for (uint64_t i = 0; i < n; i++)
        keys[i] = orc_key64(bits[i], dtype);
}

/* Merges sorted src[lo, mid) and src[mid, hi) into dst[lo, hi), left run
 * first on equal keys. */
static void merge_runs64(const uint64_t *src, uint64_t *dst, uint64_t lo, uint64_t mid,
                         uint64_t hi, int dtype)
{
    uint64_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        if (orc_key64(src[j], dtype) < orc_key64(src[i], dtype))
            dst[o++] = src[j++];
        else
            dst[o++] = src[i++];
    }
    while (i < mid)
        dst[o++] = src[i++];
    while (j < hi)
        dst[o++] = src[j++];
}

/* Keys only: out = the input 64-bit patterns in ascending orc_key64 order,
 * by the bottom-up merge sort.  Returns 0, -1 on a bad dtype, -2 when
 * scratch memory cannot be allocated. */
int orc_sort_keys64(const uint64_t *keys_in, uint64_t *keys_out, uint64_t n, int dtype)
{
    if (dtype != ORC_U64 && dtype != ORC_I64 && dtype != ORC_F64)
        return -1;
    if (n == 0)
        return 0;
    uint64_t *a = malloc(n * sizeof(uint64_t));
    uint64_t *b = malloc(n * sizeof(uint64_t));
    if (!a || !b) {
        free(a); free(b);
        return -2;
    }
    memcpy(a, keys_in, n * sizeof(uint64_t));
    for (uint64_t width = 1; width < n; width *= 2) {
        for (uint64_t lo = 0; lo < n; lo += 2 * width) {
            uint64_t mid = lo + width < n ? lo + width : n;
            uint64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            merge_runs64(a, b, lo, mid, hi, dtype);
        }
        uint64_t *t = a; a = b; b = t;
    }
    memcpy(keys_out, a, n * sizeof(uint64_t));
    free(a); free(b);
    return 0;
}
