/*
 * Huskysort oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct CPU reference for what the GPU path computes.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  It shares no code, header or constant table with
 * the CUDA library; the two are compiled from disjoint sources.
 *
 * Contents
 *   oracle_string_to_long   Algorithm 4 (stringToLong), literally.
 *   oracle_unicode_to_long  The Unicode coder (Section 4.3): Algorithm 4 over
 *                           UTF-16 code units, 4 x 16 bits, then >>> 1.
 *   oracle_encode           Algorithms 2/3 (huskyEncode over an array, with
 *                           the per-element perfection test).
 *   oracle_stable_argsort   The result the whole method must reach: the stable
 *                           argsort of the strings under unsigned-byte
 *                           lexicographic order (Section 3.1 Step 3: the final
 *                           Timsort pass is stable; a proper prefix is smaller).
 *   oracle_check_sorted     Property check usable at any size: a permutation
 *                           that is sorted and stable on ties is THE stable
 *                           argsort (unique), so this pins results too large to
 *                           re-sort on the host.
 *
 * Readings of the paper taken here:
 *   - a "char" is one byte of the input buffer (charAt on ASCII text);
 *   - perfectForLength(len) is undefined in the paper; an element is exactly
 *     represented iff len <= maxLength and (len == 0 or its last byte != 0),
 *     because "a" and "a\0" share a code;
 *   - Java shifts are taken mod 64; the only shift that can reach 64 here is
 *     the padding shift of an empty string, whose result is 0 either way.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Algorithm 4: pack min(len, max_length) chars, bit_width bits each, most
 * significant first, each ANDed with mask when mask != 0, then shift left by
 * bit_width * padding so that short strings are zero-padded on the right. */
uint64_t oracle_string_to_long(const uint8_t *s, uint64_t len, int max_length,
                               int bit_width, uint64_t mask)
{
    uint64_t length = len < (uint64_t)max_length ? len : (uint64_t)max_length;
    uint64_t padding = (uint64_t)max_length - length;
    uint64_t result = 0;
    for (uint64_t i = 0; i < length; i++) {
        uint64_t c = s[i];
        if (mask != 0)
            c = c & mask;
        result = (result << bit_width) | c;
    }
    uint64_t shift = (uint64_t)bit_width * padding;
    if (shift >= 64)
        result = 0; /* only reached when length == 0, where result is 0 */
    else
        result = result << shift;
    return result;
}

/* Algorithm 4 over 16-bit chars (a Java String's UTF-16 code units). */
uint64_t oracle_units_to_long(const uint16_t *u, uint64_t len, int max_length,
                              int bit_width, uint64_t mask)
{
    uint64_t length = len < (uint64_t)max_length ? len : (uint64_t)max_length;
    uint64_t padding = (uint64_t)max_length - length;
    uint64_t result = 0;
    for (uint64_t i = 0; i < length; i++) {
        uint64_t c = u[i];
        if (mask != 0)
            c = c & mask;
        result = (result << bit_width) | c;
    }
    uint64_t shift = (uint64_t)bit_width * padding;
    if (shift >= 64)
        result = 0;
    else
        result = result << shift;
    return result;
}

/* The paper's Unicode coder (Section 4.3, unicodeToLong and its constants):
 * 16 bits x 64/16 = 4 code units with mask 0xFFFF, then an unsigned shift
 * right by one so that Java's signed long compare keeps the order. */
uint64_t oracle_unicode_to_long(const uint16_t *u, uint64_t len)
{
    return oracle_units_to_long(u, len, 64 / 16, 16, 0xFFFF) >> 1;
}

/* Coder constants (Section 4.3 "Constants" listing): ASCII uses 7 bits per
 * char and 64/7 = 9 chars with mask 0x7F.  BYTE8 (8 bits x 8 chars, no mask)
 * is this project's order-preserving coder for arbitrary bytes. */
enum { ORACLE_CODER_ASCII7 = 1, ORACLE_CODER_BYTE8 = 2 };

static void coder_params(int coder, int *max_length, int *bit_width,
                         uint64_t *mask)
{
    if (coder == ORACLE_CODER_BYTE8) {
        *max_length = 64 / 8;
        *bit_width = 8;
        *mask = 0;
    } else {
        *max_length = 64 / 7;
        *bit_width = 7;
        *mask = 0x7F;
    }
}

/* perfectForLength (Algorithm 3), in this project's reading. */
static int exactly_represented(const uint8_t *s, uint64_t len, int max_length)
{
    if (len > (uint64_t)max_length)
        return 0;
    if (len == 0)
        return 1;
    return s[len - 1] != 0;
}

/* Algorithms 2/3: encode every element; *perfect = all elements exact.
 * exact_out (nullable) receives the per-element flag.  Returns 0. */
int oracle_encode(const uint8_t *bytes, const uint64_t *offsets, uint64_t n,
                  int coder, uint64_t *codes_out, uint8_t *exact_out,
                  int *perfect)
{
    int max_length, bit_width;
    uint64_t mask;
    coder_params(coder, &max_length, &bit_width, &mask);
    int is_perfect = 1;
    for (uint64_t i = 0; i < n; i++) {
        const uint8_t *s = bytes + offsets[i];
        uint64_t len = offsets[i + 1] - offsets[i];
        int ex = exactly_represented(s, len, max_length);
        if (!ex)
            is_perfect = 0;
        if (exact_out)
            exact_out[i] = (uint8_t)ex;
        codes_out[i] = oracle_string_to_long(s, len, max_length, bit_width, mask);
    }
    if (perfect)
        *perfect = is_perfect;
    return 0;
}

/* ---- byte-range coder -------------------------------------------------------
 * The paper notes (Section 3.2, on perfect encodings) that case-independent
 * English letters fit 5 bits and case-dependent ones 6 bits, so that more
 * characters fit in a code.  This project's coder generalises that: with lo
 * and hi the smallest and largest byte in the string data, byte c codes as
 * c - lo + 1 (0 stays the padding), packed by Algorithm 4 with bit_width
 * w = ceil(log2(hi - lo + 2)) in place of the 7-bit mask ('a'..'z': 26
 * values, 5 bits; 'A'..'z': 58 values, 6 bits).  The map keeps byte order and
 * the padding stays below every value, so the code is order preserving.
 * max_length K is a parameter.  The paper's own choice is the longest K that
 * fits 64 bits, K = floor(64 / w): 12 case-independent letters in 5 bits, 10
 * case-dependent ones in 6 bits, each string of up to K letters coded
 * perfectly.  The GPU library codes K = 8 (as many characters as BYTE8), a
 * sort key of 8*w + 1 bits (41 for letters: five 9-bit radix digits where 12
 * letters would take seven) and leaves longer strings to Step 3.  Defined for
 * w <= 6; a string is exactly represented iff its length is at most K (a NUL
 * byte inside the range has a value of its own). */

/* Algorithm 4 with a character map in place of the mask. */
uint64_t oracle_string_to_long_mapped(const uint8_t *s, uint64_t len, int max_length,
                                      int bit_width, const uint8_t *map)
{
    uint64_t length = len < (uint64_t)max_length ? len : (uint64_t)max_length;
    uint64_t padding = (uint64_t)max_length - length;
    uint64_t result = 0;
    for (uint64_t i = 0; i < length; i++)
        result = (result << bit_width) | map[s[i]];
    uint64_t shift = (uint64_t)bit_width * padding;
    return shift >= 64 ? 0 : result << shift;
}

/* Byte range of bytes[offsets[0] .. offsets[n]) and the coder parameters.
 * map_out[c] = c - lo + 1 inside the range, 0 outside.  k_req: the K to use,
 * or 0 for the paper's floor(64 / w).  Returns 0 when w <= 6 and K * w <= 64,
 * else 1 (the coder does not apply; the outputs are still written). */
int oracle_alpha_params_k(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, int k_req,
                          uint8_t *map_out, int *w_out, int *k_out)
{
    int lo = 255, hi = 0;
    if (n > 0)
        for (uint64_t q = offsets[0]; q < offsets[n]; q++) {
            if (bytes[q] < lo)
                lo = bytes[q];
            if (bytes[q] > hi)
                hi = bytes[q];
        }
    if (hi < lo)  /* no bytes at all */
        lo = hi = 0;
    int span = hi - lo + 1;
    for (int c = 0; c < 256; c++)
        map_out[c] = (c >= lo && c <= hi) ? (uint8_t)(c - lo + 1) : 0;
    int w = 1;
    while ((1 << w) < span + 1)
        w++;
    int k = k_req > 0 ? k_req : 64 / w;
    *w_out = w;
    *k_out = k;
    return (w <= 6 && k >= 1 && k * w <= 64) ? 0 : 1;
}

/* The GPU library's parameters: K = 8. */
int oracle_alpha_params(const uint8_t *bytes, const uint64_t *offsets, uint64_t n,
                        uint8_t *map_out, int *w_out, int *k_out)
{
    return oracle_alpha_params_k(bytes, offsets, n, 8, map_out, w_out, k_out);
}

/* Encode with the byte-range coder at max_length k_req (0: floor(64 / w));
 * returns 1 (nothing written) when it does not apply. */
int oracle_encode_alpha_k(const uint8_t *bytes, const uint64_t *offsets, uint64_t n, int k_req,
                          uint64_t *codes_out, uint8_t *exact_out, int *perfect,
                          int *w_out, int *k_out)
{
    uint8_t map[256];
    int w, k;
    if (oracle_alpha_params_k(bytes, offsets, n, k_req, map, &w, &k) != 0) {
        *w_out = w;
        *k_out = k;
        return 1;
    }
    int is_perfect = 1;
    for (uint64_t i = 0; i < n; i++) {
        const uint8_t *str = bytes + offsets[i];
        uint64_t len = offsets[i + 1] - offsets[i];
        int ex = len <= (uint64_t)k;
        if (!ex)
            is_perfect = 0;
        if (exact_out)
            exact_out[i] = (uint8_t)ex;
        codes_out[i] = oracle_string_to_long_mapped(str, len, k, w, map);
    }
    if (perfect)
        *perfect = is_perfect;
    *w_out = w;
    *k_out = k;
    return 0;
}

int oracle_encode_alpha(const uint8_t *bytes, const uint64_t *offsets, uint64_t n,
                        uint64_t *codes_out, uint8_t *exact_out, int *perfect,
                        int *w_out, int *k_out)
{
    return oracle_encode_alpha_k(bytes, offsets, n, 8, codes_out, exact_out, perfect, w_out, k_out);
}

/* Unsigned-byte lexicographic comparison; a proper prefix is smaller. */
static int string_compare(const uint8_t *bytes, const uint64_t *offsets,
                          uint64_t i, uint64_t j)
{
    uint64_t la = offsets[i + 1] - offsets[i];
    uint64_t lb = offsets[j + 1] - offsets[j];
    uint64_t m = la < lb ? la : lb;
    int c = memcmp(bytes + offsets[i], bytes + offsets[j], (size_t)m);
    if (c != 0)
        return c < 0 ? -1 : 1;
    if (la < lb)
        return -1;
    if (la > lb)
        return 1;
    return 0;
}

/* Public for tests: sign of the comparison of strings i and j. */
int oracle_string_compare(const uint8_t *bytes, const uint64_t *offsets,
                          uint64_t i, uint64_t j)
{
    return string_compare(bytes, offsets, i, j);
}

/* ---- stable merge sort of an index array ------------------------------- */

typedef struct {
    const uint8_t *bytes;
    const uint64_t *offsets;
} str_ctx;

/* Merge a[lo..mid) and a[mid..hi) into tmp, left side first on ties, which is
 * what makes merge sort stable. */
static void merge_runs(const str_ctx *c, uint64_t *a, uint64_t *tmp,
                       uint64_t lo, uint64_t mid, uint64_t hi)
{
    uint64_t i = lo, j = mid, k = lo;
    while (i < mid && j < hi) {
        if (string_compare(c->bytes, c->offsets, a[j], a[i]) < 0)
            tmp[k++] = a[j++];
        else
            tmp[k++] = a[i++];
    }
    while (i < mid)
        tmp[k++] = a[i++];
    while (j < hi)
        tmp[k++] = a[j++];
    memcpy(a + lo, tmp + lo, (size_t)(hi - lo) * sizeof(uint64_t));
}

/* Bottom-up merge sort of a[lo..hi): widths 1, 2, 4, ... */
static void merge_sort(const str_ctx *c, uint64_t *a, uint64_t *tmp,
                       uint64_t lo, uint64_t hi)
{
    uint64_t n = hi - lo;
    for (uint64_t width = 1; width < n; width *= 2) {
        for (uint64_t s = lo; s < hi; s += 2 * width) {
            uint64_t mid = s + width;
            if (mid >= hi)
                break;
            uint64_t e = mid + width < hi ? mid + width : hi;
            merge_runs(c, a, tmp, s, mid, e);
        }
    }
}

typedef struct {
    const str_ctx *c;
    uint64_t *a, *tmp;
    uint64_t lo, hi;
} sort_job;

static void *sort_job_run(void *p)
{
    sort_job *j = (sort_job *)p;
    merge_sort(j->c, j->a, j->tmp, j->lo, j->hi);
    return NULL;
}

typedef struct {
    const str_ctx *c;
    uint64_t *a, *tmp;
    uint64_t lo, mid, hi;
} merge_job;

static void *merge_job_run(void *p)
{
    merge_job *j = (merge_job *)p;
    merge_runs(j->c, j->a, j->tmp, j->lo, j->mid, j->hi);
    return NULL;
}

/* Stable argsort: perm receives the string indices in ascending order, equal
 * strings in input order.  The index array starts as 0..n-1 and is merge
 * sorted; with `threads` > 1, contiguous chunks are sorted concurrently and
 * then merged pairwise (lower chunk first on ties), which is still exactly a
 * stable merge sort.  perm_u64 selects a uint64 (1) or uint32 (0) output.
 * Returns 0, or -1 when memory runs out. */
int oracle_stable_argsort(const uint8_t *bytes, const uint64_t *offsets,
                          uint64_t n, void *perm, int perm_u64, int threads)
{
    if (n == 0)
        return 0;
    uint64_t *a = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint64_t *tmp = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    if (!a || !tmp) {
        free(a);
        free(tmp);
        return -1;
    }
    for (uint64_t i = 0; i < n; i++)
        a[i] = i;
    str_ctx c = {bytes, offsets};
    if (threads < 1)
        threads = 1;
    if ((uint64_t)threads > n)
        threads = (int)n;
    if (threads > 256)
        threads = 256;

    uint64_t bounds[257];
    for (int t = 0; t <= threads; t++)
        bounds[t] = n * (uint64_t)t / (uint64_t)threads;

    if (threads == 1) {
        merge_sort(&c, a, tmp, 0, n);
    } else {
        pthread_t tid[256];
        sort_job jobs[256];
        for (int t = 0; t < threads; t++) {
            jobs[t] = (sort_job){&c, a, tmp, bounds[t], bounds[t + 1]};
            pthread_create(&tid[t], NULL, sort_job_run, &jobs[t]);
        }
        for (int t = 0; t < threads; t++)
            pthread_join(tid[t], NULL);
        /* Pairwise merge tree over the sorted chunks. */
        int chunks = threads;
        while (chunks > 1) {
            merge_job mj[128];
            int pairs = 0, out = 0;
            for (int t = 0; t + 1 < chunks; t += 2) {
                mj[pairs] = (merge_job){&c, a, tmp, bounds[t], bounds[t + 1],
                                        bounds[t + 2]};
                pthread_create(&tid[pairs], NULL, merge_job_run, &mj[pairs]);
                pairs++;
            }
            for (int p = 0; p < pairs; p++)
                pthread_join(tid[p], NULL);
            for (int t = 0; t < chunks; t += 2)
                bounds[out++] = bounds[t];
            bounds[out] = n;
            chunks = out;
        }
    }

    if (perm_u64) {
        memcpy(perm, a, (size_t)n * sizeof(uint64_t));
    } else {
        uint32_t *p32 = (uint32_t *)perm;
        for (uint64_t i = 0; i < n; i++)
            p32[i] = (uint32_t)a[i];
    }
    free(a);
    free(tmp);
    return 0;
}

/* ---- property check ------------------------------------------------------
 *
 * perm is THE stable argsort iff
 *   (1) every entry is < n,
 *   (2) for every adjacent pair (p, q) = (perm[j-1], perm[j]):
 *       string(p) < string(q), or string(p) == string(q) and p < q.
 * (2) makes the sequence strictly increasing under the total order
 * (string, index), so no value repeats; n distinct values below n are a
 * permutation of 0..n-1; a strictly increasing arrangement under a total
 * order is unique.  Returns -1 when perm passes, else the first failing
 * position j (for a range failure, the position of the bad entry). */

typedef struct {
    const str_ctx *c;
    const void *perm;
    int perm_u64;
    uint64_t n, lo, hi;
    int64_t bad;
} check_job;

static inline uint64_t perm_at(const void *perm, int perm_u64, uint64_t j)
{
    return perm_u64 ? ((const uint64_t *)perm)[j] : ((const uint32_t *)perm)[j];
}

static void *check_job_run(void *p)
{
    check_job *j = (check_job *)p;
    j->bad = -1;
    for (uint64_t k = j->lo; k < j->hi; k++) {
        uint64_t q = perm_at(j->perm, j->perm_u64, k);
        if (q >= j->n) {
            j->bad = (int64_t)k;
            return NULL;
        }
        if (k == 0)
            continue;
        uint64_t p0 = perm_at(j->perm, j->perm_u64, k - 1);
        if (p0 >= j->n) {
            j->bad = (int64_t)(k - 1);
            return NULL;
        }
        int s = string_compare(j->c->bytes, j->c->offsets, p0, q);
        if (s > 0 || (s == 0 && !(p0 < q))) {
            j->bad = (int64_t)k;
            return NULL;
        }
    }
    return NULL;
}

int64_t oracle_check_sorted(const uint8_t *bytes, const uint64_t *offsets,
                            uint64_t n, const void *perm, int perm_u64,
                            int threads)
{
    if (n == 0)
        return -1;
    str_ctx c = {bytes, offsets};
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    if ((uint64_t)threads > n)
        threads = (int)n;
    pthread_t tid[256];
    check_job jobs[256];
    for (int t = 0; t < threads; t++) {
        jobs[t] = (check_job){&c, perm, perm_u64, n,
                              n * (uint64_t)t / (uint64_t)threads,
                              n * (uint64_t)(t + 1) / (uint64_t)threads, -1};
        pthread_create(&tid[t], NULL, check_job_run, &jobs[t]);
    }
    int64_t bad = -1;
    for (int t = 0; t < threads; t++) {
        pthread_join(tid[t], NULL);
        if (bad < 0 && jobs[t].bad >= 0)
            bad = jobs[t].bad;
    }
    return bad;
}

/* ---- batched instances ------------------------------------------------------
 *
 * Instance s owns strings seg_offsets[s] .. seg_offsets[s+1]-1; its result is
 * the stable argsort of those strings alone, as local indices (0-based within
 * the instance), stored at positions seg_offsets[s] .. seg_offsets[s+1]-1.
 * Threads take instances in turn; each instance is sorted exactly as
 * oracle_stable_argsort sorts a whole input. */

typedef struct {
    const uint8_t *bytes;
    const uint64_t *offsets;
    const uint64_t *seg;
    uint64_t num_segs;
    uint32_t *perm;
    const uint32_t *cperm;
    int tid, threads;
    int64_t bad;
    int oom;
} batch_job;

static void *batch_sort_run(void *p)
{
    batch_job *j = (batch_job *)p;
    for (uint64_t s = (uint64_t)j->tid; s < j->num_segs; s += (uint64_t)j->threads) {
        uint64_t lo = j->seg[s], hi = j->seg[s + 1];
        uint64_t m = hi - lo;
        if (m == 0)
            continue;
        uint64_t *a = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
        uint64_t *tmp = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
        if (!a || !tmp) {
            free(a);
            free(tmp);
            j->oom = 1;
            return NULL;
        }
        for (uint64_t i = 0; i < m; i++)
            a[i] = lo + i;
        str_ctx c = {j->bytes, j->offsets};
        merge_sort(&c, a, tmp, 0, m);
        for (uint64_t i = 0; i < m; i++)
            j->perm[lo + i] = (uint32_t)(a[i] - lo);
        free(a);
        free(tmp);
    }
    return NULL;
}

int oracle_stable_argsort_batched(const uint8_t *bytes, const uint64_t *offsets,
                                  const uint64_t *seg_offsets, uint64_t num_segs,
                                  uint32_t *perm, int threads)
{
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    pthread_t tid[256];
    batch_job jobs[256];
    for (int t = 0; t < threads; t++) {
        jobs[t] = (batch_job){bytes, offsets, seg_offsets, num_segs, perm, NULL, t, threads, -1, 0};
        pthread_create(&tid[t], NULL, batch_sort_run, &jobs[t]);
    }
    int oom = 0;
    for (int t = 0; t < threads; t++) {
        pthread_join(tid[t], NULL);
        oom |= jobs[t].oom;
    }
    return oom ? -1 : 0;
}

/* Property check per instance (see oracle_check_sorted): returns -1 if every
 * instance holds its stable argsort, else the first failing global
 * position found. */
static void *batch_check_run(void *p)
{
    batch_job *j = (batch_job *)p;
    j->bad = -1;
    for (uint64_t s = (uint64_t)j->tid; s < j->num_segs; s += (uint64_t)j->threads) {
        uint64_t lo = j->seg[s], hi = j->seg[s + 1];
        uint64_t m = hi - lo;
        for (uint64_t k = 0; k < m; k++) {
            uint64_t q = j->cperm[lo + k];
            if (q >= m) {
                if (j->bad < 0 || (int64_t)(lo + k) < j->bad)
                    j->bad = (int64_t)(lo + k);
                break;
            }
            if (k == 0)
                continue;
            uint64_t p0 = j->cperm[lo + k - 1];
            int c = string_compare(j->bytes, j->offsets, lo + p0, lo + q);
            if (c > 0 || (c == 0 && !(p0 < q))) {
                if (j->bad < 0 || (int64_t)(lo + k) < j->bad)
                    j->bad = (int64_t)(lo + k);
                break;
            }
        }
    }
    return NULL;
}

int64_t oracle_check_sorted_batched(const uint8_t *bytes, const uint64_t *offsets,
                                    const uint64_t *seg_offsets, uint64_t num_segs,
                                    const uint32_t *perm, int threads)
{
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    pthread_t tid[256];
    batch_job jobs[256];
    for (int t = 0; t < threads; t++) {
        jobs[t] = (batch_job){bytes, offsets, seg_offsets, num_segs, NULL, perm, t, threads, -1, 0};
        pthread_create(&tid[t], NULL, batch_check_run, &jobs[t]);
    }
    int64_t bad = -1;
    for (int t = 0; t < threads; t++) {
        pthread_join(tid[t], NULL);
        if (jobs[t].bad >= 0 && (bad < 0 || jobs[t].bad < bad))
            bad = jobs[t].bad;
    }
    return bad;
}
