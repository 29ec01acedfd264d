/*
 * Seeded synthetic string workloads (inputs only; no sorting or encoding).
 *
 * These stand in for the Leipzig word lists the paper benchmarks on (Section
 * 4.1), which are not available.  Every random number is a pure function of
 * (seed, stream, counter) -- a SplitMix64-style counter-based generator
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014: the 64-bit finaliser with constants 0xBF58476D1CE4E5B9 and
 * 0x94D049BB133111EB) -- so the output is identical at any thread count.
 *
 * Workload kinds (the sizes and seeds are chosen by the Python wrapper):
 *   1  random lowercase strings, length U{4..12}
 *   2  English-like tokens: Zipf(1.1) draws over a vocabulary of 50,000
 *      distinct pseudo-words (letters a-z, geometric(p=0.25) length clipped
 *      to 2..15); vocabulary rank = order of first draw
 *   3  shared prefixes: one of 100 random 16-char prefixes over [0-9A-Za-z]
 *      followed by 8 random chars over the same alphabet
 *   4  lowercase strings, length U{3..20} (instances of a batched sort; the
 *      instance sizes come from gen_instance_sizes)
 *   5  skewed: first char Zipf(1.5) over 26 letters ('a' most likely), other
 *      chars uniform a-z, length round(Normal(10, 3)) clipped to 1..24
 *
 * Two-phase use: gen_offsets() writes offsets[0..n] and returns the byte total;
 * gen_bytes() then fills the byte buffer.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    return mix64(mix64(seed ^ (stream * 0xD1B54A32D192ED03ULL)) +
                 ctr * 0x9E3779B97F4A7C15ULL);
}

/* Uniform double in (0, 1]. */
static inline double unit_open0(uint64_t r)
{
    return (double)((r >> 11) + 1) * 0x1.0p-53;
}

/* Uniform double in [0, 1). */
static inline double unit01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }

/* Uniform integer in [0, k). */
static inline uint32_t below(uint64_t r, uint32_t k)
{
    return (uint32_t)(((r >> 32) * (uint64_t)k) >> 32);
}

enum {
    ST_LEN = 1,
    ST_CHAR = 2,
    ST_PICK = 3,
    ST_AUX = 4,
    ST_LEN2 = 5,
    ST_VOCAB_LEN = 6,
    ST_VOCAB_CHAR = 7,
    ST_SIZES = 8
};

#define MAX_CHARS 64 /* counter stride per string; every kind stays below */

static const char ALNUM62[] =
    "0123456789ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz";

/* ---- kind 2 vocabulary ------------------------------------------------- */

#define VOCAB_WORDS 50000
#define VOCAB_MAXLEN 15

typedef struct {
    uint8_t words[VOCAB_WORDS][VOCAB_MAXLEN];
    uint8_t lens[VOCAB_WORDS];
    double cdf[VOCAB_WORDS];
} vocab_t;

static uint64_t word_hash(const uint8_t *w, int len)
{
    uint64_t h = 0x243F6A8885A308D3ULL ^ (uint64_t)len;
    for (int i = 0; i < len; i++)
        h = mix64(h + w[i]);
    return h;
}

static vocab_t *build_vocab(uint64_t seed)
{
    vocab_t *v = (vocab_t *)calloc(1, sizeof(vocab_t));
    if (!v)
        return NULL;
    const uint32_t cap = 1u << 17; /* open-addressing table, load < 0.4 */
    int32_t *table = (int32_t *)malloc(cap * sizeof(int32_t));
    if (!table) {
        free(v);
        return NULL;
    }
    for (uint32_t i = 0; i < cap; i++)
        table[i] = -1;
    int count = 0;
    const double ln_q = log(0.75);
    for (uint64_t attempt = 0; count < VOCAB_WORDS; attempt++) {
        /* geometric(p = 0.25) on {1, 2, ...} by inversion, clipped */
        double u = unit_open0(draw(seed, ST_VOCAB_LEN, attempt));
        int len = 1 + (int)floor(log(u) / ln_q);
        if (len < 2)
            len = 2;
        if (len > VOCAB_MAXLEN)
            len = VOCAB_MAXLEN;
        uint8_t w[VOCAB_MAXLEN];
        for (int j = 0; j < len; j++)
            w[j] = (uint8_t)('a' + below(draw(seed, ST_VOCAB_CHAR,
                                               attempt * MAX_CHARS + j), 26));
        uint32_t h = (uint32_t)word_hash(w, len) & (cap - 1);
        int dup = 0;
        while (table[h] >= 0) {
            int o = table[h];
            if (v->lens[o] == len && memcmp(v->words[o], w, len) == 0) {
                dup = 1;
                break;
            }
            h = (h + 1) & (cap - 1);
        }
        if (dup)
            continue;
        table[h] = count;
        memcpy(v->words[count], w, len);
        v->lens[count] = (uint8_t)len;
        count++;
    }
    free(table);
    /* Zipf(s = 1.1) over ranks 1..50000: cdf_k = sum_{j<=k} j^-s / H */
    double acc = 0.0;
    for (int k = 0; k < VOCAB_WORDS; k++) {
        acc += pow((double)(k + 1), -1.1);
        v->cdf[k] = acc;
    }
    for (int k = 0; k < VOCAB_WORDS; k++)
        v->cdf[k] /= acc;
    v->cdf[VOCAB_WORDS - 1] = 1.0;
    return v;
}

/* First index k with cdf[k] > u. */
static int cdf_lookup(const double *cdf, int count, double u)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (cdf[mid] > u)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

/* ---- per-kind auxiliary state ------------------------------------------- */

typedef struct {
    int kind;
    uint64_t seed;
    vocab_t *vocab;          /* kind 2 */
    uint8_t prefixes[100][16]; /* kind 3 */
    double first_cdf[26];    /* kind 5 */
} gen_state;

static int state_init(gen_state *s, int kind, uint64_t seed)
{
    memset(s, 0, sizeof(*s));
    s->kind = kind;
    s->seed = seed;
    if (kind == 2) {
        s->vocab = build_vocab(seed);
        if (!s->vocab)
            return -1;
    } else if (kind == 3) {
        for (int p = 0; p < 100; p++)
            for (int j = 0; j < 16; j++)
                s->prefixes[p][j] = (uint8_t)ALNUM62[below(
                    draw(seed, ST_AUX, (uint64_t)p * MAX_CHARS + j), 62)];
    } else if (kind == 5) {
        double acc = 0.0;
        for (int k = 0; k < 26; k++) {
            acc += pow((double)(k + 1), -1.5);
            s->first_cdf[k] = acc;
        }
        for (int k = 0; k < 26; k++)
            s->first_cdf[k] /= acc;
        s->first_cdf[25] = 1.0;
    } else if (kind != 1 && kind != 4) {
        return -2;
    }
    return 0;
}

static void state_free(gen_state *s) { free(s->vocab); }

static uint64_t string_length(const gen_state *s, uint64_t i)
{
    uint64_t seed = s->seed;
    switch (s->kind) {
    case 1:
        return 4 + below(draw(seed, ST_LEN, i), 9);
    case 2: {
        int r = cdf_lookup(s->vocab->cdf, VOCAB_WORDS,
                           unit01(draw(seed, ST_PICK, i)));
        return s->vocab->lens[r];
    }
    case 3:
        return 24;
    case 4:
        return 3 + below(draw(seed, ST_LEN, i), 18);
    case 5: {
        /* Box-Muller */
        double u1 = unit_open0(draw(seed, ST_LEN, i));
        double u2 = unit01(draw(seed, ST_LEN2, i));
        double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
        double l = floor(10.0 + 3.0 * z + 0.5);
        if (l < 1.0)
            l = 1.0;
        if (l > 24.0)
            l = 24.0;
        return (uint64_t)l;
    }
    }
    return 0;
}

static void string_fill(const gen_state *s, uint64_t i, uint8_t *dst,
                        uint64_t len)
{
    uint64_t seed = s->seed;
    switch (s->kind) {
    case 1:
    case 4:
        for (uint64_t j = 0; j < len; j++)
            dst[j] = (uint8_t)('a' + below(draw(seed, ST_CHAR, i * MAX_CHARS + j), 26));
        break;
    case 2: {
        int r = cdf_lookup(s->vocab->cdf, VOCAB_WORDS,
                           unit01(draw(seed, ST_PICK, i)));
        memcpy(dst, s->vocab->words[r], len);
        break;
    }
    case 3: {
        uint32_t p = below(draw(seed, ST_PICK, i), 100);
        memcpy(dst, s->prefixes[p], 16);
        for (uint64_t j = 16; j < len; j++)
            dst[j] = (uint8_t)ALNUM62[below(draw(seed, ST_CHAR, i * MAX_CHARS + j), 62)];
        break;
    }
    case 5: {
        int r = cdf_lookup(s->first_cdf, 26, unit01(draw(seed, ST_PICK, i)));
        dst[0] = (uint8_t)('a' + r);
        for (uint64_t j = 1; j < len; j++)
            dst[j] = (uint8_t)('a' + below(draw(seed, ST_CHAR, i * MAX_CHARS + j), 26));
        break;
    }
    }
}

/* ---- threaded drivers ---------------------------------------------------- */

typedef struct {
    const gen_state *s;
    uint64_t lo, hi;
    uint64_t *offsets;
    uint8_t *bytes;
    uint64_t total;
} gen_job;

static void *lengths_job(void *p)
{
    gen_job *j = (gen_job *)p;
    uint64_t acc = 0;
    for (uint64_t i = j->lo; i < j->hi; i++) {
        uint64_t l = string_length(j->s, i);
        j->offsets[i + 1] = l; /* lengths first, prefix-summed below */
        acc += l;
    }
    j->total = acc;
    return NULL;
}

static void *prefix_job(void *p)
{
    gen_job *j = (gen_job *)p;
    uint64_t acc = j->total; /* holds this chunk's starting offset */
    for (uint64_t i = j->lo; i < j->hi; i++) {
        acc += j->offsets[i + 1];
        j->offsets[i + 1] = acc;
    }
    return NULL;
}

static void *bytes_job(void *p)
{
    gen_job *j = (gen_job *)p;
    for (uint64_t i = j->lo; i < j->hi; i++)
        string_fill(j->s, i, j->bytes + j->offsets[i],
                    j->offsets[i + 1] - j->offsets[i]);
    return NULL;
}

static int run_jobs(gen_job *jobs, int threads, void *(*fn)(void *))
{
    pthread_t tid[256];
    for (int t = 0; t < threads; t++)
        if (pthread_create(&tid[t], NULL, fn, &jobs[t]) != 0)
            return -1;
    for (int t = 0; t < threads; t++)
        pthread_join(tid[t], NULL);
    return 0;
}

static int clamp_threads(int threads, uint64_t n)
{
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    if (n < (uint64_t)threads * 4096)
        threads = (int)(n / 4096) + 1;
    return threads;
}

/* Writes offsets[0..n] and returns the total byte count (offsets[n]); a
 * negative value on error. */
int64_t gen_offsets(int kind, uint64_t seed, uint64_t n, uint64_t *offsets,
                    int threads)
{
    gen_state s;
    if (state_init(&s, kind, seed) != 0)
        return -1;
    threads = clamp_threads(threads, n);
    gen_job jobs[256];
    offsets[0] = 0;
    for (int t = 0; t < threads; t++)
        jobs[t] = (gen_job){&s, n * (uint64_t)t / (uint64_t)threads,
                            n * (uint64_t)(t + 1) / (uint64_t)threads, offsets,
                            NULL, 0};
    if (run_jobs(jobs, threads, lengths_job) != 0) {
        state_free(&s);
        return -1;
    }
    uint64_t start = 0;
    for (int t = 0; t < threads; t++) {
        uint64_t chunk = jobs[t].total;
        jobs[t].total = start;
        start += chunk;
    }
    run_jobs(jobs, threads, prefix_job);
    state_free(&s);
    return (int64_t)offsets[n];
}

int gen_bytes(int kind, uint64_t seed, uint64_t n, const uint64_t *offsets,
              uint8_t *bytes, int threads)
{
    gen_state s;
    if (state_init(&s, kind, seed) != 0)
        return -1;
    threads = clamp_threads(threads, n);
    gen_job jobs[256];
    for (int t = 0; t < threads; t++)
        jobs[t] = (gen_job){&s, n * (uint64_t)t / (uint64_t)threads,
                            n * (uint64_t)(t + 1) / (uint64_t)threads,
                            (uint64_t *)offsets, bytes, 0};
    int rc = run_jobs(jobs, threads, bytes_job);
    state_free(&s);
    return rc;
}

/* Instance sizes for a batched workload: n_s = round(exp(U[ln lo, ln hi])). */
int gen_instance_sizes(uint64_t seed, uint64_t num, double lo, double hi,
                       uint64_t *sizes)
{
    double a = log(lo), b = log(hi);
    for (uint64_t s = 0; s < num; s++) {
        double u = unit01(draw(seed, ST_SIZES, s));
        sizes[s] = (uint64_t)floor(exp(a + u * (b - a)) + 0.5);
    }
    return 0;
}

/* The vocabulary of kind 2, for inspection by tests: copies word k (up to 15
 * bytes) into out and returns its length, or -1. */
int gen_vocab_word(uint64_t seed, int k, uint8_t *out)
{
    if (k < 0 || k >= VOCAB_WORDS)
        return -1;
    vocab_t *v = build_vocab(seed);
    if (!v)
        return -1;
    int len = v->lens[k];
    memcpy(out, v->words[k], len);
    free(v);
    return len;
}
