/*
 * Seeded synthetic workloads for the COBS query path: DNA and text documents,
 * query sets and arrival times.  This file holds none of the index or query
 * arithmetic: it only draws bytes and lengths.  Both the CUDA library and the
 * CPU oracle consume what it produces.
 *
 * Random numbers: every item (document, query, vocabulary word) draws from its
 * own stream, seeded as splitmix64(seed, item), then xoshiro256** (Blackman and
 * Vigna, "Scrambled linear pseudorandom number generators", 2018), both written
 * from their published definitions.  Items are therefore independent of the
 * order in which they are generated, and documents can be filled in parallel.
 *
 * Stand-in for the paper's corpora (Sec. 3, "Data" and "Queries"): the
 * McCortex microbial documents and the unitig-derived query sets are not
 * available, so documents are i.i.d. uniform ACGT strings (or Zipf text) with
 * log-normal lengths, and queries are mutated substrings or uniform strings.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* Stream for item `id` of a run seeded with `seed` (and a sub-stream tag). */
static void rng_stream(rng_t *r, uint64_t seed, uint64_t tag, uint64_t id) {
    uint64_t x = seed;
    uint64_t a = splitmix64_next(&x);
    x = a ^ (tag * 0xd1b54a32d192ed03ULL);
    uint64_t b = splitmix64_next(&x);
    x = b ^ (id * 0x9e3779b97f4a7c15ULL) ^ 0x2545f4914f6cdd1dULL;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

/* Uniform double in [0, 1) from the top 53 bits. */
static double rng_uniform(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* Uniform integer in [0, n), n >= 1 (multiply-shift; bias below 2^-32 for our n). */
static uint64_t rng_below(rng_t *r, uint64_t n) {
    unsigned __int128 m = (unsigned __int128)rng_next(r) * n;
    return (uint64_t)(m >> 64);
}

/* Standard normal by the Box-Muller transform. */
static double rng_normal(rng_t *r) {
    double u1 = 1.0 - rng_uniform(r); /* (0, 1] */
    double u2 = rng_uniform(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static uint64_t lognormal_len(rng_t *r, double median, double sigma, uint64_t lo, uint64_t hi) {
    double v = exp(log(median) + sigma * rng_normal(r));
    if (v < (double)lo) v = (double)lo;
    if (v > (double)hi) v = (double)hi;
    uint64_t L = (uint64_t)llround(v);
    if (L < lo) L = lo;
    if (L > hi) L = hi;
    return L;
}

static const char ACGT[4] = {'A', 'C', 'G', 'T'};

/* Stream tags, one per kind of item. */
enum { TAG_DOC_LEN = 1, TAG_DOC = 2, TAG_QUERY = 3, TAG_VOCAB = 4, TAG_ARRIVAL = 5, TAG_THR = 6 };

/* ---------------------------------------------------------------- lengths */

void synth_lengths_lognormal(uint64_t seed, uint64_t n, double median, double sigma,
                             uint64_t lo, uint64_t hi, uint64_t *out_len) {
    for (uint64_t i = 0; i < n; i++) {
        rng_t r;
        rng_stream(&r, seed, TAG_DOC_LEN, i);
        out_len[i] = lognormal_len(&r, median, sigma, lo, hi);
    }
}

/* ------------------------------------------------------- parallel filling */

typedef struct {
    int kind; /* 0 dna, 1 text */
    uint64_t seed, n;
    const uint64_t *offsets;
    uint8_t *out;
    /* text */
    const uint8_t *vocab;
    const uint64_t *vocab_off;
    const double *zipf_cdf;
    uint64_t n_words;
    /* work sharing */
    uint64_t next;
    pthread_mutex_t mu;
} fill_job;

static void fill_dna_doc(const fill_job *j, uint64_t d) {
    rng_t r;
    rng_stream(&r, j->seed, TAG_DOC, d);
    uint8_t *p = j->out + j->offsets[d];
    uint64_t L = j->offsets[d + 1] - j->offsets[d];
    uint64_t i = 0;
    while (i < L) {
        uint64_t x = rng_next(&r);
        for (int k = 0; k < 32 && i < L; k++, i++) {
            p[i] = (uint8_t)ACGT[x & 3];
            x >>= 2;
        }
    }
}

static uint64_t zipf_draw(rng_t *r, const double *cdf, uint64_t n) {
    double u = rng_uniform(r);
    uint64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        uint64_t mid = (lo + hi) / 2;
        if (cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

static void fill_text_doc(const fill_job *j, uint64_t d) {
    rng_t r;
    rng_stream(&r, j->seed, TAG_DOC, d);
    uint8_t *p = j->out + j->offsets[d];
    uint64_t L = j->offsets[d + 1] - j->offsets[d];
    uint64_t i = 0;
    while (i < L) {
        if (i > 0) p[i++] = ' ';
        uint64_t w = zipf_draw(&r, j->zipf_cdf, j->n_words);
        const uint8_t *ws = j->vocab + j->vocab_off[w];
        uint64_t wl = j->vocab_off[w + 1] - j->vocab_off[w];
        for (uint64_t k = 0; k < wl && i < L; k++) p[i++] = ws[k];
    }
}

static void *fill_worker(void *arg) {
    fill_job *j = (fill_job *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        uint64_t d0 = j->next;
        j->next += 16;
        pthread_mutex_unlock(&j->mu);
        if (d0 >= j->n) break;
        uint64_t d1 = d0 + 16 < j->n ? d0 + 16 : j->n;
        for (uint64_t d = d0; d < d1; d++) {
            if (j->kind == 0) fill_dna_doc(j, d); else fill_text_doc(j, d);
        }
    }
    return NULL;
}

static void run_fill(fill_job *j, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    j->next = 0;
    pthread_mutex_init(&j->mu, NULL);
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, fill_worker, j);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j->mu);
}

/* Document d = i.i.d. uniform ACGT bytes, offsets[d] .. offsets[d+1]. */
void synth_fill_dna(uint64_t seed, uint64_t n, const uint64_t *offsets, uint8_t *out, int nthreads) {
    fill_job j;
    memset(&j, 0, sizeof j);
    j.kind = 0; j.seed = seed; j.n = n; j.offsets = offsets; j.out = out;
    run_fill(&j, nthreads);
}

/* Vocabulary: n_words random lowercase words, lengths uniform in [minlen, maxlen].
 * Call with out_bytes == NULL to get the lengths (out_off[i+1]-out_off[i]) only. */
void synth_vocab(uint64_t seed, uint64_t n_words, uint32_t minlen, uint32_t maxlen,
                 uint8_t *out_bytes, uint64_t *out_off) {
    uint64_t pos = 0;
    out_off[0] = 0;
    for (uint64_t w = 0; w < n_words; w++) {
        rng_t r;
        rng_stream(&r, seed, TAG_VOCAB, w);
        uint64_t len = minlen + rng_below(&r, (uint64_t)(maxlen - minlen + 1));
        if (out_bytes)
            for (uint64_t k = 0; k < len; k++) out_bytes[pos + k] = (uint8_t)('a' + rng_below(&r, 26));
        pos += len;
        out_off[w + 1] = pos;
    }
}

/* Zipf(s) over ranks 1..n: cumulative distribution, cdf[n-1] == 1. */
void synth_zipf_cdf(uint64_t n, double s, double *cdf) {
    double acc = 0.0;
    for (uint64_t i = 0; i < n; i++) { acc += pow((double)(i + 1), -s); cdf[i] = acc; }
    for (uint64_t i = 0; i < n; i++) cdf[i] /= acc;
    cdf[n - 1] = 1.0;
}

/* Text document d: Zipf-drawn vocabulary words joined by single spaces, cut at
 * exactly its length. */
void synth_fill_text(uint64_t seed, uint64_t n, const uint64_t *offsets, const uint8_t *vocab,
                     const uint64_t *vocab_off, uint64_t n_words, const double *zipf_cdf,
                     uint8_t *out, int nthreads) {
    fill_job j;
    memset(&j, 0, sizeof j);
    j.kind = 1; j.seed = seed; j.n = n; j.offsets = offsets; j.out = out;
    j.vocab = vocab; j.vocab_off = vocab_off; j.zipf_cdf = zipf_cdf; j.n_words = n_words;
    run_fill(&j, nthreads);
}

/* ---------------------------------------------------------------- queries */

/*
 * DNA query plan.  Query i < n_tp is a substring of a source document with
 * per-base substitution rate drawn uniformly from [rate_lo, rate_hi] (each base
 * substituted with probability rate by one of the 3 other bases); query
 * i >= n_tp is a uniform random ACGT string.  Length: fixed_len if nonzero,
 * else log-normal(median, sigma) clipped to [lo, hi].  The source document is
 * uniform among documents at least as long as the query; if there is none the
 * length is clipped to the longest document.
 *
 * docs_by_len: document ids sorted by length ascending (ties by id).
 * Outputs per query: out_len, out_src (-1 for random), out_start, out_rate.
 */
void synth_dna_query_plan(uint64_t seed, uint64_t n, uint64_t n_tp, uint64_t fixed_len,
                          double median, double sigma, uint64_t lo, uint64_t hi,
                          double rate_lo, double rate_hi,
                          const uint64_t *doc_off, uint64_t n_docs, const uint64_t *docs_by_len,
                          uint64_t *out_len, int64_t *out_src, uint64_t *out_start, double *out_rate) {
    uint64_t maxlen = n_docs ? doc_off[docs_by_len[n_docs - 1] + 1] - doc_off[docs_by_len[n_docs - 1]] : 0;
    for (uint64_t i = 0; i < n; i++) {
        rng_t r;
        rng_stream(&r, seed, TAG_QUERY, i);
        uint64_t L = fixed_len ? fixed_len : lognormal_len(&r, median, sigma, lo, hi);
        out_rate[i] = 0.0;
        out_start[i] = 0;
        if (i < n_tp && n_docs > 0) {
            if (L > maxlen) L = maxlen;
            /* first index in docs_by_len whose length >= L */
            uint64_t a = 0, b = n_docs;
            while (a < b) {
                uint64_t m = (a + b) / 2;
                uint64_t dl = doc_off[docs_by_len[m] + 1] - doc_off[docs_by_len[m]];
                if (dl >= L) b = m; else a = m + 1;
            }
            uint64_t d = docs_by_len[a + rng_below(&r, n_docs - a)];
            uint64_t dl = doc_off[d + 1] - doc_off[d];
            out_src[i] = (int64_t)d;
            out_start[i] = rng_below(&r, dl - L + 1);
            out_rate[i] = rate_lo + (rate_hi - rate_lo) * rng_uniform(&r);
        } else {
            out_src[i] = -1;
        }
        out_len[i] = L;
    }
}

/* Fill the bytes of a DNA query plan (lengths are preserved). */
void synth_dna_query_fill(uint64_t seed, uint64_t n, const uint8_t *docs, const uint64_t *doc_off,
                          const int64_t *src, const uint64_t *start, const double *rate,
                          const uint64_t *q_off, uint8_t *out) {
    for (uint64_t i = 0; i < n; i++) {
        rng_t r;
        rng_stream(&r, seed ^ 0x5bd1e995ULL, TAG_QUERY, i);
        uint8_t *p = out + q_off[i];
        uint64_t L = q_off[i + 1] - q_off[i];
        if (src[i] >= 0) {
            const uint8_t *s = docs + doc_off[src[i]] + start[i];
            for (uint64_t k = 0; k < L; k++) {
                uint8_t c = s[k];
                if (rate[i] > 0.0 && rng_uniform(&r) < rate[i]) {
                    int b = c == 'A' ? 0 : c == 'C' ? 1 : c == 'G' ? 2 : 3;
                    b = (b + 1 + (int)rng_below(&r, 3)) & 3;
                    c = (uint8_t)ACGT[b];
                }
                p[k] = c;
            }
        } else {
            for (uint64_t k = 0; k < L; k++) p[k] = (uint8_t)ACGT[rng_next(&r) & 3];
        }
    }
}

/*
 * Text queries: query i is a substring of a uniformly drawn document, length
 * uniform in [len_lo, len_hi] (clipped to the document), then edited: every
 * position independently with probability edit_rate gets one edit, uniformly a
 * substitution, an insertion before it or a deletion, with a random lowercase
 * letter.  Output capacity must be at least 2 * sum of lengths (len_hi * 2 * n
 * is always enough).  Returns the number of bytes written; q_off has n+1 entries.
 */
uint64_t synth_text_queries(uint64_t seed, uint64_t n, uint64_t len_lo, uint64_t len_hi, double edit_rate,
                            const uint8_t *docs, const uint64_t *doc_off, uint64_t n_docs,
                            int64_t *out_src, uint8_t *out, uint64_t *q_off) {
    uint64_t pos = 0;
    q_off[0] = 0;
    for (uint64_t i = 0; i < n; i++) {
        rng_t r;
        rng_stream(&r, seed, TAG_QUERY, i);
        uint64_t L = len_lo + rng_below(&r, len_hi - len_lo + 1);
        uint64_t d = rng_below(&r, n_docs);
        uint64_t dl = doc_off[d + 1] - doc_off[d];
        if (L > dl) L = dl;
        uint64_t st = rng_below(&r, dl - L + 1);
        const uint8_t *s = docs + doc_off[d] + st;
        out_src[i] = (int64_t)d;
        for (uint64_t k = 0; k < L; k++) {
            if (rng_uniform(&r) < edit_rate) {
                uint64_t e = rng_below(&r, 3);
                uint8_t letter = (uint8_t)('a' + rng_below(&r, 26));
                if (e == 0) { out[pos++] = letter; continue; }             /* substitute */
                if (e == 1) { out[pos++] = letter; out[pos++] = s[k]; continue; } /* insert */
                continue;                                                   /* delete */
            }
            out[pos++] = s[k];
        }
        q_off[i + 1] = pos;
    }
    return pos;
}

/* Poisson arrivals: exponential gaps at `rate` per second, times in seconds. */
void synth_arrivals(uint64_t seed, uint64_t n, double rate, double *out_t) {
    rng_t r;
    rng_stream(&r, seed, TAG_ARRIVAL, 0);
    double t = 0.0;
    for (uint64_t i = 0; i < n; i++) {
        t += -log(1.0 - rng_uniform(&r)) / rate;
        out_t[i] = t;
    }
}

/* Per-query thresholds drawn uniformly from a list of permille values. */
void synth_choice_u16(uint64_t seed, uint64_t n, const uint16_t *choices, uint32_t n_choices, uint16_t *out) {
    for (uint64_t i = 0; i < n; i++) {
        rng_t r;
        rng_stream(&r, seed, TAG_THR, i);
        out[i] = choices[rng_below(&r, n_choices)];
    }
}
