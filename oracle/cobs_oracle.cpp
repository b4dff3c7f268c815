/*
 * CPU oracle for the COBS query path (Bingmann, Bradley, Gauger, Iqbal,
 * "COBS: a Compact Bit-Sliced Signature Index", arXiv:1905.09624).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark load it; the product
 * library never links, loads or calls it, and it shares no code with the CUDA
 * path (its own XXH64, term extraction, planner and query).
 *
 * Each function follows the paper's steps in order:
 *   Sec. 2.1  q-grams of a document (terms), Bloom filters with h hash functions,
 *             the false-positive bound (1-(1-1/w)^{hv})^h <= (1-e^{-hv/w})^h,
 *             q-gram score and threshold K, Theorem 1 and its Chernoff bound.
 *   Sec. 2.2  bit-sliced w x |D| layout; query = AND of h rows per term, ADD of the
 *             indicator vectors into scores, report scores >= K*|G_q(P)|;
 *             compact layout: documents sorted by size, blocks of B documents,
 *             one Bloom size per block, one wide hash reduced modulo each size.
 *   Sec. 2.3  xxHash of the q-grams; optional canonical k-mers; classic (ClaBS)
 *             vs compact (COBS) construction.
 *
 * Readings of points the paper leaves open (all also used by the CUDA path,
 * which implements them independently):
 *   - DNA k-mer code: 2 bits per base, A=0 C=1 G=2 T=3, first base in the most
 *     significant position; windows holding any byte other than A, C, G, T are
 *     skipped; canonical term = min(code, code of the reverse complement).
 *   - Byte q-gram (q <= 8): the q bytes as a little-endian integer (zero high bytes).
 *   - Hash i of term t: XXH64 over the 8 little-endian bytes of t, seed i.
 *   - Terms of a query or document are a set (distinct terms).
 *   - Bloom size of a block: w = max(1, ceil(-h * V / ln(1 - p^(1/h)))), V = the
 *     largest distinct-term count in the block (the Sec. 2.1 bound solved for w
 *     at fixed h), evaluated in IEEE double as written here.
 *   - Row of a block holds ceil(n_b/128)*16 bytes; document j of the block is
 *     bit (j & 7) of byte (j >> 3); padding bits are zero.
 *   - Compact order: stable sort by (distinct-term count, original id).
 *   - Threshold K given in permille; minimum score = ceil(K * l / 1000) in integers;
 *     a query with l = 0 reports nothing.
 *   - Hits sorted by score descending, then original id ascending.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace {

// ------------------------------------------------------------------ XXH64
// Written from the xxHash specification (XXH64 algorithm description).
const uint64_t P1 = 11400714785074694791ULL;
const uint64_t P2 = 14029467366897019727ULL;
const uint64_t P3 = 1609587929392839161ULL;
const uint64_t P4 = 9650029242287828579ULL;
const uint64_t P5 = 2870177450012600261ULL;

uint64_t rotl(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

uint64_t read64le(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}
uint32_t read32le(const uint8_t* p) {
    uint32_t v = 0;
    for (int i = 3; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}

uint64_t xx_round(uint64_t acc, uint64_t lane) {
    acc += lane * P2;
    acc = rotl(acc, 31);
    return acc * P1;
}
uint64_t xx_merge(uint64_t acc, uint64_t v) {
    acc ^= xx_round(0, v);
    return acc * P1 + P4;
}

uint64_t xxh64(const uint8_t* p, size_t len, uint64_t seed) {
    const uint8_t* end = p + len;
    uint64_t h;
    if (len >= 32) {
        uint64_t v1 = seed + P1 + P2, v2 = seed + P2, v3 = seed, v4 = seed - P1;
        while (p + 32 <= end) {
            v1 = xx_round(v1, read64le(p));
            v2 = xx_round(v2, read64le(p + 8));
            v3 = xx_round(v3, read64le(p + 16));
            v4 = xx_round(v4, read64le(p + 24));
            p += 32;
        }
        h = rotl(v1, 1) + rotl(v2, 7) + rotl(v3, 12) + rotl(v4, 18);
        h = xx_merge(h, v1);
        h = xx_merge(h, v2);
        h = xx_merge(h, v3);
        h = xx_merge(h, v4);
    } else {
        h = seed + P5;
    }
    h += (uint64_t)len;
    while (p + 8 <= end) {
        h ^= xx_round(0, read64le(p));
        h = rotl(h, 27) * P1 + P4;
        p += 8;
    }
    if (p + 4 <= end) {
        h ^= (uint64_t)read32le(p) * P1;
        h = rotl(h, 23) * P2 + P3;
        p += 4;
    }
    while (p < end) {
        h ^= (uint64_t)(*p) * P5;
        h = rotl(h, 11) * P1;
        p++;
    }
    h ^= h >> 33;
    h *= P2;
    h ^= h >> 29;
    h *= P3;
    h ^= h >> 32;
    return h;
}

// --------------------------------------------------------------- terms
enum { KIND_DNA_CANONICAL = 0, KIND_DNA_FORWARD = 1, KIND_BYTES = 2 };
enum { HASH_XXH64 = 0, HASH_IDENTITY = 1 };

int base_code(uint8_t c) {
    switch (c) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        default: return -1;
    }
}

bool kind_ok(int kind, int q) {
    if (kind == KIND_DNA_CANONICAL || kind == KIND_DNA_FORWARD) return q >= 1 && q <= 32;
    if (kind == KIND_BYTES) return q >= 1 && q <= 8;
    return false;
}

// All terms of one string in window order (with repeats).  Sec. 2.1: a string t
// with |t| >= q has |t|-q+1 consecutive q-grams.  Sec. 2.3: optional canonical form.
std::vector<uint64_t> string_terms(const uint8_t* s, size_t len, int kind, int q) {
    std::vector<uint64_t> out;
    if (len < (size_t)q) return out;
    for (size_t j = 0; j + q <= len; j++) {
        if (kind == KIND_BYTES) {
            uint64_t v = 0;
            for (int i = q - 1; i >= 0; i--) v = (v << 8) | s[j + i];
            out.push_back(v);
            continue;
        }
        uint64_t fwd = 0, rc = 0;
        bool ok = true;
        for (int i = 0; i < q; i++) {
            int c = base_code(s[j + i]);
            if (c < 0) { ok = false; break; }
            fwd = (fwd << 2) | (uint64_t)c;
        }
        if (!ok) continue;
        for (int i = q - 1; i >= 0; i--) {
            int c = base_code(s[j + i]);
            rc = (rc << 2) | (uint64_t)(3 - c);
        }
        out.push_back(kind == KIND_DNA_CANONICAL ? std::min(fwd, rc) : fwd);
    }
    return out;
}

// G_q(s) as a sorted set.
std::vector<uint64_t> distinct_terms(const uint8_t* s, size_t len, int kind, int q) {
    std::vector<uint64_t> t = string_terms(s, len, kind, q);
    std::sort(t.begin(), t.end());
    t.erase(std::unique(t.begin(), t.end()), t.end());
    return t;
}

uint64_t hash_term(uint64_t t, uint32_t i, int hash_kind) {
    if (hash_kind == HASH_IDENTITY) return t;
    uint8_t b[8];
    for (int k = 0; k < 8; k++) b[k] = (uint8_t)(t >> (8 * k));
    return xxh64(b, 8, (uint64_t)i);
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

struct orc_params {
    uint32_t term_kind;   // 0 DNA canonical, 1 DNA forward, 2 bytes
    uint32_t q;           // term length
    uint32_t num_hashes;  // h
    uint32_t hash_kind;   // 0 XXH64 (the method), 1 identity (test-only exact mode)
    double fpr;           // p
    uint64_t block_docs;  // B; 0 = classic
    uint64_t width_override;  // 0 = Bloom-size formula; else every block uses this w (test-only)
};

struct orc_block {
    uint64_t n_docs;      // documents in the block
    uint64_t doc_begin;   // first sorted position of the block
    uint64_t w;           // Bloom filter size = number of rows
    uint64_t rowbytes;    // bytes per row, ceil(n_docs/128)*16
    uint64_t row_offset;  // byte offset of row 0 of the block in the row storage
    uint64_t max_terms;   // V_b, largest distinct-term count in the block
};

struct orc_index {
    orc_params params;
    uint64_t n_docs;
    uint64_t n_blocks;
    std::vector<orc_block> blocks;
    std::vector<uint64_t> perm;   // sorted position -> original document id
    std::vector<uint64_t> nterms; // distinct terms per original document
    std::vector<uint8_t> rows;    // all blocks' rows, concatenated
};

uint64_t orc_xxh64(const void* data, uint64_t len, uint64_t seed) {
    return xxh64((const uint8_t*)data, (size_t)len, seed);
}

// Terms of one string in window order; returns the count (writes at most cap).
uint64_t orc_terms(const uint8_t* s, uint64_t len, uint32_t kind, uint32_t q, uint64_t* out, uint64_t cap) {
    if (!kind_ok((int)kind, (int)q)) return 0;
    std::vector<uint64_t> t = string_terms(s, (size_t)len, (int)kind, (int)q);
    for (size_t i = 0; i < t.size() && i < cap; i++) out[i] = t[i];
    return t.size();
}

// Distinct terms of one string, ascending; returns the count.
uint64_t orc_distinct_terms(const uint8_t* s, uint64_t len, uint32_t kind, uint32_t q, uint64_t* out,
                            uint64_t cap) {
    if (!kind_ok((int)kind, (int)q)) return 0;
    std::vector<uint64_t> t = distinct_terms(s, (size_t)len, (int)kind, (int)q);
    for (size_t i = 0; i < t.size() && i < cap; i++) out[i] = t[i];
    return t.size();
}

uint64_t orc_hash_term(uint64_t t, uint32_t i) { return hash_term(t, i, HASH_XXH64); }

// Sec. 2.1 bound solved for w at fixed h (see the header).
uint64_t orc_bloom_width(uint32_t h, uint64_t v, double p) {
    double x = -(double)h * (double)v / std::log(1.0 - std::pow(p, 1.0 / (double)h));
    double c = std::ceil(x);
    uint64_t w = c < 1.0 ? 1 : (uint64_t)c;
    return w;
}

// Distinct-term counts v_d of documents [d0, d1).
void orc_doc_counts(const uint8_t* docs, const uint64_t* doc_off, uint64_t d0, uint64_t d1, uint32_t kind,
                    uint32_t q, uint64_t* out_v) {
    for (uint64_t d = d0; d < d1; d++) {
        out_v[d - d0] = distinct_terms(docs + doc_off[d], (size_t)(doc_off[d + 1] - doc_off[d]), (int)kind,
                                       (int)q).size();
    }
}

// Plan the index from the per-document term counts v[0..n): classic = one block in
// input order; compact = stable sort by (v, id), blocks of B (Sec. 2.2, Sec. 2.3).
// Returns 0 on success, -1 on bad arguments.
int orc_plan(const orc_params* prm, const uint64_t* v, uint64_t n, orc_index** out) {
    if (!prm || !out || !kind_ok((int)prm->term_kind, (int)prm->q) || prm->num_hashes < 1) return -1;
    if (!(prm->fpr > 0.0 && prm->fpr < 1.0)) return -1;
    orc_index* ix = new orc_index();
    ix->params = *prm;
    ix->n_docs = n;
    ix->nterms.assign(v, v + n);
    ix->perm.resize(n);
    for (uint64_t i = 0; i < n; i++) ix->perm[i] = i;
    uint64_t B = prm->block_docs;
    if (B == 0) {
        B = n > 0 ? n : 1;
    } else {
        std::stable_sort(ix->perm.begin(), ix->perm.end(), [&](uint64_t a, uint64_t b) {
            if (v[a] != v[b]) return v[a] < v[b];
            return a < b;
        });
    }
    uint64_t off = 0;
    for (uint64_t begin = 0; begin < n; begin += B) {
        orc_block b;
        b.doc_begin = begin;
        b.n_docs = std::min(B, n - begin);
        b.max_terms = 0;
        for (uint64_t j = 0; j < b.n_docs; j++) b.max_terms = std::max(b.max_terms, v[ix->perm[begin + j]]);
        b.w = prm->width_override ? prm->width_override
                                  : orc_bloom_width(prm->num_hashes, b.max_terms, prm->fpr);
        b.rowbytes = (b.n_docs + 127) / 128 * 16;
        b.row_offset = off;
        off += b.w * b.rowbytes;
        ix->blocks.push_back(b);
    }
    ix->n_blocks = ix->blocks.size();
    ix->rows.assign(off, 0);
    *out = ix;
    return 0;
}

// Set the Bloom bits of the documents at positions [j0, j1) of block `blk`
// (Sec. 2.1: bit h_i(s) for every q-gram s and every i < h; Sec. 2.2: row-major
// bit-sliced storage).  Disjoint column ranges that are multiples of 8 touch
// disjoint bytes.
int orc_fill_columns(orc_index* ix, const uint8_t* docs, const uint64_t* doc_off, uint64_t blk, uint64_t j0,
                     uint64_t j1) {
    if (blk >= ix->n_blocks) return -1;
    const orc_block& b = ix->blocks[blk];
    if (j1 > b.n_docs) j1 = b.n_docs;
    const orc_params& P = ix->params;
    for (uint64_t j = j0; j < j1; j++) {
        uint64_t d = ix->perm[b.doc_begin + j];
        std::vector<uint64_t> T = distinct_terms(docs + doc_off[d], (size_t)(doc_off[d + 1] - doc_off[d]),
                                                 (int)P.term_kind, (int)P.q);
        for (uint64_t t : T) {
            for (uint32_t i = 0; i < P.num_hashes; i++) {
                uint64_t r = hash_term(t, i, (int)P.hash_kind) % b.w;
                ix->rows[b.row_offset + r * b.rowbytes + (j >> 3)] |= (uint8_t)(1u << (j & 7));
            }
        }
    }
    return 0;
}

// Whole build: counts, plan, bits (single-threaded).
int orc_build(const orc_params* prm, const uint8_t* docs, const uint64_t* doc_off, uint64_t n, orc_index** out) {
    if (!prm || !kind_ok((int)prm->term_kind, (int)prm->q)) return -1;
    std::vector<uint64_t> v(n);
    if (n) orc_doc_counts(docs, doc_off, 0, n, prm->term_kind, prm->q, v.data());
    int rc = orc_plan(prm, v.data(), n, out);
    if (rc) return rc;
    for (uint64_t b = 0; b < (*out)->n_blocks; b++)
        orc_fill_columns(*out, docs, doc_off, b, 0, (*out)->blocks[b].n_docs);
    return 0;
}

void orc_index_free(orc_index* ix) { delete ix; }
uint64_t orc_index_n_blocks(const orc_index* ix) { return ix->n_blocks; }
uint64_t orc_index_n_docs(const orc_index* ix) { return ix->n_docs; }
void orc_index_block(const orc_index* ix, uint64_t b, orc_block* out) { *out = ix->blocks[b]; }
const uint64_t* orc_index_perm(const orc_index* ix) { return ix->perm.data(); }
const uint64_t* orc_index_nterms(const orc_index* ix) { return ix->nterms.data(); }
uint8_t* orc_index_rows(orc_index* ix) { return ix->rows.data(); }
uint64_t orc_index_rows_bytes(const orc_index* ix) { return ix->rows.size(); }

// Scores of one query against every document, indexed by ORIGINAL document id
// (Sec. 2.2: for every distinct term, AND of the h rows, ADD into the scores).
// Returns l = |G_q(P)|.
uint64_t orc_scores(const orc_index* ix, const uint8_t* qs, uint64_t qlen, uint32_t* scores_by_id) {
    const orc_params& P = ix->params;
    std::vector<uint64_t> T = distinct_terms(qs, (size_t)qlen, (int)P.term_kind, (int)P.q);
    for (uint64_t d = 0; d < ix->n_docs; d++) scores_by_id[d] = 0;
    std::vector<uint64_t> r(P.num_hashes);
    for (const orc_block& b : ix->blocks) {
        std::vector<uint32_t> score(b.n_docs, 0);
        for (uint64_t t : T) {
            for (uint32_t i = 0; i < P.num_hashes; i++) r[i] = hash_term(t, i, (int)P.hash_kind) % b.w;
            for (uint64_t j = 0; j < b.n_docs; j++) {
                bool all = true;
                for (uint32_t i = 0; i < P.num_hashes; i++) {
                    uint8_t byte = ix->rows[b.row_offset + r[i] * b.rowbytes + (j >> 3)];
                    if (!((byte >> (j & 7)) & 1)) { all = false; break; }
                }
                if (all) score[j] += 1;
            }
        }
        for (uint64_t j = 0; j < b.n_docs; j++) scores_by_id[ix->perm[b.doc_begin + j]] = score[j];
    }
    return T.size();
}

// One query: hits with score >= ceil(K*l/1000), sorted by (score desc, id asc).
// Writes at most cap hits; returns the number of hits.  *ell = l, *min_score = threshold.
uint64_t orc_query(const orc_index* ix, const uint8_t* qs, uint64_t qlen, uint32_t thr_permille, uint64_t* ell,
                   uint64_t* min_score, uint32_t* ids, uint32_t* scores, uint64_t cap) {
    std::vector<uint32_t> s(ix->n_docs);
    uint64_t l = orc_scores(ix, qs, qlen, s.data());
    uint64_t mn = ((uint64_t)thr_permille * l + 999) / 1000;
    if (ell) *ell = l;
    if (min_score) *min_score = mn;
    if (l == 0) return 0;
    std::vector<std::pair<uint32_t, uint32_t>> hits;  // (score, id)
    for (uint64_t d = 0; d < ix->n_docs; d++)
        if (s[d] >= mn) hits.push_back({s[d], (uint32_t)d});
    std::sort(hits.begin(), hits.end(), [](const std::pair<uint32_t, uint32_t>& a,
                                           const std::pair<uint32_t, uint32_t>& b) {
        if (a.first != b.first) return a.first > b.first;
        return a.second < b.second;
    });
    for (size_t i = 0; i < hits.size() && i < cap; i++) {
        ids[i] = hits[i].second;
        scores[i] = hits[i].first;
    }
    return hits.size();
}

// Exact q-gram containment |G_q(P) ∩ G_q(d)| for every document (the lower bound
// the Bloom scores must respect, Sec. 2.2: no false negatives).
uint64_t orc_exact_scores(const uint8_t* docs, const uint64_t* doc_off, uint64_t n, uint32_t kind, uint32_t q,
                          const uint8_t* qs, uint64_t qlen, uint32_t* out) {
    std::vector<uint64_t> T = distinct_terms(qs, (size_t)qlen, (int)kind, (int)q);
    for (uint64_t d = 0; d < n; d++) {
        std::vector<uint64_t> D = distinct_terms(docs + doc_off[d], (size_t)(doc_off[d + 1] - doc_off[d]),
                                                 (int)kind, (int)q);
        uint64_t c = 0;
        for (uint64_t t : T)
            if (std::binary_search(D.begin(), D.end(), t)) c++;
        out[d] = (uint32_t)c;
    }
    return T.size();
}

// ---------------------------------------------------------------- FP theory
// log C(n, k) via lgamma.
static double log_choose(uint64_t n, uint64_t k) {
    return std::lgamma((double)n + 1.0) - std::lgamma((double)k + 1.0) - std::lgamma((double)(n - k) + 1.0);
}

// P[X >= t] for X ~ Binomial(l, p), summed in log space.  Theorem 1 (Sec. 2.1)
// states P[X > floor(K l)] = 1 - sum_{i <= floor(K l)} C(l,i) p^i (1-p)^(l-i),
// which is orc_binom_tail_ge(l, p, floor(K l) + 1).
double orc_binom_tail_ge(uint64_t l, double p, uint64_t t) {
    if (t == 0) return 1.0;
    if (t > l) return 0.0;
    if (p <= 0.0) return 0.0;
    if (p >= 1.0) return 1.0;
    double mx = -INFINITY;
    std::vector<double> lt;
    for (uint64_t i = t; i <= l; i++) {
        double v = log_choose(l, i) + (double)i * std::log(p) + (double)(l - i) * std::log1p(-p);
        lt.push_back(v);
        mx = std::max(mx, v);
    }
    double s = 0.0;
    for (double v : lt) s += std::exp(v - mx);
    return std::exp(mx) * s;
}

// Binomial pmf, for distribution checks.
double orc_binom_pmf(uint64_t l, double p, uint64_t i) {
    if (i > l) return 0.0;
    return std::exp(log_choose(l, i) + (double)i * std::log(p) + (double)(l - i) * std::log1p(-p));
}

// Chernoff bound of Sec. 2.1 for K >= p: exp(-l (K-p)^2 / (2 (1-p))).
double orc_chernoff(uint64_t l, double K, double p) {
    return std::exp(-(double)l * (K - p) * (K - p) / (2.0 * (1.0 - p)));
}

// Single-term false-positive rate of a Bloom filter, Sec. 2.1: exact form and bound.
double orc_bloom_fpr(uint32_t h, uint64_t v, uint64_t w) {
    return std::pow(1.0 - std::pow(1.0 - 1.0 / (double)w, (double)h * (double)v), (double)h);
}
double orc_bloom_fpr_bound(uint32_t h, uint64_t v, uint64_t w) {
    return std::pow(1.0 - std::exp(-(double)h * (double)v / (double)w), (double)h);
}

}  // extern "C"
