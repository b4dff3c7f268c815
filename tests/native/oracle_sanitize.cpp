// Drives the CPU oracle (oracle/cobs_oracle.cpp) over small seeded inputs with
// every term kind, classic and compact layouts and 1-3 hashes, including empty
// documents, documents shorter than a term, non-ACGT bytes and empty queries.
// The tests build it with -fsanitize=address,undefined and expect exit status 0
// and no sanitizer report; it also checks the oracle's own invariants (no false
// negatives, scores bounded by the distinct query terms, hits sorted).
#include <cstdint>
#include <cstdio>
#include <vector>

extern "C" {
struct orc_params {
    uint32_t term_kind, q, num_hashes, hash_kind;
    double fpr;
    uint64_t block_docs, width_override;
};
struct orc_index;
int orc_build(const orc_params *prm, const uint8_t *docs, const uint64_t *doc_off, uint64_t n, orc_index **out);
void orc_index_free(orc_index *ix);
uint64_t orc_query(const orc_index *ix, const uint8_t *qs, uint64_t qlen, uint32_t thr_permille, uint64_t *ell,
                   uint64_t *min_score, uint32_t *ids, uint32_t *scores, uint64_t cap);
uint64_t orc_exact_scores(const uint8_t *docs, const uint64_t *doc_off, uint64_t n, uint32_t kind, uint32_t q,
                          const uint8_t *qs, uint64_t qlen, uint32_t *out);
uint64_t orc_terms(const uint8_t *s, uint64_t len, uint32_t kind, uint32_t q, uint64_t *out, uint64_t cap);
double orc_binom_tail_ge(uint64_t l, double p, uint64_t t);
double orc_chernoff(uint64_t l, double K, double p);
}

static uint64_t g_x = 0x243F6A8885A308D3ULL;
static uint64_t rnd() {
    g_x ^= g_x << 13;
    g_x ^= g_x >> 7;
    g_x ^= g_x << 17;
    return g_x;
}

int main() {
    int errors = 0;
    const struct { uint32_t kind, q; } kinds[] = {{0, 5}, {0, 31}, {1, 7}, {2, 1}, {2, 4}, {2, 8}};
    for (auto K : kinds) {
        for (uint32_t h = 1; h <= 3; h++) {
            for (uint64_t B : {0ULL, 8ULL, 20ULL}) {
                // documents: random lengths 0..300, DNA with occasional N, or bytes
                const uint64_t n = 37;
                std::vector<uint8_t> docs;
                std::vector<uint64_t> off = {0};
                for (uint64_t d = 0; d < n; d++) {
                    const uint64_t len = rnd() % 300;
                    for (uint64_t i = 0; i < len; i++) {
                        uint64_t r = rnd();
                        docs.push_back(K.kind == 2 ? (uint8_t)(r % 7) : (r % 50 == 0 ? 'N' : "ACGT"[r & 3]));
                    }
                    off.push_back(docs.size());
                }
                orc_params P = {K.kind, K.q, h, 0, 0.3, B, 0};
                orc_index *ix = nullptr;
                if (orc_build(&P, docs.data(), off.data(), n, &ix) != 0) { errors++; continue; }
                std::vector<uint32_t> ids(n), sc(n), exact(n);
                for (int t = 0; t < 12; t++) {
                    // a substring of a document (t even) or random bytes
                    const uint64_t d = rnd() % n, dl = off[d + 1] - off[d];
                    std::vector<uint8_t> qv;
                    if (t % 2 == 0 && dl) {
                        const uint64_t a = rnd() % dl, l = rnd() % (dl - a + 1);
                        qv.assign(docs.begin() + off[d] + a, docs.begin() + off[d] + a + l);
                    } else {
                        qv.resize(rnd() % 80);
                        for (auto &c : qv) c = K.kind == 2 ? (uint8_t)(rnd() % 7) : "ACGT"[rnd() & 3];
                    }
                    const uint8_t *qp = qv.empty() ? nullptr : qv.data();
                    uint64_t ell = 0, mn = 0;
                    const uint32_t thr = t % 3 == 0 ? 1000 : 500;
                    uint64_t nh = orc_query(ix, qp, qv.size(), thr, &ell, &mn, ids.data(), sc.data(), n);
                    orc_exact_scores(docs.data(), off.data(), n, K.kind, K.q, qp, qv.size(), exact.data());
                    std::vector<int> hit(n, 0);
                    for (uint64_t i = 0; i < nh && i < n; i++) {
                        if (ids[i] >= n || sc[i] > ell || sc[i] < mn) errors++;
                        if (i && (sc[i] > sc[i - 1] || (sc[i] == sc[i - 1] && ids[i] <= ids[i - 1]))) errors++;
                        hit[ids[i]] = 1;
                    }
                    for (uint64_t e = 0; e < n; e++)  // no false negatives
                        if (ell && exact[e] >= mn && !hit[e]) errors++;
                    std::vector<uint64_t> tv(qv.size() + 1);
                    orc_terms(qp, qv.size(), K.kind, K.q, tv.data(), tv.size());
                }
                orc_index_free(ix);
            }
        }
    }
    // Theorem 1 worked example: l = 70, p = 0.3, more than floor(0.5 * 70) terms
    const double tail = orc_binom_tail_ge(70, 0.3, 36);
    if (tail < 1.4e-4 || tail > 1.46e-4) errors++;
    if (orc_chernoff(70, 0.5, 0.3) < tail) errors++;
    std::printf("oracle sanitize run: %d errors\n", errors);
    return errors ? 1 : 0;
}
