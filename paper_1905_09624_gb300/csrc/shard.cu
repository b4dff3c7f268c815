// Document-block sharding across devices (Sec. 4 lists distributed query
// processing as future work; by Sec. 2.2 the blocks of a compact index are
// independent column groups, and the score of a document only involves its own
// block's rows).  Whole blocks are assigned to shards; every shard answers a
// query over its documents; the hit lists are merged into the order of the
// unsharded index.  Host code only: each shard is an ordinary index that a
// device loads and queries with the unchanged kernels.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <queue>
#include <vector>

#include "host_internal.h"

using namespace cobs;

namespace {

constexpr uint32_t MAX_SHARDS = 1u << 16;

uint64_t block_bytes(const cobs_block_info &b) { return b.w * b.rowbytes; }

}  // namespace

// Greedy balance of the index bytes: blocks by decreasing bytes (ties: lower
// block first), each to the shard holding the fewest bytes so far (ties: lower
// shard).
extern "C" cobs_status cobs_shard_plan(const cobs_index *ix, uint32_t n_shards, uint32_t *block_shard,
                                       uint64_t *shard_bytes) {
    if (!ix || (!block_shard && !ix->blocks.empty())) return set_error(COBS_ERR_ARG, "NULL argument");
    if (n_shards == 0 || n_shards > MAX_SHARDS) return set_error(COBS_ERR_ARG, "n_shards must be 1..65536");
    const size_t nb = ix->blocks.size();
    std::vector<uint32_t> order(nb);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        return block_bytes(ix->blocks[a]) > block_bytes(ix->blocks[b]);
    });
    std::vector<uint64_t> load(n_shards, 0);
    for (uint32_t b : order) {
        uint32_t best = 0;
        for (uint32_t s = 1; s < n_shards; s++)
            if (load[s] < load[best]) best = s;
        block_shard[b] = best;
        load[best] += block_bytes(ix->blocks[b]);
    }
    if (shard_bytes) memcpy(shard_bytes, load.data(), n_shards * sizeof(uint64_t));
    return COBS_OK;
}

// The shard's blocks in their order, rows copied; documents renumbered 0..n-1
// in increasing order of their ids in ix.
extern "C" cobs_status cobs_index_shard(const cobs_index *ix, const uint32_t *block_shard, uint32_t shard,
                                        cobs_index **out, uint64_t *global_ids, uint64_t *n_docs_out) {
    if (!ix || !out || (!block_shard && !ix->blocks.empty())) return set_error(COBS_ERR_ARG, "NULL argument");
    std::vector<uint64_t> ids;  // ids in ix of the shard's documents
    for (size_t b = 0; b < ix->blocks.size(); b++) {
        if (block_shard[b] != shard) continue;
        const cobs_block_info &B = ix->blocks[b];
        for (uint64_t j = 0; j < B.n_docs; j++) ids.push_back(ix->perm[B.doc_begin + j]);
    }
    std::sort(ids.begin(), ids.end());
    std::vector<uint64_t> local(ix->n_docs, ~0ULL);
    for (uint64_t i = 0; i < ids.size(); i++) local[ids[i]] = i;
    cobs_index *sx = new cobs_index();
    sx->params = ix->params;
    sx->n_docs = ids.size();
    sx->nterms.resize(ids.size());
    for (uint64_t i = 0; i < ids.size(); i++) sx->nterms[i] = ix->nterms[ids[i]];
    uint64_t rows_bytes = 0;
    for (size_t b = 0; b < ix->blocks.size(); b++)
        if (block_shard[b] == shard) rows_bytes += block_bytes(ix->blocks[b]);
    sx->rows.reserve(rows_bytes);
    for (size_t b = 0; b < ix->blocks.size(); b++) {
        if (block_shard[b] != shard) continue;
        cobs_block_info B = ix->blocks[b];
        const uint8_t *src = ix->rows.data() + B.row_offset;
        for (uint64_t j = 0; j < B.n_docs; j++) sx->perm.push_back(local[ix->perm[B.doc_begin + j]]);
        B.doc_begin = sx->perm.size() - B.n_docs;
        B.row_offset = sx->rows.size();
        sx->rows.insert(sx->rows.end(), src, src + block_bytes(B));
        sx->blocks.push_back(B);
    }
    if (global_ids && !ids.empty()) memcpy(global_ids, ids.data(), ids.size() * sizeof(uint64_t));
    if (n_docs_out) *n_docs_out = ids.size();
    *out = sx;
    return COBS_OK;
}

// k-way merge by (score descending, id in ix ascending), query by query.  Each
// shard's list of a query is already in that order: its local ids increase
// with the ids in ix.
extern "C" cobs_status cobs_hits_merge(uint32_t n_shards, uint64_t n_queries, const uint64_t *const *hit_offsets,
                                       const uint32_t *const *ids, const uint32_t *const *scores,
                                       const uint64_t *const *global_ids, uint64_t *hit_offsets_out,
                                       uint32_t *ids_out, uint32_t *scores_out) {
    if (!hit_offsets_out || (n_shards && (!hit_offsets || !ids || !scores || !global_ids)))
        return set_error(COBS_ERR_ARG, "NULL argument");
    if (n_shards > MAX_SHARDS) return set_error(COBS_ERR_ARG, "n_shards must be at most 65536");
    uint64_t total = 0;
    for (uint32_t s = 0; s < n_shards; s++) {
        if (!hit_offsets[s]) return set_error(COBS_ERR_ARG, "NULL hit offsets of shard %u", s);
        const uint64_t n = hit_offsets[s][n_queries] - hit_offsets[s][0];
        if (n && (!ids[s] || !scores[s] || !global_ids[s]))
            return set_error(COBS_ERR_ARG, "NULL hit list of shard %u", s);
        total += n;
    }
    if (total && (!ids_out || !scores_out)) return set_error(COBS_ERR_ARG, "NULL output");
    struct Head {
        uint32_t score;
        uint64_t id;
        uint32_t shard;
    };
    auto after = [](const Head &a, const Head &b) {  // a comes after b in the merged order
        return a.score != b.score ? a.score < b.score : a.id > b.id;
    };
    std::vector<Head> store;
    store.reserve(n_shards);
    std::priority_queue<Head, std::vector<Head>, decltype(after)> heap(after, std::move(store));
    std::vector<uint64_t> pos(n_shards, 0), end(n_shards, 0);
    uint64_t k = 0;
    hit_offsets_out[0] = 0;
    for (uint64_t q = 0; q < n_queries; q++) {
        for (uint32_t s = 0; s < n_shards; s++) {
            pos[s] = hit_offsets[s][q];
            end[s] = hit_offsets[s][q + 1];
            if (end[s] < pos[s]) return set_error(COBS_ERR_ARG, "hit offsets of shard %u decrease", s);
            if (pos[s] < end[s]) heap.push(Head{scores[s][pos[s]], global_ids[s][ids[s][pos[s]]], s});
        }
        while (!heap.empty()) {
            const Head h = heap.top();
            heap.pop();
            if (h.id > 0xFFFFFFFFULL) return set_error(COBS_ERR_ARG, "document id beyond 32 bits");
            ids_out[k] = (uint32_t)h.id;
            scores_out[k] = h.score;
            k++;
            const uint64_t p = ++pos[h.shard];
            if (p < end[h.shard]) heap.push(Head{scores[h.shard][p], global_ids[h.shard][ids[h.shard][p]], h.shard});
        }
        hit_offsets_out[q + 1] = k;
    }
    return COBS_OK;
}
