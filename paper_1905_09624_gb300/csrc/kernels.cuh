// Launch wrappers of the COBS kernels (host-callable, defined in the .cu files).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <mutex>

#include "device_common.cuh"

namespace cobs {

// Runs f once per device and call site (kernel attributes are set per device);
// safe from several host threads.
struct PerDeviceOnce {
    std::mutex m;
    uint64_t done = 0;  // bit d: done on device d (devices 0..63)
    template <class F>
    void operator()(F f) {
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> g(m);
        const uint64_t bit = dev < 64 ? 1ULL << dev : 0;
        if (bit && (done & bit)) return;
        f();
        done |= bit;
    }
};

// Query-term table: shared-memory slots per CTA before the set spills to global memory.
constexpr uint32_t TERMS_SMEM_SLOTS = 4096;   // 32 KB: largest distinct set kept in shared memory
#ifndef COBS_TERMS_THREADS
#define COBS_TERMS_THREADS 256
#endif
constexpr uint32_t TERMS_THREADS = COBS_TERMS_THREADS;
constexpr uint32_t TERMS_SEG = 8;             // windows rolled by one thread per round
constexpr uint32_t TERMS_BUCKET_BITS = 6;     // terms are emitted in 64 row buckets per block
constexpr uint32_t TERMS_BUCKETS = 1u << TERMS_BUCKET_BITS;
#ifndef COBS_TERMS_BP
#define COBS_TERMS_BP 4
#endif
constexpr uint32_t TERMS_BLOCKS_PER_PASS = COBS_TERMS_BP;  // blocks whose rows one pass over the terms computes
// An on-chip set of a short query takes up to TERMS_SET_SPREAD slots per window
// (at least 2, the size every set is correct with): a sparser table means fewer
// probes and less divergence among a warp's insertions.  The launch gives the
// table region as much of a shared-memory budget of TERMS_SMEM_BUDGET bytes per
// CTA (set and list) as the spread can use.
constexpr uint32_t TERMS_SET_SPREAD = 4;
#ifndef COBS_TERMS_SMEM_BUDGET
#define COBS_TERMS_SMEM_BUDGET 40960
#endif
constexpr uint32_t TERMS_SMEM_BUDGET = COBS_TERMS_SMEM_BUDGET;
// table slots of the on-chip region for a launch whose largest on-chip set has
// `slots` = set_slots(windows) slots (its list holds slots / 2 terms)
inline uint32_t terms_smem_table(uint32_t slots) {
    const uint32_t budget = TERMS_SMEM_BUDGET / 8 > slots / 2 ? TERMS_SMEM_BUDGET / 8 - slots / 2 : 0u;
    const uint32_t spread = slots / 2 * TERMS_SET_SPREAD;
    const uint32_t t = budget < spread ? budget : spread;
    return t > slots ? t : slots;
}

struct TermsArgs {
    const uint8_t *bytes;          // queries concatenated
    const uint64_t *offsets;       // n + 1 (device)
    const uint64_t *term_base;     // per query: first slot in the term arrays (multiple of TERM_ALIGN)
    const uint64_t *table_base;    // per query: first slot of its global set (if it spills)
    unsigned long long *tables;    // global sets
    uint32_t *ell;                 // out: distinct terms per query
    uint32_t *rows_idx;            // out: row of term t for (block b, hash i) at [(b*h+i)*tcap + base + t]
    unsigned long long *codes;     // scratch: distinct term codes, tcap entries
    uint64_t tcap;
    const DevBlock *blocks;
    uint32_t n_blocks, h, kind, k;
    uint32_t q0;                   // first query handled by blockIdx.x == 0
    uint32_t smem_slots;           // sets of up to this many slots (<= TERMS_SMEM_SLOTS) and their lists live in shared memory
    uint32_t smem_table;           // slots of the on-chip table region (>= smem_slots; 0: smem_slots); an on-chip
                                   // set spreads over up to TERMS_SET_SPREAD slots per window of this region
    // Chunk plan of the long queries (more windows than one round): with
    // n_chunks > 0 every long query is processed by one CTA per round (its set
    // at tables + table_base[q] filled with EMPTY_KEY, ell[q] and long_flag[q]
    // zero before the launch), then one CTA per (query, group of blocks).
    const uint32_t *long_q;        // n_long long queries
    const uint32_t *chunk_q;       // per chunk: query
    const uint32_t *chunk_w0;      // per chunk: first window (a multiple of the round)
    uint32_t *long_flag;           // per query: the EMPTY_KEY code was seen
    uint32_t n_long, n_chunks;
};
void launch_query_terms(const TermsArgs &a, uint32_t n_queries, cudaStream_t s);
// The three parts of launch_query_terms, for callers that clear the long
// queries' sets group by group: the one-CTA-per-query kernel (long queries of
// the chunk plan return at once), the insertion of a.n_chunks chunks, the row
// pass of a.n_long long queries.
void launch_terms_short(const TermsArgs &a, uint32_t n_queries, cudaStream_t s);
void launch_terms_long_insert(const TermsArgs &a, cudaStream_t s);
void launch_terms_long_rows(const TermsArgs &a, cudaStream_t s);
uint32_t terms_round_windows();    // windows per round (long queries have more)
// The global sets of a batch's long queries are filled group by group in one
// region of this many slots (64 MB: it stays in L2 while a group inserts), or
// of the largest single set when that is larger.
constexpr uint64_t TERMS_TABLE_REGION_SLOTS = 8ULL << 20;

// Batched gather/AND/ADD with fused threshold (persistent).
struct SliceDesc {
    uint32_t block;      // block index
    uint32_t byte_off;   // byte offset of the slice within a row
};
struct GatherArgs {
    const uint8_t *rows;
    const DevBlock *blocks;
    const uint32_t *perm;          // sorted position -> original id
    const uint32_t *rows_idx;
    uint64_t tcap;
    const uint64_t *term_base;
    const uint32_t *ell;
    const uint16_t *thr;
    // Work items in processing order (longest first): x = query, y = first term,
    // z = term limit (the item covers terms [y, min(l, z))), w = partial slot, or
    // ITEM_WHOLE when the item is the whole query (threshold in the epilogue).
    const uint4 *items;
    uint32_t n_queries;            // items in this launch
    uint32_t h;
    const SliceDesc *slices;
    uint32_t n_slices;
    uint32_t n_groups;             // ceil(n_queries / queries-per-warp)
    unsigned long long *work_counter;
    unsigned long long *hit_count;
    uint32_t *qcount;              // hits per query
    uint32_t *raw_q;               // raw hits: query
    unsigned long long *raw_key;   // raw hits: (~score << 32) | original id
    uint64_t hit_cap;
    uint32_t l2_idx_policy;        // L2 eviction priority of row-index loads: 0 normal, 1 first, 2 last
    uint32_t l2_row_policy;        // same for the gathered index rows
    uint16_t *partials;            // split items: counts per (partial slot, sorted position)
    uint32_t n_docs;
    // TMA form (h == 1, 128-byte slices): one 128-byte tensor map per block
    // (w rows x rowbytes bytes, box 1 x 128), or null for the cp.async ring
    const void *tmaps;
    uint32_t *err;                 // set when a bounded wait ran out (results invalid)
};
constexpr uint32_t ITEM_WHOLE = 0xFFFFFFFFu;
// Long queries of small batches are split into items of SPLIT_TERMS terms (a
// multiple of TERM_ALIGN below 2^12, so a part counts in 12 bit-sliced levels).
constexpr uint32_t SPLIT_TERMS = 4080;
constexpr uint32_t SPLIT_MIN_TERMS = 256;   // smallest part of the adaptive split

// Split queries: sum the partial counts of their items, threshold, emit hits.
struct SplitArgs {
    const uint4 *split;            // x = query, y = first partial slot, z = slots
    uint32_t n_split;
    const uint16_t *partials;
    uint32_t n_docs;
    const uint32_t *perm;
    const uint32_t *ell;
    const uint16_t *thr;
    unsigned long long *hit_count;
    uint32_t *qcount;
    uint32_t *raw_q;
    unsigned long long *raw_key;
    uint64_t hit_cap;
};
void launch_split_finish(const SplitArgs &a, cudaStream_t s);
// lanes_per_query in {2, 4, 8}: slice = 16 * lanes_per_query bytes.  L = counter
// levels (8, 12, 16 or 24): every query of the launch has fewer than 2^L terms.
void launch_gather_batched_L(const GatherArgs &a, uint32_t lanes_per_query, uint32_t L, uint32_t grid,
                             cudaStream_t s);
uint32_t counter_levels_for(uint32_t max_terms);
int gather_batched_max_blocks_per_sm(uint32_t lanes_per_query, uint32_t h);
int gather_batched_warps_per_cta(uint32_t lanes_per_query, uint32_t h);
// the forms launch_gather_batched_L dispatches to (128-byte slices)
void launch_gather_pipe_h(const GatherArgs &a, uint32_t L, uint32_t grid, cudaStream_t s);  // h = 2..4
int gather_pipe_h_blocks_per_sm(uint32_t h);
void launch_gather_tma(const GatherArgs &a, uint32_t L, uint32_t grid, cudaStream_t s);     // h = 1, TMA feed
// Term arrays: every query's region starts at a multiple of TERM_ALIGN slots and
// spans a multiple of TERM_ALIGN slots (the gather reads row indices 16 at a time).
constexpr uint64_t TERM_ALIGN = 16;

// Plain form: one query per launch after its terms kernel, over tiles of
// (128-byte column group of a block's rows) x (chunk of the query's terms); the
// last tile of a column group adds the chunks' counts and thresholds.
constexpr uint32_t PLAIN_WARPS = 4;
constexpr uint32_t PLAIN_THREADS = PLAIN_WARPS * 32;
constexpr uint32_t PLAIN_STREAMS = PLAIN_WARPS * 4;   // streams of 8 lanes per CTA
constexpr uint32_t PLAIN_GROUP_BYTES = 128;           // a column group: 8 lanes x 16 bytes
constexpr uint32_t PLAIN_MAX_CHUNKS = 64;
constexpr uint32_t PLAIN_FUSED_MAX_H = 4;             // hashes of the fused form (its rows in shared memory)
struct PlainArgs {
    const uint8_t *rows;
    const DevBlock *blocks;
    const SliceDesc *groups;       // column groups (block, byte offset), PLAIN_GROUP_BYTES wide
    uint32_t n_groups;
    uint32_t h;
    const uint32_t *perm;          // sorted position -> original id
    const uint32_t *rows_idx;
    uint64_t tcap;
    const uint64_t *term_base;     // two-kernel form: the terms kernel's regions
    uint32_t *ell;                 // l per query (written by the fused form)
    const uint16_t *thr;
    const uint8_t *bytes;          // fused form: the queries' bytes and n + 1 offsets
    const uint64_t *offsets;
    uint32_t kind, k;              // fused form: term kind and length
    uint32_t q;                    // the query (index into offsets, term_base, ell, thr, qcount)
    uint32_t n_chunks;             // grid.y; chunk c holds terms [c * chunk_terms, (c + 1) * chunk_terms)
    uint32_t chunk_terms;          // a multiple of 16
    uint32_t _pad;
    uint32_t *partials;            // n_chunks > 1: [group][chunk][L][4][8] counter words
    uint32_t *tickets;             // per group: chunks done; zero before the launch, zero after it
    unsigned long long *hit_count;
    uint32_t *qcount;
    uint32_t *raw_q;
    unsigned long long *raw_key;
    uint64_t hit_cap;
};
// Two-kernel form, after the terms kernel of the query (a programmatic dependent
// of it).  L: counter levels, the query has fewer than 2^L terms.
cudaError_t launch_plain_query(const PlainArgs &a, uint32_t L, cudaStream_t s);
// Fused form (terms, gather, threshold in one launch) for a query of npos
// windows; pdl: a programmatic dependent of the stream's previous kernel, which
// must then be a plain kernel of the same stream or have completed the inputs.
bool plain_fused_fits(uint64_t npos, uint32_t h);
cudaError_t launch_plain_fused(const PlainArgs &a, uint32_t npos, bool pdl, cudaStream_t s);
// Chunks (and terms per chunk) of a query of npos windows over n_groups column groups.
uint32_t plain_chunks(uint64_t npos, uint32_t n_groups, uint32_t n_sm, uint32_t max_chunks, uint32_t *chunk_terms);
// Words of the partials array for n_groups x n_chunks tiles (any L).
uint64_t plain_partial_words(uint32_t n_groups, uint32_t n_chunks);

// Hit finalisation: per-query offsets, scatter, sort (score desc, id asc), unpack.
struct HitsArgs {
    uint32_t n_queries;
    const uint32_t *ell;
    const uint16_t *thr;
    uint32_t *min_score;
    const uint32_t *qcount;
    uint32_t *qcursor;
    uint64_t *hit_off;             // n + 1
    const unsigned long long *hit_count;
    uint64_t hit_cap;
    const uint32_t *raw_q;
    const unsigned long long *raw_key;
    unsigned long long *keys;      // scattered keys
    unsigned long long *tmp;       // sort scratch (same size)
    uint32_t *out_ids;
    uint32_t *out_scores;
    uint32_t *big_list;            // scratch, n_queries entries: queries with many hits from the front,
                                   // queries with a few hits from the back
    unsigned long long *big_count; // list lengths, written by the offset scan
    unsigned long long *mid_count;
};
void launch_hits_finalize(const HitsArgs &a, cudaStream_t s);

// Device build: distinct-term counts, Bloom bit-setting.
// Windows per CTA.  Small counting chunks put many CTAs on each document, so
// few documents' sets are live at once; bit-setting runs in column order, so
// CTAs that run together update the same words.
constexpr uint32_t COUNT_CHUNK = 4096;
constexpr uint32_t SETBITS_CHUNK = 8192;
constexpr uint32_t BUILD_THREADS = 256;
struct CountArgs {
    const uint8_t *docs;
    const uint64_t *doc_off;
    const uint32_t *chunk_doc;     // per CTA: document
    const uint64_t *chunk_p0;      // per CTA: first window position
    const uint64_t *table_base;    // per document (in slots), relative to `tables`
    const uint32_t *table_cap;     // per document: set_slots(windows)
    unsigned long long *tables;
    unsigned long long *v;         // out: distinct terms per document (zeroed before)
    uint32_t *has_empty;           // per document flag for the EMPTY code (bytes kind)
    uint32_t kind, k;
};
void launch_doc_count(const CountArgs &a, uint32_t n_chunks, cudaStream_t s);

// Distinct counts by hash partitions: every window's term goes to one of P_d
// partitions of its document by the high bits of its hash (a scatter pass, one
// CTA per COUNT_CHUNK windows, shared-memory ranks and one global atomic per
// partition and CTA); then one CTA per partition counts its distinct terms in a
// shared-memory set.  Documents of more than PART_MAX partitions, and any whose
// partition overflowed its capacity, are counted with global sets instead.
#ifndef COBS_PART_SET_SLOTS
#define COBS_PART_SET_SLOTS 8192
#endif
constexpr uint32_t PART_SET_SLOTS = COBS_PART_SET_SLOTS;  // shared-memory set of one partition (8 B a slot)
constexpr uint32_t PART_WINDOWS = PART_SET_SLOTS * 3 / 8;  // windows per partition (target): load <= 0.44
constexpr uint32_t PART_MAX = 2048;                        // partitions of a document
constexpr uint32_t PART_THREADS = 256;
#ifndef COBS_PART_COUNT_THREADS
#define COBS_PART_COUNT_THREADS 512
#endif
constexpr uint32_t PART_COUNT_THREADS = COBS_PART_COUNT_THREADS;  // threads of a partition's count CTA
struct PartArgs {
    const uint8_t *docs;
    const uint64_t *doc_off;
    const uint32_t *chunk_doc;     // scatter: per CTA, document
    const uint64_t *chunk_p0;      // scatter: per CTA, first window
    const uint32_t *part_doc;      // count: per CTA (partition of the wave), document
    const uint32_t *part_idx;      // count: per CTA, partition within the document
    const uint32_t *n_parts;       // per document: P_d
    const uint64_t *part0;         // per document: first partition (relative to the wave)
    const uint32_t *part_cap;      // per document: terms a partition holds
    const uint64_t *code0;         // per document: first term slot (relative to the wave)
    uint32_t *part_count;          // per partition of the wave: terms appended (zeroed before)
    unsigned long long *codes;     // the wave's partitions
    unsigned long long *v;         // out: distinct terms per document (added to)
    uint32_t *has_empty;           // per document flag for the EMPTY code (bytes kind)
    uint32_t *overflow;            // per document: a partition overflowed
    uint32_t kind, k;
    uint32_t max_parts;            // scatter: the largest P_d of the launch's documents
};
void launch_part_scatter(const PartArgs &a, uint32_t n_chunks, cudaStream_t s);
void launch_part_count(const PartArgs &a, uint32_t n_parts, cudaStream_t s);

struct SetBitsArgs {
    const uint8_t *docs;
    const uint64_t *doc_off;
    const uint32_t *chunk_doc;
    const uint64_t *chunk_p0;
    const uint32_t *doc_block;     // per original document: block
    const uint32_t *doc_col;       // per original document: column within the block
    const DevBlock *blocks;
    uint32_t *rows32;
    uint32_t kind, k, h;
};
void launch_doc_setbits(const SetBitsArgs &a, uint32_t n_chunks, cudaStream_t s);

// Bit-set by per-document filters: a CTA builds one document's whole filter of
// w bits in shared memory, writes it out column-major (`pitch_words` 32-bit words
// per document, a multiple of 8); a transpose turns tiles of 256 documents x 256
// rows into the row-major rows.  For blocks whose filter fits in shared memory.
#ifndef COBS_FILTER_THREADS
#define COBS_FILTER_THREADS 1024
#endif
constexpr uint32_t FILTER_THREADS = COBS_FILTER_THREADS;
constexpr uint32_t FILTER_TILE = 8192;               // windows staged at a time
constexpr uint32_t FILTER_SMEM_MAX = 212u * 1024u;   // largest filter kept in shared memory (w <= 1,736,704)
constexpr uint32_t TRANSPOSE_DOCS = 256, TRANSPOSE_WORDS = 8;
struct FilterArgs {
    const uint8_t *docs;
    const uint64_t *doc_off;
    const uint32_t *col_doc;       // per CTA (column of the wave): original document
    uint32_t *filters;             // out: [columns of the wave][pitch_words]
    uint32_t pitch_words;
    uint32_t w;
    uint64_t barrett_m;
    uint32_t kind, k, h;
};
void launch_doc_filter(const FilterArgs &a, uint32_t n_cols, cudaStream_t s);
struct TransposeArgs {
    const uint32_t *filters;       // [n_cols][pitch_words]
    uint32_t pitch_words;
    uint32_t n_cols;               // documents of the wave
    uint32_t col0;                 // first column of the wave in the block (a multiple of 256)
    uint32_t w, rowbytes;
    uint8_t *rows;                 // row 0 of the block
};
void launch_filter_transpose(const TransposeArgs &a, cudaStream_t s);

}  // namespace cobs
