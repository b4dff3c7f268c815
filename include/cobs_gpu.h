/*
 * cobs_gpu.h -- C ABI of the GB300 (sm_103a) COBS query engine.
 *
 * COBS (Bingmann, Bradley, Gauger, Iqbal, "COBS: a Compact Bit-Sliced Signature
 * Index", arXiv:1905.09624) indexes a list of documents by one Bloom filter per
 * document, stored bit-sliced: row r of a block holds bit r of every filter of the
 * block (Sec. 2.2).  A query hashes its distinct q-grams ("terms", Sec. 2.1),
 * gathers h rows per term in every block, ANDs them, adds the resulting bits into
 * per-document scores and reports the documents whose score is at least
 * ceil(K * l), l = number of distinct query terms (Sec. 2.1, Sec. 2.2).  The
 * compact layout sorts documents by size and gives every block of B documents its
 * own Bloom size; one wide hash is reduced modulo each block's size (Sec. 2.2).
 *
 * Conventions for every call:
 *   - Every call returns a cobs_status; nothing throws across the ABI.  On an error
 *     cobs_last_error() returns a message (thread-local, valid until the next call
 *     on the same thread).  Out-parameters are untouched on error.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *     memory on the index's device.  Input arrays are borrowed for the duration of
 *     the call only (device inputs: until the work queued on the stream has run).
 *   - Objects returned through `**out` are owned by the library and released by
 *     their matching *_free call.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); work is
 *     queued on it.  Calls that return host results synchronise that stream.
 *   - Term kinds: 0 = DNA canonical k-mer (min of the 2-bit code of the k-mer and
 *     of its reverse complement, first base most significant, A=0 C=1 G=2 T=3),
 *     1 = DNA forward k-mer, 2 = byte q-gram (q bytes read little-endian).  Windows
 *     of DNA kinds that contain a byte other than 'A','C','G','T' are skipped
 *     (Sec. 2.1 q-grams; Sec. 2.3 canonical k-mers).
 *   - Hash i of a term t is XXH64 of the 8 little-endian bytes of t with seed i
 *     (Sec. 2.3 names xxHash); its row in block b is that hash modulo w_b (Sec. 2.2).
 */
#ifndef COBS_GPU_H
#define COBS_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    COBS_OK = 0,
    COBS_PENDING = 1,        /* serve: the ticket's result is not ready yet */
    COBS_ERR_ARG = -1,       /* invalid argument (message says which) */
    COBS_ERR_OOM = -2,       /* a device or host allocation failed */
    COBS_ERR_CUDA = -3,      /* a CUDA runtime call failed (message has the CUDA error) */
    COBS_ERR_TIMEOUT = -4,   /* a bounded wait ran out */
    COBS_ERR_BUDGET = -5,    /* serve: request can never fit the score-buffer budget */
    COBS_ERR_FORMAT = -6,    /* index file is not a cobs_gpu index or is truncated */
    COBS_ERR_OVERFLOW = -7,  /* a query has more terms than the score width can count */
    COBS_ERR_NOT_FOUND = -8, /* serve: unknown or already released ticket */
    COBS_ERR_CANCELLED = -9  /* serve: the ticket was cancelled (cobs_serve_cancel) */
} cobs_status;

/* Index parameters (Sec. 2.1-2.3). */
typedef struct cobs_params {
    uint32_t term_kind;   /* 0 DNA canonical, 1 DNA forward, 2 byte q-gram */
    uint32_t q;           /* term length: 1..32 for DNA kinds, 1..8 for bytes */
    uint32_t num_hashes;  /* h >= 1 hash functions per filter (Sec. 2.1 "k") */
    uint32_t score_bits;  /* 16 or 32: width of the reported score counters */
    double fpr;           /* target false-positive rate p of every filter, 0 < p < 1 */
    uint64_t block_docs;  /* B documents per block (compact); 0 = classic, one block in input order */
    uint64_t width;       /* 0 = every block's Bloom size from the Sec. 2.1 bound; else every block
                             gets w = width (classic indexes built over batches of documents with
                             one common w merge by concatenation, Sec. 2.3); at most 2^32 - 1 */
} cobs_params;

/* One block of the index; same meaning on host and device.  Sec. 2.2: documents at
 * sorted positions [doc_begin, doc_begin + n_docs) share one Bloom size w, stored
 * as w rows of rowbytes bytes; document j of the block is bit (j & 7) of byte
 * (j >> 3) of each row; padding bits are zero. */
typedef struct cobs_block_info {
    uint64_t n_docs;      /* documents in the block */
    uint64_t doc_begin;   /* first sorted position */
    uint64_t w;           /* Bloom filter size = rows; w = max(1, ceil(-h V / ln(1 - p^(1/h)))) */
    uint64_t rowbytes;    /* ceil(n_docs / 128) * 16 */
    uint64_t row_offset;  /* byte offset of the block's row 0 in the row storage */
    uint64_t max_terms;   /* V: largest distinct-term count of a document in the block */
} cobs_block_info;

typedef struct cobs_index cobs_index;               /* host copy of an index */
typedef struct cobs_device_index cobs_device_index; /* index resident in device memory */
typedef struct cobs_engine cobs_engine;             /* query workspace bound to a device index */
typedef struct cobs_server cobs_server;             /* continuous-batching serve loop */

/* Per-query result: hits sorted by score descending, then document id ascending. */
typedef struct cobs_hits {
    uint32_t n_terms;     /* l = distinct terms of the query; 0 => no hits */
    uint32_t min_score;   /* ceil(K * l), K in permille: (K * l + 999) / 1000 */
    uint32_t n_hits;
    uint32_t _pad;
    const uint32_t *doc_ids;  /* original document ids (input order of the build) */
    const uint32_t *scores;   /* score of each hit (number of terms present) */
} cobs_hits;

/* The hit lists of all queries of one result are stored back to back in query
 * order: hits[i].doc_ids == hits[0].doc_ids + (hits of queries 0..i-1), and the
 * same for scores, so a caller can copy them in one piece. */
typedef struct cobs_result {
    uint64_t n_queries;
    const cobs_hits *hits;    /* hits[i] for query i; storage owned by the result */
} cobs_result;

/* Query forms (flags of cobs_query_batch / cobs_engine_query*). */
#define COBS_PLAIN   1u  /* one query per kernel sequence, queries one after another */
#define COBS_BATCHED 2u  /* all queries in one persistent launch (row slices shared through L2) */
#define COBS_GRAPH   4u  /* COBS_BATCHED, replayed from a captured CUDA graph */

/* ------------------------------------------------------------------ build */

/* Build an index on the device from host documents (Sec. 2.3 "Classic and
 * Compact").  docs: all documents concatenated (host); doc_offsets: n_docs + 1
 * host offsets, document d = docs[doc_offsets[d] .. doc_offsets[d+1]).
 * Steps on the device: distinct-term count per document, host planning (sort by
 * (count, id) for compact, Bloom size per block), Bloom bit-setting into the
 * row-major blocks.  n_docs may be 0.  Errors: ARG (bad params, w_b >= 2^32,
 * n_docs >= 2^32), OOM, CUDA. */
cobs_status cobs_build_device(const cobs_params *params, const uint8_t *docs, const uint64_t *doc_offsets,
                              uint64_t n_docs, int device, void *stream, cobs_device_index **out);

/* Same as cobs_build_device, but docs and doc_offsets are DEVICE pointers on the
 * current device, already resident; doc_offsets_host is a host copy of the offsets
 * (used to plan the work; must equal the device array). */
cobs_status cobs_build_device_resident(const cobs_params *params, const uint8_t *docs_dev,
                                       const uint64_t *doc_offsets_dev, const uint64_t *doc_offsets_host,
                                       uint64_t n_docs, void *stream, cobs_device_index **out);

/* Build on the device and return a host copy (cobs_build_device + download). */
cobs_status cobs_build(const cobs_params *params, const uint8_t *docs, const uint64_t *doc_offsets,
                       uint64_t n_docs, cobs_index **out);

/* Copy a device index to the host (bit-exact: blocks, permutation, rows). */
cobs_status cobs_device_index_download(const cobs_device_index *dix, cobs_index **out);

/* Upload a host index to `device`; the index stays resident until freed. */
cobs_status cobs_load_device(const cobs_index *ix, int device, void *stream, cobs_device_index **out);

/* Streamed device index, for indexes larger than device memory (Sec. 2.3: the
 * compact index is queried block by block from external memory).  The rows of
 * `ix` are copied into pinned host memory owned by the returned object; the block
 * table and permutation go to `device`.  Engines created on it copy each block's
 * rows into a ring of device staging slots (cobs_engine_cfg.stage_bytes) on a
 * second stream while the previous block is gathered, so a query batch reads the
 * whole index over the host link once.  Only the batched and graph forms run on
 * a streamed index (COBS_PLAIN: ARG).  Errors: ARG, OOM (pinned memory), CUDA. */
cobs_status cobs_load_device_streamed(const cobs_index *ix, int device, void *stream, cobs_device_index **out);

/* Multi-index querying (Sec. 4: a front end queries several index files at once
 * and selects datasets by the indexes it combines): a device index that borrows
 * the rows of n_parts device indexes (no copy) and presents their blocks as one
 * index, queried by the same kernels in one launch sequence.  Document j of part
 * i gets id offset_i + j, offset_i = the documents of parts 0..i-1; every
 * document scores exactly as on its own part.  Parts must be on one device,
 * agree in term kind, q and number of hashes, and not be streamed (ARG
 * otherwise); a part may itself be a multi-index.  score_bits is the widest of
 * the parts.  The parts must outlive the view; free it with
 * cobs_device_index_free.  cobs_device_index_download of a view returns the
 * merged host index (cobs_index_merge layout: the parts' blocks in order). */
cobs_status cobs_multi_index_create(cobs_device_index *const *parts, uint64_t n_parts, cobs_device_index **out);

/* Save / load the library's own file format (header, block table, permutation,
 * per-document term counts, rows; little-endian).  load: FORMAT on a bad file. */
cobs_status cobs_index_save(const cobs_index *ix, const char *path);
cobs_status cobs_index_load(const char *path, cobs_index **out);

/* Merge two host indexes into a new one (Sec. 2.3: classic indexes with the same
 * parameters are concatenated; compact ones stay separate sub-indexes).  The
 * documents of b follow those of a: document j of b gets id n_docs(a) + j.
 *  - a and b classic (block_docs 0, one block each) with the same w: one classic
 *    block whose rows are a's document bits followed by b's -- bit-identical to
 *    the classic index built over both document lists with width = w;
 *  - otherwise: a's blocks, then b's (row offsets and sorted positions shifted);
 *    queries score every document exactly as on a and b separately.
 * term_kind, q and num_hashes must agree (ARG); score_bits is the wider of the
 * two.  Host memory only; a and b are unchanged. */
cobs_status cobs_index_merge(const cobs_index *a, const cobs_index *b, cobs_index **out);

/* Incremental insertion (Sec. 2.3: new documents packed into the best block
 * with free room): a new host index holding ix's documents and n_docs more
 * (document j of the new list gets id n_docs(ix) + j).  The distinct-term count
 * v of every new document is computed on `device`; in input order each goes to
 * a free column of the block whose largest count is the smallest one still at
 * least v (the block's Bloom size then keeps the false-positive rate; free
 * columns are the row padding up to a multiple of 128 documents), ties to the
 * lower block, appended after the block's documents.  The documents no block
 * takes form new blocks after the old ones, planned as a build over them alone
 * (the block size, p and width of ix's parameters).  Bits are set on the device
 * by the build kernels; ix is unchanged.  Errors: ARG, OOM, CUDA. */
cobs_status cobs_index_insert(const cobs_index *ix, const uint8_t *docs, const uint64_t *doc_offsets,
                              uint64_t n_docs, int device, cobs_index **out);

/* ------------------------------------------------- sharding across devices */

/* Document-block sharding (Sec. 4 names distributed query processing as future
 * work; by Sec. 2.2 the blocks of a compact index are independent column groups
 * and a document's score only involves its own block's rows, so whole blocks can
 * sit on different devices and a query's hits are the union of the shards').
 *
 * cobs_shard_plan assigns every block of ix to one of n_shards shards, balancing
 * the index bytes sum(w_b * rowbytes_b): blocks in decreasing order of bytes
 * (ties: lower block first), each to the shard with the fewest bytes so far
 * (ties: lower shard).  block_shard: n_blocks entries (host, caller-owned);
 * shard_bytes (may be NULL): n_shards entries receiving each shard's bytes.
 * Errors: ARG (n_shards 0 or above 65,536). */
cobs_status cobs_shard_plan(const cobs_index *ix, uint32_t n_shards, uint32_t *block_shard, uint64_t *shard_bytes);

/* The index of shard `shard` under block_shard: its blocks in their order with
 * their rows byte for byte; its documents are those of its blocks, renumbered
 * 0..n-1 in increasing order of their ids in ix (so a shard's hit order, by
 * score then id, is the order of ix).  global_ids (may be NULL; capacity >=
 * n_docs of ix) receives the id in ix of shard document j at [j]; *n_docs_out
 * (may be NULL) = n.  A shard without blocks is an index of no documents.
 * Host memory only; ix is unchanged.  Errors: ARG. */
cobs_status cobs_index_shard(const cobs_index *ix, const uint32_t *block_shard, uint32_t shard, cobs_index **out,
                             uint64_t *global_ids, uint64_t *n_docs_out);

/* Merge the hit lists of n_queries queries from n_shards shards into the order
 * of the unsharded index: per query, score descending, then id in ix ascending.
 * Shard s gives its results as a shard query returns them: hit_offsets[s]
 * (n_queries + 1 offsets), ids[s] (shard-local ids) and scores[s], with
 * global_ids[s] its id map (cobs_index_shard).  Output: hit_offsets_out
 * (n_queries + 1, starting at 0), ids_out (ids in ix) and scores_out, each of
 * capacity sum over shards of their hits.  l and ceil(K l) of a query are the
 * same on every shard.  Host memory only.  Errors: ARG (NULL arrays, decreasing
 * offsets, an id beyond 32 bits). */
cobs_status cobs_hits_merge(uint32_t n_shards, uint64_t n_queries, const uint64_t *const *hit_offsets,
                            const uint32_t *const *ids, const uint32_t *const *scores,
                            const uint64_t *const *global_ids, uint64_t *hit_offsets_out, uint32_t *ids_out,
                            uint32_t *scores_out);

/* Inspect a host index.  Pointers stay valid until cobs_index_free.
 * perm[i] = original id of the document at sorted position i;
 * nterms[d] = distinct terms of original document d. */
cobs_status cobs_index_info(const cobs_index *ix, cobs_params *params, uint64_t *n_docs, uint64_t *n_blocks,
                            const cobs_block_info **blocks, const uint64_t **perm, const uint64_t **nterms,
                            const uint8_t **rows, uint64_t *rows_bytes);

/* Inspect a device index (host copies of the table; device pointer to the rows,
 * or NULL for a streamed index, whose rows are in pinned host memory, and for a
 * multi-index view, whose rows stay in its parts). */
cobs_status cobs_device_index_info(const cobs_device_index *dix, cobs_params *params, uint64_t *n_docs,
                                   uint64_t *n_blocks, const cobs_block_info **blocks,
                                   const void **rows_dev, uint64_t *rows_bytes);

void cobs_index_free(cobs_index *ix);
void cobs_device_index_free(cobs_device_index *dix);

/* ------------------------------------------------------------------ query */

/* Query a device index from HOST buffers: copies the queries to the device, runs
 * the query path (Sec. 2.2: terms, hash, AND of h rows, ADD into scores,
 * threshold), copies the hits back.  queries: all queries concatenated;
 * query_offsets: n + 1 offsets; threshold_permille[i] in 1..1000 is K of query i.
 * flags: one of COBS_PLAIN, COBS_BATCHED, COBS_GRAPH.  Results are identical for
 * every flag.  Errors: ARG (threshold 0 or > 1000, bad flags), OVERFLOW (a query
 * has more than 2^score_bits - 1 windows), OOM, CUDA. */
cobs_status cobs_query_batch(cobs_device_index *dix, const uint8_t *queries, const uint64_t *query_offsets,
                             const uint16_t *threshold_permille, uint64_t n, uint32_t flags, void *stream,
                             cobs_result **out);
void cobs_result_free(cobs_result *res);

/* Engine: a reusable workspace for repeated query batches on one device index.
 * max_queries / max_query_bytes size the initial buffers (they grow on demand,
 * except inside a captured graph).  The engine queues all work on `stream`. */
typedef struct cobs_engine_cfg {
    uint64_t max_queries;
    uint64_t max_query_bytes;
    uint64_t max_hits;        /* initial hit capacity (0 = 1M); grows and re-runs on overflow */
    uint32_t slice_bytes;     /* batched row-slice width: 32, 64, 128, or 256 with one hash;
                                 0 = default (256 with one hash when the blocks' rows pad to at most
                                 2 % more bytes than with 128, else 128; 128 for gather_feed 2) */
    uint32_t ctas_per_sm;     /* persistent grid = SMs * ctas_per_sm; 0 = full occupancy */
    uint32_t l2_hints;        /* L2 eviction priority of the batched gather's loads:
                                 0 = default (4), 1 = none, 2 = row indices evict-first,
                                 3 = row indices evict-first and index rows evict-last,
                                 4 = index rows evict-last */
    uint32_t split;           /* long-query split of the batched form (single-hash indexes):
                                 0 = auto (batches too small to give every resident warp
                                 several tiles split their long queries into parts of
                                 256..4080 terms, sized so the tiles cover the resident
                                 warps about twice; the parts' counts are summed before
                                 the threshold), 1 = never, 2 = always */
    uint64_t stage_bytes;     /* streamed index only: device bytes of the staging ring, split
                                 into slots of the largest block's bytes (0 = two slots;
                                 at least one slot, at most one per block) */
    uint32_t gather_feed;     /* single-hash batched gather at 128-byte slices on a resident
                                 index: 0 = default, 1 = cp.async ring (16-byte pieces per
                                 lane), 2 = TMA gather (tile::gather4, four indexed rows per
                                 copy, one tensor map per block); others use the ring */
    uint32_t split_part;      /* terms per part of a split query (the query-term chunk of a
                                 work tile): 0 = sized per batch (see split); else a multiple
                                 of 16 in 256..4080 */
    uint32_t class_streams;   /* counter classes of a batch (queries grouped by length): 0 or 1 =
                                 each class's gather on a stream of its own, overlapping;
                                 2 = all on the engine stream, one after another */
    uint32_t tuned_from_cache;/* cobs_engine_autotune output: 1 when the choice came from the
                                 process-wide cache of earlier sweeps (ignored on input) */
} cobs_engine_cfg;

cobs_status cobs_engine_create(cobs_device_index *dix, const cobs_engine_cfg *cfg, void *stream,
                               cobs_engine **out);
void cobs_engine_free(cobs_engine *eng);

/* Query from DEVICE-resident inputs (bytes, offsets, thresholds on the device);
 * offsets_host is a host copy of the offsets used to plan tiles (must equal the
 * device array).  Asynchronous: results stay on the device (see
 * cobs_engine_results_device) and are complete when the engine stream reaches
 * this point.  A batch still in flight on the engine is waited for first (its
 * results, if not collected, are dropped).  After a failed call (e.g. OOM) the
 * engine stays usable; the calls that collect results return ARG until a batch
 * has been queued in full. */
cobs_status cobs_engine_query_device(cobs_engine *eng, const uint8_t *queries_dev, const uint64_t *offsets_dev,
                                     const uint64_t *offsets_host, const uint16_t *thr_dev, uint64_t n,
                                     uint32_t flags);

/* Query from HOST inputs through the engine (H2D, query, D2H; synchronises). */
cobs_status cobs_engine_query_host(cobs_engine *eng, const uint8_t *queries, const uint64_t *offsets,
                                   const uint16_t *thr, uint64_t n, uint32_t flags, cobs_result **out);

/* The same without waiting: queues the copies of the host inputs and the query
 * on the engine stream and returns; cobs_engine_download (or _results_device,
 * _stats) waits and collects.  Offsets and thresholds are copied before the
 * call returns; query bytes in page-locked memory are read by DMA from the
 * caller's buffer, which must stay unchanged until the results are collected
 * (pageable bytes are staged before the call returns).  Engines on different
 * streams pipeline batches: one engine's copies and host planning overlap
 * another's kernels. */
cobs_status cobs_engine_submit_host(cobs_engine *eng, const uint8_t *queries, const uint64_t *offsets,
                                    const uint16_t *thr, uint64_t n, uint32_t flags);

/* Device pointers to the last query's results (valid until the next query):
 * n_terms[n], min_score[n], hit_offsets[n+1] (u64), hit_ids[total], hit_scores[total]. */
cobs_status cobs_engine_results_device(cobs_engine *eng, const uint32_t **n_terms, const uint32_t **min_score,
                                       const uint64_t **hit_offsets, const uint32_t **hit_ids,
                                       const uint32_t **hit_scores);

/* Copy the last query's results to the host (synchronises the engine stream). */
cobs_status cobs_engine_download(cobs_engine *eng, cobs_result **out);

/* Timing of the last query's kernels, measured with CUDA events on the engine
 * stream: ms of the term kernel, the gather/AND/ADD kernel(s), the hit kernels,
 * and the whole sequence; plus algorithmic row bytes gathered (h * rowbytes_b per
 * term and block) and distinct terms.  Synchronises the engine stream. */
typedef struct cobs_query_stats {
    double ms_terms, ms_gather, ms_hits, ms_total;
    uint64_t row_bytes, terms, n_tiles, gather_launches, launches;
    uint32_t slice_bytes, ctas_per_sm, l2_hints;
    uint32_t split_queries;   /* queries of the last batch that ran as split parts */
    double ms_host;           /* host time of the last query call: planning and enqueueing */
    uint64_t h2d_index_bytes; /* streamed index: row bytes copied to the staging ring */
    uint32_t split_part;      /* terms per part of the split queries (0: none split) */
    int32_t stream_numa_node; /* streamed index: host NUMA node its rows are bound to (the one
                                 nearest the device); -1 = none (no NUMA, or not streamed) */
} cobs_query_stats;
cobs_status cobs_engine_stats(cobs_engine *eng, cobs_query_stats *out);

/* Autotune the batched form's work tiles on a sample batch (device inputs as in
 * cobs_engine_query_device; Sec. 2.3 scores documents in parallel partitions,
 * here tiles of a row slice x a chunk of a query's terms).  Dimensions, swept one
 * after another from the engine's current choice (coordinate descent): slice
 * width, resident CTAs per SM, L2 hints, the query-term chunk (split: none, the
 * batch-sized part, parts of 4,080 and 1,024 terms; single-hash indexes), and the
 * counter-class streams (overlapping or serial).  Each candidate runs the whole
 * batch from a cold L2, best of two; the fastest by the time of its kernels
 * (terms to hits) is kept by the engine and written to cfg_out.  The choice is
 * cached process-wide under the index's block shape and the batch's
 * query-length histogram (log2 buckets); a later call with the same key applies
 * the cached choice without sweeping (cfg_out->tuned_from_cache = 1). */
cobs_status cobs_engine_autotune(cobs_engine *eng, const uint8_t *queries_dev, const uint64_t *offsets_dev,
                                 const uint64_t *offsets_host, const uint16_t *thr_dev, uint64_t n,
                                 cobs_engine_cfg *cfg_out);

/* ------------------------------------------------------------------ serve */

typedef struct cobs_serve_cfg {
    uint64_t score_budget_bytes; /* admission budget for in-flight work (0 = 4 GiB) */
    uint32_t max_inflight_waves; /* waves on the device at once (0 = 2) */
    uint32_t max_wave_queries;   /* queries per wave (0 = 4096) */
    uint32_t wait_timeout_ms;    /* bounded waits for completions (0 = 10000) */
    uint32_t form;               /* query form of every wave: 0 or COBS_BATCHED = one batched launch
                                    sequence per wave; COBS_PLAIN = the plain form (one query per
                                    launch; with max_wave_queries 1, one query per wave) */
} cobs_serve_cfg;

typedef struct cobs_serve_stats {
    uint64_t completed, waves, rejected;
    double p50_ms, p99_ms, max_ms, qps, seconds;  /* latency: submit to result visible to poll */
    double mean_wave_queries;                     /* queries per wave */
    double mean_wave_ms, max_wave_ms;             /* wave launch to its results collected */
    uint64_t cancelled;                           /* tickets cancelled before their result was read */
    uint64_t failed;                              /* tickets that ended with an error status */
} cobs_serve_stats;

/* Start a serve loop on a device index (one scheduler thread; waves overlap on the
 * device on separate streams).  submit copies the query; poll returns COBS_PENDING
 * until the result is ready, then fills *out (valid until cobs_hits_release).
 * submit returns BUDGET if the query can never be admitted.  A wave that does not
 * finish within wait_timeout_ms fails its tickets with COBS_ERR_TIMEOUT.
 * cancel: a queued ticket is never launched; one already on the device has its
 * result dropped when its wave ends (its budget returns then).  Either way poll
 * returns COBS_ERR_CANCELLED until cobs_hits_release; NOT_FOUND for a ticket that
 * is unknown or released.  A finished ticket's result is dropped the same way. */
cobs_status cobs_serve_start(cobs_device_index *dix, const cobs_serve_cfg *cfg, cobs_server **out);
cobs_status cobs_serve_submit(cobs_server *srv, const uint8_t *q, uint64_t len, uint16_t thr_permille,
                              uint64_t *ticket);
cobs_status cobs_serve_poll(cobs_server *srv, uint64_t ticket, cobs_hits *out);
cobs_status cobs_serve_cancel(cobs_server *srv, uint64_t ticket);
void cobs_hits_release(cobs_server *srv, uint64_t ticket);
cobs_status cobs_serve_stop(cobs_server *srv, cobs_serve_stats *out);

/* ------------------------------------------------------ no allocation */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory.  Examples: a process whose memory pool (such as
 * a framework's caching allocator) already holds all the device memory it may
 * use, and latency-critical request threads that must not call cudaMalloc or
 * cudaFree, which can synchronise the whole device and stall other streams.
 *
 * cobs_query_one_noalloc runs ONE query through the plain kernels (terms,
 * gather/AND/ADD, threshold, sorted hits) and allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library routine.  Its scratch is a fixed array in
 * the library's device code, about 7.1 MiB, which every GPU that loads the
 * library holds until the process exits.  Limits: at most
 * COBS_NOALLOC_MAX_WINDOWS windows in the query, COBS_NOALLOC_MAX_DOCS documents
 * in the index and COBS_NOALLOC_MAX_ROW_LISTS (blocks x hashes); beyond them the
 * call returns COBS_ERR_ARG with a message.
 *
 * Arguments: query_dev / len: the query bytes (device); thr_permille: K in
 * 1..1000; out_meta_dev: 3 device uint32 receiving (n_terms, min_score, n_hits);
 * out_ids_dev / out_scores_dev: device arrays of out_capacity >= n_docs entries
 * receiving the hits sorted by score descending, then id ascending.  The current
 * device must be the index's device.  Asynchronous on `stream`: the outputs are
 * complete when the stream reaches this point.
 *
 * The first call on a device looks up the scratch array's device address (once
 * per device); make that first call before any stream capture.  Every call
 * shares the one scratch array and leaves its contents behind (each call clears
 * what must start at zero), so calls that overlap on the GPU -- on different
 * streams, or from different threads -- race with each other and give wrong
 * results: serialise them.  A streamed index is refused (ARG). */
#define COBS_NOALLOC_MAX_WINDOWS 16384u
#define COBS_NOALLOC_MAX_DOCS 131072u
#define COBS_NOALLOC_MAX_ROW_LISTS 32u
cobs_status cobs_query_one_noalloc(cobs_device_index *dix, const uint8_t *query_dev, uint64_t len,
                                   uint16_t thr_permille, uint32_t *out_meta_dev, uint32_t *out_ids_dev,
                                   uint32_t *out_scores_dev, uint64_t out_capacity, void *stream);

/* -------------------------------------------------------- measurement */

/* L2 read-bandwidth probe (the paper has no counterpart; it measures the ceiling
 * of a gather whose rows are reused through the L2 cache).  Reads the device
 * buffer buf_dev of `bytes` bytes (16-byte aligned; sized well inside the L2)
 * `reps` times with 16-byte loads that bypass L1, from (SMs x ctas_per_sm) CTAs
 * of 256 threads (ctas_per_sm 0 = 8), queued on `stream`.  The caller times it
 * with CUDA events: bandwidth = reps x bytes / time.  sink_dev: one device
 * uint64 the kernel may add to (its value means nothing).  Errors: ARG, CUDA. */
cobs_status cobs_probe_l2_read(const void *buf_dev, uint64_t bytes, uint32_t reps, uint32_t ctas_per_sm,
                               void *sink_dev, void *stream);

/* Test hook (the paper has no counterpart): out_dev[i] = x_dev[i] mod w for
 * i < n, computed by the device's Barrett reduction with the constant an index
 * uses for a block of Bloom size w -- the reduction behind every row index
 * (Sec. 2.2: one wide hash, then modulo each filter size).  x_dev (uint64) and
 * out_dev (uint32) are device arrays; w in 1..2^32 - 1; queued on `stream`.
 * Errors: ARG (w out of range, NULL arrays), CUDA. */
cobs_status cobs_debug_barrett_mod(const uint64_t *x_dev, uint64_t n, uint64_t w, uint32_t *out_dev, void *stream);

/* --------------------------------------------------------------- misc */

const char *cobs_last_error(void);

/* Bloom size used by the planner: max(1, ceil(-h * v / ln(1 - p^(1/h)))), the
 * Sec. 2.1 bound (1 - e^{-hv/w})^h = p solved for w at fixed h. */
uint64_t cobs_bloom_width(uint32_t h, uint64_t v, double p);

/* Library version string. */
const char *cobs_version(void);

/* Version of this header's types and entry points; it changes whenever a struct
 * layout or a signature changes.  A caller built against this header checks
 * cobs_abi_version() == COBS_GPU_ABI_VERSION before using the library. */
#define COBS_GPU_ABI_VERSION 4u
uint32_t cobs_abi_version(void);

/* Host-side fault injection for tests (the paper has no counterpart).  After
 * `after` more successful device or pinned-host allocations by the library, every
 * allocation fails as if memory were exhausted, until this is called with a
 * negative value: the calls that needed memory return COBS_ERR_OOM and leave
 * their objects freeable and usable.  The failing allocation is never attempted,
 * so nothing reaches the device.  Process-wide; default off. */
void cobs_debug_fail_alloc(int64_t after);

/* Test hook (the paper has no counterpart): scratch budget in bytes of the device
 * build's waves (the distinct-term sets of a wave of documents, the filters of a
 * wave of 256-column tiles); 0 restores the library's choice.  A small budget
 * makes a small build run in many waves.  Process-wide; results do not depend
 * on it. */
void cobs_debug_build_scratch(uint64_t bytes);

#ifdef __cplusplus
}
#endif
#endif /* COBS_GPU_H */
