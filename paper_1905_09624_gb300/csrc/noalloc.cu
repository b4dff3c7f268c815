// One query through the plain kernels with no allocation of any kind: every
// scratch buffer the kernels need lives in one file-scope device array.
//
// Some callers cannot call cudaMalloc: a process whose memory pool (for example
// a framework's caching allocator) already holds the device memory it is allowed
// to use, and latency-critical request threads that must not pay for cudaMalloc
// and cudaFree, which can synchronise the whole device and stall every other
// stream.  They pass their own input and output buffers; the scratch below is
// reserved once per device when the library is loaded and kept until the process
// exits.
#include <cstring>
#include <mutex>

#include "host_internal.h"

using namespace cobs;

namespace {

constexpr uint64_t NA_MAX_WINDOWS = COBS_NOALLOC_MAX_WINDOWS;
constexpr uint64_t NA_MAX_DOCS = COBS_NOALLOC_MAX_DOCS;
constexpr uint64_t NA_MAX_ROW_LISTS = COBS_NOALLOC_MAX_ROW_LISTS;
constexpr uint64_t NA_TCAP = (NA_MAX_WINDOWS + TERM_ALIGN - 1) / TERM_ALIGN * TERM_ALIGN;
// column groups of the plain kernel: one per 1,024 documents of a block, plus
// one ragged group per block (blocks <= row lists)
constexpr uint64_t NA_MAX_GROUPS = NA_MAX_DOCS / (PLAIN_GROUP_BYTES * 8) + NA_MAX_ROW_LISTS;
constexpr uint32_t NA_MAX_CHUNKS = 4;  // term chunks of the plain kernel
constexpr uint64_t NA_LEVELS = 16;      // counter levels: fewer than 2^16 terms
static_assert(NA_MAX_WINDOWS < (1u << NA_LEVELS), "a query's counts fit NA_LEVELS levels");

constexpr uint64_t al(uint64_t x) { return (x + 255) / 256 * 256; }

// scratch layout (byte offsets, 256-aligned)
constexpr uint64_t OFF_HDR = 0;                                          // offsets[2], term_base, table_base, thr
constexpr uint64_t OFF_CTR = OFF_HDR + al(64);                           // qcount | counters (cleared per call)
constexpr uint64_t CTR_BYTES = 256;
constexpr uint64_t OFF_TICKETS = OFF_CTR + al(CTR_BYTES);                // per column group (cleared per call)
constexpr uint64_t OFF_CURSOR = OFF_TICKETS + al(NA_MAX_GROUPS * 4);     // qcursor[1]
constexpr uint64_t OFF_HITOFF = OFF_CURSOR + al(8);                      // hit_off[2]
constexpr uint64_t OFF_ROWS = OFF_HITOFF + al(16);                       // row indices
constexpr uint64_t OFF_CODES = OFF_ROWS + al(NA_MAX_ROW_LISTS * NA_TCAP * 4);
constexpr uint64_t OFF_TABLE = OFF_CODES + al(NA_TCAP * 8);
constexpr uint64_t OFF_PART = OFF_TABLE + al(2 * NA_MAX_WINDOWS * 8 + 128);  // plain kernel's chunk sums
constexpr uint64_t OFF_RAWQ = OFF_PART + al(NA_MAX_GROUPS * NA_MAX_CHUNKS * NA_LEVELS * 32 * 4);
constexpr uint64_t OFF_RAWKEY = OFF_RAWQ + al(NA_MAX_DOCS * 4);
constexpr uint64_t OFF_KEYS = OFF_RAWKEY + al(NA_MAX_DOCS * 8);
constexpr uint64_t OFF_TMP = OFF_KEYS + al(NA_MAX_DOCS * 8);
constexpr uint64_t NA_BYTES = OFF_TMP + al(NA_MAX_DOCS * 8);

static_assert(NA_BYTES < (16ULL << 20), "the no-allocation scratch stays modest");

__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct Header {
    uint64_t offsets[2];
    uint64_t term_base;
    uint64_t table_base;
    uint16_t thr;
    uint16_t pad[3];
};

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_scratch[MAX_DEVICES] = {nullptr};
int g_n_sm[MAX_DEVICES] = {0};

// Device address of the scratch array on the current device and its SM count
// (looked up once per device).  In host code g_noalloc_scratch names a host-side
// stand-in, not the device array: only this address may be given to a kernel.
cobs_status scratch_of(int dev, unsigned char **out, int *n_sm) {
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(COBS_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(COBS_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return set_error(COBS_ERR_CUDA, "SM count: %s", cudaGetErrorString(e));
        g_n_sm[dev] = sms;
        g_scratch[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch[dev];
    *n_sm = g_n_sm[dev];
    return COBS_OK;
}

// Per-call state, written on the device (no host buffer is read by the copy
// engine): the query's offsets and threshold, zeroed counters and tickets.
__global__ void k_noalloc_begin(unsigned char *S, uint64_t len, uint16_t thr, uint32_t n_tickets) {
    if (threadIdx.x == 0) {
        Header *h = reinterpret_cast<Header *>(S + OFF_HDR);
        h->offsets[0] = 0;
        h->offsets[1] = len;
        h->term_base = 0;
        h->table_base = 0;
        h->thr = thr;
    }
    uint32_t *ctr = reinterpret_cast<uint32_t *>(S + OFF_CTR);
    for (uint32_t i = threadIdx.x; i < CTR_BYTES / 4; i += blockDim.x) ctr[i] = 0u;
    uint32_t *tk = reinterpret_cast<uint32_t *>(S + OFF_TICKETS);
    for (uint32_t i = threadIdx.x; i < n_tickets; i += blockDim.x) tk[i] = 0u;
}

}  // namespace

#define NA_CU(call)                                                                            \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return set_error(COBS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" cobs_status cobs_query_one_noalloc(cobs_device_index *dix, const uint8_t *query_dev, uint64_t len,
                                              uint16_t thr_permille, uint32_t *out_meta_dev, uint32_t *out_ids_dev,
                                              uint32_t *out_scores_dev, uint64_t out_capacity, void *stream) {
    if (!dix || !out_meta_dev || (len && !query_dev) || (dix->n_docs && (!out_ids_dev || !out_scores_dev)))
        return set_error(COBS_ERR_ARG, "NULL argument");
    if (thr_permille == 0 || thr_permille > 1000) return set_error(COBS_ERR_ARG, "threshold must be 1..1000 permille");
    if (dix->streamed) return set_error(COBS_ERR_ARG, "this entry point needs a resident index");
    const cobs_params &P = dix->params;
    const uint64_t np = len >= P.q ? len - P.q + 1 : 0;
    if (np > (P.score_bits == 16 ? 0xFFFFULL : 0xFFFFFFFFULL))
        return set_error(COBS_ERR_OVERFLOW, "query has more windows than the score width counts");
    if (np > NA_MAX_WINDOWS)
        return set_error(COBS_ERR_ARG, "query has %llu windows; this entry point takes at most %llu",
                         (unsigned long long)np, (unsigned long long)NA_MAX_WINDOWS);
    if (dix->n_docs > NA_MAX_DOCS)
        return set_error(COBS_ERR_ARG, "index has %llu documents; this entry point takes at most %llu",
                         (unsigned long long)dix->n_docs, (unsigned long long)NA_MAX_DOCS);
    const uint64_t lists = (uint64_t)dix->blocks.size() * P.num_hashes;
    if (lists > NA_MAX_ROW_LISTS)
        return set_error(COBS_ERR_ARG, "index has %llu blocks x hashes; this entry point takes at most %llu",
                         (unsigned long long)lists, (unsigned long long)NA_MAX_ROW_LISTS);
    if (out_capacity < dix->n_docs)
        return set_error(COBS_ERR_ARG, "out_capacity must be at least the number of documents (%llu)",
                         (unsigned long long)dix->n_docs);
    int dev = 0;
    NA_CU(cudaGetDevice(&dev));
    if (dev != dix->device) return set_error(COBS_ERR_ARG, "current device %d is not the index's device %d", dev, dix->device);
    if (dix->n_pgroups > NA_MAX_GROUPS)
        return set_error(COBS_ERR_ARG, "index has %u column groups; this entry point takes at most %llu",
                         dix->n_pgroups, (unsigned long long)NA_MAX_GROUPS);
    unsigned char *S = nullptr;
    int n_sm = 0;
    cobs_status st = scratch_of(dev, &S, &n_sm);
    if (st != COBS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;

    k_noalloc_begin<<<1, 256, 0, s>>>(S, len, thr_permille, dix->n_pgroups);
    NA_CU(cudaGetLastError());
    Header *dh = reinterpret_cast<Header *>(S + OFF_HDR);
    uint32_t *qcount = reinterpret_cast<uint32_t *>(S + OFF_CTR);
    unsigned long long *hit_count = reinterpret_cast<unsigned long long *>(S + OFF_CTR + 64);

    PlainArgs pa{};
    pa.rows = dix->dev_rows();
    pa.blocks = dix->dblocks.as<DevBlock>();
    pa.groups = dix->pgroups.as<SliceDesc>();
    pa.n_groups = dix->n_pgroups;
    pa.h = P.num_hashes;
    pa.perm = dix->dperm.as<uint32_t>();
    pa.rows_idx = reinterpret_cast<uint32_t *>(S + OFF_ROWS);
    pa.tcap = NA_TCAP;
    pa.term_base = &dh->term_base;
    pa.ell = out_meta_dev;
    pa.thr = &dh->thr;
    pa.bytes = query_dev;
    pa.offsets = dh->offsets;
    pa.kind = P.term_kind;
    pa.k = P.q;
    pa.q = 0;
    pa.n_chunks = plain_chunks(np, dix->n_pgroups, (uint32_t)n_sm, NA_MAX_CHUNKS, &pa.chunk_terms);
    pa.partials = reinterpret_cast<uint32_t *>(S + OFF_PART);
    pa.tickets = reinterpret_cast<uint32_t *>(S + OFF_TICKETS);
    pa.hit_count = hit_count;
    pa.qcount = qcount;
    pa.raw_q = reinterpret_cast<uint32_t *>(S + OFF_RAWQ);
    pa.raw_key = reinterpret_cast<unsigned long long *>(S + OFF_RAWKEY);
    pa.hit_cap = NA_MAX_DOCS;
    const uint32_t levels = counter_levels_for((uint32_t)np);  // <= NA_LEVELS
    if (plain_fused_fits(np, P.num_hashes)) {
        // terms, gather and threshold in one launch; an ordinary launch, since it
        // reads the offsets k_noalloc_begin wrote
        NA_CU(launch_plain_fused(pa, (uint32_t)np, false, s));
    } else {
        TermsArgs ta{};
        ta.bytes = query_dev;
        ta.offsets = dh->offsets;
        ta.term_base = &dh->term_base;
        ta.table_base = &dh->table_base;
        ta.tables = reinterpret_cast<unsigned long long *>(S + OFF_TABLE);
        ta.ell = out_meta_dev;
        ta.rows_idx = reinterpret_cast<uint32_t *>(S + OFF_ROWS);
        ta.codes = reinterpret_cast<unsigned long long *>(S + OFF_CODES);
        ta.tcap = NA_TCAP;
        ta.blocks = dix->dblocks.as<DevBlock>();
        ta.n_blocks = (uint32_t)dix->blocks.size();
        ta.h = P.num_hashes;
        ta.kind = P.term_kind;
        ta.k = P.q;
        ta.q0 = 0;
        ta.smem_slots = TERMS_SMEM_SLOTS;
        launch_query_terms(ta, 1, s);
        NA_CU(launch_plain_query(pa, levels, s));
    }

    HitsArgs ha{};
    ha.n_queries = 1;
    ha.ell = out_meta_dev;
    ha.thr = &dh->thr;
    ha.min_score = out_meta_dev + 1;
    ha.qcount = qcount;
    ha.qcursor = reinterpret_cast<uint32_t *>(S + OFF_CURSOR);
    ha.hit_off = reinterpret_cast<uint64_t *>(S + OFF_HITOFF);
    ha.hit_count = hit_count;
    ha.hit_cap = NA_MAX_DOCS;
    ha.raw_q = pa.raw_q;
    ha.raw_key = pa.raw_key;
    ha.keys = reinterpret_cast<unsigned long long *>(S + OFF_KEYS);
    ha.tmp = reinterpret_cast<unsigned long long *>(S + OFF_TMP);
    ha.out_ids = out_ids_dev;
    ha.out_scores = out_scores_dev;
    ha.big_list = reinterpret_cast<uint32_t *>(S + OFF_CURSOR + 4);
    ha.big_count = reinterpret_cast<unsigned long long *>(S + OFF_CTR + 128);  // cleared above
    ha.mid_count = reinterpret_cast<unsigned long long *>(S + OFF_CTR + 136);
    launch_hits_finalize(ha, s);
    // number of hits = hit_off[1] (low 32 bits; at most the number of documents)
    NA_CU(cudaMemcpyAsync(out_meta_dev + 2, S + OFF_HITOFF + 8, 4, cudaMemcpyDeviceToDevice, s));
    NA_CU(cudaGetLastError());
    return COBS_OK;
}
