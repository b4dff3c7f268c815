// Host-side objects of the library (index, device index, engine), shared by the
// runtime and the serve loop.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "cobs_gpu.h"
#include "kernels.cuh"
#include "status.h"

// Return a status from a CUDA call that failed (OOM for an allocation) or from a
// library call that failed, with the message recorded.
#define CU(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return set_error(e_ == cudaErrorMemoryAllocation ? COBS_ERR_OOM : COBS_ERR_CUDA, "%s: %s", \
                             #call, cudaGetErrorString(e_));                                            \
    } while (0)

#define TRY(expr)                         \
    do {                                  \
        cobs_status s_ = (expr);          \
        if (s_ != COBS_OK) return s_;     \
    } while (0)

namespace cobs {

// NVTX range over a host scope: shows planning, enqueueing and waiting on a
// profiler's timeline (NVTX is header-only; without a tool attached a range
// costs a few nanoseconds).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Device allocation that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t n) {
        if (n == 0) n = 16;
        if (n <= bytes) return cudaSuccess;
        release();
        if (alloc_injected_failure()) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        else p = nullptr;
        return e;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Pinned host allocation that only grows.  ensure() takes it from the CUDA
// allocator; ensure_on_node() maps pages bound to one host NUMA node and pins
// them (the node nearest a device, so its copies cross no socket link).
struct PinBuf {
    void *p = nullptr;
    size_t bytes = 0;
    size_t mapped = 0;  // ensure_on_node: bytes of the mapping (0: from cudaMallocHost)
    int node = -1;      // ensure_on_node: the NUMA node the pages are bound to
    PinBuf() = default;
    PinBuf(const PinBuf &) = delete;
    PinBuf &operator=(const PinBuf &) = delete;
    ~PinBuf() { release(); }
    void release();
    cudaError_t ensure_on_node(size_t n, int numa_node);
    cudaError_t ensure(size_t n) {
        if (n == 0) n = 16;
        if (n <= bytes) return cudaSuccess;
        release();
        if (alloc_injected_failure()) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMallocHost(&p, n);
        if (e == cudaSuccess) bytes = n;
        else p = nullptr;
        return e;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Query batch plan (host): term regions, set regions, processing order and the
// counter-width classes of the batched kernel.
struct BatchPlan {
    uint64_t n = 0;
    std::vector<uint64_t> npos;
    std::vector<uint64_t> term_base, table_base;
    struct Class {
        uint32_t begin, count, L;  // a run of items with the same counter width
    };
    std::vector<Class> classes;
    struct Item {
        uint32_t q, t0, lim, slot;  // same layout as the device's uint4 items
    };
    std::vector<Item> items;        // work items of the batched kernel
    std::vector<Item> split;        // split queries: (query, first slot, slots, 0)
    uint64_t n_parts = 0;           // partial slots
    uint32_t part_terms = 0;        // terms per part of the split queries
    uint32_t plain_max_chunks = 1;  // plain form: most term chunks of a query of the batch
    // long queries (more windows than one round of the term kernel): one term
    // CTA per round (chunk), then one row CTA per (query, block group)
    std::vector<uint32_t> long_q, chunk_q, chunk_w0;
    // consecutive long queries whose sets share the table region in turn: the
    // sets of a group sit at table_base[q] within the region (cleared before the
    // group inserts)
    struct LongGroup {
        uint32_t long0, n_long, chunk0, n_chunks;
        uint64_t slots;
    };
    std::vector<LongGroup> long_groups;
    uint64_t tcap = 0, total_slots = 0, sum_npos = 0, max_npos = 0;
    uint32_t smem_slots = 16;  // largest distinct set of the batch kept in shared memory
};

struct ResultStore;

// Barrett constant floor(2^64 / w) of a Bloom size w (UINT64_MAX for w <= 1),
// the per-block modulus constant of barrett_mod.
uint64_t barrett_m_of(uint64_t w);

// The engine's table of row slices of lpq 16-byte lanes (made anew when the
// width changes).
cobs_status ensure_slices(cobs_engine *eng, uint32_t lpq);

}  // namespace cobs

struct cobs_index {
    cobs_params params{};
    uint64_t n_docs = 0;
    std::vector<cobs_block_info> blocks;
    std::vector<uint64_t> perm, nterms;
    std::vector<uint8_t> rows;
};

struct cobs_device_index {
    cobs_params params{};
    int device = 0;
    uint64_t n_docs = 0;
    std::vector<cobs_block_info> blocks;
    std::vector<uint64_t> perm, nterms;
    uint64_t rows_bytes = 0;
    uint32_t n_pgroups = 0;  // 128-byte column groups over all blocks (plain kernel)
    cobs::DevBuf rows, dblocks, dperm, pgroups;
    // streamed index: rows in pinned host memory, copied block by block per batch
    bool streamed = false;
    cobs::PinBuf host_rows;            // on the device's nearest host NUMA node where the system reports one
    uint64_t max_block_bytes = 0;
    // multi-index view: rows borrowed from resident parts; block b's rows start at
    // rows_view + dev_row_offset[b] on the device (blocks[].row_offset stays the
    // packed offset of the merged layout)
    const uint8_t *rows_view = nullptr;
    std::vector<uint64_t> dev_row_offset;
    const uint8_t *dev_rows() const { return rows_view ? rows_view : rows.as<uint8_t>(); }
};

struct cobs_engine {
    cobs_device_index *dix = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cobs_engine_cfg cfg{};
    int n_sm = 0;
    uint32_t lanes_per_query = 8;
    uint32_t l2_hints = 3;
    uint32_t ctas_per_sm = 1;
    uint64_t hit_cap = 0;

    // per batch
    cobs::DevBuf qbytes, qoff, thr;          // staging of host queries
    cobs::DevBuf plan;                        // term_base | table_base | items | split
    cobs::DevBuf partials;                    // split items: counts per (slot, document)
    cobs::DevBuf long_flag;                   // per query: EMPTY_KEY code seen (long queries)
    cobs::DevBuf tmaps;                       // TMA gather: one 128-byte tensor map per block
    bool use_tma = false;
    cobs::DevBuf ell, minsc, qcount, qcursor, hitoff, biglist;
    cobs::DevBuf counters;                    // [0] hit count, [1..] work counters
    cobs::DevBuf rows_idx, tables, codes;
    cobs::DevBuf raw_q, raw_key, keys, tmp, out_ids, out_scores;
    cobs::DevBuf plain_part;                  // plain form: per-chunk counter sums of the column groups
    cobs::DevBuf tickets;                     // plain form: per column group, chunks done
    cobs::DevBuf slices;
    uint32_t n_slices = 0, slice_lpq = 0;
    std::vector<uint32_t> block_slice0;       // per block: first slice (n_blocks + 1 entries)

    // streamed index: staging ring of device slots, filled on a second stream
    cobs::DevBuf stage;
    uint32_t n_stage = 0;
    uint64_t stage_slot_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_up, ev_free;  // per slot: rows copied / per (slot, class): slot read
    // counter classes of a batch run on their own streams, so a class of a few
    // long queries overlaps the others instead of running alone
    static constexpr int MAX_CLASSES = 4;
    static constexpr int ERR_SLOT = 14;       // counter slot of the gather's wait-limit flag
    cudaStream_t cls_stream[MAX_CLASSES] = {};
    cudaEvent_t ev_cls[MAX_CLASSES] = {};
    cudaEvent_t ev_terms = nullptr;
    uint64_t stat_h2d_index_bytes = 0;
    cobs::PinBuf pin_plan, pin_count, pin_in;

    cobs::BatchPlan bp;
    // last batch (for re-runs after a hit-capacity overflow)
    const uint8_t *last_bytes = nullptr;
    const uint64_t *last_off = nullptr;
    const uint16_t *last_thr = nullptr;
    std::vector<uint64_t> last_off_host;
    uint32_t last_flags = 0;
    bool pending = false;
    bool has_results = false;  // the last batch was enqueued in full (its buffers hold its results)

    // CUDA graph of the batched sequence
    cudaGraphExec_t gexec = nullptr;
    std::vector<uint64_t> gsig;
    uint64_t graph_stats[3] = {0, 0, 0};  // kernels, gather kernels, tiles in the graph

    // timing
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_done = nullptr;
    uint64_t stat_launches = 0, stat_gather_launches = 0, stat_tiles = 0;
    double stat_host_ms = 0;
    uint64_t hit_off_cache = 0;
};

namespace cobs {
// Engine operations used by the serve loop.
cobs_status engine_query(cobs_engine *eng, const uint8_t *d_bytes, const uint64_t *d_off, const uint64_t *h_off,
                         const uint16_t *d_thr, uint64_t n, uint32_t flags);
cobs_status engine_finish(cobs_engine *eng);
}  // namespace cobs
