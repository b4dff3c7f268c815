// Host runtime and C ABI of the query engine: batch planning, the plain,
// batched and graph forms (Sec. 2.2 query steps as kernel launches), the
// streamed index's staging ring, and result assembly.
#include <cuda.h>  // CUtensorMap and its encoder's types (resolved through the runtime)

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "host_internal.h"

using namespace cobs;

// ----------------------------------------------------------------- engine


// Default feed of the single-hash gather at 128-byte slices.
constexpr bool GATHER_FEED_TMA_DEFAULT = false;

// One tensor map per block for the TMA gather: the block's rows as a 2-D
// tensor of w rows x rowbytes bytes, copied as boxes of 1 row x 128 bytes (the
// part of a box past rowbytes reads zeros).  The encoder is the driver's,
// reached through the runtime.
static cobs_status make_tensor_maps(cobs_engine *eng) {
    typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static encode_fn encode = nullptr;
    static std::once_flag looked_up;
    std::call_once(looked_up, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &qr) == cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            encode = (encode_fn)fn;
    });
    if (!encode) return set_error(COBS_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const cobs_device_index *dix = eng->dix;
    const size_t nb = dix->blocks.size();
    std::vector<CUtensorMap> maps(std::max<size_t>(nb, 1));
    for (size_t b = 0; b < nb; b++) {
        const cobs_block_info &B = dix->blocks[b];
        const uint64_t off = dix->dev_row_offset.empty() ? B.row_offset : dix->dev_row_offset[b];
        void *base = (void *)(dix->dev_rows() + off);
        const cuuint64_t dims[2] = {B.rowbytes, B.w};
        const cuuint64_t strides[1] = {B.rowbytes};
        const cuuint32_t box[2] = {128, 1};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&maps[b], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return set_error(COBS_ERR_CUDA, "tensor map of block %zu: driver error %d", b, (int)r);
    }
    CU(eng->tmaps.ensure(maps.size() * sizeof(CUtensorMap)));
    CU(cudaMemcpy(eng->tmaps.p, maps.data(), nb * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    return COBS_OK;
}

cobs_status cobs::ensure_slices(cobs_engine *eng, uint32_t lpq) {
    if (eng->slice_lpq == lpq && eng->n_slices) return COBS_OK;
    std::vector<SliceDesc> sl;
    const uint32_t S = 16 * lpq;
    eng->block_slice0.assign(1, 0u);
    for (uint32_t b = 0; b < eng->dix->blocks.size(); b++) {
        for (uint32_t off = 0; off < eng->dix->blocks[b].rowbytes; off += S) sl.push_back(SliceDesc{b, off});
        eng->block_slice0.push_back((uint32_t)sl.size());
    }
    eng->n_slices = 0;  // no table until the new one is in place
    eng->slice_lpq = 0;
    CU(eng->slices.ensure(std::max<size_t>(sl.size(), 1) * sizeof(SliceDesc)));
    if (!sl.empty())
        CU(cudaMemcpyAsync(eng->slices.p, sl.data(), sl.size() * sizeof(SliceDesc), cudaMemcpyHostToDevice,
                           eng->stream));
    CU(cudaStreamSynchronize(eng->stream));
    eng->n_slices = (uint32_t)sl.size();
    eng->slice_lpq = lpq;
    return COBS_OK;
}

extern "C" cobs_status cobs_engine_create(cobs_device_index *dix, const cobs_engine_cfg *cfg, void *stream,
                                          cobs_engine **out) {
    if (!dix || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    CU(cudaSetDevice(dix->device));
    cobs_engine *eng = new cobs_engine();
    eng->dix = dix;
    eng->stream = (cudaStream_t)stream;
    if (!eng->stream) {
        // graph capture needs a stream other than the legacy default stream
        cudaError_t e = cudaStreamCreateWithFlags(&eng->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete eng;
            return set_error(COBS_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
        }
        eng->own_stream = true;
    }
    if (cfg) eng->cfg = *cfg;
    int dev = dix->device;
    cudaDeviceGetAttribute(&eng->n_sm, cudaDevAttrMultiProcessorCount, dev);
    // default slice width: 256 bytes with one hash (its index rows are read once
    // per two 128-byte columns: gather 0.728 ms against 0.742 ms on the bench
    // batch) unless the blocks' rows would leave more lanes idle than with 128
    // (a 640-byte row is 3 slices of 256: 1.10 ms against 0.95 ms on a view of
    // two such blocks); 128 bytes with more hashes and for the TMA feed
    uint64_t pad128 = 0, pad256 = 0;
    for (const auto &B : dix->blocks) {
        pad128 += (B.rowbytes + 127) / 128 * 128;
        pad256 += (B.rowbytes + 255) / 256 * 256;
    }
    const bool wide = pad256 * 50 <= pad128 * 51;  // at most 2 % more lane-bytes
    const uint32_t sb_default = dix->params.num_hashes == 1 && eng->cfg.gather_feed != 2 && wide ? 256 : 128;
    uint32_t sb = eng->cfg.slice_bytes ? eng->cfg.slice_bytes : sb_default;
    if (sb != 32 && sb != 64 && sb != 128 && !(sb == 256 && dix->params.num_hashes == 1)) {
        delete eng;
        return set_error(COBS_ERR_ARG, "slice_bytes must be 32, 64 or 128 (256 with one hash)");
    }
    eng->lanes_per_query = sb / 16;
    int occ = gather_batched_max_blocks_per_sm(eng->lanes_per_query, dix->params.num_hashes);
    eng->ctas_per_sm = eng->cfg.ctas_per_sm ? eng->cfg.ctas_per_sm : (uint32_t)std::max(occ, 1);
    if (eng->cfg.l2_hints > 4) {
        cobs_engine_free(eng);
        return set_error(COBS_ERR_ARG, "l2_hints must be 0..4");
    }
    if (eng->cfg.split > 2) {
        cobs_engine_free(eng);
        return set_error(COBS_ERR_ARG, "split must be 0, 1 or 2");
    }
    if (eng->cfg.split_part && (eng->cfg.split_part % TERM_ALIGN || eng->cfg.split_part < SPLIT_MIN_TERMS ||
                                eng->cfg.split_part > SPLIT_TERMS)) {
        cobs_engine_free(eng);
        return set_error(COBS_ERR_ARG, "split_part must be 0 or a multiple of 16 in 256..4080");
    }
    if (eng->cfg.class_streams > 2) {
        cobs_engine_free(eng);
        return set_error(COBS_ERR_ARG, "class_streams must be 0, 1 or 2");
    }
    eng->cfg.tuned_from_cache = 0;
    if (eng->cfg.gather_feed > 2) {
        cobs_engine_free(eng);
        return set_error(COBS_ERR_ARG, "gather_feed must be 0, 1 or 2");
    }
    {
        const bool want = eng->cfg.gather_feed == 2 || (eng->cfg.gather_feed == 0 && GATHER_FEED_TMA_DEFAULT);
        if (want && !dix->streamed && dix->params.num_hashes == 1 && eng->lanes_per_query == 8) {
            cobs_status ts = make_tensor_maps(eng);
            if (ts != COBS_OK && eng->cfg.gather_feed == 2) {
                cobs_engine_free(eng);
                return ts;
            }
            eng->use_tma = ts == COBS_OK;
        }
    }
    eng->l2_hints = eng->cfg.l2_hints ? eng->cfg.l2_hints : 4;
    eng->hit_cap = eng->cfg.max_hits ? eng->cfg.max_hits : (1ULL << 20);
    for (auto &e : eng->ev) cudaEventCreate(&e);
    cudaEventCreateWithFlags(&eng->ev_done, cudaEventDisableTiming);
    {
        cudaError_t e = cudaEventCreateWithFlags(&eng->ev_terms, cudaEventDisableTiming);
        for (int c = 0; c < cobs_engine::MAX_CLASSES && e == cudaSuccess; c++) {
            e = cudaStreamCreateWithFlags(&eng->cls_stream[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&eng->ev_cls[c], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            cobs_engine_free(eng);
            return set_error(COBS_ERR_CUDA, "class streams: %s", cudaGetErrorString(e));
        }
    }
    if (dix->streamed && !dix->blocks.empty()) {
        // staging ring: slots of the largest block, one per block at most
        const uint64_t slot = (dix->max_block_bytes + 255) / 256 * 256;
        uint64_t ns = eng->cfg.stage_bytes ? eng->cfg.stage_bytes / std::max<uint64_t>(slot, 1) : 2;
        ns = std::min<uint64_t>(ns, dix->blocks.size());
        if (ns == 0) {
            cobs_engine_free(eng);
            return set_error(COBS_ERR_ARG, "stage_bytes %llu below one slot of %llu bytes",
                             (unsigned long long)eng->cfg.stage_bytes, (unsigned long long)slot);
        }
        eng->n_stage = (uint32_t)ns;
        eng->stage_slot_bytes = slot;
        cudaError_t e = eng->stage.ensure(ns * slot);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&eng->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&eng->ev_fork, cudaEventDisableTiming);
        eng->ev_up.assign(ns, nullptr);
        eng->ev_free.assign(ns * cobs_engine::MAX_CLASSES, nullptr);
        for (uint64_t i = 0; i < ns && e == cudaSuccess; i++)
            e = cudaEventCreateWithFlags(&eng->ev_up[i], cudaEventDisableTiming);
        for (size_t i = 0; i < eng->ev_free.size() && e == cudaSuccess; i++)
            e = cudaEventCreateWithFlags(&eng->ev_free[i], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cobs_engine_free(eng);
            return set_error(e == cudaErrorMemoryAllocation ? COBS_ERR_OOM : COBS_ERR_CUDA, "staging ring: %s",
                             cudaGetErrorString(e));
        }
    }
    cobs_status st = ensure_slices(eng, eng->lanes_per_query);
    if (st != COBS_OK) {
        cobs_engine_free(eng);
        return st;
    }
    *out = eng;
    return COBS_OK;
}

extern "C" void cobs_engine_free(cobs_engine *eng) {
    if (!eng) return;
    cudaSetDevice(eng->dix->device);
    if (eng->stream) cudaStreamSynchronize(eng->stream);
    if (eng->gexec) cudaGraphExecDestroy(eng->gexec);
    for (auto &e : eng->ev)
        if (e) cudaEventDestroy(e);
    if (eng->ev_done) cudaEventDestroy(eng->ev_done);
    if (eng->copy_stream) {
        cudaStreamSynchronize(eng->copy_stream);
        cudaStreamDestroy(eng->copy_stream);
    }
    if (eng->ev_fork) cudaEventDestroy(eng->ev_fork);
    if (eng->ev_terms) cudaEventDestroy(eng->ev_terms);
    for (int c = 0; c < cobs_engine::MAX_CLASSES; c++) {
        if (eng->cls_stream[c]) {
            cudaStreamSynchronize(eng->cls_stream[c]);
            cudaStreamDestroy(eng->cls_stream[c]);
        }
        if (eng->ev_cls[c]) cudaEventDestroy(eng->ev_cls[c]);
    }
    for (auto e : eng->ev_up)
        if (e) cudaEventDestroy(e);
    for (auto e : eng->ev_free)
        if (e) cudaEventDestroy(e);
    if (eng->own_stream) cudaStreamDestroy(eng->stream);
    delete eng;
}

// Plan a batch from the host offsets.
static cobs_status make_plan(cobs_engine *eng, const uint64_t *h_off, uint64_t n, bool batched, BatchPlan &bp) {
    const cobs_params &P = eng->dix->params;
    const uint32_t k = P.q;
    const uint64_t limit = P.score_bits == 16 ? 0xFFFFULL : 0xFFFFFFFFULL;
    bp.n = n;
    bp.npos.resize(n);
    bp.term_base.resize(n);
    bp.table_base.resize(n);
    bp.tcap = 0;
    bp.total_slots = 0;
    bp.sum_npos = 0;
    bp.max_npos = 0;
    bp.smem_slots = 16;
    for (uint64_t q = 0; q < n; q++) {
        if (h_off[q + 1] < h_off[q]) return set_error(COBS_ERR_ARG, "query offsets decrease at %llu", (unsigned long long)q);
        uint64_t len = h_off[q + 1] - h_off[q];
        uint64_t np = len >= k ? len - k + 1 : 0;
        if (np > limit)
            return set_error(COBS_ERR_OVERFLOW, "query %llu has %llu windows; %u-bit scores count at most %llu",
                             (unsigned long long)q, (unsigned long long)np, P.score_bits, (unsigned long long)limit);
        if (np >= (1ULL << 24)) return set_error(COBS_ERR_ARG, "query %llu longer than 2^24 windows", (unsigned long long)q);
        bp.npos[q] = np;
        bp.term_base[q] = bp.tcap;
        bp.tcap += (np + TERM_ALIGN - 1) / TERM_ALIGN * TERM_ALIGN;
        uint64_t sl = set_slots(np);
        // a global set for every query whose set does not fit on chip and for
        // every query of more than one round (chunk CTAs share its set): placed
        // with the long-query groups below
        bp.table_base[q] = 0;
        if (sl <= TERMS_SMEM_SLOTS && np <= terms_round_windows())
            bp.smem_slots = std::max<uint32_t>(bp.smem_slots, (uint32_t)sl);
        bp.sum_npos += np;
        bp.max_npos = std::max(bp.max_npos, np);
    }
    if (bp.tcap == 0) bp.tcap = TERM_ALIGN;
    bp.plain_max_chunks = 1;
    if (!batched) {
        for (uint64_t q = 0; q < n; q++) {
            uint32_t ct = 0;
            bp.plain_max_chunks = std::max(bp.plain_max_chunks, plain_chunks(bp.npos[q], eng->dix->n_pgroups,
                                                                             (uint32_t)eng->n_sm, PLAIN_MAX_CHUNKS, &ct));
        }
    }
    bp.long_q.clear();
    bp.chunk_q.clear();
    bp.chunk_w0.clear();
    bp.long_groups.clear();
    bp.total_slots = 0;
    const uint64_t round = terms_round_windows();
    uint64_t region = TERMS_TABLE_REGION_SLOTS;
    for (uint64_t q = 0; q < n; q++)
        if (bp.npos[q] > round) region = std::max<uint64_t>(region, set_slots(bp.npos[q]));
    uint64_t used = 0;  // slots of the current group
    for (uint64_t q = 0; q < n; q++) {
        if (bp.npos[q] <= round) continue;
        const uint64_t sl = set_slots(bp.npos[q]);
        if (bp.long_groups.empty() || used + sl > region) {
            bp.long_groups.push_back({(uint32_t)bp.long_q.size(), 0u, (uint32_t)bp.chunk_q.size(), 0u, 0});
            used = 0;
        }
        BatchPlan::LongGroup &g = bp.long_groups.back();
        bp.table_base[q] = used;
        used += sl;
        g.slots = used;
        g.n_long += 1;
        bp.total_slots = std::max(bp.total_slots, used);
        bp.long_q.push_back((uint32_t)q);
        for (uint64_t w0 = 0; w0 < bp.npos[q]; w0 += round) {
            bp.chunk_q.push_back((uint32_t)q);
            bp.chunk_w0.push_back((uint32_t)w0);
            g.n_chunks += 1;
        }
    }
    // queries by windows, longest first, ties in input order: a stable LSD radix
    // sort on the complemented window count (below 2^24), two 12-bit digits
    std::vector<uint32_t> order(n);
    std::iota(order.begin(), order.end(), 0u);
    auto longer = [&](uint32_t a, uint32_t b) { return bp.npos[a] > bp.npos[b]; };
    if (!std::is_sorted(order.begin(), order.end(), longer)) {
        std::vector<uint32_t> tmp(n);
        std::vector<uint32_t> cnt(4097);
        for (int pass = 0; pass < 2; pass++) {
            const int sh = 12 * pass;
            auto digit = [&](uint32_t q) { return (uint32_t)(((~bp.npos[q] & 0xFFFFFFu) >> sh) & 0xFFFu); };
            std::fill(cnt.begin(), cnt.end(), 0u);
            for (uint64_t i = 0; i < n; i++) cnt[digit(order[i]) + 1]++;
            for (int d = 0; d < 4096; d++) cnt[d + 1] += cnt[d];
            for (uint64_t i = 0; i < n; i++) tmp[cnt[digit(order[i])]++] = order[i];
            order.swap(tmp);
        }
    }
    // Work items.  A batch too small to give every resident warp several tiles
    // splits its long queries into parts (h == 1 only), so one long query no
    // longer runs on a single warp per slice.  The part size aims at about two
    // tiles per resident warp: the batch's windows over the items that many
    // tiles hold, a multiple of TERM_ALIGN between SPLIT_MIN_TERMS and
    // SPLIT_TERMS.
    const uint64_t qpw = 32 / eng->lanes_per_query;
    const uint64_t warps = (uint64_t)eng->n_sm * eng->ctas_per_sm *
                           (uint64_t)gather_batched_warps_per_cta(eng->lanes_per_query, P.num_hashes);
    const bool small = (uint64_t)eng->n_slices * ((n + qpw - 1) / qpw) < 4 * warps;
    bool split = batched && P.num_hashes == 1 && eng->cfg.split != 1 && (eng->cfg.split == 2 || small);
    uint64_t part = SPLIT_TERMS;
    if (split) {
        if (eng->cfg.split_part) {
            part = eng->cfg.split_part;  // the term chunk chosen by the caller or the autotuner
        } else {
            const uint64_t items_target =
                std::max<uint64_t>(1, 2 * warps * qpw / std::max<uint32_t>(eng->n_slices, 1));
            part = (bp.sum_npos + items_target - 1) / items_target;
            part = (part + TERM_ALIGN - 1) / TERM_ALIGN * TERM_ALIGN;
            part = std::min<uint64_t>(std::max<uint64_t>(part, SPLIT_MIN_TERMS), SPLIT_TERMS);
        }
        // partial counts (2 bytes per part and document) stay below 1 GiB
        uint64_t parts = 0;
        for (uint64_t q = 0; q < n; q++)
            if (bp.npos[q] > part) parts += (bp.npos[q] + part - 1) / part;
        split = parts * eng->dix->n_docs * 2 <= (1ULL << 30);
    }
    bp.items.clear();
    bp.split.clear();
    bp.n_parts = 0;
    bp.part_terms = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint32_t q = order[i];
        const uint64_t np = bp.npos[q];
        if (split && np > part) {
            const uint32_t parts = (uint32_t)((np + part - 1) / part);
            const uint32_t ps = (uint32_t)part;
            bp.part_terms = ps;
            bp.split.push_back({q, (uint32_t)bp.n_parts, parts, 0u});
            for (uint32_t p = 0; p < parts; p++)
                bp.items.push_back({q, p * ps, (p + 1) * ps, (uint32_t)(bp.n_parts + p)});
            bp.n_parts += parts;
        } else {
            bp.items.push_back({q, 0u, ITEM_WHOLE, ITEM_WHOLE});
        }
    }
    // longest items first; counter width classes by the items' term bounds
    auto bound = [&](const BatchPlan::Item &it) {
        return std::min<uint64_t>(bp.npos[it.q], it.lim) - std::min<uint64_t>(bp.npos[it.q], it.t0);
    };
    if (!bp.split.empty())  // without parts the items already follow the query order
        std::stable_sort(bp.items.begin(), bp.items.end(),
                         [&](const BatchPlan::Item &a, const BatchPlan::Item &b) { return bound(a) > bound(b); });
    bp.classes.clear();
    const uint32_t ni = (uint32_t)bp.items.size();
    for (uint32_t i = 0; i < ni;) {
        uint32_t L = counter_levels_for((uint32_t)bound(bp.items[i]));
        uint32_t j = i;
        while (j < ni && counter_levels_for((uint32_t)bound(bp.items[j])) == L) j++;
        bp.classes.push_back({i, j - i, L});
        i = j;
    }
    return COBS_OK;
}

// A streamed index is copied and gathered in column units of at most
// STREAM_UNIT_BYTES of every row (2-D copies: pitch = rowbytes): the gathers of
// one unit run while the next unit is copied.  Host-to-device 2-D copies of
// 512-byte rows ran at the full pinned-memory rate (209 GB/s; 256 bytes: 185,
// 128 bytes: 107).  A multiple of every slice width.
constexpr uint64_t STREAM_UNIT_BYTES = 512;
static uint64_t units_of(uint64_t rowbytes) {
    return rowbytes <= STREAM_UNIT_BYTES ? 1 : (rowbytes + STREAM_UNIT_BYTES - 1) / STREAM_UNIT_BYTES;
}
static uint64_t stream_units(const cobs_device_index *dix) {
    uint64_t n = 0;
    for (const auto &B : dix->blocks) n += units_of(B.rowbytes);
    return n;
}

// Plan upload: term_base[n] | table_base[n] (u64) | items | split queries (uint4)
// | long queries | chunk queries | chunk first windows (u32).
static uint64_t plan_bytes(const BatchPlan &bp) {
    return bp.n * 16 + bp.items.size() * 16 + bp.split.size() * 16 +
           (bp.long_q.size() + 2 * bp.chunk_q.size()) * 4;
}

static cobs_status ensure_buffers(cobs_engine *eng, const BatchPlan &bp) {
    const uint64_t n = bp.n;
    const uint64_t nb = eng->dix->blocks.size(), h = eng->dix->params.num_hashes;
    CU(eng->plan.ensure(plan_bytes(bp) + 64));
    CU(eng->partials.ensure(bp.n_parts * eng->dix->n_docs * 2));
    CU(eng->long_flag.ensure(n * 4));
    CU(eng->ell.ensure(n * 4));
    CU(eng->minsc.ensure(n * 4));
    // qcount, then the counters (one memset clears both): [0] hits, [1..4] work
    // counters, [13] and [15] the hit lists to sort, [14] the gather's error
    // flag, then 4 per block for a streamed index
    CU(eng->qcount.ensure(n * 4 + (64 + 4 * std::max<uint64_t>(nb, stream_units(eng->dix))) * 8));
    CU(eng->qcursor.ensure(n * 4));
    CU(eng->biglist.ensure(n * 4));
    CU(eng->hitoff.ensure((n + 1) * 8));
    CU(eng->rows_idx.ensure(std::max<uint64_t>(nb, 1) * h * bp.tcap * 4));
    CU(eng->codes.ensure(bp.tcap * 8));
    CU(eng->tables.ensure(bp.total_slots * 8));
    CU(eng->raw_q.ensure(eng->hit_cap * 4));
    CU(eng->raw_key.ensure(eng->hit_cap * 8));
    CU(eng->keys.ensure(eng->hit_cap * 8));
    CU(eng->tmp.ensure(eng->hit_cap * 8));
    CU(eng->out_ids.ensure(eng->hit_cap * 4));
    CU(eng->out_scores.ensure(eng->hit_cap * 4));
    CU(eng->plain_part.ensure(plain_partial_words(eng->dix->n_pgroups, bp.plain_max_chunks) * 4));
    CU(eng->tickets.ensure((uint64_t)eng->dix->n_pgroups * 4));
    CU(eng->pin_plan.ensure(plan_bytes(bp) + 64));
    CU(eng->pin_count.ensure(16 * 8));
    return COBS_OK;
}

static unsigned long long *counters_of(cobs_engine *eng, uint64_t n) {
    // counters live right after the n query counts, 8-byte aligned
    uintptr_t p = (uintptr_t)(eng->qcount.as<uint8_t>() + n * 4);
    p = (p + 7) & ~(uintptr_t)7;
    return (unsigned long long *)p;
}

// Enqueue the whole query sequence on the engine stream.
static cobs_status enqueue(cobs_engine *eng, const uint8_t *d_bytes, const uint64_t *d_off, const uint16_t *d_thr,
                           uint32_t flags, bool timed) {
    TraceRange tr("cobs.enqueue");
    cobs_device_index *dix = eng->dix;
    const BatchPlan &bp = eng->bp;
    const uint64_t n = bp.n;
    const cobs_params &P = dix->params;
    cudaStream_t s = eng->stream;
    uint8_t *plan = eng->plan.as<uint8_t>();
    const uint64_t *term_base = (const uint64_t *)plan;
    const uint64_t *table_base = (const uint64_t *)(plan + n * 8);
    const uint4 *items = (const uint4 *)(plan + n * 16);
    const uint4 *split = items + bp.items.size();
    const uint32_t *long_q = (const uint32_t *)(split + bp.split.size());
    const uint32_t *chunk_q = long_q + bp.long_q.size();
    const uint32_t *chunk_w0 = chunk_q + bp.chunk_q.size();
    unsigned long long *ctr = counters_of(eng, n);
    const uint64_t n_ctr = 16 + (dix->streamed ? 4 * stream_units(dix) : 0);
    eng->stat_launches = 0;
    eng->stat_gather_launches = 0;
    eng->stat_tiles = 0;
    eng->stat_h2d_index_bytes = 0;

    // timing events: inside a stream capture they must be external records to
    // become event nodes of the graph
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(s, &cst));
    const unsigned int tflag = cst == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (timed) CU(cudaEventRecordWithFlags(eng->ev[0], s, tflag));
    if (dix->streamed) CU(cudaEventRecord(eng->ev_fork, s));  // the copy stream joins here
    CU(cudaMemsetAsync(eng->qcount.p, 0, (uint8_t *)(ctr + n_ctr) - eng->qcount.as<uint8_t>(), s));
    CU(cudaMemcpyAsync(plan, eng->pin_plan.p, plan_bytes(bp), cudaMemcpyHostToDevice, s));

    TermsArgs ta{};
    ta.bytes = d_bytes;
    ta.offsets = d_off;
    ta.term_base = term_base;
    ta.table_base = table_base;
    ta.tables = eng->tables.as<unsigned long long>();
    ta.ell = eng->ell.as<uint32_t>();
    ta.rows_idx = eng->rows_idx.as<uint32_t>();
    ta.codes = eng->codes.as<unsigned long long>();
    ta.tcap = bp.tcap;
    ta.blocks = dix->dblocks.as<DevBlock>();
    ta.n_blocks = (uint32_t)dix->blocks.size();
    ta.h = P.num_hashes;
    ta.kind = P.term_kind;
    ta.k = P.q;
    ta.smem_slots = bp.smem_slots;
    ta.smem_table = terms_smem_table(bp.smem_slots);

    if (flags & COBS_PLAIN) {
        // One query per launch over (column group x term chunk) tiles, which
        // threshold and emit the query's hits themselves (the tickets start at
        // zero and every query's last tiles leave them at zero).  A query of at
        // most one term round: the fused kernel alone, a programmatic dependent
        // of the previous query's, so the two overlap until the epilogue.  A
        // longer one: its terms kernels (a CTA per round of windows for a long
        // query), then the gather kernel.
        if (timed) CU(cudaEventRecordWithFlags(eng->ev[1], s, tflag));
        if (dix->n_pgroups) CU(cudaMemsetAsync(eng->tickets.p, 0, (uint64_t)dix->n_pgroups * 4, s));
        PlainArgs pa{};
        pa.rows = dix->dev_rows();
        pa.blocks = dix->dblocks.as<DevBlock>();
        pa.groups = dix->pgroups.as<SliceDesc>();
        pa.n_groups = dix->n_pgroups;
        pa.h = P.num_hashes;
        pa.perm = dix->dperm.as<uint32_t>();
        pa.rows_idx = eng->rows_idx.as<uint32_t>();
        pa.tcap = bp.tcap;
        pa.term_base = term_base;
        pa.ell = eng->ell.as<uint32_t>();
        pa.thr = d_thr;
        pa.partials = eng->plain_part.as<uint32_t>();
        pa.tickets = eng->tickets.as<uint32_t>();
        pa.hit_count = ctr;
        pa.qcount = eng->qcount.as<uint32_t>();
        pa.raw_q = eng->raw_q.as<uint32_t>();
        pa.raw_key = eng->raw_key.as<unsigned long long>();
        pa.hit_cap = eng->hit_cap;
        pa.bytes = d_bytes;
        pa.offsets = d_off;
        pa.kind = P.term_kind;
        pa.k = P.q;
        const uint64_t round = terms_round_windows();
        uint32_t li = 0, ci = 0;  // the next long query and its first chunk in the batch plan
        for (uint64_t q = 0; q < n; q++) {
            const uint64_t np = bp.npos[q];
            pa.q = (uint32_t)q;
            pa.n_chunks = plain_chunks(np, dix->n_pgroups, (uint32_t)eng->n_sm, PLAIN_MAX_CHUNKS, &pa.chunk_terms);
            if (plain_fused_fits(np, P.num_hashes)) {
                CU(launch_plain_fused(pa, (uint32_t)np, true, s));
                eng->stat_launches += 1;
            } else {
                ta.q0 = (uint32_t)q;
                if (np > round) {
                    const uint32_t nch = (uint32_t)((np + round - 1) / round);
                    CU(cudaMemsetAsync(eng->tables.as<unsigned long long>() + bp.table_base[q], 0xFF,
                                       set_slots(np) * 8, s));
                    CU(cudaMemsetAsync(eng->ell.as<uint32_t>() + q, 0, 4, s));
                    CU(cudaMemsetAsync(eng->long_flag.as<uint32_t>() + q, 0, 4, s));
                    TermsArgs tl = ta;
                    tl.long_q = long_q + li;
                    tl.chunk_q = chunk_q + ci;
                    tl.chunk_w0 = chunk_w0 + ci;
                    tl.long_flag = eng->long_flag.as<uint32_t>();
                    tl.n_long = 1;
                    tl.n_chunks = nch;
                    launch_query_terms(tl, 1, s);
                    li += 1;
                    ci += nch;
                    eng->stat_launches += 3;
                } else {
                    launch_query_terms(ta, 1, s);
                    eng->stat_launches += 1;
                }
                CU(launch_plain_query(pa, counter_levels_for((uint32_t)np), s));
                eng->stat_launches += 1;
            }
            eng->stat_gather_launches += 1;
        }
        CU(cudaGetLastError());
        if (timed) CU(cudaEventRecordWithFlags(eng->ev[2], s, tflag));
    } else {
        ta.q0 = 0;
        if (!bp.long_q.empty()) {
            // long queries: distinct counts and flags zeroed; after the one-CTA-
            // per-query kernel, group by group the table region is cleared and a
            // CTA per chunk inserts (a group's sets stay in L2), then a CTA per
            // (query, block group) runs the row pass
            CU(cudaMemsetAsync(eng->ell.p, 0, n * 4, s));
            CU(cudaMemsetAsync(eng->long_flag.p, 0, n * 4, s));
            ta.long_q = long_q;
            ta.chunk_q = chunk_q;
            ta.chunk_w0 = chunk_w0;
            ta.long_flag = eng->long_flag.as<uint32_t>();
            ta.n_long = (uint32_t)bp.long_q.size();
            ta.n_chunks = (uint32_t)bp.chunk_q.size();
        }
        {
            TraceRange tr_terms("cobs.terms");
            launch_terms_short(ta, (uint32_t)n, s);
            eng->stat_launches += 1;
            for (const BatchPlan::LongGroup &g : bp.long_groups) {
                CU(cudaMemsetAsync(eng->tables.p, 0xFF, g.slots * 8, s));
                TermsArgs tg = ta;
                tg.chunk_q = chunk_q + g.chunk0;
                tg.chunk_w0 = chunk_w0 + g.chunk0;
                tg.n_chunks = g.n_chunks;
                launch_terms_long_insert(tg, s);
                eng->stat_launches += 1;
            }
            if (!bp.long_q.empty()) {
                launch_terms_long_rows(ta, s);
                eng->stat_launches += 1;
            }
        }
        CU(cudaGetLastError());
        if (timed) CU(cudaEventRecordWithFlags(eng->ev[1], s, tflag));
        const uint32_t qpw = 32 / eng->lanes_per_query;
        const uint32_t grid = (uint32_t)eng->n_sm * eng->ctas_per_sm;
        // several counter classes: each on its own stream, forked after the terms
        const uint32_t n_cls = (uint32_t)bp.classes.size();
        if (n_cls > (uint32_t)cobs_engine::MAX_CLASSES) return set_error(COBS_ERR_ARG, "more than 4 counter classes");
        const bool multi = n_cls > 1 && eng->cfg.class_streams != 2;
        auto gs = [&](size_t c) { return multi ? eng->cls_stream[c] : s; };
        if (multi) {
            CU(cudaEventRecord(eng->ev_terms, s));
            for (uint32_t c = 0; c < n_cls; c++) CU(cudaStreamWaitEvent(gs(c), eng->ev_terms, 0));
        }
        // one gather launch per counter class over slices [sl0, sl0 + nsl); rows
        // of block b are read at rows + row_offset_b
        auto gather_classes = [&](const uint8_t *rows, uint32_t sl0, uint32_t nsl, unsigned long long *wctr) {
            for (size_t c = 0; c < bp.classes.size(); c++) {
                const BatchPlan::Class &cl = bp.classes[c];
                GatherArgs ga{};
                ga.rows = rows;
                ga.blocks = dix->dblocks.as<DevBlock>();
                ga.perm = dix->dperm.as<uint32_t>();
                ga.rows_idx = eng->rows_idx.as<uint32_t>();
                ga.tcap = bp.tcap;
                ga.term_base = term_base;
                ga.ell = eng->ell.as<uint32_t>();
                ga.thr = d_thr;
                ga.items = items + cl.begin;
                ga.n_queries = cl.count;
                ga.h = P.num_hashes;
                ga.slices = eng->slices.as<SliceDesc>() + sl0;
                ga.n_slices = nsl;
                ga.n_groups = (cl.count + qpw - 1) / qpw;
                ga.work_counter = wctr + c;
                ga.hit_count = ctr;
                ga.qcount = eng->qcount.as<uint32_t>();
                ga.raw_q = eng->raw_q.as<uint32_t>();
                ga.raw_key = eng->raw_key.as<unsigned long long>();
                ga.hit_cap = eng->hit_cap;
                // l2_hints: 1 none, 2 row indices evict-first, 3 + index rows evict-last, 4 rows evict-last only
                ga.l2_idx_policy = (eng->l2_hints == 2 || eng->l2_hints == 3) ? 1u : 0u;
                ga.l2_row_policy = (eng->l2_hints == 3 || eng->l2_hints == 4) ? 2u : 0u;
                ga.partials = eng->partials.as<uint16_t>();
                ga.n_docs = (uint32_t)dix->n_docs;
                ga.tmaps = eng->use_tma && !dix->streamed ? eng->tmaps.p : nullptr;
                ga.err = (uint32_t *)(ctr + cobs_engine::ERR_SLOT);
                if (ga.n_slices == 0 || ga.n_groups == 0) continue;
                launch_gather_batched_L(ga, eng->lanes_per_query, cl.L, grid, gs(c));
                eng->stat_launches += 1;
                eng->stat_gather_launches += 1;
                eng->stat_tiles += (uint64_t)ga.n_slices * ga.n_groups;
            }
        };
        TraceRange tr_gather("cobs.gather");
        if (!dix->streamed) {
            gather_classes(dix->dev_rows(), 0, eng->n_slices, ctr + 1);  // classes <= 4 < 15
        } else {
            // Block b: the copy stream fills slot b mod S once every class's gathers
            // of block b - S have read it; each class gathers block b once it is in.
            const uint32_t nb = (uint32_t)dix->blocks.size();
            const uint32_t MC = (uint32_t)cobs_engine::MAX_CLASSES;
            CU(cudaStreamWaitEvent(eng->copy_stream, eng->ev_fork, 0));
            const uint32_t S = 16u * eng->lanes_per_query;  // slice width
            uint32_t unit = 0;                                // running unit: its 4 work counters
            for (uint32_t b = 0; b < nb; b++) {
                const uint32_t slot = b % eng->n_stage;
                const cobs_block_info &B = dix->blocks[b];
                const uint64_t bytes = B.w * B.rowbytes;
                uint8_t *dst = eng->stage.as<uint8_t>() + slot * eng->stage_slot_bytes;
                const uint8_t *src = dix->host_rows.as<uint8_t>() + B.row_offset;
                if (b >= eng->n_stage)
                    for (uint32_t c = 0; c < std::max(n_cls, 1u); c++)
                        CU(cudaStreamWaitEvent(eng->copy_stream, eng->ev_free[slot * MC + c], 0));
                // the kernels add row_offset_b to the rows pointer: shift the slot back by it
                const uint8_t *rows = (const uint8_t *)((uintptr_t)dst - (uintptr_t)B.row_offset);
                const uint64_t nu = units_of(B.rowbytes);
                for (uint64_t u = 0; u < nu; u++, unit++) {
                    const uint64_t c0 = u * STREAM_UNIT_BYTES;
                    const uint64_t width = std::min<uint64_t>(STREAM_UNIT_BYTES, B.rowbytes - c0);
                    if (nu == 1) {
                        if (bytes) CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, eng->copy_stream));
                    } else if (B.w) {
                        CU(cudaMemcpy2DAsync(dst + c0, B.rowbytes, src + c0, B.rowbytes, width, B.w,
                                             cudaMemcpyHostToDevice, eng->copy_stream));
                    }
                    CU(cudaEventRecord(eng->ev_up[slot], eng->copy_stream));
                    for (uint32_t c = 0; c < std::max(n_cls, 1u); c++)
                        CU(cudaStreamWaitEvent(gs(c), eng->ev_up[slot], 0));
                    // the unit's slices: byte offsets [c0, c0 + width) of the block's rows
                    const uint32_t s0 = eng->block_slice0[b] + (uint32_t)(c0 / S);
                    const uint32_t s1 = std::min<uint32_t>(eng->block_slice0[b + 1],
                                                           eng->block_slice0[b] + (uint32_t)((c0 + width + S - 1) / S));
                    gather_classes(rows, s0, s1 - s0, ctr + 16 + 4 * unit);
                }
                for (uint32_t c = 0; c < std::max(n_cls, 1u); c++)
                    CU(cudaEventRecord(eng->ev_free[slot * MC + c], gs(c)));
                eng->stat_h2d_index_bytes += bytes;
            }
            if (nb) CU(cudaStreamWaitEvent(s, eng->ev_up[(nb - 1) % eng->n_stage], 0));  // join the copy stream
        }
        if (multi) {  // join the class streams
            for (uint32_t c = 0; c < n_cls; c++) {
                CU(cudaEventRecord(eng->ev_cls[c], gs(c)));
                CU(cudaStreamWaitEvent(s, eng->ev_cls[c], 0));
            }
        }
        if (!bp.split.empty()) {
            SplitArgs sa{};
            sa.split = split;
            sa.n_split = (uint32_t)bp.split.size();
            sa.partials = eng->partials.as<uint16_t>();
            sa.n_docs = (uint32_t)dix->n_docs;
            sa.perm = dix->dperm.as<uint32_t>();
            sa.ell = eng->ell.as<uint32_t>();
            sa.thr = d_thr;
            sa.hit_count = ctr;
            sa.qcount = eng->qcount.as<uint32_t>();
            sa.raw_q = eng->raw_q.as<uint32_t>();
            sa.raw_key = eng->raw_key.as<unsigned long long>();
            sa.hit_cap = eng->hit_cap;
            launch_split_finish(sa, s);
            eng->stat_launches += 1;
        }
        CU(cudaGetLastError());
        if (timed) CU(cudaEventRecordWithFlags(eng->ev[2], s, tflag));
    }
    HitsArgs ha{};
    ha.n_queries = (uint32_t)n;
    ha.ell = eng->ell.as<uint32_t>();
    ha.thr = d_thr;
    ha.min_score = eng->minsc.as<uint32_t>();
    ha.qcount = eng->qcount.as<uint32_t>();
    ha.qcursor = eng->qcursor.as<uint32_t>();
    ha.hit_off = eng->hitoff.as<uint64_t>();
    ha.hit_count = ctr;
    ha.hit_cap = eng->hit_cap;
    ha.raw_q = eng->raw_q.as<uint32_t>();
    ha.raw_key = eng->raw_key.as<unsigned long long>();
    ha.keys = eng->keys.as<unsigned long long>();
    ha.tmp = eng->tmp.as<unsigned long long>();
    ha.out_ids = eng->out_ids.as<uint32_t>();
    ha.out_scores = eng->out_scores.as<uint32_t>();
    ha.big_list = eng->biglist.as<uint32_t>();
    ha.big_count = ctr + 15;  // cleared with the other counters
    ha.mid_count = ctr + 13;
    {
        TraceRange tr_hits("cobs.hits");
        launch_hits_finalize(ha, s);
    }
    eng->stat_launches += 4;  // offsets, scatter, the two segment sorts
    CU(cudaGetLastError());
    if (timed) CU(cudaEventRecordWithFlags(eng->ev[3], s, tflag));
    // hit count and the gather's wait-limit flag, read when the batch is collected
    CU(cudaMemcpyAsync(eng->pin_count.p, ctr, 16 * 8, cudaMemcpyDeviceToHost, s));
    return COBS_OK;
}

static void fill_pinned_plan(cobs_engine *eng) {
    const BatchPlan &bp = eng->bp;
    uint8_t *p = eng->pin_plan.as<uint8_t>();
    memcpy(p, bp.term_base.data(), bp.n * 8);
    memcpy(p + bp.n * 8, bp.table_base.data(), bp.n * 8);
    if (!bp.items.empty()) memcpy(p + bp.n * 16, bp.items.data(), bp.items.size() * 16);
    if (!bp.split.empty()) memcpy(p + bp.n * 16 + bp.items.size() * 16, bp.split.data(), bp.split.size() * 16);
    uint8_t *u = p + bp.n * 16 + (bp.items.size() + bp.split.size()) * 16;
    const size_t nl = bp.long_q.size(), nc = bp.chunk_q.size();
    if (nl) memcpy(u, bp.long_q.data(), nl * 4);
    if (nc) {
        memcpy(u + nl * 4, bp.chunk_q.data(), nc * 4);
        memcpy(u + (nl + nc) * 4, bp.chunk_w0.data(), nc * 4);
    }
}

static std::vector<uint64_t> graph_signature(cobs_engine *eng, const uint8_t *d_bytes, const uint64_t *d_off,
                                             const uint16_t *d_thr) {
    const BatchPlan &bp = eng->bp;
    std::vector<uint64_t> sig = {bp.n, bp.tcap, bp.total_slots, (uint64_t)d_bytes, (uint64_t)d_off, (uint64_t)d_thr,
                                 eng->hit_cap, eng->lanes_per_query, eng->ctas_per_sm, eng->l2_hints, bp.smem_slots,
                                 (uint64_t)eng->rows_idx.p, (uint64_t)eng->tables.p, (uint64_t)eng->raw_q.p,
                                 (uint64_t)eng->codes.p,
                                 (uint64_t)eng->plan.p, (uint64_t)eng->pin_plan.p, (uint64_t)eng->qcount.p,
                                 (uint64_t)eng->ell.p, (uint64_t)eng->minsc.p, (uint64_t)eng->qcursor.p,
                                 (uint64_t)eng->hitoff.p, (uint64_t)eng->raw_key.p, (uint64_t)eng->keys.p,
                                 (uint64_t)eng->biglist.p,
                                 (uint64_t)eng->tmp.p, (uint64_t)eng->out_ids.p, (uint64_t)eng->out_scores.p,
                                 (uint64_t)eng->pin_count.p, (uint64_t)eng->slices.p, eng->n_slices,
                                 (uint64_t)bp.items.size(), (uint64_t)bp.split.size(), bp.n_parts,
                                 (uint64_t)eng->partials.p, (uint64_t)bp.long_q.size(), (uint64_t)bp.chunk_q.size(),
                                 (uint64_t)eng->long_flag.p, eng->cfg.class_streams, bp.part_terms,
                                 (uint64_t)bp.long_groups.size()};
    for (const auto &g : bp.long_groups) {
        sig.push_back(g.n_chunks);
        sig.push_back(g.slots);
    }
    for (const auto &c : bp.classes) {
        sig.push_back(c.begin);
        sig.push_back(c.count);
        sig.push_back(c.L);
    }
    return sig;
}

namespace cobs {

cobs_status engine_query(cobs_engine *eng, const uint8_t *d_bytes, const uint64_t *d_off, const uint64_t *h_off,
                         const uint16_t *d_thr, uint64_t n, uint32_t flags) {
    if (!eng || (n && (!d_bytes || !d_off || !h_off || !d_thr))) return set_error(COBS_ERR_ARG, "NULL argument");
    if (flags != COBS_PLAIN && flags != COBS_BATCHED && flags != COBS_GRAPH && flags != (COBS_GRAPH | COBS_BATCHED))
        return set_error(COBS_ERR_ARG, "flags must be COBS_PLAIN, COBS_BATCHED or COBS_GRAPH");
    if (n >= 0x7FFFFFFFULL) return set_error(COBS_ERR_ARG, "too many queries in one batch");
    if (eng->dix->streamed && flags == COBS_PLAIN)
        return set_error(COBS_ERR_ARG, "a streamed index runs the batched or graph form only");
    const auto t_host = std::chrono::steady_clock::now();
    CU(cudaSetDevice(eng->dix->device));
    if (eng->pending) {
        // the previous batch may still read the pinned plan this call refills: wait
        // for it (its results were never collected and are dropped)
        CU(cudaEventSynchronize(eng->ev_done));
        eng->pending = false;
    }
    eng->has_results = false;  // until this batch is enqueued in full
    TRY(ensure_slices(eng, eng->lanes_per_query));  // (re)made if an earlier call failed to make it
    {
        TraceRange tr("cobs.plan");
        TRY(make_plan(eng, h_off, n, flags != COBS_PLAIN, eng->bp));
        TRY(ensure_buffers(eng, eng->bp));
    }
    eng->last_bytes = d_bytes;
    eng->last_off = d_off;
    eng->last_thr = d_thr;
    eng->last_off_host.assign(h_off, h_off + n + 1);
    eng->last_flags = flags;
    if (n == 0) {
        eng->pending = false;
        eng->has_results = true;
        return COBS_OK;
    }
    fill_pinned_plan(eng);
    if (flags & COBS_GRAPH) {
        std::vector<uint64_t> sig = graph_signature(eng, d_bytes, d_off, d_thr);
        if (!eng->gexec || sig != eng->gsig) {
            if (eng->gexec) {
                cudaGraphExecDestroy(eng->gexec);
                eng->gexec = nullptr;
            }
            cudaGraph_t g = nullptr;
            CU(cudaStreamBeginCapture(eng->stream, cudaStreamCaptureModeThreadLocal));
            // the phase events become event-record nodes of the graph
            cobs_status st = enqueue(eng, d_bytes, d_off, d_thr, COBS_BATCHED, true);
            cudaError_t ce = cudaStreamEndCapture(eng->stream, &g);
            if (st != COBS_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (ce != cudaSuccess) return set_error(COBS_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&eng->gexec, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                eng->gexec = nullptr;
                return set_error(COBS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
            }
            eng->gsig = sig;
            eng->graph_stats[0] = eng->stat_launches;
            eng->graph_stats[1] = eng->stat_gather_launches;
            eng->graph_stats[2] = eng->stat_tiles;
        }
        CU(cudaGraphLaunch(eng->gexec, eng->stream));
        // kernels inside the graph
        eng->stat_launches = eng->graph_stats[0];
        eng->stat_gather_launches = eng->graph_stats[1];
        eng->stat_tiles = eng->graph_stats[2];
    } else {
        TRY(enqueue(eng, d_bytes, d_off, d_thr, flags, true));
    }
    CU(cudaEventRecord(eng->ev_done, eng->stream));
    eng->pending = true;
    eng->has_results = true;
    eng->stat_host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host).count();
    return COBS_OK;
}

// Wait for the last batch; if its hits overflowed the capacity, grow and re-run.
cobs_status engine_finish(cobs_engine *eng) {
    if (!eng->pending) return COBS_OK;
    TraceRange tr("cobs.finish");
    for (int attempt = 0; attempt < 4; attempt++) {
        CU(cudaEventSynchronize(eng->ev_done));
        if (eng->pin_count.as<uint32_t>()[2 * cobs_engine::ERR_SLOT] != 0) {
            eng->pending = false;
            eng->has_results = false;
            return set_error(COBS_ERR_TIMEOUT, "gather: a bounded wait on a TMA barrier ran out; results invalid");
        }
        unsigned long long cnt = *eng->pin_count.as<unsigned long long>();
        if (cnt <= eng->hit_cap) {
            eng->pending = false;
            return COBS_OK;
        }
        uint64_t cap = eng->hit_cap;
        while (cap < cnt) cap *= 2;
        eng->hit_cap = cap;
        eng->pending = false;
        eng->has_results = false;  // truncated hits: valid again only once the re-run is enqueued
        TRY(ensure_buffers(eng, eng->bp));
        const uint32_t fl = eng->last_flags;
        const std::vector<uint64_t> off = eng->last_off_host;  // engine_query refills last_off_host
        TRY(engine_query(eng, eng->last_bytes, eng->last_off, off.data(), eng->last_thr, eng->bp.n, fl));
    }
    return set_error(COBS_ERR_CUDA, "hit capacity kept overflowing");
}

}  // namespace cobs

extern "C" cobs_status cobs_engine_query_device(cobs_engine *eng, const uint8_t *queries_dev,
                                                const uint64_t *offsets_dev, const uint64_t *offsets_host,
                                                const uint16_t *thr_dev, uint64_t n, uint32_t flags) {
    return engine_query(eng, queries_dev, offsets_dev, offsets_host, thr_dev, n, flags);
}

extern "C" cobs_status cobs_engine_results_device(cobs_engine *eng, const uint32_t **n_terms,
                                                  const uint32_t **min_score, const uint64_t **hit_offsets,
                                                  const uint32_t **hit_ids, const uint32_t **hit_scores) {
    if (!eng) return set_error(COBS_ERR_ARG, "NULL engine");
    TRY(engine_finish(eng));
    if (!eng->has_results) return set_error(COBS_ERR_ARG, "no results: no batch ran, or the last one failed");
    if (n_terms) *n_terms = eng->ell.as<uint32_t>();
    if (min_score) *min_score = eng->minsc.as<uint32_t>();
    if (hit_offsets) *hit_offsets = eng->hitoff.as<uint64_t>();
    if (hit_ids) *hit_ids = eng->out_ids.as<uint32_t>();
    if (hit_scores) *hit_scores = eng->out_scores.as<uint32_t>();
    return COBS_OK;
}

namespace cobs {
struct ResultStore {
    cobs_result pub;
    std::vector<cobs_hits> hits;
    std::vector<uint32_t> ids, scores;
};
}  // namespace cobs

extern "C" cobs_status cobs_engine_download(cobs_engine *eng, cobs_result **out) {
    if (!eng || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    TRY(engine_finish(eng));
    if (!eng->has_results) return set_error(COBS_ERR_ARG, "no results: no batch ran, or the last one failed");
    const uint64_t n = eng->bp.n;
    ResultStore *rs = new ResultStore();
    std::vector<uint32_t> ell(n), mn(n);
    std::vector<uint64_t> off(n + 1, 0);
    cudaStream_t s = eng->stream;
    cudaError_t e = cudaSuccess;
    if (n) {
        e = cudaMemcpyAsync(ell.data(), eng->ell.p, n * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(mn.data(), eng->minsc.p, n * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(off.data(), eng->hitoff.p, (n + 1) * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    const uint64_t total = off[n];
    if (e == cudaSuccess && total) {
        rs->ids.resize(total);
        rs->scores.resize(total);
        e = cudaMemcpyAsync(rs->ids.data(), eng->out_ids.p, total * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rs->scores.data(), eng->out_scores.p, total * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) {
        delete rs;
        return set_error(COBS_ERR_CUDA, "download results: %s", cudaGetErrorString(e));
    }
    rs->hits.resize(n);
    for (uint64_t q = 0; q < n; q++) {
        cobs_hits &h = rs->hits[q];
        h.n_terms = ell[q];
        h.min_score = mn[q];
        h.n_hits = (uint32_t)(off[q + 1] - off[q]);
        h._pad = 0;
        h.doc_ids = total ? rs->ids.data() + off[q] : nullptr;
        h.scores = total ? rs->scores.data() + off[q] : nullptr;
    }
    rs->pub.n_queries = n;
    rs->pub.hits = rs->hits.data();
    *out = &rs->pub;
    return COBS_OK;
}

extern "C" void cobs_result_free(cobs_result *res) {
    if (!res) return;
    delete reinterpret_cast<ResultStore *>(reinterpret_cast<char *>(res) - offsetof(ResultStore, pub));
}

static cobs_status check_thresholds(const uint16_t *thr, uint64_t n) {
    for (uint64_t i = 0; i < n; i++)
        if (thr[i] == 0 || thr[i] > 1000)
            return set_error(COBS_ERR_ARG, "threshold of query %llu is %u permille (must be 1..1000)",
                             (unsigned long long)i, thr[i]);
    return COBS_OK;
}

extern "C" cobs_status cobs_engine_query_host(cobs_engine *eng, const uint8_t *queries, const uint64_t *offsets,
                                              const uint16_t *thr, uint64_t n, uint32_t flags, cobs_result **out) {
    if (!out) return set_error(COBS_ERR_ARG, "NULL argument");
    TRY(cobs_engine_submit_host(eng, queries, offsets, thr, n, flags));
    return cobs_engine_download(eng, out);
}

extern "C" cobs_status cobs_engine_submit_host(cobs_engine *eng, const uint8_t *queries, const uint64_t *offsets,
                                               const uint16_t *thr, uint64_t n, uint32_t flags) {
    if (!eng || !offsets || (n && (!thr || !queries))) return set_error(COBS_ERR_ARG, "NULL argument");
    TRY(engine_finish(eng));  // the staging buffers of a previous batch are free again
    TRY(check_thresholds(thr, n));
    CU(cudaSetDevice(eng->dix->device));
    const uint64_t total = offsets[n];
    const uint64_t in_bytes = total + (n + 1) * 8 + n * 2 + 64;
    CU(eng->pin_in.ensure(in_bytes));
    CU(eng->qbytes.ensure(total));
    CU(eng->qoff.ensure((n + 1) * 8));
    CU(eng->thr.ensure(n * 2 + 16));
    // Query bytes in page-locked memory are copied by DMA straight from the
    // caller's buffer; pageable bytes go through the engine's pinned staging.
    cudaPointerAttributes pa{};
    const bool pinned = total && cudaPointerGetAttributes(&pa, queries) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();  // clear a lookup failure on pageable memory
    uint8_t *pin = eng->pin_in.as<uint8_t>();
    if (total && !pinned) memcpy(pin, queries, total);
    uint64_t o1 = (total + 15) / 16 * 16, o2 = o1 + (n + 1) * 8;
    memcpy(pin + o1, offsets, (n + 1) * 8);
    if (n) memcpy(pin + o2, thr, n * 2);
    cudaStream_t s = eng->stream;
    if (total) CU(cudaMemcpyAsync(eng->qbytes.p, pinned ? queries : pin, total, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(eng->qoff.p, pin + o1, (n + 1) * 8, cudaMemcpyHostToDevice, s));
    if (n) CU(cudaMemcpyAsync(eng->thr.p, pin + o2, n * 2, cudaMemcpyHostToDevice, s));
    return engine_query(eng, eng->qbytes.as<uint8_t>(), eng->qoff.as<uint64_t>(), offsets, eng->thr.as<uint16_t>(), n,
                        flags);
}

extern "C" cobs_status cobs_query_batch(cobs_device_index *dix, const uint8_t *queries, const uint64_t *query_offsets,
                                        const uint16_t *threshold_permille, uint64_t n, uint32_t flags, void *stream,
                                        cobs_result **out) {
    if (!dix || !query_offsets || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    cobs_engine_cfg cfg{};
    cfg.max_queries = n;
    cfg.max_query_bytes = query_offsets[n];
    cobs_engine *eng = nullptr;
    TRY(cobs_engine_create(dix, &cfg, stream, &eng));
    cobs_status st = cobs_engine_query_host(eng, queries, query_offsets, threshold_permille, n, flags, out);
    cobs_engine_free(eng);
    return st;
}

extern "C" cobs_status cobs_engine_stats(cobs_engine *eng, cobs_query_stats *out) {
    if (!eng || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    TRY(engine_finish(eng));
    if (!eng->has_results) return set_error(COBS_ERR_ARG, "no statistics: no batch ran, or the last one failed");
    memset(out, 0, sizeof *out);
    float t = 0;
    if (eng->bp.n) {  // batched and graph forms: phase events; plain: ev[1] after the last terms launch
        cudaEventElapsedTime(&t, eng->ev[0], eng->ev[1]); out->ms_terms = t;
        cudaEventElapsedTime(&t, eng->ev[1], eng->ev[2]); out->ms_gather = t;
        cudaEventElapsedTime(&t, eng->ev[2], eng->ev[3]); out->ms_hits = t;
        cudaEventElapsedTime(&t, eng->ev[0], eng->ev[3]); out->ms_total = t;
    }
    const cobs_device_index *dix = eng->dix;
    uint64_t rb = 0;
    for (const auto &b : dix->blocks) rb += b.rowbytes;
    std::vector<uint32_t> ell(eng->bp.n);
    if (eng->bp.n) CU(cudaMemcpy(ell.data(), eng->ell.p, eng->bp.n * 4, cudaMemcpyDeviceToHost));
    uint64_t terms = 0;
    for (uint32_t e : ell) terms += e;
    out->terms = terms;
    out->row_bytes = terms * rb * dix->params.num_hashes;
    out->n_tiles = eng->stat_tiles;
    out->gather_launches = eng->stat_gather_launches;
    out->launches = eng->stat_launches;
    out->slice_bytes = eng->lanes_per_query * 16;
    out->ctas_per_sm = eng->ctas_per_sm;
    out->l2_hints = eng->l2_hints;
    out->split_queries = (uint32_t)eng->bp.split.size();
    out->ms_host = eng->stat_host_ms;
    out->h2d_index_bytes = eng->stat_h2d_index_bytes;
    out->split_part = eng->bp.part_terms;
    out->stream_numa_node = eng->dix->streamed ? eng->dix->host_rows.node : -1;
    return COBS_OK;
}
