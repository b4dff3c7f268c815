// Host runtime and C ABI of the COBS query engine: index planning and device
// build (Sec. 2.3 "Classic and Compact"), index transfer and files, the query
// engine with its plain, batched and graph forms, and result assembly.
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

extern "C" const char *cobs_version(void) { return "cobs_gpu 0.1 (sm_103a)"; }
extern "C" uint32_t cobs_abi_version(void) { return COBS_GPU_ABI_VERSION; }

// --------------------------------------------------------------- planning

// Sec. 2.1: the false-positive rate of a filter with w cells, h hashes and v
// elements is about (1 - e^{-hv/w})^h; solved for w at the target p.
extern "C" uint64_t cobs_bloom_width(uint32_t h, uint64_t v, double p) {
    double x = -(double)h * (double)v / std::log(1.0 - std::pow(p, 1.0 / (double)h));
    double c = std::ceil(x);
    return c < 1.0 ? 1 : (uint64_t)c;
}

static cobs_status check_params(const cobs_params *P) {
    if (!P) return set_error(COBS_ERR_ARG, "params is NULL");
    if (P->term_kind > 2) return set_error(COBS_ERR_ARG, "term_kind must be 0, 1 or 2");
    if (P->term_kind == 2 ? (P->q < 1 || P->q > 8) : (P->q < 1 || P->q > 32))
        return set_error(COBS_ERR_ARG, "q out of range for the term kind");
    if (P->num_hashes < 1 || P->num_hashes > 16) return set_error(COBS_ERR_ARG, "num_hashes must be 1..16");
    if (!(P->fpr > 0.0 && P->fpr < 1.0)) return set_error(COBS_ERR_ARG, "fpr must be in (0, 1)");
    if (P->score_bits != 16 && P->score_bits != 32) return set_error(COBS_ERR_ARG, "score_bits must be 16 or 32");
    if (P->width > 0xFFFFFFFFULL) return set_error(COBS_ERR_ARG, "width must be below 2^32");
    return COBS_OK;
}

// Classic: one block, input order.  Compact: documents ordered by (distinct
// terms, id), blocks of B consecutive documents, Bloom size of the largest
// document of each block (Sec. 2.2, Sec. 2.3).
static cobs_status plan_index(const cobs_params &P, const std::vector<uint64_t> &v,
                              std::vector<cobs_block_info> &blocks, std::vector<uint64_t> &perm) {
    const uint64_t n = v.size();
    perm.resize(n);
    std::iota(perm.begin(), perm.end(), 0ULL);
    if (P.block_docs)
        std::sort(perm.begin(), perm.end(), [&](uint64_t a, uint64_t b) { return v[a] != v[b] ? v[a] < v[b] : a < b; });
    const uint64_t B = P.block_docs ? P.block_docs : (n ? n : 1);
    blocks.clear();
    uint64_t off = 0;
    for (uint64_t begin = 0; begin < n; begin += B) {
        cobs_block_info b{};
        b.doc_begin = begin;
        b.n_docs = std::min(B, n - begin);
        for (uint64_t j = 0; j < b.n_docs; j++) b.max_terms = std::max(b.max_terms, v[perm[begin + j]]);
        b.w = P.width ? P.width : cobs_bloom_width(P.num_hashes, b.max_terms, P.fpr);
        if (b.w > 0xFFFFFFFFULL) return set_error(COBS_ERR_ARG, "block %llu needs %llu rows (limit 2^32-1)",
                                                  (unsigned long long)blocks.size(), (unsigned long long)b.w);
        b.rowbytes = (b.n_docs + 127) / 128 * 16;
        b.row_offset = off;
        off += b.w * b.rowbytes;
        blocks.push_back(b);
    }
    return COBS_OK;
}

uint64_t cobs::barrett_m_of(uint64_t w) {
    if (w <= 1) return ~0ULL;
    unsigned __int128 one = (unsigned __int128)1 << 64;
    return (uint64_t)(one / w);
}

// Upload the block table, permutation and column groups of a device index.
static cobs_status upload_tables(cobs_device_index *dix, cudaStream_t s) {
    const uint64_t nb = dix->blocks.size();
    std::vector<DevBlock> db(nb);
    std::vector<SliceDesc> pg;
    for (uint64_t b = 0; b < nb; b++) {
        const cobs_block_info &B = dix->blocks[b];
        db[b].row_offset = dix->dev_row_offset.empty() ? B.row_offset : dix->dev_row_offset[b];
        db[b].barrett_m = barrett_m_of(B.w);
        db[b].w = (uint32_t)B.w;
        db[b].rowbytes = (uint32_t)B.rowbytes;
        db[b].n_docs = (uint32_t)B.n_docs;
        db[b].doc_begin = (uint32_t)B.doc_begin;
        for (uint64_t c = 0; c < B.rowbytes; c += PLAIN_GROUP_BYTES) pg.push_back(SliceDesc{(uint32_t)b, (uint32_t)c});
    }
    dix->n_pgroups = (uint32_t)pg.size();
    std::vector<uint32_t> p32(dix->n_docs);
    for (uint64_t i = 0; i < dix->n_docs; i++) p32[i] = (uint32_t)dix->perm[i];
    CU(dix->dblocks.ensure(nb * sizeof(DevBlock)));
    CU(dix->dperm.ensure(dix->n_docs * 4));
    CU(dix->pgroups.ensure(pg.size() * sizeof(SliceDesc)));
    if (nb) CU(cudaMemcpyAsync(dix->dblocks.p, db.data(), nb * sizeof(DevBlock), cudaMemcpyHostToDevice, s));
    if (dix->n_docs) CU(cudaMemcpyAsync(dix->dperm.p, p32.data(), dix->n_docs * 4, cudaMemcpyHostToDevice, s));
    if (!pg.empty())
        CU(cudaMemcpyAsync(dix->pgroups.p, pg.data(), pg.size() * sizeof(SliceDesc), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    return COBS_OK;
}

// ------------------------------------------------------------ device build

// Distinct-term counts of the documents `docs` with one open-addressing set per
// document in global memory (cleared by a memset), in waves of documents whose
// sets fit a budget; every wave reuses the same set memory.  Adds to dv.
static cobs_status count_global(const cobs_params *P, const uint8_t *d_docs, const uint64_t *d_off,
                                const std::vector<uint64_t> &npos, const std::vector<uint32_t> &docs,
                                DevBuf &dv, DevBuf &dempty, cudaStream_t s) {
    if (docs.empty()) return COBS_OK;
    const uint64_t n_docs = npos.size();
    const uint32_t k = P->q;
    std::vector<uint32_t> chunk_doc;
    std::vector<uint64_t> chunk_p0;
    for (uint32_t d : docs)
        for (uint64_t p = 0; p < npos[d]; p += COUNT_CHUNK) {
            chunk_doc.push_back(d);
            chunk_p0.push_back(p);
        }
    const uint64_t n_chunks = chunk_doc.size();
    if (n_chunks > 0x7FFFFFFFULL) return set_error(COBS_ERR_ARG, "documents too large for one build");
    DevBuf dchunk_doc, dchunk_p0, dtbase, dtcap, dtables;
    CU(dchunk_doc.ensure(n_chunks * 4));
    CU(dchunk_p0.ensure(n_chunks * 8));
    CU(dtbase.ensure(n_docs * 8));
    CU(dtcap.ensure(n_docs * 4));
    if (n_chunks) {
        CU(cudaMemcpyAsync(dchunk_doc.p, chunk_doc.data(), n_chunks * 4, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(dchunk_p0.p, chunk_p0.data(), n_chunks * 8, cudaMemcpyHostToDevice, s));
    }
    // Build of 10,000 DNA documents (1 GB) with every document here: waves of
    // 8 GB 43.8 ms, 512 MB 40.0 ms, 128 MB 43.3 ms, 32 MB 61.1 ms.
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    uint64_t budget = std::min<uint64_t>(free_b / 4, 512ULL << 20) / 8;  // in slots
    if (budget < (1u << 20)) budget = 1u << 20;
    if (build_scratch_override()) budget = std::max<uint64_t>(build_scratch_override() / 8, 16);
    std::vector<uint64_t> tbase(n_docs, 0);
    std::vector<uint32_t> tcap(n_docs, 0);
    struct Wave { uint64_t i0, i1, c0, c1, slots; };  // docs[i0, i1), chunks [c0, c1)
    std::vector<Wave> waves;
    {
        uint64_t i = 0, c = 0;
        while (i < docs.size()) {
            Wave wv{i, i, c, c, 0};
            while (i < docs.size()) {
                const uint32_t d = docs[i];
                const uint64_t sl = set_slots(npos[d]);
                if (sl > 0xFFFFFFFFULL) return set_error(COBS_ERR_ARG, "document %u too long", d);
                if (wv.i1 > wv.i0 && wv.slots + sl > budget) break;
                tbase[d] = wv.slots;
                tcap[d] = (uint32_t)sl;
                wv.slots += sl;
                while (c < n_chunks && chunk_doc[c] == d) c++;
                i++;
                wv.i1 = i;
                wv.c1 = c;
            }
            waves.push_back(wv);
        }
    }
    uint64_t max_slots = 16;
    for (const Wave &wv : waves) max_slots = std::max(max_slots, wv.slots);
    CU(dtables.ensure(max_slots * 8));
    CU(cudaMemcpyAsync(dtbase.p, tbase.data(), n_docs * 8, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(dtcap.p, tcap.data(), n_docs * 4, cudaMemcpyHostToDevice, s));
    for (const Wave &wv : waves) {
        CU(cudaMemsetAsync(dtables.p, 0xFF, wv.slots * 8, s));
        CountArgs ca{};
        ca.docs = d_docs;
        ca.doc_off = d_off;
        ca.chunk_doc = dchunk_doc.as<uint32_t>() + wv.c0;
        ca.chunk_p0 = dchunk_p0.as<uint64_t>() + wv.c0;
        ca.table_base = dtbase.as<uint64_t>();
        ca.table_cap = dtcap.as<uint32_t>();
        ca.tables = dtables.as<unsigned long long>();
        ca.v = dv.as<unsigned long long>();
        ca.has_empty = dempty.as<uint32_t>();
        ca.kind = P->term_kind;
        ca.k = k;
        launch_doc_count(ca, (uint32_t)(wv.c1 - wv.c0), s);
        CU(cudaGetLastError());
    }
    CU(cudaStreamSynchronize(s));  // the staging buffers above are freed on return
    return COBS_OK;
}

// Distinct-term counts of the documents `docs` by hash partitions (scatter, then
// a shared-memory set per partition), in waves whose partitions fit a budget.
// Adds to dv; returns in `overflowed` the documents whose count is incomplete
// (a partition got more terms than its capacity) and must come from elsewhere.
static cobs_status count_partitioned(const cobs_params *P, const uint8_t *d_docs, const uint64_t *d_off,
                                     const std::vector<uint64_t> &npos, const std::vector<uint32_t> &docs,
                                     DevBuf &dv, DevBuf &dempty, cudaStream_t s, std::vector<uint32_t> &overflowed) {
    overflowed.clear();
    if (docs.empty()) return COBS_OK;
    const uint64_t n_docs = npos.size();
    std::vector<uint32_t> n_parts(n_docs, 0), part_cap(n_docs, 0);
    std::vector<uint64_t> part0(n_docs, 0), code0(n_docs, 0);
    std::vector<uint32_t> chunk_doc, part_doc, part_idx;
    std::vector<uint64_t> chunk_p0;
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    uint64_t budget = std::min<uint64_t>(free_b / 4, 2ULL << 30);  // bytes of partitions per wave
    if (build_scratch_override()) budget = build_scratch_override();
    struct Wave { uint64_t c0, c1, q0, q1, slots; };  // chunks [c0, c1), partitions [q0, q1), term slots
    std::vector<Wave> waves;
    Wave wv{0, 0, 0, 0, 0};
    for (uint32_t d : docs) {
        const uint64_t np = npos[d];
        const uint64_t pd = std::max<uint64_t>(1, (np + PART_WINDOWS - 1) / PART_WINDOWS);
        const uint64_t mean = (np + pd - 1) / pd;
        // mean + 8 standard deviations of a binomial partition size, + 64
        const uint64_t cap = mean + 8 * (uint64_t)std::ceil(std::sqrt((double)mean)) + 64;
        const uint64_t need = pd * cap;
        if (wv.q1 > wv.q0 && (wv.slots + need) * 8 > budget) {
            waves.push_back(wv);
            wv = Wave{wv.c1, wv.c1, wv.q1, wv.q1, 0};
        }
        n_parts[d] = (uint32_t)pd;
        part_cap[d] = (uint32_t)cap;
        part0[d] = wv.q1 - wv.q0;
        code0[d] = wv.slots;
        for (uint64_t p = 0; p < np; p += COUNT_CHUNK) {
            chunk_doc.push_back(d);
            chunk_p0.push_back(p);
        }
        for (uint32_t i = 0; i < pd; i++) {
            part_doc.push_back(d);
            part_idx.push_back(i);
        }
        wv.c1 = chunk_doc.size();
        wv.q1 = part_doc.size();
        wv.slots += need;
    }
    waves.push_back(wv);
    const uint64_t n_chunks = chunk_doc.size(), n_part = part_doc.size();
    if (n_chunks > 0x7FFFFFFFULL || n_part > 0x7FFFFFFFULL)
        return set_error(COBS_ERR_ARG, "documents too large for one build");
    uint64_t max_slots = 1, max_parts = 1;
    for (const Wave &w : waves) {
        max_slots = std::max(max_slots, w.slots);
        max_parts = std::max(max_parts, w.q1 - w.q0);
    }
    DevBuf dchunk_doc, dchunk_p0, dpart_doc, dpart_idx, dn_parts, dpart0, dcap, dcode0, dcount, dcodes, dover;
    CU(dchunk_doc.ensure(n_chunks * 4));
    CU(dchunk_p0.ensure(n_chunks * 8));
    CU(dpart_doc.ensure(n_part * 4));
    CU(dpart_idx.ensure(n_part * 4));
    CU(dn_parts.ensure(n_docs * 4));
    CU(dpart0.ensure(n_docs * 8));
    CU(dcap.ensure(n_docs * 4));
    CU(dcode0.ensure(n_docs * 8));
    CU(dover.ensure(n_docs * 4));
    CU(dcount.ensure(max_parts * 4));
    CU(dcodes.ensure(max_slots * 8));
    if (n_chunks) {
        CU(cudaMemcpyAsync(dchunk_doc.p, chunk_doc.data(), n_chunks * 4, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(dchunk_p0.p, chunk_p0.data(), n_chunks * 8, cudaMemcpyHostToDevice, s));
    }
    CU(cudaMemcpyAsync(dpart_doc.p, part_doc.data(), n_part * 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(dpart_idx.p, part_idx.data(), n_part * 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(dn_parts.p, n_parts.data(), n_docs * 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(dpart0.p, part0.data(), n_docs * 8, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(dcap.p, part_cap.data(), n_docs * 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(dcode0.p, code0.data(), n_docs * 8, cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(dover.p, 0, n_docs * 4, s));
    for (const Wave &w : waves) {
        CU(cudaMemsetAsync(dcount.p, 0, (w.q1 - w.q0) * 4, s));
        PartArgs pa{};
        pa.docs = d_docs;
        pa.doc_off = d_off;
        pa.chunk_doc = dchunk_doc.as<uint32_t>() + w.c0;
        pa.chunk_p0 = dchunk_p0.as<uint64_t>() + w.c0;
        pa.part_doc = dpart_doc.as<uint32_t>() + w.q0;
        pa.part_idx = dpart_idx.as<uint32_t>() + w.q0;
        pa.n_parts = dn_parts.as<uint32_t>();
        pa.part0 = dpart0.as<uint64_t>();
        pa.part_cap = dcap.as<uint32_t>();
        pa.code0 = dcode0.as<uint64_t>();
        pa.part_count = dcount.as<uint32_t>();
        pa.codes = dcodes.as<unsigned long long>();
        pa.v = dv.as<unsigned long long>();
        pa.has_empty = dempty.as<uint32_t>();
        pa.overflow = dover.as<uint32_t>();
        pa.kind = P->term_kind;
        pa.k = P->q;
        launch_part_scatter(pa, (uint32_t)(w.c1 - w.c0), s);
        launch_part_count(pa, (uint32_t)(w.q1 - w.q0), s);
        CU(cudaGetLastError());
    }
    std::vector<uint32_t> over(n_docs);
    CU(cudaMemcpyAsync(over.data(), dover.p, n_docs * 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (uint32_t d : docs)
        if (over[d]) overflowed.push_back(d);
    return COBS_OK;
}

// Distinct-term counts v[d] of documents on the device (the sizes of Sec. 2.3,
// determined before the blocks are planned), and their window counts npos[d].
static cobs_status count_terms(const cobs_params *P, const uint8_t *d_docs, const uint64_t *d_off,
                               const uint64_t *h_off, uint64_t n_docs, cudaStream_t s, std::vector<uint64_t> &npos,
                               std::vector<uint64_t> &v) {
    if (n_docs >= 0xFFFFFFFFULL) return set_error(COBS_ERR_ARG, "n_docs must be < 2^32");
    const uint32_t k = P->q;
    npos.assign(n_docs, 0);
    std::vector<uint32_t> part_docs, global_docs;
    for (uint64_t d = 0; d < n_docs; d++) {
        if (h_off[d + 1] < h_off[d]) return set_error(COBS_ERR_ARG, "document offsets decrease at %llu",
                                                      (unsigned long long)d);
        const uint64_t len = h_off[d + 1] - h_off[d];
        npos[d] = len >= k ? len - k + 1 : 0;
        if (npos[d] == 0) continue;  // no terms: v = 0
        if ((npos[d] + PART_WINDOWS - 1) / PART_WINDOWS <= PART_MAX) part_docs.push_back((uint32_t)d);
        else global_docs.push_back((uint32_t)d);
    }
    // counts and EMPTY flags of the two methods kept apart: a document counted
    // again with a global set takes that count
    DevBuf dv_p, de_p, dv_g, de_g;
    CU(dv_p.ensure(n_docs * 8));
    CU(de_p.ensure(n_docs * 4));
    CU(dv_g.ensure(n_docs * 8));
    CU(de_g.ensure(n_docs * 4));
    if (n_docs) {
        CU(cudaMemsetAsync(dv_p.p, 0, n_docs * 8, s));
        CU(cudaMemsetAsync(de_p.p, 0, n_docs * 4, s));
        CU(cudaMemsetAsync(dv_g.p, 0, n_docs * 8, s));
        CU(cudaMemsetAsync(de_g.p, 0, n_docs * 4, s));
    }
    std::vector<uint32_t> overflowed;
    TRY(count_partitioned(P, d_docs, d_off, npos, part_docs, dv_p, de_p, s, overflowed));
    global_docs.insert(global_docs.end(), overflowed.begin(), overflowed.end());
    TRY(count_global(P, d_docs, d_off, npos, global_docs, dv_g, de_g, s));
    std::vector<uint64_t> vg(n_docs);
    v.assign(n_docs, 0);
    if (n_docs) {
        CU(cudaMemcpyAsync(v.data(), dv_p.p, n_docs * 8, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(vg.data(), dv_g.p, n_docs * 8, cudaMemcpyDeviceToHost, s));
    }
    CU(cudaStreamSynchronize(s));
    for (uint32_t d : global_docs) v[d] = vg[d];
    return COBS_OK;
}

// Bloom bits of documents: document d goes to column doc_col[d] of block
// doc_block[d] of the rows at rows32 (block table at dblocks).  Work in the
// order `order` (documents by column: CTAs that run together set bits of
// neighbouring columns, i.e. of the same 32-bit words of every row, so the words
// being updated stay in L2).
static cobs_status set_doc_bits(const cobs_params *P, const uint8_t *d_docs, const uint64_t *d_off,
                                const std::vector<uint64_t> &npos, const std::vector<uint64_t> &order,
                                const std::vector<uint32_t> &doc_block, const std::vector<uint32_t> &doc_col,
                                const DevBlock *dblocks, uint32_t *rows32, cudaStream_t s) {
    const uint64_t n_docs = npos.size();
    DevBuf ddocblk, ddoccol, dchunk_doc, dchunk_p0;
    CU(ddocblk.ensure(n_docs * 4));
    CU(ddoccol.ensure(n_docs * 4));
    if (n_docs) {
        CU(cudaMemcpyAsync(ddocblk.p, doc_block.data(), n_docs * 4, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(ddoccol.p, doc_col.data(), n_docs * 4, cudaMemcpyHostToDevice, s));
    }
    std::vector<uint32_t> sb_doc;
    std::vector<uint64_t> sb_p0;
    for (uint64_t d : order)
        for (uint64_t p = 0; p < npos[d]; p += SETBITS_CHUNK) {
            sb_doc.push_back((uint32_t)d);
            sb_p0.push_back(p);
        }
    const uint64_t n_sb = sb_doc.size();
    if (n_sb > 0x7FFFFFFFULL) return set_error(COBS_ERR_ARG, "documents too large for one build");
    CU(dchunk_doc.ensure(n_sb * 4));
    CU(dchunk_p0.ensure(n_sb * 8));
    if (n_sb) {
        CU(cudaMemcpyAsync(dchunk_doc.p, sb_doc.data(), n_sb * 4, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(dchunk_p0.p, sb_p0.data(), n_sb * 8, cudaMemcpyHostToDevice, s));
    }
    SetBitsArgs sa{};
    sa.docs = d_docs;
    sa.doc_off = d_off;
    sa.chunk_doc = dchunk_doc.as<uint32_t>();
    sa.chunk_p0 = dchunk_p0.as<uint64_t>();
    sa.doc_block = ddocblk.as<uint32_t>();
    sa.doc_col = ddoccol.as<uint32_t>();
    sa.blocks = dblocks;
    sa.rows32 = rows32;
    sa.kind = P->term_kind;
    sa.k = P->q;
    sa.h = P->num_hashes;
    launch_doc_setbits(sa, (uint32_t)n_sb, s);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(s));  // the staging buffers above are freed on return
    return COBS_OK;
}

// Bloom bits of a freshly planned index (rows zeroed, tables uploaded): blocks
// whose filter fits in shared memory by per-document filters and a transpose,
// in waves of whole 256-column tiles whose filters fit a scratch budget; the
// other blocks by the atomic bit-set.
static cobs_status set_block_bits(const cobs_params *P, const uint8_t *d_docs, const uint64_t *d_off,
                                  const std::vector<uint64_t> &npos, cobs_device_index *dix,
                                  const std::vector<uint32_t> &doc_block, const std::vector<uint32_t> &doc_col,
                                  cudaStream_t s) {
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    const uint64_t budget = build_scratch_override() ? build_scratch_override() : std::min<uint64_t>(free_b / 4, 1ULL << 30);
    std::vector<uint64_t> rest;  // documents of the other blocks, by column
    DevBuf dfilt;
    for (uint64_t b = 0; b < dix->blocks.size(); b++) {
        const cobs_block_info &B = dix->blocks[b];
        const uint64_t pitch = (B.w + 255) / 256 * 8;  // ceil(w / 32) words, rounded up to 8
        if (pitch * 4 > FILTER_SMEM_MAX) {
            for (uint64_t j = 0; j < B.n_docs; j++) rest.push_back(dix->perm[B.doc_begin + j]);
            continue;
        }
        uint64_t C = budget / (pitch * 4) / TRANSPOSE_DOCS * TRANSPOSE_DOCS;
        if (C < TRANSPOSE_DOCS) C = TRANSPOSE_DOCS;
        if (C > B.n_docs) C = (B.n_docs + TRANSPOSE_DOCS - 1) / TRANSPOSE_DOCS * TRANSPOSE_DOCS;
        CU(dfilt.ensure(C * pitch * 4));
        for (uint64_t c = 0; c < B.n_docs; c += C) {
            const uint32_t n_cols = (uint32_t)std::min<uint64_t>(C, B.n_docs - c);
            FilterArgs fa{};
            fa.docs = d_docs;
            fa.doc_off = d_off;
            fa.col_doc = dix->dperm.as<uint32_t>() + B.doc_begin + c;  // column -> original document
            fa.filters = dfilt.as<uint32_t>();
            fa.pitch_words = (uint32_t)pitch;
            fa.w = (uint32_t)B.w;
            fa.barrett_m = barrett_m_of(B.w);
            fa.kind = P->term_kind;
            fa.k = P->q;
            fa.h = P->num_hashes;
            launch_doc_filter(fa, n_cols, s);
            TransposeArgs ta{};
            ta.filters = dfilt.as<uint32_t>();
            ta.pitch_words = (uint32_t)pitch;
            ta.n_cols = n_cols;
            ta.col0 = (uint32_t)c;
            ta.w = (uint32_t)B.w;
            ta.rowbytes = (uint32_t)B.rowbytes;
            ta.rows = dix->rows.as<uint8_t>() + B.row_offset;
            launch_filter_transpose(ta, s);
            CU(cudaGetLastError());
        }
    }
    if (!rest.empty())
        TRY(set_doc_bits(P, d_docs, d_off, npos, rest, doc_block, doc_col, dix->dblocks.as<DevBlock>(),
                         dix->rows.as<uint32_t>(), s));
    CU(cudaStreamSynchronize(s));  // the filter scratch is freed on return
    return COBS_OK;
}

static cobs_status build_impl(const cobs_params *P, const uint8_t *d_docs, const uint64_t *d_off,
                              const uint64_t *h_off, uint64_t n_docs, int device, cudaStream_t s,
                              cobs_device_index **out) {
    TraceRange tr("cobs.build");
    TRY(check_params(P));
    std::vector<uint64_t> npos, v;
    {
        TraceRange tr_count("cobs.build.count");
        TRY(count_terms(P, d_docs, d_off, h_off, n_docs, s, npos, v));
    }

    // Plan on the host, then set the Bloom bits on the device.
    cobs_device_index *dix = new cobs_device_index();
    dix->params = *P;
    dix->device = device;
    dix->n_docs = n_docs;
    dix->nterms = v;
    cobs_status st = plan_index(*P, v, dix->blocks, dix->perm);
    if (st != COBS_OK) { delete dix; return st; }
    dix->rows_bytes = dix->blocks.empty() ? 0 : dix->blocks.back().row_offset + dix->blocks.back().w * dix->blocks.back().rowbytes;
    auto fail = [&](cobs_status e) {
        cudaStreamSynchronize(s);  // work already queued may still use the buffers
        delete dix;
        return e;
    };
    cudaError_t ce = dix->rows.ensure(dix->rows_bytes);
    if (ce != cudaSuccess) return fail(set_error(COBS_ERR_OOM, "index rows (%llu bytes): %s",
                                                 (unsigned long long)dix->rows_bytes, cudaGetErrorString(ce)));
    if (dix->rows_bytes && (ce = cudaMemsetAsync(dix->rows.p, 0, dix->rows_bytes, s)) != cudaSuccess)
        return fail(set_error(COBS_ERR_CUDA, "memset rows: %s", cudaGetErrorString(ce)));
    st = upload_tables(dix, s);
    if (st != COBS_OK) return fail(st);
    std::vector<uint32_t> doc_block(n_docs), doc_col(n_docs);
    for (uint64_t b = 0; b < dix->blocks.size(); b++)
        for (uint64_t j = 0; j < dix->blocks[b].n_docs; j++) {
            uint64_t d = dix->perm[dix->blocks[b].doc_begin + j];
            doc_block[d] = (uint32_t)b;
            doc_col[d] = (uint32_t)j;
        }
    {
        TraceRange tr_bits("cobs.build.bits");
        st = set_block_bits(P, d_docs, d_off, npos, dix, doc_block, doc_col, s);
    }
    if (st != COBS_OK) return fail(st);
    *out = dix;
    return COBS_OK;
}

extern "C" cobs_status cobs_build_device_resident(const cobs_params *params, const uint8_t *docs_dev,
                                                  const uint64_t *doc_offsets_dev, const uint64_t *doc_offsets_host,
                                                  uint64_t n_docs, void *stream, cobs_device_index **out) {
    if (!out || (n_docs && (!docs_dev || !doc_offsets_dev || !doc_offsets_host)))
        return set_error(COBS_ERR_ARG, "NULL argument");
    int dev = 0;
    CU(cudaGetDevice(&dev));
    return build_impl(params, docs_dev, doc_offsets_dev, doc_offsets_host, n_docs, dev, (cudaStream_t)stream, out);
}

extern "C" cobs_status cobs_build_device(const cobs_params *params, const uint8_t *docs, const uint64_t *doc_offsets,
                                         uint64_t n_docs, int device, void *stream, cobs_device_index **out) {
    if (!out || !doc_offsets || (n_docs && !docs)) return set_error(COBS_ERR_ARG, "NULL argument");
    TRY(check_params(params));
    CU(cudaSetDevice(device));
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t total = doc_offsets[n_docs];
    DevBuf dd, doff;
    CU(dd.ensure(total));
    CU(doff.ensure((n_docs + 1) * 8));
    if (total) CU(cudaMemcpyAsync(dd.p, docs, total, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(doff.p, doc_offsets, (n_docs + 1) * 8, cudaMemcpyHostToDevice, s));
    return build_impl(params, dd.as<uint8_t>(), doff.as<uint64_t>(), doc_offsets, n_docs, device, s, out);
}

extern "C" cobs_status cobs_device_index_download(const cobs_device_index *dix, cobs_index **out) {
    if (!dix || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    CU(cudaSetDevice(dix->device));
    cobs_index *ix = new cobs_index();
    ix->params = dix->params;
    ix->n_docs = dix->n_docs;
    ix->blocks = dix->blocks;
    ix->perm = dix->perm;
    ix->nterms = dix->nterms;
    ix->rows.resize(dix->rows_bytes);
    if (dix->rows_bytes && dix->streamed) {
        memcpy(ix->rows.data(), dix->host_rows.p, dix->rows_bytes);
    } else if (dix->rows_bytes && dix->rows_view) {
        for (size_t b = 0; b < dix->blocks.size(); b++) {
            const cobs_block_info &B = dix->blocks[b];
            cudaError_t e = cudaMemcpy(ix->rows.data() + B.row_offset, dix->rows_view + dix->dev_row_offset[b],
                                       B.w * B.rowbytes, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                delete ix;
                return set_error(COBS_ERR_CUDA, "download rows: %s", cudaGetErrorString(e));
            }
        }
    } else if (dix->rows_bytes) {
        cudaError_t e = cudaMemcpy(ix->rows.data(), dix->rows.p, dix->rows_bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            delete ix;
            return set_error(COBS_ERR_CUDA, "download rows: %s", cudaGetErrorString(e));
        }
    }
    *out = ix;
    return COBS_OK;
}

extern "C" cobs_status cobs_build(const cobs_params *params, const uint8_t *docs, const uint64_t *doc_offsets,
                                  uint64_t n_docs, cobs_index **out) {
    cobs_device_index *dix = nullptr;
    int dev = 0;
    CU(cudaGetDevice(&dev));
    TRY(cobs_build_device(params, docs, doc_offsets, n_docs, dev, nullptr, &dix));
    cobs_status s = cobs_device_index_download(dix, out);
    delete dix;
    return s;
}

// Resident: rows copied to device memory.  Streamed: rows copied to pinned host
// memory, streamed block by block by the engines.
static cobs_status load_impl(const cobs_index *ix, int device, void *stream, bool streamed, cobs_device_index **out) {
    TraceRange tr("cobs.load");
    if (!ix || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    TRY(check_params(&ix->params));
    CU(cudaSetDevice(device));
    cobs_device_index *dix = new cobs_device_index();
    dix->params = ix->params;
    dix->device = device;
    dix->n_docs = ix->n_docs;
    dix->blocks = ix->blocks;
    dix->perm = ix->perm;
    dix->nterms = ix->nterms;
    dix->rows_bytes = ix->rows.size();
    dix->streamed = streamed;
    for (const auto &b : ix->blocks) dix->max_block_bytes = std::max<uint64_t>(dix->max_block_bytes, b.w * b.rowbytes);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (streamed) {
        e = dix->host_rows.ensure(dix->rows_bytes);
        if (e == cudaSuccess && dix->rows_bytes) memcpy(dix->host_rows.p, ix->rows.data(), dix->rows_bytes);
    } else {
        e = dix->rows.ensure(dix->rows_bytes);
        if (e == cudaSuccess && dix->rows_bytes)
            e = cudaMemcpyAsync(dix->rows.p, ix->rows.data(), dix->rows_bytes, cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) {
        delete dix;
        return set_error(e == cudaErrorMemoryAllocation ? COBS_ERR_OOM : COBS_ERR_CUDA, "load rows: %s",
                         cudaGetErrorString(e));
    }
    cobs_status st = upload_tables(dix, s);
    if (st != COBS_OK) {
        delete dix;
        return st;
    }
    *out = dix;
    return COBS_OK;
}

extern "C" cobs_status cobs_load_device(const cobs_index *ix, int device, void *stream, cobs_device_index **out) {
    return load_impl(ix, device, stream, false, out);
}

extern "C" cobs_status cobs_load_device_streamed(const cobs_index *ix, int device, void *stream,
                                                 cobs_device_index **out) {
    return load_impl(ix, device, stream, true, out);
}

extern "C" cobs_status cobs_multi_index_create(cobs_device_index *const *parts, uint64_t n_parts,
                                               cobs_device_index **out) {
    if (!parts || !n_parts || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    for (uint64_t i = 0; i < n_parts; i++) {
        const cobs_device_index *p = parts[i];
        if (!p) return set_error(COBS_ERR_ARG, "part %llu is NULL", (unsigned long long)i);
        if (p->streamed) return set_error(COBS_ERR_ARG, "part %llu is streamed; parts must be resident",
                                          (unsigned long long)i);
        const cobs_params &A = parts[0]->params, &B = p->params;
        if (p->device != parts[0]->device) return set_error(COBS_ERR_ARG, "parts on different devices");
        if (A.term_kind != B.term_kind || A.q != B.q || A.num_hashes != B.num_hashes)
            return set_error(COBS_ERR_ARG, "parts differ in term kind, q or number of hashes");
    }
    CU(cudaSetDevice(parts[0]->device));
    cobs_device_index *dix = new cobs_device_index();
    dix->params = parts[0]->params;
    dix->device = parts[0]->device;
    std::vector<uintptr_t> addr;  // device address of every block's rows
    for (uint64_t i = 0; i < n_parts; i++) {
        const cobs_device_index *p = parts[i];
        dix->params.score_bits = std::max(dix->params.score_bits, p->params.score_bits);
        dix->params.block_docs = std::max(dix->params.block_docs, p->params.block_docs);
        if (p->params.width != dix->params.width) dix->params.width = 0;
        for (size_t b = 0; b < p->blocks.size(); b++) {
            cobs_block_info B = p->blocks[b];
            addr.push_back((uintptr_t)p->dev_rows() + (p->dev_row_offset.empty() ? B.row_offset : p->dev_row_offset[b]));
            B.row_offset = dix->rows_bytes;
            B.doc_begin += dix->n_docs;
            dix->rows_bytes += B.w * B.rowbytes;
            dix->max_block_bytes = std::max<uint64_t>(dix->max_block_bytes, B.w * B.rowbytes);
            dix->blocks.push_back(B);
        }
        for (uint64_t id : p->perm) dix->perm.push_back(id + dix->n_docs);
        dix->nterms.insert(dix->nterms.end(), p->nterms.begin(), p->nterms.end());
        dix->n_docs += p->n_docs;
    }
    if (dix->blocks.size() > 1 && dix->params.block_docs == 0) {
        uint64_t bmax = 0;
        for (const auto &b : dix->blocks) bmax = std::max(bmax, b.n_docs);
        dix->params.block_docs = bmax;  // several blocks: no longer one classic block
    }
    if (!addr.empty()) {
        const uintptr_t base = *std::min_element(addr.begin(), addr.end());
        dix->rows_view = (const uint8_t *)base;
        for (uintptr_t x : addr) dix->dev_row_offset.push_back((uint64_t)(x - base));
    }
    cobs_status st = upload_tables(dix, nullptr);
    if (st != COBS_OK) {
        delete dix;
        return st;
    }
    *out = dix;
    return COBS_OK;
}

extern "C" void cobs_index_free(cobs_index *ix) { delete ix; }
extern "C" void cobs_device_index_free(cobs_device_index *dix) {
    if (!dix) return;
    cudaSetDevice(dix->device);
    delete dix;
}

extern "C" cobs_status cobs_index_info(const cobs_index *ix, cobs_params *params, uint64_t *n_docs,
                                       uint64_t *n_blocks, const cobs_block_info **blocks, const uint64_t **perm,
                                       const uint64_t **nterms, const uint8_t **rows, uint64_t *rows_bytes) {
    if (!ix) return set_error(COBS_ERR_ARG, "NULL index");
    if (params) *params = ix->params;
    if (n_docs) *n_docs = ix->n_docs;
    if (n_blocks) *n_blocks = ix->blocks.size();
    if (blocks) *blocks = ix->blocks.data();
    if (perm) *perm = ix->perm.data();
    if (nterms) *nterms = ix->nterms.data();
    if (rows) *rows = ix->rows.data();
    if (rows_bytes) *rows_bytes = ix->rows.size();
    return COBS_OK;
}

extern "C" cobs_status cobs_device_index_info(const cobs_device_index *dix, cobs_params *params, uint64_t *n_docs,
                                              uint64_t *n_blocks, const cobs_block_info **blocks,
                                              const void **rows_dev, uint64_t *rows_bytes) {
    if (!dix) return set_error(COBS_ERR_ARG, "NULL index");
    if (params) *params = dix->params;
    if (n_docs) *n_docs = dix->n_docs;
    if (n_blocks) *n_blocks = dix->blocks.size();
    if (blocks) *blocks = dix->blocks.data();
    if (rows_dev) *rows_dev = (dix->streamed || dix->rows_view) ? nullptr : dix->rows.p;
    if (rows_bytes) *rows_bytes = dix->rows_bytes;
    return COBS_OK;
}

// ------------------------------------------------------------------ insert
extern "C" cobs_status cobs_index_insert(const cobs_index *ix, const uint8_t *docs, const uint64_t *doc_offsets,
                                         uint64_t n_new, int device, cobs_index **out) {
    if (!ix || !out || !doc_offsets || (n_new && !docs)) return set_error(COBS_ERR_ARG, "NULL argument");
    TRY(check_params(&ix->params));
    if (ix->n_docs + n_new >= 0xFFFFFFFFULL) return set_error(COBS_ERR_ARG, "n_docs must be < 2^32");
    const cobs_params &P = ix->params;
    CU(cudaSetDevice(device));
    cudaStream_t s = nullptr;
    const uint64_t total = doc_offsets[n_new];
    DevBuf dd, doff;
    CU(dd.ensure(total));
    CU(doff.ensure((n_new + 1) * 8));
    if (total) CU(cudaMemcpyAsync(dd.p, docs, total, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(doff.p, doc_offsets, (n_new + 1) * 8, cudaMemcpyHostToDevice, s));
    std::vector<uint64_t> npos, v;
    TRY(count_terms(&P, dd.as<uint8_t>(), doff.as<uint64_t>(), doc_offsets, n_new, s, npos, v));

    // Best free block: the one with the smallest largest-document count that is
    // still at least the new document's (its Bloom size keeps the rate) and has
    // a free column; ties to the lower block.  New documents in input order.
    const uint64_t n_old = ix->n_docs, nb_old = ix->blocks.size();
    std::vector<uint64_t> free_cols(nb_old);
    for (uint64_t b = 0; b < nb_old; b++) free_cols[b] = ix->blocks[b].rowbytes * 8 - ix->blocks[b].n_docs;
    std::vector<std::vector<uint64_t>> added(nb_old);
    std::vector<uint64_t> left;  // new documents no block takes
    std::vector<uint32_t> doc_block(n_new), doc_col(n_new);
    for (uint64_t j = 0; j < n_new; j++) {
        int64_t best = -1;
        for (uint64_t b = 0; b < nb_old; b++)
            if (free_cols[b] && ix->blocks[b].max_terms >= v[j] &&
                (best < 0 || ix->blocks[b].max_terms < ix->blocks[best].max_terms))
                best = (int64_t)b;
        if (best < 0) {
            left.push_back(j);
            continue;
        }
        doc_block[j] = (uint32_t)best;
        doc_col[j] = (uint32_t)(ix->blocks[best].n_docs + added[best].size());
        added[best].push_back(j);
        free_cols[best]--;
    }
    // the rest form blocks of their own, planned like a build over them alone
    std::vector<uint64_t> vl(left.size());
    for (size_t i = 0; i < left.size(); i++) vl[i] = v[left[i]];
    std::vector<cobs_block_info> nblocks;
    std::vector<uint64_t> nperm;
    TRY(plan_index(P, vl, nblocks, nperm));

    cobs_index *res = new cobs_index();
    res->params = P;
    res->n_docs = n_old + n_new;
    res->nterms = ix->nterms;
    res->nterms.insert(res->nterms.end(), v.begin(), v.end());
    uint64_t pos = 0;
    for (uint64_t b = 0; b < nb_old; b++) {
        cobs_block_info B = ix->blocks[b];
        for (uint64_t i = 0; i < B.n_docs; i++) res->perm.push_back(ix->perm[B.doc_begin + i]);
        for (uint64_t j : added[b]) res->perm.push_back(n_old + j);
        B.doc_begin = pos;
        B.n_docs += added[b].size();
        pos += B.n_docs;
        res->blocks.push_back(B);
    }
    const uint64_t old_bytes = ix->rows.size();
    for (size_t nbi = 0; nbi < nblocks.size(); nbi++) {
        cobs_block_info B = nblocks[nbi];
        for (uint64_t i = 0; i < B.n_docs; i++) {
            const uint64_t j = left[nperm[B.doc_begin + i]];
            res->perm.push_back(n_old + j);
            doc_block[j] = (uint32_t)(nb_old + nbi);
            doc_col[j] = (uint32_t)i;
        }
        B.doc_begin = pos;
        B.row_offset += old_bytes;
        pos += B.n_docs;
        res->blocks.push_back(B);
    }
    if (res->blocks.size() > 1 && res->params.block_docs == 0) {
        uint64_t bmax = 0;
        for (const auto &b : res->blocks) bmax = std::max(bmax, b.n_docs);
        res->params.block_docs = bmax;  // several blocks: no longer one classic block
    }
    const uint64_t new_bytes = nblocks.empty() ? 0 : nblocks.back().row_offset + nblocks.back().w * nblocks.back().rowbytes;

    // rows on the device: the old ones, the new blocks cleared, then the new bits
    cobs_device_index tmp;
    tmp.params = res->params;
    tmp.device = device;
    tmp.n_docs = res->n_docs;
    tmp.blocks = res->blocks;
    tmp.perm = res->perm;
    tmp.rows_bytes = old_bytes + new_bytes;
    auto fail = [&](cobs_status e) {
        cudaStreamSynchronize(s);  // work already queued may still use the buffers
        delete res;
        return e;
    };
    cudaError_t ce = tmp.rows.ensure(tmp.rows_bytes);
    if (ce == cudaSuccess && old_bytes) ce = cudaMemcpyAsync(tmp.rows.p, ix->rows.data(), old_bytes, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess && new_bytes) ce = cudaMemsetAsync(tmp.rows.as<uint8_t>() + old_bytes, 0, new_bytes, s);
    if (ce != cudaSuccess) return fail(set_error(COBS_ERR_OOM, "insert rows: %s", cudaGetErrorString(ce)));
    cobs_status st = upload_tables(&tmp, s);
    if (st != COBS_OK) return fail(st);
    std::vector<uint64_t> order;  // by column: old blocks' new documents, then the new blocks
    for (uint64_t b = 0; b < nb_old; b++) order.insert(order.end(), added[b].begin(), added[b].end());
    for (size_t nbi = 0; nbi < nblocks.size(); nbi++)
        for (uint64_t i = 0; i < nblocks[nbi].n_docs; i++) order.push_back(left[nperm[nblocks[nbi].doc_begin + i]]);
    st = set_doc_bits(&P, dd.as<uint8_t>(), doff.as<uint64_t>(), npos, order, doc_block, doc_col,
                      tmp.dblocks.as<DevBlock>(), tmp.rows.as<uint32_t>(), s);
    if (st != COBS_OK) return fail(st);
    res->rows.resize(tmp.rows_bytes);
    if (tmp.rows_bytes &&
        (ce = cudaMemcpy(res->rows.data(), tmp.rows.p, tmp.rows_bytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(set_error(COBS_ERR_CUDA, "insert download: %s", cudaGetErrorString(ce)));
    *out = res;
    return COBS_OK;
}

// ------------------------------------------------------------------ merge
extern "C" cobs_status cobs_index_merge(const cobs_index *a, const cobs_index *b, cobs_index **out) {
    if (!a || !b || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    const cobs_params &A = a->params, &B = b->params;
    if (A.term_kind != B.term_kind || A.q != B.q || A.num_hashes != B.num_hashes)
        return set_error(COBS_ERR_ARG, "indexes differ in term kind, q or number of hashes");
    cobs_index *ix = new cobs_index();
    ix->params = A;
    ix->params.score_bits = std::max(A.score_bits, B.score_bits);
    ix->n_docs = a->n_docs + b->n_docs;
    ix->nterms = a->nterms;
    ix->nterms.insert(ix->nterms.end(), b->nterms.begin(), b->nterms.end());
    const bool classic = A.block_docs == 0 && B.block_docs == 0 && a->blocks.size() == 1 && b->blocks.size() == 1 &&
                         a->blocks[0].w == b->blocks[0].w;
    if (classic) {
        // one block: row r = a's bits of row r, then b's bits shifted to column n_a
        const cobs_block_info &ba = a->blocks[0], &bb = b->blocks[0];
        cobs_block_info m{};
        m.n_docs = ix->n_docs;
        m.doc_begin = 0;
        m.w = ba.w;
        m.rowbytes = (m.n_docs + 127) / 128 * 16;
        m.row_offset = 0;
        m.max_terms = std::max(ba.max_terms, bb.max_terms);
        ix->blocks.push_back(m);
        ix->params.width = m.w;
        ix->perm.resize(ix->n_docs);
        std::iota(ix->perm.begin(), ix->perm.end(), 0ULL);
        ix->rows.assign(m.w * m.rowbytes, 0);
        const uint64_t na = ba.n_docs, nbytes_a = (na + 7) / 8, nbytes_b = (bb.n_docs + 7) / 8;
        const uint32_t sh = (uint32_t)(na & 7);
        for (uint64_t r = 0; r < m.w; r++) {
            uint8_t *dst = ix->rows.data() + r * m.rowbytes;
            const uint8_t *ra = a->rows.data() + ba.row_offset + r * ba.rowbytes;
            const uint8_t *rb = b->rows.data() + bb.row_offset + r * bb.rowbytes;
            memcpy(dst, ra, nbytes_a);  // padding bits of a's last byte are zero
            for (uint64_t k = 0; k < nbytes_b; k++) {
                const uint64_t at = (na >> 3) + k;
                dst[at] |= (uint8_t)(rb[k] << sh);
                if (sh && at + 1 < m.rowbytes) dst[at + 1] |= (uint8_t)(rb[k] >> (8 - sh));
            }
        }
    } else {
        ix->blocks = a->blocks;
        for (cobs_block_info blk : b->blocks) {
            blk.row_offset += a->rows.size();
            blk.doc_begin += a->n_docs;
            ix->blocks.push_back(blk);
        }
        uint64_t bmax = 0;
        for (const auto &blk : ix->blocks) bmax = std::max(bmax, blk.n_docs);
        if (ix->blocks.size() > 1 || A.block_docs) ix->params.block_docs = std::max(bmax, std::max(A.block_docs, B.block_docs));
        if (A.width != B.width) ix->params.width = 0;
        ix->perm = a->perm;
        for (uint64_t p : b->perm) ix->perm.push_back(p + a->n_docs);
        ix->rows = a->rows;
        ix->rows.insert(ix->rows.end(), b->rows.begin(), b->rows.end());
    }
    *out = ix;
    return COBS_OK;
}

// ------------------------------------------------------------------ files
static const char MAGIC[8] = {'C', 'O', 'B', 'S', 'G', 'P', 'U', '2'};

extern "C" cobs_status cobs_index_save(const cobs_index *ix, const char *path) {
    if (!ix || !path) return set_error(COBS_ERR_ARG, "NULL argument");
    FILE *f = fopen(path, "wb");
    if (!f) return set_error(COBS_ERR_ARG, "cannot open %s for writing", path);
    uint64_t nb = ix->blocks.size(), rb = ix->rows.size();
    bool ok = fwrite(MAGIC, 8, 1, f) == 1 && fwrite(&ix->params, sizeof(cobs_params), 1, f) == 1 &&
              fwrite(&ix->n_docs, 8, 1, f) == 1 && fwrite(&nb, 8, 1, f) == 1 && fwrite(&rb, 8, 1, f) == 1;
    if (ok && nb) ok = fwrite(ix->blocks.data(), sizeof(cobs_block_info), nb, f) == nb;
    if (ok && ix->n_docs) ok = fwrite(ix->perm.data(), 8, ix->n_docs, f) == ix->n_docs &&
                               fwrite(ix->nterms.data(), 8, ix->n_docs, f) == ix->n_docs;
    if (ok && rb) ok = fwrite(ix->rows.data(), 1, rb, f) == rb;
    if (fclose(f) != 0) ok = false;
    return ok ? COBS_OK : set_error(COBS_ERR_ARG, "write to %s failed", path);
}

extern "C" cobs_status cobs_index_load(const char *path, cobs_index **out) {
    if (!path || !out) return set_error(COBS_ERR_ARG, "NULL argument");
    FILE *f = fopen(path, "rb");
    if (!f) return set_error(COBS_ERR_ARG, "cannot open %s", path);
    cobs_index *ix = new cobs_index();
    char magic[8];
    uint64_t nb = 0, rb = 0;
    bool ok = fread(magic, 8, 1, f) == 1 && memcmp(magic, MAGIC, 8) == 0 &&
              fread(&ix->params, sizeof(cobs_params), 1, f) == 1 && fread(&ix->n_docs, 8, 1, f) == 1 &&
              fread(&nb, 8, 1, f) == 1 && fread(&rb, 8, 1, f) == 1;
    ok = ok && nb <= (1ULL << 32) && ix->n_docs < (1ULL << 32) && rb < (1ULL << 44);
    if (ok) {
        ix->blocks.resize(nb);
        ix->perm.resize(ix->n_docs);
        ix->nterms.resize(ix->n_docs);
        ix->rows.resize(rb);
        ok = (!nb || fread(ix->blocks.data(), sizeof(cobs_block_info), nb, f) == nb) &&
             (!ix->n_docs || (fread(ix->perm.data(), 8, ix->n_docs, f) == ix->n_docs &&
                              fread(ix->nterms.data(), 8, ix->n_docs, f) == ix->n_docs)) &&
             (!rb || fread(ix->rows.data(), 1, rb, f) == rb);
    }
    // consistency of the table with the row storage
    if (ok) {
        uint64_t off = 0, docs = 0;
        for (const cobs_block_info &b : ix->blocks) {
            ok = ok && b.row_offset == off && b.doc_begin == docs && b.rowbytes == (b.n_docs + 127) / 128 * 16 &&
                 b.w >= 1 && b.w <= 0xFFFFFFFFULL;
            off += b.w * b.rowbytes;
            docs += b.n_docs;
        }
        ok = ok && off == rb && docs == ix->n_docs;
        for (uint64_t i = 0; ok && i < ix->n_docs; i++) ok = ix->perm[i] < ix->n_docs;
    }
    fclose(f);
    if (!ok) {
        delete ix;
        return set_error(COBS_ERR_FORMAT, "%s is not a complete cobs_gpu index", path);
    }
    *out = ix;
    return COBS_OK;
}

// ----------------------------------------------------------------- engine

static const uint32_t MAX_CLASSES = 4;

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

static cobs_status ensure_slices(cobs_engine *eng, uint32_t lpq) {
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
        // every query of more than one round (chunk CTAs share its set)
        if (sl > TERMS_SMEM_SLOTS || np > terms_round_windows()) {
            bp.table_base[q] = bp.total_slots;
            bp.total_slots += sl;
        } else {
            bp.table_base[q] = 0;
            bp.smem_slots = std::max<uint32_t>(bp.smem_slots, (uint32_t)sl);
        }
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
    const uint64_t round = terms_round_windows();
    for (uint64_t q = 0; q < n; q++) {
        if (bp.npos[q] <= round) continue;
        bp.long_q.push_back((uint32_t)q);
        for (uint64_t w0 = 0; w0 < bp.npos[q]; w0 += round) {
            bp.chunk_q.push_back((uint32_t)q);
            bp.chunk_w0.push_back((uint32_t)w0);
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
    // qcount, then the counters (one memset clears both): [0] hits, [1..14] work
    // counters, [15] big segments, then 4 per block for a streamed index
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
            // long queries: sets cleared, distinct counts and flags zeroed, then a
            // CTA per chunk and a CTA per (query, block group)
            CU(cudaMemsetAsync(eng->tables.p, 0xFF, bp.total_slots * 8, s));
            CU(cudaMemsetAsync(eng->ell.p, 0, n * 4, s));
            CU(cudaMemsetAsync(eng->long_flag.p, 0, n * 4, s));
            ta.long_q = long_q;
            ta.chunk_q = chunk_q;
            ta.chunk_w0 = chunk_w0;
            ta.long_flag = eng->long_flag.as<uint32_t>();
            ta.n_long = (uint32_t)bp.long_q.size();
            ta.n_chunks = (uint32_t)bp.chunk_q.size();
            eng->stat_launches += 2;
        }
        {
            TraceRange tr_terms("cobs.terms");
            launch_query_terms(ta, (uint32_t)n, s);
        }
        eng->stat_launches += 1;
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
    {
        TraceRange tr_hits("cobs.hits");
        launch_hits_finalize(ha, s);
    }
    eng->stat_launches += 3;
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
                                 (uint64_t)eng->long_flag.p, eng->cfg.class_streams, bp.part_terms};
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
    return COBS_OK;
}

namespace {

// One point of the autotuner's space.
struct TuneChoice {
    uint32_t lpq, ctas, hints, split, part, class_streams;
};

// Process-wide cache of autotuner choices, keyed by the index's block shape and
// the batch's query-length histogram.
std::mutex g_tune_mu;
std::map<std::vector<uint64_t>, TuneChoice> g_tune_cache;

std::vector<uint64_t> tune_key(const cobs_engine *eng, const uint64_t *h_off, uint64_t n) {
    const cobs_device_index *dix = eng->dix;
    const cobs_params &P = dix->params;
    std::vector<uint64_t> key = {(uint64_t)dix->device, P.num_hashes, P.term_kind, P.q, dix->streamed ? 1u : 0u,
                                 dix->blocks.size()};
    for (const auto &B : dix->blocks) {
        key.push_back(B.w);
        key.push_back(B.rowbytes);
    }
    // queries: log2 of their number, then per log2 bucket of windows the share
    // of the queries in sixteenths
    uint64_t hist[26] = {0};
    for (uint64_t q = 0; q < n; q++) {
        const uint64_t len = h_off[q + 1] - h_off[q];
        const uint64_t np = len >= P.q ? len - P.q + 1 : 0;
        hist[np ? std::min<uint64_t>(64 - (uint64_t)__builtin_clzll(np), 25) : 0]++;
    }
    key.push_back(n ? 64 - (uint64_t)__builtin_clzll(n) : 0);
    for (uint64_t b = 0; b < 26; b++) key.push_back(n ? (hist[b] * 16 + n / 2) / n : 0);
    return key;
}

}  // namespace

extern "C" cobs_status cobs_engine_autotune(cobs_engine *eng, const uint8_t *queries_dev, const uint64_t *offsets_dev,
                                            const uint64_t *offsets_host, const uint16_t *thr_dev, uint64_t n,
                                            cobs_engine_cfg *cfg_out) {
    if (!eng) return set_error(COBS_ERR_ARG, "NULL engine");
    if (n && !offsets_host) return set_error(COBS_ERR_ARG, "NULL offsets");
    const cobs_params &P = eng->dix->params;
    const TuneChoice old{eng->lanes_per_query, eng->ctas_per_sm, eng->l2_hints, eng->cfg.split, eng->cfg.split_part,
                         eng->cfg.class_streams};
    auto apply = [&](const TuneChoice &c) -> cobs_status {
        TRY(ensure_slices(eng, c.lpq));
        eng->lanes_per_query = c.lpq;
        eng->ctas_per_sm = c.ctas;
        eng->l2_hints = c.hints;
        eng->cfg.split = c.split;
        eng->cfg.split_part = c.part;
        eng->cfg.class_streams = c.class_streams;
        return COBS_OK;
    };
    auto finish = [&](const TuneChoice &c, bool cached) -> cobs_status {
        TRY(apply(c));
        if (eng->gexec) {
            cudaGraphExecDestroy(eng->gexec);
            eng->gexec = nullptr;
        }
        if (cfg_out) {
            *cfg_out = eng->cfg;
            cfg_out->slice_bytes = c.lpq * 16;
            cfg_out->ctas_per_sm = c.ctas;
            cfg_out->l2_hints = c.hints;
            cfg_out->tuned_from_cache = cached ? 1u : 0u;
        }
        return COBS_OK;
    };
    const std::vector<uint64_t> key = tune_key(eng, offsets_host, n);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return finish(it->second, true);
    }
    // Coordinate descent from the current choice: every candidate runs the whole
    // batch from a cold L2 (a 256 MB write first), twice; its time is the best of
    // the two, measured with the engine's events from the first kernel to the
    // end of the hit kernels.
    DevBuf flush;
    CU(flush.ensure(256ULL << 20));
    bool verbose = getenv("COBS_AUTOTUNE_VERBOSE") != nullptr;
    auto measure = [&](const TuneChoice &c, double *ms) -> cobs_status {
        TRY(apply(c));
        double tbest = 1e30;
        for (int rep = 0; rep < 2; rep++) {
            if (cudaMemsetAsync(flush.p, rep, flush.bytes, eng->stream) != cudaSuccess)
                return set_error(COBS_ERR_CUDA, "autotune: L2 flush");
            TRY(engine_query(eng, queries_dev, offsets_dev, offsets_host, thr_dev, n, COBS_BATCHED));
            TRY(engine_finish(eng));
            float t = 0;
            cudaEventElapsedTime(&t, eng->ev[0], eng->ev[3]);
            tbest = std::min(tbest, (double)t);
        }
        if (verbose)
            fprintf(stderr, "autotune slice=%u ctas=%u l2_hints=%u split=%u part=%u class_streams=%u ms=%.4f\n",
                    c.lpq * 16, c.ctas, c.hints, c.split, c.part, c.class_streams, tbest);
        *ms = tbest;
        return COBS_OK;
    };
    TuneChoice best = old;
    double best_ms = 0;
    cobs_status st = measure(best, &best_ms);
    auto try_all = [&](const std::vector<TuneChoice> &cands) -> cobs_status {
        for (const TuneChoice &c : cands) {
            double ms = 0;
            TRY(measure(c, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        return COBS_OK;
    };
    std::vector<TuneChoice> cands;
    // 1. slice width
    if (st == COBS_OK) {
        cands.clear();
        for (uint32_t lpq : {2u, 4u, 8u, 16u}) {
            if (lpq == 16 && P.num_hashes != 1) continue;
            if (lpq == best.lpq) continue;
            TuneChoice c = best;
            c.lpq = lpq;
            cands.push_back(c);
        }
        st = try_all(cands);
    }
    // 2. resident CTAs per SM
    if (st == COBS_OK) {
        cands.clear();
        const uint32_t occ = (uint32_t)std::max(1, gather_batched_max_blocks_per_sm(best.lpq, P.num_hashes));
        for (uint32_t ct : {occ, std::max(occ / 2, 1u), 1u}) {
            if (ct == best.ctas) continue;
            bool dup = false;
            for (const auto &c : cands) dup |= c.ctas == ct;
            if (dup) continue;
            TuneChoice c = best;
            c.ctas = ct;
            cands.push_back(c);
        }
        st = try_all(cands);
    }
    // 3. L2 hints (single-hash kernels take them)
    if (st == COBS_OK && P.num_hashes == 1) {
        cands.clear();
        for (uint32_t hnt : {1u, 2u, 3u, 4u}) {
            if (hnt == best.hints) continue;
            TuneChoice c = best;
            c.hints = hnt;
            cands.push_back(c);
        }
        st = try_all(cands);
    }
    // 4. the query-term chunk of the tiles (single-hash indexes split long queries)
    if (st == COBS_OK && P.num_hashes == 1) {
        cands.clear();
        const TuneChoice opts[4] = {{0, 0, 0, 0, 0, 0}, {0, 0, 0, 1, 0, 0}, {0, 0, 0, 2, SPLIT_TERMS, 0},
                                    {0, 0, 0, 2, 1024, 0}};
        for (const TuneChoice &o : opts) {
            if (o.split == best.split && o.part == best.part) continue;
            TuneChoice c = best;
            c.split = o.split;
            c.part = o.part;
            cands.push_back(c);
        }
        st = try_all(cands);
    }
    // 5. counter classes overlapping on their own streams or one after another
    if (st == COBS_OK && eng->bp.classes.size() > 1) {
        TuneChoice c = best;
        c.class_streams = best.class_streams == 2 ? 0u : 2u;
        st = try_all({c});
    }
    if (st != COBS_OK) {
        (void)apply(old);  // on a failure the engine keeps the shape it had
        return st;
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    return finish(best, false);
}
