// Host runtime and C ABI of the COBS indexes: planning and device build
// (Sec. 2.3 "Classic and Compact"), transfer to and from the device, the
// streamed and multi-index forms, insertion, merge and the index file format.
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

#ifndef COBS_COUNT_WAVE_MB
#define COBS_COUNT_WAVE_MB 2048  // partition bytes of one wave of the distinct count, MB
#endif

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
    // bytes of partitions per wave: fewer, larger waves cost fewer launches,
    // memsets and tails (a quarter of the free memory at most)
    uint64_t budget = std::min<uint64_t>(free_b / 4, (uint64_t)COBS_COUNT_WAVE_MB << 20);
    if (build_scratch_override()) budget = build_scratch_override();
    struct Wave { uint64_t c0, c1, q0, q1, slots, max_parts; };  // chunks [c0, c1), partitions [q0, q1), term slots
    std::vector<Wave> waves;
    Wave wv{0, 0, 0, 0, 0, 1};
    for (uint32_t d : docs) {
        const uint64_t np = npos[d];
        const uint64_t pd = std::max<uint64_t>(1, (np + PART_WINDOWS - 1) / PART_WINDOWS);
        const uint64_t mean = (np + pd - 1) / pd;
        // mean + 8 standard deviations of a binomial partition size, + 64
        const uint64_t cap = mean + 8 * (uint64_t)std::ceil(std::sqrt((double)mean)) + 64;
        const uint64_t need = pd * cap;
        if (wv.q1 > wv.q0 && (wv.slots + need) * 8 > budget) {
            waves.push_back(wv);
            wv = Wave{wv.c1, wv.c1, wv.q1, wv.q1, 0, 1};
        }
        wv.max_parts = std::max<uint64_t>(wv.max_parts, pd);
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
        pa.max_parts = (uint32_t)w.max_parts;
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
        int numa = -1;  // the host node nearest the device, if the system has NUMA
        if (cudaDeviceGetAttribute(&numa, cudaDevAttrHostNumaId, device) != cudaSuccess) {
            numa = -1;
            cudaGetLastError();
        }
        e = dix->host_rows.ensure_on_node(dix->rows_bytes, numa);
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
