// K1: query terms.  For every query: all windows of length q (Sec. 2.1),
// canonical form (Sec. 2.3), the distinct set G_q(P) via an open-addressing set,
// then for every distinct term and every block b and hash i < h its row
// XXH64(term, i) mod w_b (Sec. 2.2), written as a u32 row index.
//
// A query is processed in rounds of TERMS_ROUND windows.  For DNA each round
// packs its bytes straight from global memory into a 2-bit base stream and a
// mask of non-ACGT bytes, 16 bases per word (every thread packs 4 bytes, four
// lanes merge a word); byte q-grams stage the bytes in shared memory.  Every
// thread then takes one window at a time: its k bases are a funnel shift of
// three packed words, its validity a shift of the mask, its reverse complement a
// bit reversal of the complemented code with the bits of each base swapped back.
// The window is hashed, inserted into the set and appended to the distinct list
// when it is new (warp-aggregated).  A final pass writes the rows in row-bucket
// order.
//
// Short queries (one round) run fused in one CTA with the set in shared memory.
// With one hash and at most two blocks the rows of a new term are computed at
// insertion: the list holds them (block 1 in the high word) and the bucket
// histogram is counted on the way, so the final pass only scatters.  Otherwise
// the list holds hash 0 when h == 1, else the code, and the final pass
// recomputes the rows.
//
// Long queries, when the caller supplies a chunk plan, are spread over many
// CTAs: one CTA per round inserts into the query's set in global memory
// (cleared by the caller) and appends to its global list, counting the
// distinct terms with a global atomic; then one CTA per (query, group of
// blocks) runs the row pass.  Without a chunk plan one CTA walks all rounds.
#include <algorithm>

#include "terms_common.cuh"

namespace cobs {

// Shared-memory helpers of the rows-at-insertion path (h == 1, at most two blocks).
struct FastRows {
    bool on;
    uint32_t nb;
    const uint64_t *m;   // Barrett constants
    const uint32_t *w;   // row counts
    const uint32_t *shift;
    uint32_t *hist;      // 2 x TERMS_BUCKETS
};

// Windows [0, rn) of a staged round: extract, hash, insert into `table` (cap
// slots) and append each new term to `list` at a slot counted by *ell_ctr
// (shared or global; one atomic per warp and iteration).  *has_empty flags the
// one code the set cannot hold.
__device__ __forceinline__ void insert_round(const TermsArgs &a, uint32_t rn, uint32_t k, uint64_t mask, bool dna,
                                             const uint8_t *s_bytes, const uint32_t *s_pk, const uint16_t *s_inv,
                                             unsigned long long *table, uint32_t cap, unsigned long long *list,
                                             uint32_t *ell_ctr, uint32_t *has_empty, const FastRows &fr) {
    const uint32_t lane = threadIdx.x & 31u;
    // one window per thread and iteration; every lane of a warp runs the same
    // number of iterations, for the warp-level append
    for (uint32_t p = threadIdx.x; p < ((rn + 31u) & ~31u); p += blockDim.x) {
        uint64_t code = 0;
        bool term = false;
        if (p < rn) {
            if (dna) {
                term = packed_kmer(s_pk, s_inv, p, k, a.kind == KIND_DNA_CANONICAL, mask, &code);
            } else {
                code = bytes_qgram(s_bytes, p, k);
                term = true;
            }
        }
        bool fresh = false;
        uint64_t h0 = 0;
        if (term) {
            h0 = xxh64_u64(code, 0);
            if (code == EMPTY_KEY) fresh = atomicExch(has_empty, 1u) == 0u;
            else fresh = set_insert(table, cap, h0, code);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, fresh);
        if (m) {
            uint32_t slot0 = 0;
            const uint32_t leader = __ffs(m) - 1;
            if (lane == leader) slot0 = atomicAdd(ell_ctr, (uint32_t)__popc(m));
            slot0 = __shfl_sync(0xffffffffu, slot0, leader);
            if (fresh) {
                uint64_t entry = a.h == 1 ? h0 : code;
                if (fr.on) {
                    const uint32_t rw0 = barrett_mod(h0, fr.m[0], fr.w[0]);
                    atomicAdd(&fr.hist[rw0 >> fr.shift[0]], 1u);
                    uint32_t rw1 = 0;
                    if (fr.nb > 1) {
                        rw1 = barrett_mod(h0, fr.m[1], fr.w[1]);
                        atomicAdd(&fr.hist[TERMS_BUCKETS + (rw1 >> fr.shift[1])], 1u);
                    }
                    entry = ((uint64_t)rw1 << 32) | rw0;
                }
                list[slot0 + __popc(m & ((1u << lane) - 1u))] = entry;
            }
        }
    }
}

// Exclusive scan of the 64 bucket counts at hj, by one warp.
__device__ __forceinline__ void scan_hist(uint32_t *hj) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < TERMS_BUCKETS; c0 += 32) {
        const uint32_t v = hj[c0 + lane];
        uint32_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += y;
        }
        hj[c0 + lane] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
}

// Row pass for blocks [b0, b0 + nbp), nbp <= NB: the distinct terms' rows in
// row-bucket order (a counting sort by the top bits of the hash-0 row).  Scores
// do not depend on the order of the terms; bucketed order makes all warps of
// the gather sweep the rows of a slice together, so the rows in use at any
// moment form a narrow band.  list[t] is hash 0 (h == 1) or the code.  Every
// thread of the CTA calls it.
template <uint32_t NB>
__device__ __forceinline__ void row_pass(const TermsArgs &a, const unsigned long long *list, uint32_t ell,
                                         uint64_t base, uint32_t b0, uint32_t nbp, uint32_t *s_hist,
                                         uint32_t *s_shift) {
    const uint32_t warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    // every distinct term once, spread over the threads: f(code, hash 0); the code
    // is only meaningful (and only used) when h > 1
    auto each_distinct = [&](auto &&f) {
        for (uint32_t t = threadIdx.x; t < ell; t += blockDim.x) {
            const uint64_t key = list[t];
            f(key, a.h == 1 ? key : xxh64_u64(key, 0));
        }
    };
    for (uint32_t i = threadIdx.x; i < nbp * TERMS_BUCKETS; i += blockDim.x) s_hist[i] = 0;
    if (threadIdx.x < nbp) {
        const uint32_t w = a.blocks[b0 + threadIdx.x].w;
        const int lg = 32 - __clz(w > 1 ? w - 1 : 0);  // bits of the largest row
        s_shift[threadIdx.x] = lg > (int)TERMS_BUCKET_BITS ? (uint32_t)(lg - TERMS_BUCKET_BITS) : 0u;
    }
    __syncthreads();
    each_distinct([&](uint64_t, uint64_t h0) {
#pragma unroll
        for (uint32_t j = 0; j < NB; j++) {
            if (j < nbp) {
                const DevBlock blk = a.blocks[b0 + j];
                const uint32_t r0 = barrett_mod(h0, blk.barrett_m, blk.w);
                atomicAdd(&s_hist[j * TERMS_BUCKETS + (r0 >> s_shift[j])], 1u);
            }
        }
    });
    __syncthreads();
    for (uint32_t j = warp; j < nbp; j += n_warps) scan_hist(s_hist + j * TERMS_BUCKETS);
    __syncthreads();
    each_distinct([&](uint64_t code, uint64_t h0) {
        uint32_t pos[NB];
#pragma unroll
        for (uint32_t j = 0; j < NB; j++) {
            if (j < nbp) {
                const DevBlock blk = a.blocks[b0 + j];
                const uint32_t r0 = barrett_mod(h0, blk.barrett_m, blk.w);
                pos[j] = atomicAdd(&s_hist[j * TERMS_BUCKETS + (r0 >> s_shift[j])], 1u);
                a.rows_idx[(uint64_t)((b0 + j) * a.h) * a.tcap + base + pos[j]] = r0;
            }
        }
        for (uint32_t i2 = 1; i2 < a.h; i2++) {
            const uint64_t hv = xxh64_u64(code, i2);
#pragma unroll
            for (uint32_t j = 0; j < NB; j++) {
                if (j < nbp) {
                    const DevBlock blk = a.blocks[b0 + j];
                    a.rows_idx[(uint64_t)((b0 + j) * a.h + i2) * a.tcap + base + pos[j]] =
                        barrett_mod(hv, blk.barrett_m, blk.w);
                }
            }
        }
    });
    __syncthreads();
}

__device__ __forceinline__ uint64_t windows_of(const TermsArgs &a, uint32_t q, uint64_t *off0) {
    *off0 = a.offsets[q];
    const uint64_t len = a.offsets[q + 1] - *off0;
    return len >= a.k ? len - a.k + 1 : 0;
}

// FAST: one hash and at most two blocks (rows at insertion).  The general form
// runs the row pass TERMS_GENERAL_BP blocks at a time, so every term is hashed
// once per pass whatever the number of blocks; it is a kernel of its own so its
// registers do not weigh on the fast form.
#ifndef COBS_TERMS_GENERAL_BP
#define COBS_TERMS_GENERAL_BP 8
#endif
constexpr uint32_t TERMS_GENERAL_BP = COBS_TERMS_GENERAL_BP;
template <bool FAST>
__global__ void __launch_bounds__(TERMS_THREADS) k_query_terms(TermsArgs a) {
    constexpr uint32_t NBH = FAST ? 2 : TERMS_GENERAL_BP;  // histograms in shared memory
    // dynamic shared memory: the on-chip table region (smem_table slots) and the
    // distinct list (a set of set_slots(windows) <= smem_slots slots is for at
    // most smem_slots / 2 windows)
    extern __shared__ unsigned long long s_table[];
    const uint32_t table_slots = a.smem_table > a.smem_slots ? a.smem_table : a.smem_slots;
    unsigned long long *s_list = s_table + table_slots;
    __shared__ __align__(16) uint8_t s_bytes[TERMS_STAGE_BYTES];
    __shared__ uint32_t s_pk[TERMS_PK_WORDS];   // 2-bit bases, 16 per word
    __shared__ uint16_t s_inv[TERMS_PK_WORDS];  // non-ACGT bytes, 16 per word
    __shared__ uint32_t s_ell;
    __shared__ uint32_t s_has_empty;
    __shared__ uint32_t s_hist[NBH * TERMS_BUCKETS];
    __shared__ uint32_t s_shift[NBH];

    // a kernel launched after this one as a programmatic dependent (the plain
    // form's gather) may be scheduled now; it waits for this grid's completion
    // before it reads anything written here (no effect without such a kernel)
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const uint32_t q = a.q0 + blockIdx.x;
    uint64_t off0;
    const uint64_t npos = windows_of(a, q, &off0);
    if (a.n_chunks && npos > TERMS_ROUND) return;  // a long query of the chunk plan
    const uint32_t k = a.k;
    // a set that fits on chip holds at most TERMS_ROUND distinct terms (one round);
    // on chip it spreads over up to TERMS_SET_SPREAD slots per window
    const bool in_smem = set_slots(npos) <= a.smem_slots;
    uint32_t cap = (uint32_t)set_slots(npos);
    if (in_smem) {
        const uint32_t sparse = (uint32_t)npos * TERMS_SET_SPREAD;
        const uint32_t wide = sparse < table_slots ? sparse : table_slots;
        cap = wide > cap ? wide : cap;
    }
    unsigned long long *table = in_smem ? s_table : a.tables + a.table_base[q];
    const uint64_t base = a.term_base[q];
    unsigned long long *list = in_smem ? s_list : a.codes + base;

    for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) table[i] = EMPTY_KEY;
    if (threadIdx.x == 0) { s_ell = 0; s_has_empty = 0; }

    // rows at insertion (one hash, at most two blocks): block moduli in shared memory
    const bool rows_in_list = FAST;
    const uint32_t nb_fast = rows_in_list ? a.n_blocks : 0u;
    __shared__ uint64_t s_fm[2];
    __shared__ uint32_t s_fw[2];
    if (threadIdx.x < nb_fast) {
        const DevBlock blk = a.blocks[threadIdx.x];
        s_fm[threadIdx.x] = blk.barrett_m;
        s_fw[threadIdx.x] = blk.w;
        const int lg = 32 - __clz(blk.w > 1 ? blk.w - 1 : 0);  // bits of the largest row
        s_shift[threadIdx.x] = lg > (int)TERMS_BUCKET_BITS ? (uint32_t)(lg - TERMS_BUCKET_BITS) : 0u;
    }
    if (rows_in_list)
        for (uint32_t i = threadIdx.x; i < 2 * TERMS_BUCKETS; i += blockDim.x) s_hist[i] = 0;
    const FastRows fr{rows_in_list, nb_fast, s_fm, s_fw, s_shift, s_hist};

    const uint8_t *src = a.bytes + off0;
    const uint64_t mask = kmer_mask(k);
    const bool dna = a.kind != KIND_BYTES;
    for (uint64_t r0 = 0; r0 < npos; r0 += TERMS_ROUND) {
        const uint32_t rn = (uint32_t)(npos - r0 < TERMS_ROUND ? npos - r0 : TERMS_ROUND);
        __syncthreads();  // previous round finished with the staged bases (and the table init)
        stage_round(src, r0, rn, k, dna, s_bytes, s_pk, s_inv);
        __syncthreads();
        insert_round(a, rn, k, mask, dna, s_bytes, s_pk, s_inv, table, cap, list, &s_ell, &s_has_empty, fr);
    }
    __syncthreads();
    const uint32_t ell = s_ell;
    if (threadIdx.x == 0) a.ell[q] = ell;
    if (rows_in_list) {
        const uint32_t warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
        for (uint32_t j = warp; j < nb_fast; j += n_warps) scan_hist(s_hist + j * TERMS_BUCKETS);
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < ell; t += blockDim.x) {
            const uint64_t e = list[t];
#pragma unroll
            for (uint32_t j = 0; j < 2; j++) {
                if (j < nb_fast) {
                    const uint32_t r = (uint32_t)(e >> (32 * j));
                    const uint32_t pos = atomicAdd(&s_hist[j * TERMS_BUCKETS + (r >> s_shift[j])], 1u);
                    a.rows_idx[(uint64_t)j * a.tcap + base + pos] = r;
                }
            }
        }
        return;
    }
    if constexpr (!FAST) {
        constexpr uint32_t G = TERMS_GENERAL_BP;
        for (uint32_t b0 = 0; b0 < a.n_blocks; b0 += G)
            row_pass<G>(a, list, ell, base, b0, a.n_blocks - b0 < G ? a.n_blocks - b0 : G, s_hist, s_shift);
    }
}

// Long queries, insertion: one CTA per round (chunk) of a long query.  The
// query's set and distinct count start cleared; the list is the query's global
// term region.
__global__ void __launch_bounds__(TERMS_THREADS) k_terms_long_insert(TermsArgs a) {
    __shared__ __align__(16) uint8_t s_bytes[TERMS_STAGE_BYTES];
    __shared__ uint32_t s_pk[TERMS_PK_WORDS];
    __shared__ uint16_t s_inv[TERMS_PK_WORDS];
    const uint32_t q = a.chunk_q[blockIdx.x];
    const uint64_t r0 = a.chunk_w0[blockIdx.x];
    uint64_t off0;
    const uint64_t npos = windows_of(a, q, &off0);
    const uint32_t rn = (uint32_t)(npos - r0 < TERMS_ROUND ? npos - r0 : TERMS_ROUND);
    const uint32_t cap = (uint32_t)set_slots(npos);
    stage_round(a.bytes + off0, r0, rn, a.k, a.kind != KIND_BYTES, s_bytes, s_pk, s_inv);
    __syncthreads();
    const FastRows fr{false, 0u, nullptr, nullptr, nullptr, nullptr};
    insert_round(a, rn, a.k, kmer_mask(a.k), a.kind != KIND_BYTES, s_bytes, s_pk, s_inv,
                 a.tables + a.table_base[q], cap, a.codes + a.term_base[q], &a.ell[q], &a.long_flag[q], fr);
}

// Long queries, rows: one CTA per (long query, group of BP blocks).  With one
// hash the scatter runs in chunks of LR_CHUNK terms: the chunk's rows of a block
// are sorted by bucket in shared memory, and each bucket's run is written to its
// place in one contiguous piece (the plain scatter writes one 4-byte row per
// lane to 32 places).
constexpr uint32_t LR_PER_THREAD = 4;
constexpr uint32_t LR_CHUNK = TERMS_THREADS * LR_PER_THREAD;
__global__ void __launch_bounds__(TERMS_THREADS) k_terms_long_rows(TermsArgs a) {
    __shared__ uint32_t s_hist[BP * TERMS_BUCKETS];
    __shared__ uint32_t s_shift[BP];
    __shared__ uint32_t s_lh[TERMS_BUCKETS];   // chunk: bucket counts, then exclusive offsets
    __shared__ uint32_t s_stage[LR_CHUNK];     // chunk rows in bucket order
    const uint32_t q = a.long_q[blockIdx.x];
    const uint32_t b0 = blockIdx.y * BP;
    const uint32_t nbp = a.n_blocks - b0 < BP ? a.n_blocks - b0 : BP;
    const uint64_t base = a.term_base[q];
    const unsigned long long *list = a.codes + base;
    const uint32_t ell = a.ell[q];
    if (a.h != 1) {
        row_pass<BP>(a, list, ell, base, b0, nbp, s_hist, s_shift);
        return;
    }
    // bucket counts of every block of the group, then global offsets
    for (uint32_t i = threadIdx.x; i < nbp * TERMS_BUCKETS; i += blockDim.x) s_hist[i] = 0;
    if (threadIdx.x < nbp) {
        const uint32_t w = a.blocks[b0 + threadIdx.x].w;
        const int lg = 32 - __clz(w > 1 ? w - 1 : 0);
        s_shift[threadIdx.x] = lg > (int)TERMS_BUCKET_BITS ? (uint32_t)(lg - TERMS_BUCKET_BITS) : 0u;
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < ell; t += blockDim.x) {
        const uint64_t h0 = list[t];
#pragma unroll
        for (uint32_t j = 0; j < BP; j++) {
            if (j < nbp) {
                const DevBlock blk = a.blocks[b0 + j];
                atomicAdd(&s_hist[j * TERMS_BUCKETS + (barrett_mod(h0, blk.barrett_m, blk.w) >> s_shift[j])], 1u);
            }
        }
    }
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (uint32_t j = warp; j < nbp; j += n_warps) scan_hist(s_hist + j * TERMS_BUCKETS);
    __syncthreads();
    for (uint32_t c0 = 0; c0 < ell; c0 += LR_CHUNK) {
        const uint32_t cn = ell - c0 < LR_CHUNK ? ell - c0 : LR_CHUNK;
        uint64_t h0[LR_PER_THREAD];
#pragma unroll
        for (uint32_t i = 0; i < LR_PER_THREAD; i++) {
            const uint32_t t = c0 + i * blockDim.x + threadIdx.x;
            h0[i] = t < ell ? list[t] : 0ULL;
        }
        for (uint32_t j = 0; j < nbp; j++) {
            const DevBlock blk = a.blocks[b0 + j];
            const uint32_t sh = s_shift[j];
            uint32_t *gh = s_hist + j * TERMS_BUCKETS;  // next free position of each bucket
            if (threadIdx.x < TERMS_BUCKETS) s_lh[threadIdx.x] = 0;
            __syncthreads();
            uint32_t r[LR_PER_THREAD], rank[LR_PER_THREAD];
#pragma unroll
            for (uint32_t i = 0; i < LR_PER_THREAD; i++) {
                const uint32_t t = c0 + i * blockDim.x + threadIdx.x;
                r[i] = barrett_mod(h0[i], blk.barrett_m, blk.w);
                rank[i] = t < ell ? atomicAdd(&s_lh[r[i] >> sh], 1u) : 0u;
            }
            __syncthreads();
            if (warp == 0) scan_hist(s_lh);  // counts -> exclusive offsets
            __syncthreads();
#pragma unroll
            for (uint32_t i = 0; i < LR_PER_THREAD; i++) {
                const uint32_t t = c0 + i * blockDim.x + threadIdx.x;
                if (t < ell) s_stage[s_lh[r[i] >> sh] + rank[i]] = r[i];
            }
            __syncthreads();
            // staged position x of bucket b goes to gh[b] + (x - s_lh[b])
            uint32_t *dst = a.rows_idx + (uint64_t)(b0 + j) * a.tcap + base;
            for (uint32_t x = threadIdx.x; x < cn; x += blockDim.x) {
                const uint32_t rv = s_stage[x];
                const uint32_t b = rv >> sh;
                dst[gh[b] + (x - s_lh[b])] = rv;
            }
            __syncthreads();
            if (threadIdx.x < TERMS_BUCKETS) {  // advance each bucket by the chunk's count
                const uint32_t b = threadIdx.x;
                const uint32_t next = b + 1 < TERMS_BUCKETS ? s_lh[b + 1] : cn;
                gh[b] += next - s_lh[b];
            }
            __syncthreads();
        }
    }
}

void launch_terms_short(const TermsArgs &a, uint32_t n_queries, cudaStream_t s) {
    if (n_queries == 0) return;
    static PerDeviceOnce once;
    once([] {
        const int most = (int)std::max<size_t>(TERMS_SMEM_SLOTS * 3 / 2 * sizeof(unsigned long long),
                                               TERMS_SMEM_BUDGET);
        cudaFuncSetAttribute(k_query_terms<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        cudaFuncSetAttribute(k_query_terms<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    });
    // shared memory: the on-chip table region (at least the largest set of the
    // launch that is kept on chip), plus a list of half that set's slots
    const uint32_t table_slots = a.smem_table > a.smem_slots ? a.smem_table : a.smem_slots;
    const size_t dyn = (size_t)(table_slots + a.smem_slots / 2) * sizeof(unsigned long long);
    if (a.h == 1 && a.n_blocks <= 2) k_query_terms<true><<<n_queries, TERMS_THREADS, dyn, s>>>(a);
    else k_query_terms<false><<<n_queries, TERMS_THREADS, dyn, s>>>(a);
}

void launch_terms_long_insert(const TermsArgs &a, cudaStream_t s) {
    if (a.n_chunks) k_terms_long_insert<<<a.n_chunks, TERMS_THREADS, 0, s>>>(a);
}

void launch_terms_long_rows(const TermsArgs &a, cudaStream_t s) {
    const uint32_t groups = (a.n_blocks + BP - 1) / BP;
    if (a.n_long && groups) k_terms_long_rows<<<dim3(a.n_long, groups), TERMS_THREADS, 0, s>>>(a);
}

void launch_query_terms(const TermsArgs &a, uint32_t n_queries, cudaStream_t s) {
    if (n_queries == 0) return;
    launch_terms_short(a, n_queries, s);
    if (a.n_chunks) {
        launch_terms_long_insert(a, s);
        launch_terms_long_rows(a, s);
    }
}

uint32_t terms_round_windows() { return TERMS_ROUND; }

}  // namespace cobs
