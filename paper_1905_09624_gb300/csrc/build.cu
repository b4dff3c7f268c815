// Device index construction (Sec. 2.3 "Classic and Compact"): distinct-term
// count of every document (its "size", which orders the compact layout), and
// the Bloom bit-setting of every (term, hash) pair into the row-major blocks
// (Sec. 2.1 Bloom filters, Sec. 2.2 bit-sliced rows).
//
// Each CTA takes a chunk of one document's windows, stages the chunk's bytes in
// shared memory (packing DNA into a 2-bit stream) and gives every thread one
// window at a time.
#include "kernels.cuh"

namespace cobs {

template <uint32_t W>
struct ChunkStage {
    uint8_t bytes[W + 32];             // W windows need W + k - 1 <= W + 31 bytes
    uint32_t pk[(W + 32) / 16 + 3];
    uint16_t inv[(W + 32) / 16 + 3];
};

// Stage the windows [p0, p0 + nwin) of one document.  Cooperative (NT threads);
// every thread issues all of its byte loads before it stores any, so they are
// in flight together; ends with a barrier.
template <uint32_t NT, uint32_t W>
__device__ __forceinline__ void stage_chunk(ChunkStage<W> &st, const uint8_t *doc, uint64_t p0, uint32_t nwin,
                                            uint32_t k, bool dna) {
    constexpr uint32_t PER = (W + 32 + NT - 1) / NT;
    const uint32_t nbytes = nwin + k - 1;
    uint8_t v[PER];
#pragma unroll
    for (uint32_t j = 0; j < PER; j++) {
        const uint32_t i = threadIdx.x + j * NT;
        v[j] = i < nbytes ? doc[p0 + i] : (uint8_t)0;
    }
#pragma unroll
    for (uint32_t j = 0; j < PER; j++) {
        const uint32_t i = threadIdx.x + j * NT;
        if (i < nbytes) st.bytes[i] = v[j];
    }
    __syncthreads();
    if (dna) {
        pack_bases(st.bytes, nbytes, st.pk, st.inv);
        __syncthreads();
    }
}

// Term code of window p of the staged chunk; false for a DNA window with a
// non-ACGT byte.
template <uint32_t W>
__device__ __forceinline__ bool chunk_term(const ChunkStage<W> &st, uint32_t p, uint32_t kind, uint32_t k,
                                           uint64_t mask, uint64_t *code) {
    if (kind == KIND_BYTES) {
        *code = bytes_qgram(st.bytes, p, k);
        return true;
    }
    return packed_kmer(st.pk, st.inv, p, k, kind == KIND_DNA_CANONICAL, mask, code);
}

__global__ void __launch_bounds__(BUILD_THREADS) k_doc_count(CountArgs a) {
    __shared__ ChunkStage<COUNT_CHUNK> st;
    const uint32_t d = a.chunk_doc[blockIdx.x];
    const uint64_t len = a.doc_off[d + 1] - a.doc_off[d];
    const uint64_t npos = len >= a.k ? len - a.k + 1 : 0;
    const uint64_t p0 = a.chunk_p0[blockIdx.x];
    const uint32_t nwin = (uint32_t)(npos - p0 < COUNT_CHUNK ? npos - p0 : COUNT_CHUNK);
    stage_chunk<BUILD_THREADS>(st, a.docs + a.doc_off[d], p0, nwin, a.k, a.kind != KIND_BYTES);
    unsigned long long *table = a.tables + a.table_base[d];
    const uint32_t cap = a.table_cap[d];
    const uint64_t mask = kmer_mask(a.k);
    uint32_t fresh = 0;
    for (uint32_t p = threadIdx.x; p < nwin; p += blockDim.x) {
        uint64_t code;
        if (!chunk_term(st, p, a.kind, a.k, mask, &code)) continue;
        if (code == EMPTY_KEY) {
            if (atomicExch(&a.has_empty[d], 1u) == 0u) fresh++;
        } else if (set_insert(table, cap, xxh64_u64(code, 0), code)) {
            fresh++;
        }
    }
    fresh = __reduce_add_sync(0xffffffffu, fresh);
    if ((threadIdx.x & 31u) == 0 && fresh) atomicAdd(&a.v[d], (unsigned long long)fresh);
}

__global__ void __launch_bounds__(BUILD_THREADS) k_doc_setbits(SetBitsArgs a) {
    __shared__ ChunkStage<SETBITS_CHUNK> st;
    const uint32_t d = a.chunk_doc[blockIdx.x];
    const uint64_t len = a.doc_off[d + 1] - a.doc_off[d];
    const uint64_t npos = len >= a.k ? len - a.k + 1 : 0;
    const uint64_t p0 = a.chunk_p0[blockIdx.x];
    const uint32_t nwin = (uint32_t)(npos - p0 < SETBITS_CHUNK ? npos - p0 : SETBITS_CHUNK);
    stage_chunk<BUILD_THREADS>(st, a.docs + a.doc_off[d], p0, nwin, a.k, a.kind != KIND_BYTES);
    const DevBlock blk = a.blocks[a.doc_block[d]];
    const uint32_t j = a.doc_col[d];
    const uint32_t bit = 1u << (j & 31u);
    uint32_t *base = a.rows32 + blk.row_offset / 4 + (j >> 5);
    const uint32_t words_per_row = blk.rowbytes / 4;
    const uint64_t mask = kmer_mask(a.k);
    for (uint32_t p = threadIdx.x; p < nwin; p += blockDim.x) {
        uint64_t code;
        if (!chunk_term(st, p, a.kind, a.k, mask, &code)) continue;
        for (uint32_t i = 0; i < a.h; i++) {
            const uint32_t r = barrett_mod(xxh64_u64(code, i), blk.barrett_m, blk.w);
            atomicOr(base + (uint64_t)r * words_per_row, bit);
        }
    }
}

// ------------------------------------------------ partitioned distinct count
// Scatter: the CTA's windows get their partition (multiply-shift of the high 32
// bits of mix64 of the term) and a rank within it from shared-memory counters; one
// global atomic per partition reserves the CTA's run, then every term -- taken
// again from the staged bases -- is written to its slot.  Slots past the
// partition's capacity are not written: the count pass sees the overflow and the
// document is recounted with a global set.  Shared memory: the stage, a word per
// window and two counters per partition (max_parts), so several CTAs fit an SM.
__global__ void __launch_bounds__(PART_THREADS) k_part_scatter(PartArgs a) {
    __shared__ ChunkStage<COUNT_CHUNK> st;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t *s_pr = reinterpret_cast<uint32_t *>(s_dyn);  // COUNT_CHUNK: partition << 12 | rank
    uint32_t *s_hist = s_pr + COUNT_CHUNK;                  // max_parts
    uint32_t *s_base = s_hist + a.max_parts;                // max_parts
    const uint32_t d = a.chunk_doc[blockIdx.x];
    const uint64_t len = a.doc_off[d + 1] - a.doc_off[d];
    const uint64_t npos = len >= a.k ? len - a.k + 1 : 0;
    const uint64_t p0 = a.chunk_p0[blockIdx.x];
    const uint32_t nwin = (uint32_t)(npos - p0 < COUNT_CHUNK ? npos - p0 : COUNT_CHUNK);
    const uint32_t P = a.n_parts[d];
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) s_hist[i] = 0u;
    stage_chunk<PART_THREADS>(st, a.docs + a.doc_off[d], p0, nwin, a.k, a.kind != KIND_BYTES);  // barriers order the zeroing
    const uint64_t mask = kmer_mask(a.k);
    for (uint32_t w = threadIdx.x; w < nwin; w += blockDim.x) {
        uint64_t code;
        uint32_t pr = 0xFFFFFFFFu;
        if (chunk_term(st, w, a.kind, a.k, mask, &code)) {
            if (code == EMPTY_KEY) {  // kept out of the sets: a flag per document
                if (atomicExch(&a.has_empty[d], 1u) == 0u) atomicAdd(&a.v[d], 1ULL);
            } else {
                const uint64_t h = mix64(code);
                const uint32_t part = (uint32_t)(((h >> 32) * (uint64_t)P) >> 32);
                pr = (part << 12) | atomicAdd(&s_hist[part], 1u);
            }
        }
        s_pr[w] = pr;
    }
    __syncthreads();
    const uint64_t pbase = a.part0[d];
    for (uint32_t i = threadIdx.x; i < P; i += blockDim.x)
        if (s_hist[i]) s_base[i] = atomicAdd(&a.part_count[pbase + i], s_hist[i]);
    __syncthreads();
    const uint32_t cap = a.part_cap[d];
    unsigned long long *out = a.codes + a.code0[d];
    for (uint32_t w = threadIdx.x; w < nwin; w += blockDim.x) {
        const uint32_t pr = s_pr[w];
        if (pr == 0xFFFFFFFFu) continue;
        const uint32_t part = pr >> 12;
        const uint32_t slot = s_base[part] + (pr & 4095u);
        uint64_t code = 0;
        chunk_term(st, w, a.kind, a.k, mask, &code);  // a term: pr was set for it
        if (slot < cap) out[(uint64_t)part * cap + slot] = code;
    }
}

// Count: the distinct terms of one partition in a shared-memory open-addressing
// set (home slot from the low 32 bits of the hash: the high bits chose the
// partition), added to the document's count once per warp.
__global__ void __launch_bounds__(PART_COUNT_THREADS) k_part_count(PartArgs a) {
    extern __shared__ __align__(16) unsigned long long s_set[];  // PART_SET_SLOTS
    const uint32_t d = a.part_doc[blockIdx.x];
    const uint32_t n = a.part_count[blockIdx.x];
    const uint32_t cap = a.part_cap[d];
    if (n > cap) {  // the scatter dropped terms: recounted with a global set
        if (threadIdx.x == 0) atomicExch(&a.overflow[d], 1u);
        return;
    }
    for (uint32_t i = threadIdx.x; i < PART_SET_SLOTS; i += blockDim.x) s_set[i] = EMPTY_KEY;
    __syncthreads();
    const unsigned long long *src = a.codes + a.code0[d] + (uint64_t)a.part_idx[blockIdx.x] * cap;
    uint32_t fresh = 0;
    // PART_BATCH loads in flight per thread before the first insertion waits on one
    constexpr uint32_t PART_BATCH = 8;
    for (uint32_t base = threadIdx.x; base < n; base += blockDim.x * PART_BATCH) {
        unsigned long long key[PART_BATCH];
#pragma unroll
        for (uint32_t j = 0; j < PART_BATCH; j++) {
            const uint32_t i = base + j * blockDim.x;
            key[j] = i < n ? src[i] : (unsigned long long)EMPTY_KEY;
        }
#pragma unroll
        for (uint32_t j = 0; j < PART_BATCH; j++) {
            if (key[j] == EMPTY_KEY) continue;  // past the partition's terms (the set never holds EMPTY)
            const uint64_t h = mix64(key[j]);
            uint32_t slot = (uint32_t)(((h & 0xFFFFFFFFULL) * PART_SET_SLOTS) >> 32);
            for (uint32_t probe = 0; probe < PART_SET_SLOTS; probe++) {
                const unsigned long long old = atomicCAS(&s_set[slot], (unsigned long long)EMPTY_KEY, key[j]);
                if (old == EMPTY_KEY) {
                    fresh++;
                    break;
                }
                if (old == key[j]) break;
                slot = (slot + 1u) & (PART_SET_SLOTS - 1u);
            }
        }
    }
    fresh = __reduce_add_sync(0xffffffffu, fresh);
    if ((threadIdx.x & 31u) == 0 && fresh) atomicAdd(&a.v[d], (unsigned long long)fresh);
}

void launch_part_scatter(const PartArgs &a, uint32_t n_chunks, cudaStream_t s) {
    constexpr int most = (int)(COUNT_CHUNK * 4 + 2 * PART_MAX * 4);
    static PerDeviceOnce once;
    once([] { cudaFuncSetAttribute(k_part_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, most); });
    const size_t dyn = (size_t)COUNT_CHUNK * 4 + 2 * (size_t)a.max_parts * 4;
    if (n_chunks) k_part_scatter<<<n_chunks, PART_THREADS, dyn, s>>>(a);
}

void launch_part_count(const PartArgs &a, uint32_t n_parts, cudaStream_t s) {
    constexpr int dyn = (int)(PART_SET_SLOTS * 8);
    static PerDeviceOnce once;
    once([] { cudaFuncSetAttribute(k_part_count, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn); });
    if (n_parts) k_part_count<<<n_parts, PART_COUNT_THREADS, dyn, s>>>(a);
}

// ------------------------------------------------- per-document filters
// Sec. 2.1 builds one Bloom filter per document and Sec. 2.2 stores the filters
// bit-sliced.  Here a CTA sets the bits of one document's whole filter in shared
// memory (atomicOr on shared words: no global atomics), staging the document's
// windows FILTER_TILE at a time, then writes the filter out column-major.
__global__ void __launch_bounds__(FILTER_THREADS) k_doc_filter(FilterArgs a) {
    extern __shared__ __align__(16) uint32_t s_filt[];  // pitch_words
    __shared__ ChunkStage<FILTER_TILE> st;
    const uint32_t d = a.col_doc[blockIdx.x];
    const uint64_t len = a.doc_off[d + 1] - a.doc_off[d];
    const uint64_t npos = len >= a.k ? len - a.k + 1 : 0;
    for (uint32_t i = threadIdx.x; i < a.pitch_words; i += blockDim.x) s_filt[i] = 0u;
    __syncthreads();
    const uint64_t mask = kmer_mask(a.k);
    const bool dna = a.kind != KIND_BYTES;
    const uint8_t *doc = a.docs + a.doc_off[d];
    // the bytes of the next tile are loaded into registers while this tile's
    // windows are processed (PRE bytes per thread), then staged
    constexpr uint32_t PRE = (FILTER_TILE + 32 + FILTER_THREADS - 1) / FILTER_THREADS;
    if (npos) stage_chunk<FILTER_THREADS>(st, doc, 0, (uint32_t)(npos < FILTER_TILE ? npos : FILTER_TILE), a.k, dna);
    for (uint64_t p0 = 0; p0 < npos; p0 += FILTER_TILE) {
        const uint32_t nwin = (uint32_t)(npos - p0 < FILTER_TILE ? npos - p0 : FILTER_TILE);
        const uint64_t q0 = p0 + FILTER_TILE;
        const uint32_t nnext = q0 < npos ? (uint32_t)(npos - q0 < FILTER_TILE ? npos - q0 : FILTER_TILE) : 0u;
        const uint32_t nbytes_next = nnext ? nnext + a.k - 1 : 0u;
        uint8_t pre[PRE];
#pragma unroll
        for (uint32_t j = 0; j < PRE; j++) {
            const uint32_t i = threadIdx.x + j * FILTER_THREADS;
            pre[j] = i < nbytes_next ? doc[q0 + i] : (uint8_t)0;
        }
        for (uint32_t p = threadIdx.x; p < nwin; p += blockDim.x) {
            uint64_t code;
            if (!chunk_term(st, p, a.kind, a.k, mask, &code)) continue;
            for (uint32_t i = 0; i < a.h; i++) {
                const uint32_t r = barrett_mod(xxh64_u64(code, i), a.barrett_m, a.w);
                atomicOr(&s_filt[r >> 5], 1u << (r & 31u));
            }
        }
        __syncthreads();  // the stage is refilled next; the last barrier also orders the copy-out
        if (nnext) {
#pragma unroll
            for (uint32_t j = 0; j < PRE; j++) {
                const uint32_t i = threadIdx.x + j * FILTER_THREADS;
                if (i < nbytes_next) st.bytes[i] = pre[j];
            }
            __syncthreads();
            if (dna) {
                pack_bases(st.bytes, nbytes_next, st.pk, st.inv);
                __syncthreads();
            }
        }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(a.filters + (uint64_t)blockIdx.x * a.pitch_words);
    const uint4 *src = reinterpret_cast<const uint4 *>(s_filt);
    for (uint32_t i = threadIdx.x; i < a.pitch_words / 4; i += blockDim.x) dst[i] = src[i];
}

// 32 x 32 bit-matrix transpose across a warp: lane l holds row l (bit c =
// column c); afterwards lane l holds column l (bit c = row c).  Five rounds swap
// the off-diagonal j x j blocks of every 2j x 2j block with the partner lane
// l ^ j (the recursive block transpose of Warren, "Hacker's Delight", 2nd ed.,
// Sec. 7-3, with the rows in lanes instead of an array).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, uint32_t lane) {
    uint32_t m = 0x0000FFFFu;
#pragma unroll
    for (uint32_t j = 16; j != 0; j >>= 1, m ^= m << j) {
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y << j) & ~m));
    }
    return x;
}

// Tile of 256 filters (documents c0.., one per thread) x 8 filter words (256
// rows): each warp turns its 32 documents x 32 rows sub-tiles around (afterwards
// lane i holds row i of the sub-tile, bit l = document l), then every thread
// writes one row's 32 bytes (documents c0..c0+255, LSB-first) in two 16-byte
// stores, the second only if the row is that wide.
__global__ void __launch_bounds__(TRANSPOSE_DOCS) k_filter_transpose(TransposeArgs a) {
    __shared__ uint32_t s_in[TRANSPOSE_DOCS][TRANSPOSE_WORDS + 1];       // [document][word]
    __shared__ uint32_t s_out[TRANSPOSE_WORDS * 32][TRANSPOSE_WORDS + 1];  // [row][32-document word]
    const uint32_t t = threadIdx.x, warp = t >> 5, lane = t & 31u;
    const uint32_t wi0 = blockIdx.x * TRANSPOSE_WORDS;
    const uint32_t c0 = blockIdx.y * TRANSPOSE_DOCS;
    uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
    if (c0 + t < a.n_cols) {  // documents past the wave: zero bits (padding columns stay zero)
        const uint4 *src = reinterpret_cast<const uint4 *>(a.filters + (uint64_t)(c0 + t) * a.pitch_words + wi0);
        lo = src[0];
        hi = src[1];
    }
    s_in[t][0] = lo.x; s_in[t][1] = lo.y; s_in[t][2] = lo.z; s_in[t][3] = lo.w;
    s_in[t][4] = hi.x; s_in[t][5] = hi.y; s_in[t][6] = hi.z; s_in[t][7] = hi.w;
    __syncthreads();
#pragma unroll 1
    for (uint32_t word = 0; word < TRANSPOSE_WORDS; word++) {
        s_out[32u * word + lane][warp] = warp_transpose32(s_in[32u * warp + lane][word], lane);
    }
    __syncthreads();
    const uint32_t r = 32u * wi0 + t;
    const uint32_t byte0 = (a.col0 + c0) / 8u;
    if (r < a.w && byte0 < a.rowbytes) {
        uint8_t *dst = a.rows + (uint64_t)r * a.rowbytes + byte0;
        *reinterpret_cast<uint4 *>(dst) = make_uint4(s_out[t][0], s_out[t][1], s_out[t][2], s_out[t][3]);
        if (byte0 + 16u < a.rowbytes)
            *reinterpret_cast<uint4 *>(dst + 16) = make_uint4(s_out[t][4], s_out[t][5], s_out[t][6], s_out[t][7]);
    }
}

void launch_doc_filter(const FilterArgs &a, uint32_t n_cols, cudaStream_t s) {
    static PerDeviceOnce once;
    once([] {
        cudaFuncSetAttribute(k_doc_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FILTER_SMEM_MAX);
    });
    if (n_cols) k_doc_filter<<<n_cols, FILTER_THREADS, (size_t)a.pitch_words * 4, s>>>(a);
}

void launch_filter_transpose(const TransposeArgs &a, cudaStream_t s) {
    if (!a.n_cols) return;
    const dim3 grid(a.pitch_words / TRANSPOSE_WORDS, (a.n_cols + TRANSPOSE_DOCS - 1) / TRANSPOSE_DOCS);
    k_filter_transpose<<<grid, TRANSPOSE_DOCS, 0, s>>>(a);
}

void launch_doc_count(const CountArgs &a, uint32_t n_chunks, cudaStream_t s) {
    if (n_chunks) k_doc_count<<<n_chunks, BUILD_THREADS, 0, s>>>(a);
}

void launch_doc_setbits(const SetBitsArgs &a, uint32_t n_chunks, cudaStream_t s) {
    if (n_chunks) k_doc_setbits<<<n_chunks, BUILD_THREADS, 0, s>>>(a);
}

}  // namespace cobs
