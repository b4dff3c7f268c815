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

// Stage the windows [p0, p0 + nwin) of one document.  Cooperative; ends with a
// barrier.
template <uint32_t W>
__device__ __forceinline__ void stage_chunk(ChunkStage<W> &st, const uint8_t *doc, uint64_t p0, uint32_t nwin,
                                            uint32_t k, bool dna) {
    const uint32_t nbytes = nwin + k - 1;
    for (uint32_t i = threadIdx.x; i < nbytes; i += blockDim.x) st.bytes[i] = doc[p0 + i];
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
    stage_chunk(st, a.docs + a.doc_off[d], p0, nwin, a.k, a.kind != KIND_BYTES);
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
    stage_chunk(st, a.docs + a.doc_off[d], p0, nwin, a.k, a.kind != KIND_BYTES);
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

void launch_doc_count(const CountArgs &a, uint32_t n_chunks, cudaStream_t s) {
    if (n_chunks) k_doc_count<<<n_chunks, BUILD_THREADS, 0, s>>>(a);
}

void launch_doc_setbits(const SetBitsArgs &a, uint32_t n_chunks, cudaStream_t s) {
    if (n_chunks) k_doc_setbits<<<n_chunks, BUILD_THREADS, 0, s>>>(a);
}

}  // namespace cobs
