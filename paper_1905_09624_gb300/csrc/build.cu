// Device index construction (Sec. 2.3 "Classic and Compact"): distinct-term
// count of every document (its "size", which orders the compact layout), and
// the Bloom bit-setting of every (term, hash) pair into the row-major blocks
// (Sec. 2.1 Bloom filters, Sec. 2.2 bit-sliced rows).
#include "kernels.cuh"

namespace cobs {

// Walk the windows [p0, p1) of document d with one thread per segment of
// segment positions; f(code) is called for every term.
template <typename F>
__device__ __forceinline__ void walk_segment(const uint8_t *src, uint64_t p0, uint64_t p1, uint32_t kind, uint32_t k,
                                             F &&f) {
    if (p1 <= p0) return;
    const uint64_t mask = kmer_mask(k);
    Roller r;
    roll_init(r);
    const uint64_t ie = p1 + k - 1;
    for (uint64_t i = p0; i < ie; i++) {
        uint64_t code;
        if (roll_push(r, src[i], kind, k, mask, &code)) f(code);
    }
}

constexpr uint32_t BUILD_SEG = BUILD_CHUNK / BUILD_THREADS;  // 64 positions per thread

__global__ void __launch_bounds__(BUILD_THREADS) k_doc_count(CountArgs a) {
    const uint32_t d = a.chunk_doc[blockIdx.x];
    const uint64_t len = a.doc_off[d + 1] - a.doc_off[d];
    const uint64_t npos = len >= a.k ? len - a.k + 1 : 0;
    const uint64_t p0 = a.chunk_p0[blockIdx.x] + (uint64_t)threadIdx.x * BUILD_SEG;
    const uint64_t p1 = p0 + BUILD_SEG < npos ? p0 + BUILD_SEG : npos;
    unsigned long long *table = a.tables + a.table_base[d];
    const uint32_t cap = a.table_cap[d];
    uint32_t fresh = 0;
    walk_segment(a.docs + a.doc_off[d], p0, p1, a.kind, a.k, [&](uint64_t code) {
        if (code == EMPTY_KEY) {
            if (atomicExch(&a.has_empty[d], 1u) == 0u) fresh++;
        } else if (set_insert(table, cap, xxh64_u64(code, 0), code)) {
            fresh++;
        }
    });
    fresh = __reduce_add_sync(0xffffffffu, fresh);
    if ((threadIdx.x & 31u) == 0 && fresh) atomicAdd(&a.v[d], (unsigned long long)fresh);
}

__global__ void __launch_bounds__(BUILD_THREADS) k_doc_setbits(SetBitsArgs a) {
    const uint32_t d = a.chunk_doc[blockIdx.x];
    const uint64_t len = a.doc_off[d + 1] - a.doc_off[d];
    const uint64_t npos = len >= a.k ? len - a.k + 1 : 0;
    const uint64_t p0 = a.chunk_p0[blockIdx.x] + (uint64_t)threadIdx.x * BUILD_SEG;
    const uint64_t p1 = p0 + BUILD_SEG < npos ? p0 + BUILD_SEG : npos;
    const DevBlock blk = a.blocks[a.doc_block[d]];
    const uint32_t j = a.doc_col[d];
    const uint32_t bit = 1u << (j & 31u);
    uint32_t *base = a.rows32 + blk.row_offset / 4 + (j >> 5);
    const uint32_t words_per_row = blk.rowbytes / 4;
    walk_segment(a.docs + a.doc_off[d], p0, p1, a.kind, a.k, [&](uint64_t code) {
        for (uint32_t i = 0; i < a.h; i++) {
            uint32_t r = barrett_mod(xxh64_u64(code, i), blk.barrett_m, blk.w);
            atomicOr(base + (uint64_t)r * words_per_row, bit);
        }
    });
}

void launch_doc_count(const CountArgs &a, uint32_t n_chunks, cudaStream_t s) {
    if (n_chunks) k_doc_count<<<n_chunks, BUILD_THREADS, 0, s>>>(a);
}

void launch_doc_setbits(const SetBitsArgs &a, uint32_t n_chunks, cudaStream_t s) {
    if (n_chunks) k_doc_setbits<<<n_chunks, BUILD_THREADS, 0, s>>>(a);
}

}  // namespace cobs
