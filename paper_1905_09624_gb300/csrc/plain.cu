// The plain form (one query per kernel sequence), its threshold, and the
// threshold of split queries (sum of their parts' counts).
#include "gather_common.cuh"

namespace cobs {

// ------------------------------------------------------------------ plain
// One query: thread = (16-byte column over all blocks, chunk of PLAIN_CHUNK terms);
// partial counts of a chunk are added to the score array with atomics.
template <int G>
__global__ void __launch_bounds__(PLAIN_THREADS) k_gather_plain(PlainArgs a) {
    const uint32_t x = blockIdx.y * blockDim.x + threadIdx.x;
    const uint32_t ell = a.ell[a.q];
    const uint32_t t0 = blockIdx.x * PLAIN_CHUNK;
    if (x >= a.n_cols || t0 >= ell) return;
    const uint32_t t1 = t0 + PLAIN_CHUNK < ell ? t0 + PLAIN_CHUNK : ell;
    const uint32_t b = a.col_block[x];
    const uint32_t col = a.col_byte[x];
    const DevBlock blk = a.blocks[b];
    constexpr int L = 8;  // a chunk counts at most 128
    uint32_t lv[4][L];
#pragma unroll
    for (int w = 0; w < 4; w++)
#pragma unroll
        for (int l = 0; l < L; l++) lv[w][l] = 0u;
    const uint32_t *ridx = a.rows_idx + (uint64_t)(b * a.h) * a.tcap + a.term_base[a.q];
    accumulate<L, G>(lv, a.rows + blk.row_offset + col, blk.rowbytes, ridx, a.tcap, a.h, t0, t1);
    const uint32_t doc0 = col * 8u;
#pragma unroll
    for (int w = 0; w < 4; w++) {
        uint32_t any = 0;
#pragma unroll
        for (int l = 0; l < L; l++) any |= lv[w][l];
        while (any) {
            uint32_t bit = __ffs(any) - 1u;
            any &= any - 1u;
            uint32_t j = doc0 + 32u * w + bit;
            if (j < blk.n_docs) atomicAdd(&a.scores[blk.doc_begin + j], count_of<L>(lv[w], bit));
        }
    }
}

void launch_gather_plain(const PlainArgs &a, uint32_t n_chunks, cudaStream_t s) {
    if (n_chunks == 0 || a.n_cols == 0) return;
    // x: term chunks (up to 2^31 - 1), y: column groups (n_cols / 128 stays far below 65536)
    dim3 grid(n_chunks, (a.n_cols + PLAIN_THREADS - 1) / PLAIN_THREADS);
    if (a.h == 1) k_gather_plain<16><<<grid, PLAIN_THREADS, 0, s>>>(a);
    else k_gather_plain<8><<<grid, PLAIN_THREADS, 0, s>>>(a);
}

// Threshold of the plain form: scan the score array, compact the hits with a
// warp ballot and one atomic per warp.
__global__ void k_plain_threshold(ThresholdArgs a) {
    const uint32_t ell = a.ell[a.q];
    if (ell == 0u) return;
    const uint32_t mn = (uint32_t)(((uint64_t)a.thr[a.q] * ell + 999u) / 1000u);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t iters = (a.n_docs + stride - 1) / stride;
    for (uint32_t it = 0; it < iters; it++) {
        uint32_t p = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
        uint32_t sc = p < a.n_docs ? a.scores[p] : 0u;
        bool hit = p < a.n_docs && sc >= mn;
        uint32_t m = __ballot_sync(FULL, hit);
        if (!m) continue;
        unsigned long long base = 0;
        uint32_t leader = __ffs(m) - 1u;
        if (lane == leader) {
            base = atomicAdd(a.hit_count, (unsigned long long)__popc(m));
            atomicAdd(&a.qcount[a.q], (uint32_t)__popc(m));
        }
        base = __shfl_sync(FULL, base, leader);
        if (hit) {
            unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
            if (pos < a.hit_cap) {
                a.raw_q[pos] = a.q;
                a.raw_key[pos] = ((unsigned long long)(~sc) << 32) | a.perm[p];
            }
        }
    }
}

// Split queries: score of a sorted position = sum of its items' partial counts;
// the threshold and the warp-ballot compaction follow the plain form.
__global__ void k_split_finish(SplitArgs a) {
    for (uint32_t si = blockIdx.y; si < a.n_split; si += gridDim.y) {
        const uint4 sp = a.split[si];
        const uint32_t q = sp.x;
        const uint32_t ell = a.ell[q];
        if (ell == 0u) continue;
        const uint32_t mn = (uint32_t)(((uint64_t)a.thr[q] * ell + 999u) / 1000u);
        const uint32_t lane = threadIdx.x & 31u;
        const uint32_t stride = gridDim.x * blockDim.x;
        const uint32_t iters = (a.n_docs + stride - 1) / stride;
        for (uint32_t it = 0; it < iters; it++) {
            const uint32_t p = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
            uint32_t sc = 0;
            if (p < a.n_docs)
                for (uint32_t i = 0; i < sp.z; i++) sc += a.partials[(uint64_t)(sp.y + i) * a.n_docs + p];
            const bool hit = p < a.n_docs && sc >= mn;
            const uint32_t m = __ballot_sync(FULL, hit);
            if (!m) continue;
            unsigned long long base = 0;
            const uint32_t leader = __ffs(m) - 1u;
            if (lane == leader) {
                base = atomicAdd(a.hit_count, (unsigned long long)__popc(m));
                atomicAdd(&a.qcount[q], (uint32_t)__popc(m));
            }
            base = __shfl_sync(FULL, base, leader);
            if (hit) {
                const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
                if (pos < a.hit_cap) {
                    a.raw_q[pos] = q;
                    a.raw_key[pos] = ((unsigned long long)(~sc) << 32) | a.perm[p];
                }
            }
        }
    }
}

void launch_split_finish(const SplitArgs &a, cudaStream_t s) {
    if (a.n_split == 0 || a.n_docs == 0) return;
    uint32_t bx = (a.n_docs + 255) / 256;
    if (bx > 64) bx = 64;
    const uint32_t by = a.n_split < 65535u ? a.n_split : 65535u;
    k_split_finish<<<dim3(bx, by), 256, 0, s>>>(a);
}

void launch_plain_threshold(const ThresholdArgs &a, cudaStream_t s) {
    uint32_t blocks = (a.n_docs + 255) / 256;
    if (blocks == 0) return;
    if (blocks > 1024) blocks = 1024;
    k_plain_threshold<<<blocks, 256, 0, s>>>(a);
}

}  // namespace cobs
