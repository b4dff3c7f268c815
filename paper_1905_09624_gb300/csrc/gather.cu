// K2/K4: gather the h rows of every query term in a block, AND them, ADD the
// indicator bits into per-document scores (Sec. 2.2), threshold (Sec. 2.1).
//
// Counters are bit-sliced ("vertical"): a lane owns 128 documents (one 16-byte
// column of a row) and keeps, for each of its four 32-document words, L words
// lv[0..L-1] such that the score of document bit j is sum_l bit_j(lv[l]) 2^l.
// Indicator words are added 16 (or 8) at a time by a carry-save adder tree
// (Harley and Seal's population-count scheme: each full adder is two 3-input
// logic operations), the carry out of the tree is rippled into the upper levels.
// This replaces the paper's byte-lookup expansion into 16-bit counters with SIMD
// adds (Sec. 2.3), which needs about one add per 8 documents; the adder tree
// needs about three logic operations per 32 documents.
#include "gather_common.cuh"

namespace cobs {

// One warp-tile of the register kernel: QPW queries x one row slice of one block.
template <int LPQ, int G, int L>
__device__ __forceinline__ void tile_body(const GatherArgs &a, const DevBlock &blk, uint32_t block_idx,
                                          uint32_t col, bool active, uint32_t q, uint32_t ell) {
    uint32_t lv[4][L];
#pragma unroll
    for (int w = 0; w < 4; w++)
#pragma unroll
        for (int l = 0; l < L; l++) lv[w][l] = 0u;
    const uint32_t n = active ? ell : 0u;
    const uint32_t *ridx = a.rows_idx + (uint64_t)(block_idx * a.h) * a.tcap + a.term_base[q];
    const uint8_t *colbase = a.rows + blk.row_offset + col;
    accumulate<L, G>(lv, colbase, blk.rowbytes, ridx, a.tcap, a.h, 0u, n);
    emit_hits<L, LPQ>(a, blk, col, q, ell, lv, n != 0u);  // every lane of the warp
}

// Persistent batched kernel.  Tiles are (row slice, group of QPW queries), slice
// major, so the CTAs resident at any moment read the same few slices and the
// slices stay in L2; within a slice the groups run longest query first.
template <int LPQ, int G, int L>
__global__ void __launch_bounds__(GATHER_THREADS) k_gather_batched(GatherArgs a) {
    constexpr uint32_t QPW = 32 / LPQ;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t qslot = lane / LPQ;
    const uint32_t c = lane % LPQ;
    const unsigned long long n_tiles = (unsigned long long)a.n_slices * a.n_groups;
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(a.work_counter, 1ULL);
        tile = __shfl_sync(FULL, tile, 0);
        if (tile >= n_tiles) break;
        const uint32_t s = (uint32_t)(tile / a.n_groups);
        const uint32_t g = (uint32_t)(tile % a.n_groups);
        const SliceDesc sd = a.slices[s];
        const DevBlock blk = a.blocks[sd.block];
        const uint32_t qi = g * QPW + qslot;
        const bool valid = qi < a.n_queries;
        const uint32_t q = valid ? a.items[qi].x : 0u;  // items of this kernel are whole queries
        const uint32_t ell = valid ? a.ell[q] : 0u;
        const uint32_t col = sd.byte_off + c * 16u;
        const bool active = valid && col < blk.rowbytes;
        tile_body<LPQ, G, L>(a, blk, sd.block, col, active, q, ell);
    }
}

// ------------------------------------------------------- cp.async pipeline
// h == 1 form of the batched kernel: every lane streams its query's row slices
// through a ring of PIPE_D stages of PIPE_G rows in shared memory (cp.async,
// 16 bytes per lane and row, L2 only), so up to PIPE_D - 1 groups of loads are
// in flight while the adder tree consumes the oldest group.  Row indices are
// prefetched in registers.  The default geometry (16 rows x 2 stages, 2 warps
// per CTA, 6 CTAs per SM) was the fastest of the measured variants: more
// resident warps beat deeper rings per warp (the profile record in profiles/
// lists the sweep).
#ifndef COBS_PIPE_G
#define COBS_PIPE_G 16
#endif
#ifndef COBS_PIPE_D
#define COBS_PIPE_D 2
#endif
#ifndef COBS_PIPE_WARPS
#define COBS_PIPE_WARPS 2
#endif
#ifndef COBS_PIPE_IDX_AHEAD
#define COBS_PIPE_IDX_AHEAD 1  // row indices are loaded 1 or 2 stages before they are issued
#endif
#ifndef COBS_PIPE_MINB
#define COBS_PIPE_MINB 0  // 0: let the compiler choose the register count
#endif
constexpr int PIPE_WARPS = COBS_PIPE_WARPS;
constexpr int PIPE_THREADS = PIPE_WARPS * 32;
constexpr int PIPE_G = COBS_PIPE_G;  // rows per stage (8 or 16)
constexpr int PIPE_D = COBS_PIPE_D;  // stages in the ring
static_assert(PIPE_G == 8 || PIPE_G == 16, "stages of 8 or 16 rows");
// A one-warp CTA variant of this kernel stopped with "illegal instruction" once
// and its cause was not found; it is excluded.
static_assert(PIPE_WARPS >= 2, "CTAs of at least two warps");

__device__ __forceinline__ void issue_stage(uint4 *stage_lane, const uint8_t *colbase, uint32_t rowbytes,
                                            const uint32_t (&r)[PIPE_G], uint32_t t0, uint32_t n, uint64_t pol) {
    if (t0 + PIPE_G <= n) {  // a full group: no per-row predicates
#pragma unroll
        for (int j = 0; j < PIPE_G; j++) cp_async16(stage_lane + j * 32, colbase + (uint64_t)r[j] * rowbytes, 16u, pol);
        return;
    }
#pragma unroll
    for (int j = 0; j < PIPE_G; j++) {
        const bool ok = t0 + j < n;
        const uint8_t *src = ok ? colbase + (uint64_t)r[j] * rowbytes : colbase;
        cp_async16(stage_lane + j * 32, src, ok ? 16u : 0u, pol);  // past the terms: zero fill
    }
}

template <int LPQ, int L>
#if COBS_PIPE_MINB > 0
__global__ void __launch_bounds__(PIPE_THREADS, COBS_PIPE_MINB) k_gather_pipe(GatherArgs a) {
#else
__global__ void __launch_bounds__(PIPE_THREADS) k_gather_pipe(GatherArgs a) {
#endif
    __shared__ __align__(16) uint4 s_stage[PIPE_WARPS][PIPE_D][PIPE_G][32];
    constexpr uint32_t QPW = 32 / LPQ;
    constexpr int LV0 = PIPE_G == 16 ? 4 : 3;
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t qslot = lane / LPQ;
    const uint32_t c = lane % LPQ;
    const unsigned long long n_tiles = (unsigned long long)a.n_slices * a.n_groups;
    const uint64_t pol_idx = l2_policy(a.l2_idx_policy);
    const uint64_t pol_row = l2_policy(a.l2_row_policy);
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(a.work_counter, 1ULL);
        tile = __shfl_sync(FULL, tile, 0);
        if (tile >= n_tiles) break;
        const uint32_t s = (uint32_t)(tile / a.n_groups);
        const uint32_t g0 = (uint32_t)(tile % a.n_groups);
        const SliceDesc sd = a.slices[s];
        const DevBlock blk = a.blocks[sd.block];
        const uint32_t qi = g0 * QPW + qslot;
        const bool valid = qi < a.n_queries;
        const uint4 it = valid ? a.items[qi] : make_uint4(0u, 0u, 0u, ITEM_WHOLE);
        const uint32_t q = it.x;
        const uint32_t ell = valid ? a.ell[q] : 0u;
        const uint32_t tend = ell < it.z ? ell : it.z;  // terms [it.y, tend) of the query
        const uint32_t col = sd.byte_off + c * 16u;
        const bool active = valid && col < blk.rowbytes;
        const uint32_t n = active && tend > it.y ? tend - it.y : 0u;
        const uint32_t ng = (n + PIPE_G - 1) / PIPE_G;
        const uint32_t *ridx = a.rows_idx + (uint64_t)sd.block * a.tcap + a.term_base[q] + it.y;
        const uint8_t *colbase = a.rows + blk.row_offset + col;
        const uint32_t rowbytes = blk.rowbytes;

        uint32_t lv[4][L];
#pragma unroll
        for (int w = 0; w < 4; w++)
#pragma unroll
            for (int l = 0; l < L; l++) lv[w][l] = 0u;
        uint32_t ra[PIPE_G];
        load_idx(ridx, 0, ng, ra, pol_idx);
#if COBS_PIPE_IDX_AHEAD == 2
        uint32_t rb[PIPE_G];
        load_idx(ridx, 1, ng, rb, pol_idx);
#endif
        // after issuing group gi: ra <- indices of gi + 1 (and rb <- gi + 2)
        auto advance_idx = [&](uint32_t gnext) {
#if COBS_PIPE_IDX_AHEAD == 2
#pragma unroll
            for (int j = 0; j < PIPE_G; j++) ra[j] = rb[j];
            load_idx(ridx, gnext + 1, ng, rb, pol_idx);
#else
            load_idx(ridx, gnext, ng, ra, pol_idx);
#endif
        };
        uint32_t gi = 0, si = 0;  // next group to issue, its stage
#pragma unroll
        for (int p = 0; p < PIPE_D - 1; p++) {
            if (gi < ng) issue_stage(&s_stage[warp][si][0][lane], colbase, rowbytes, ra, gi * PIPE_G, n, pol_row);
            cp_async_commit();
            gi++;
            si = si + 1 == PIPE_D ? 0 : si + 1;
            advance_idx(gi);
        }
        uint32_t sc = 0;  // stage being consumed
        CarryPairs<LV0, L> carry;
        for (uint32_t g = 0; g < ng; g++) {
            if (gi < ng) issue_stage(&s_stage[warp][si][0][lane], colbase, rowbytes, ra, gi * PIPE_G, n, pol_row);
            cp_async_commit();
            gi++;
            si = si + 1 == PIPE_D ? 0 : si + 1;
            advance_idx(gi);
            cp_async_wait<PIPE_D - 1>();
            if constexpr (PIPE_G == 16) carry.add(lv, hs16_stage<L>(lv, &s_stage[warp][sc][0][lane]));
            else carry.add(lv, hs8_stage<L>(lv, &s_stage[warp][sc][0][lane]));
            sc = sc + 1 == PIPE_D ? 0 : sc + 1;
        }
        carry.flush(lv);
        cp_async_wait<0>();
        emit_hits<L, LPQ>(a, blk, col, q, ell, lv, it.w == ITEM_WHOLE && n != 0u);  // every lane of the warp
        if (it.w != ITEM_WHOLE && active) write_partials<L>(a, blk, col, it.w, lv);  // every part writes, zeros included
    }
}

template <int LPQ>
static void launch_pipe_L(const GatherArgs &a, uint32_t L, uint32_t grid, cudaStream_t s) {
    switch (L) {
        case 8: k_gather_pipe<LPQ, 8><<<grid, PIPE_THREADS, 0, s>>>(a); break;
        case 12: k_gather_pipe<LPQ, 12><<<grid, PIPE_THREADS, 0, s>>>(a); break;
        case 16: k_gather_pipe<LPQ, 16><<<grid, PIPE_THREADS, 0, s>>>(a); break;
        default: k_gather_pipe<LPQ, 24><<<grid, PIPE_THREADS, 0, s>>>(a); break;
    }
}

template <int LPQ, int G>
static void launch_L(const GatherArgs &a, uint32_t L, uint32_t grid, cudaStream_t s) {
    switch (L) {
        case 8: k_gather_batched<LPQ, G, 8><<<grid, GATHER_THREADS, 0, s>>>(a); break;
        case 12: k_gather_batched<LPQ, G, 12><<<grid, GATHER_THREADS, 0, s>>>(a); break;
        case 16: k_gather_batched<LPQ, G, 16><<<grid, GATHER_THREADS, 0, s>>>(a); break;
        default: k_gather_batched<LPQ, G, 24><<<grid, GATHER_THREADS, 0, s>>>(a); break;
    }
}

uint32_t counter_levels_for(uint32_t max_terms) {
    const uint32_t bits = max_terms ? 32u - (uint32_t)__builtin_clz(max_terms) : 0u;  // bits of max_terms
    if (bits <= 8) return 8;
    if (bits <= 12) return 12;
    if (bits <= 16) return 16;
    return 24;
}

void launch_gather_batched_L(const GatherArgs &a, uint32_t lanes_per_query, uint32_t L, uint32_t grid,
                             cudaStream_t s) {
    if (a.h == 1 && a.tmaps && lanes_per_query == 8) {  // TMA gather ring
        launch_gather_tma(a, L, grid, s);
        return;
    }
    if (a.h == 1) {
        // cp.async pipeline
        switch (lanes_per_query) {
            case 2: launch_pipe_L<2>(a, L, grid, s); break;
            case 4: launch_pipe_L<4>(a, L, grid, s); break;
            case 16: launch_pipe_L<16>(a, L, grid, s); break;
            default: launch_pipe_L<8>(a, L, grid, s); break;
        }
        return;
    }
    if (lanes_per_query == 8 && a.h >= 2 && a.h <= 4) {  // pipelined, 128-byte slices
        launch_gather_pipe_h(a, L, grid, s);
        return;
    }
    switch (lanes_per_query) {
        case 2: launch_L<2, 8>(a, L, grid, s); break;
        case 4: launch_L<4, 8>(a, L, grid, s); break;
        default: launch_L<8, 8>(a, L, grid, s); break;
    }
}

// Warps per CTA of the batched kernel used for h hashes: the single-hash ring
// PIPE_WARPS, the TMA feed and the multi-hash ring 2, the register kernel
// GATHER_THREADS / 32.
int gather_batched_warps_per_cta(uint32_t lanes_per_query, uint32_t h) {
    if (h == 1) return PIPE_WARPS;
    if (lanes_per_query == 8 && h <= 4) return 2;
    return GATHER_THREADS / 32;
}

// Resident CTAs per SM of the batched kernel used for h hashes (persistent grid
// = SMs x this).
int gather_batched_max_blocks_per_sm(uint32_t lanes_per_query, uint32_t h) {
    int nb = 0;
    if (h == 1) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_pipe<8, 12>, PIPE_THREADS, 0);
    } else if (lanes_per_query == 8 && h <= 4) {
        nb = gather_pipe_h_blocks_per_sm(h);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_batched<8, 8, 12>, GATHER_THREADS, 0);
    }
    return nb;
}

}  // namespace cobs
