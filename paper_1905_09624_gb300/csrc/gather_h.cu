// K2 for h = 2..4 hashes: the pipelined gather whose stages hold every term's
// h rows; the consumer ANDs them (Sec. 2.2) before the carry-save tree.
#include "gather_common.cuh"

namespace cobs {

// ---------------------------------------------------------- pipe, h > 1
// The pipelined kernel for H = 2..4 hashes: a stage holds PH_G terms x H rows
// per lane (row i of term j at position j * H + i); the consumer ANDs the H
// rows of each term (Sec. 2.2) and feeds the PH_G indicator words to a
// Harley-Seal tree.  The ring lives in dynamic shared memory.  Stages of 4
// terms keep the ring at 24 KB per CTA for h = 3 (8 CTAs/SM); stages of 8
// (48 KB, 4 CTAs/SM) were 13 % slower on the text workload.
#ifndef COBS_PH_G
#define COBS_PH_G 4
#endif
constexpr int PH_G = COBS_PH_G, PH_D = 2, PH_WARPS = 2, PH_THREADS = PH_WARPS * 32;
static_assert(PH_G == 4 || PH_G == 8, "stages of 4 or 8 terms");
template <int H>
constexpr size_t pipe_h_smem() { return (size_t)PH_WARPS * PH_D * PH_G * H * 32 * sizeof(uint4); }

template <int H>
__device__ __forceinline__ W4 and_rows(const uint4 *st, int j) {
    W4 x = w4(st[(j * H) * 32]);
#pragma unroll
    for (int i = 1; i < H; i++) {
        const W4 y = w4(st[(j * H + i) * 32]);
#pragma unroll
        for (int w = 0; w < 4; w++) x.v[w] &= y.v[w];
    }
    return x;
}
template <int L, int H>
__device__ __forceinline__ W4 hs4_and_stage(uint32_t (&lv)[4][L], const uint4 *st) {
    const W4 tA = csa_lv<0>(lv, and_rows<H>(st, 0), and_rows<H>(st, 1));
    const W4 tB = csa_lv<0>(lv, and_rows<H>(st, 2), and_rows<H>(st, 3));
    return csa_lv<1>(lv, tA, tB);
}
template <int L, int H>
__device__ __forceinline__ W4 hs8_and_stage(uint32_t (&lv)[4][L], const uint4 *st) {
    W4 tA = csa_lv<0>(lv, and_rows<H>(st, 0), and_rows<H>(st, 1));
    W4 tB = csa_lv<0>(lv, and_rows<H>(st, 2), and_rows<H>(st, 3));
    W4 fA = csa_lv<1>(lv, tA, tB);
    tA = csa_lv<0>(lv, and_rows<H>(st, 4), and_rows<H>(st, 5));
    tB = csa_lv<0>(lv, and_rows<H>(st, 6), and_rows<H>(st, 7));
    W4 fB = csa_lv<1>(lv, tA, tB);
    return csa_lv<2>(lv, fA, fB);
}

template <int H>
__device__ __forceinline__ void load_idx_h(const uint32_t *const (&ridx)[H], uint32_t g, uint32_t ng,
                                           uint32_t (&r)[H][PH_G], uint64_t pol) {
    if (g < ng) {
#pragma unroll
        for (int i = 0; i < H; i++)
#pragma unroll
            for (int j = 0; j < PH_G; j += 4) {
                uint4 v = ldg_hint(ridx[i] + g * (uint32_t)PH_G + j, pol);
                r[i][j] = v.x; r[i][j + 1] = v.y; r[i][j + 2] = v.z; r[i][j + 3] = v.w;
            }
    }
}

template <int H>
__device__ __forceinline__ void issue_stage_h(uint4 *stage_lane, const uint8_t *colbase, uint32_t rowbytes,
                                              const uint32_t (&r)[H][PH_G], uint32_t t0, uint32_t n, uint64_t pol) {
    if (t0 + PH_G <= n) {
#pragma unroll
        for (int j = 0; j < PH_G; j++)
#pragma unroll
            for (int i = 0; i < H; i++)
                cp_async16(stage_lane + (j * H + i) * 32, colbase + (uint64_t)r[i][j] * rowbytes, 16u, pol);
        return;
    }
#pragma unroll
    for (int j = 0; j < PH_G; j++) {
        const bool ok = t0 + j < n;
#pragma unroll
        for (int i = 0; i < H; i++) {
            const uint8_t *src = ok ? colbase + (uint64_t)r[i][j] * rowbytes : colbase;
            cp_async16(stage_lane + (j * H + i) * 32, src, ok ? 16u : 0u, pol);  // past the terms: zero fill
        }
    }
}

template <int LPQ, int L, int H>
__global__ void __launch_bounds__(PH_THREADS) k_gather_pipe_h(GatherArgs a) {
    extern __shared__ __align__(16) uint4 s_ring[];  // [PH_WARPS][PH_D][PH_G * H][32]
    constexpr uint32_t QPW = 32 / LPQ;
    constexpr uint32_t STAGE = PH_G * H * 32;  // uint4 per stage
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t qslot = lane / LPQ;
    const uint32_t c = lane % LPQ;
    uint4 *ring = s_ring + (size_t)warp * PH_D * STAGE + lane;
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
        const uint32_t q = valid ? a.items[qi].x : 0u;  // items of this kernel are whole queries
        const uint32_t ell = valid ? a.ell[q] : 0u;
        const uint32_t col = sd.byte_off + c * 16u;
        const bool active = valid && col < blk.rowbytes;
        const uint32_t n = active ? ell : 0u;
        const uint32_t ng = (n + PH_G - 1) / PH_G;
        const uint32_t *ridx[H];
#pragma unroll
        for (int i = 0; i < H; i++)
            ridx[i] = a.rows_idx + ((uint64_t)sd.block * H + i) * a.tcap + a.term_base[q];
        const uint8_t *colbase = a.rows + blk.row_offset + col;
        const uint32_t rowbytes = blk.rowbytes;

        uint32_t lv[4][L];
#pragma unroll
        for (int w = 0; w < 4; w++)
#pragma unroll
            for (int l = 0; l < L; l++) lv[w][l] = 0u;
        uint32_t ra[H][PH_G];
        load_idx_h<H>(ridx, 0, ng, ra, pol_idx);
        uint32_t gi = 0, si = 0;  // next group to issue, its stage
#pragma unroll
        for (int p = 0; p < PH_D - 1; p++) {
            if (gi < ng) issue_stage_h<H>(ring + si * STAGE, colbase, rowbytes, ra, gi * PH_G, n, pol_row);
            cp_async_commit();
            gi++;
            si = si + 1 == PH_D ? 0 : si + 1;
            load_idx_h<H>(ridx, gi, ng, ra, pol_idx);
        }
        uint32_t sc = 0;  // stage being consumed
        CarryPairs<PH_G == 8 ? 3 : 2, L> carry;
        for (uint32_t g = 0; g < ng; g++) {
            if (gi < ng) issue_stage_h<H>(ring + si * STAGE, colbase, rowbytes, ra, gi * PH_G, n, pol_row);
            cp_async_commit();
            gi++;
            si = si + 1 == PH_D ? 0 : si + 1;
            load_idx_h<H>(ridx, gi, ng, ra, pol_idx);
            cp_async_wait<PH_D - 1>();
            if constexpr (PH_G == 8) carry.add(lv, hs8_and_stage<L, H>(lv, ring + sc * STAGE));
            else carry.add(lv, hs4_and_stage<L, H>(lv, ring + sc * STAGE));
            sc = sc + 1 == PH_D ? 0 : sc + 1;
        }
        carry.flush(lv);
        cp_async_wait<0>();
        emit_hits<L, LPQ>(a, blk, col, q, ell, lv, n != 0u);  // every lane of the warp
    }
}

// Every instantiation for H opts in to its ring size (once; engines call this
// when they are created, before any stream capture).
template <int H>
static void pipe_h_prepare() {
    static PerDeviceOnce once;
    once([] {
        constexpr int smem = (int)pipe_h_smem<H>();
        cudaFuncSetAttribute(k_gather_pipe_h<8, 8, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_gather_pipe_h<8, 12, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_gather_pipe_h<8, 16, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_gather_pipe_h<8, 24, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
}

template <int H>
static void launch_pipe_h(const GatherArgs &a, uint32_t L, uint32_t grid, cudaStream_t s) {
    constexpr size_t smem = pipe_h_smem<H>();
    pipe_h_prepare<H>();
    switch (L) {
        case 8: k_gather_pipe_h<8, 8, H><<<grid, PH_THREADS, smem, s>>>(a); break;
        case 12: k_gather_pipe_h<8, 12, H><<<grid, PH_THREADS, smem, s>>>(a); break;
        case 16: k_gather_pipe_h<8, 16, H><<<grid, PH_THREADS, smem, s>>>(a); break;
        default: k_gather_pipe_h<8, 24, H><<<grid, PH_THREADS, smem, s>>>(a); break;
    }
}

void launch_gather_pipe_h(const GatherArgs &a, uint32_t L, uint32_t grid, cudaStream_t s) {
    if (a.h == 2) launch_pipe_h<2>(a, L, grid, s);
    else if (a.h == 3) launch_pipe_h<3>(a, L, grid, s);
    else launch_pipe_h<4>(a, L, grid, s);
}

int gather_pipe_h_blocks_per_sm(uint32_t h) {
    int nb = 0;
    // the ring size must be allowed before the occupancy query sees it
    if (h == 2) {
        pipe_h_prepare<2>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_pipe_h<8, 12, 2>, PH_THREADS, pipe_h_smem<2>());
    } else if (h == 3) {
        pipe_h_prepare<3>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_pipe_h<8, 12, 3>, PH_THREADS, pipe_h_smem<3>());
    } else {
        pipe_h_prepare<4>();
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_pipe_h<8, 12, 4>, PH_THREADS, pipe_h_smem<4>());
    }
    return nb;
}

}  // namespace cobs
