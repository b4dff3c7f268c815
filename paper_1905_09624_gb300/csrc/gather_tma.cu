// K2, single hash, fed by the tensor memory accelerator (an alternative to the
// cp.async ring of the default kernel; selected per engine).
#include "gather_common.cuh"

namespace cobs {

// ------------------------------------------------------ pipe, TMA gather
// The single-hash kernel fed by the tensor memory accelerator: per stage and
// query, one lane issues four tile::gather4 copies, each bringing four indexed
// rows' 128-byte slices of the block (a 2-D tensor map of w rows x rowbytes
// bytes, box 1 x 128) into shared memory; the stage's mbarrier counts the
// bytes.  Rows of the ring are [query][row][16-byte piece], so lane c of a
// query reads piece c of every row (rows 8 uint4 apart).  The rows past a
// query's last term repeat its group's first row and are cleared before the
// carry-save tree reads them.  Every wait on an mbarrier is bounded; a wait
// that runs out sets the error flag, drains the stages and ends the CTA.
constexpr int TG_G = 16, TG_D = 2, TG_WARPS = 2, TG_THREADS = TG_WARPS * 32;
// A wait suspends the thread for up to TG_SUSPEND_NS per try (the hardware wakes
// it when the phase completes); TG_WAIT_TRIES tries bound it (about 1.6 s).
constexpr uint32_t TG_WAIT_TRIES = 1u << 14;
constexpr uint32_t TG_SUSPEND_NS = 100000;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(TG_SUSPEND_NS)
        : "memory");
    return ok != 0;
}
// Bounded wait of every lane of the warp; false (on all lanes) if any gave up.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity) {
    bool ok = false;
    for (uint32_t i = 0; i < TG_WAIT_TRIES && !ok; i++) ok = mbar_try_wait(bar, parity);
    return __all_sync(FULL, ok);
}
__device__ __forceinline__ void tma_gather4(void *dst, const void *tmap, int x, const int (&r)[4], uint64_t *bar,
                                            uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

template <int L>
__global__ void __launch_bounds__(TG_THREADS) k_gather_tma(GatherArgs a) {
    constexpr uint32_t QPW = 4, G = TG_G;
    __shared__ __align__(128) uint4 s_ring[TG_WARPS][TG_D][QPW][G][8];
    __shared__ __align__(8) uint64_t s_bar[TG_WARPS][TG_D];
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t qslot = lane >> 3;
    const uint32_t c = lane & 7u;
    if (lane == 0) {
        for (int st = 0; st < TG_D; st++) mbar_init(&s_bar[warp][st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    const unsigned long long n_tiles = (unsigned long long)a.n_slices * a.n_groups;
    const uint64_t pol_idx = l2_policy(a.l2_idx_policy);
    const uint64_t pol_row = l2_policy(a.l2_row_policy);
    uint32_t parity = 0;  // bit st: parity of stage st's next phase
    uint32_t si = 0;      // next stage of the ring (continues across tiles)
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
        const uint32_t nq = valid && tend > it.y ? tend - it.y : 0u;
        const uint32_t col = sd.byte_off + c * 16u;
        const bool active = valid && col < blk.rowbytes;
        const uint32_t ngq = (nq + G - 1) / G;
        const uint32_t ngmax = __reduce_max_sync(FULL, ngq);
        const uint32_t *ridx = a.rows_idx + (uint64_t)sd.block * a.tcap + a.term_base[q] + it.y;
        const void *tmap = (const uint8_t *)a.tmaps + (size_t)sd.block * 128;
        const int x = (int)sd.byte_off;

        uint32_t lv[4][L];
#pragma unroll
        for (int w = 0; w < 4; w++)
#pragma unroll
            for (int l = 0; l < L; l++) lv[w][l] = 0u;
        uint32_t ra[G];
        if (c == 0) load_idx(ridx, 0, ngq, ra, pol_idx);
        // queue group g of every query of the warp into stage st
        auto issue = [&](uint32_t st, uint32_t g) {
            __syncwarp();  // every lane has read the stage's previous contents
            const bool me = c == 0 && g < ngq;
            const uint32_t cnt = __popc(__ballot_sync(FULL, me));
            if (lane == 0) mbar_arrive_expect(&s_bar[warp][st], cnt * G * 128u);
            if (me) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const uint32_t t0 = g * G;
#pragma unroll
                for (int k4 = 0; k4 < (int)G; k4 += 4) {
                    int r[4];
#pragma unroll
                    for (int kk = 0; kk < 4; kk++) r[kk] = (int)(t0 + k4 + kk < nq ? ra[k4 + kk] : ra[0]);
                    tma_gather4(&s_ring[warp][st][qslot][k4][0], tmap, x, r, &s_bar[warp][st], pol_row);
                }
            }
        };
        bool failed = false;
        if (ngmax) {
            issue(si, 0);
            if (c == 0) load_idx(ridx, 1, ngq, ra, pol_idx);
        }
        CarryPairs<4, L> carry;
        for (uint32_t g = 0; g < ngmax; g++) {
            const uint32_t cur = si, nxt = si ^ 1u;
            if (g + 1 < ngmax) {
                issue(nxt, g + 1);
                if (c == 0) load_idx(ridx, g + 2, ngq, ra, pol_idx);
            }
            if (!mbar_wait_warp(&s_bar[warp][cur], (parity >> cur) & 1u)) {
                failed = true;
                break;
            }
            parity ^= 1u << cur;
            if (active && g < ngq) {
                uint4 *rows = &s_ring[warp][cur][qslot][0][c];
                const uint32_t t0 = g * G;
                if (t0 + G > nq)  // rows past the query's last term: cleared (this lane's piece)
                    for (uint32_t j = nq - t0; j < G; j++) rows[j * 8] = make_uint4(0u, 0u, 0u, 0u);
                carry.add(lv, hs16_stage<L, 8>(lv, rows));
            }
            si = nxt;
        }
        if (failed) {
            if (lane == 0) atomicExch(a.err, 1u);
            // both stages may still have copies in flight: wait for them (bounded), then stop
            for (int st = 0; st < TG_D; st++) (void)mbar_wait_warp(&s_bar[warp][st], (parity >> st) & 1u);
            return;
        }
        carry.flush(lv);
        const uint32_t n = active ? nq : 0u;
        emit_hits<L, 8>(a, blk, col, q, ell, lv, it.w == ITEM_WHOLE && n != 0u);  // every lane of the warp
        if (it.w != ITEM_WHOLE && active) write_partials<L>(a, blk, col, it.w, lv);  // every part writes, zeros included
    }
}

void launch_gather_tma(const GatherArgs &a, uint32_t L, uint32_t grid, cudaStream_t s) {
    switch (L) {
        case 8: k_gather_tma<8><<<grid, TG_THREADS, 0, s>>>(a); break;
        case 12: k_gather_tma<12><<<grid, TG_THREADS, 0, s>>>(a); break;
        case 16: k_gather_tma<16><<<grid, TG_THREADS, 0, s>>>(a); break;
        default: k_gather_tma<24><<<grid, TG_THREADS, 0, s>>>(a); break;
    }
}

}  // namespace cobs
