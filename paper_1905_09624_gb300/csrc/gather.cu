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
#include "kernels.cuh"

namespace cobs {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int GATHER_THREADS = 128;

__device__ __forceinline__ void csa(uint32_t &hi, uint32_t &lo, uint32_t a, uint32_t b, uint32_t c) {
    uint32_t u = a ^ b;
    hi = (a & b) | (u & c);
    lo = u ^ c;
}

// Add G indicator words (G = 16 or 8) into the vertical counter lv[0..L-1].
template <int L, int G>
__device__ __forceinline__ void hs_add(uint32_t (&lv)[L], const uint32_t (&x)[G]) {
    static_assert(G == 16 || G == 8, "group of 8 or 16");
    if constexpr (G == 16) {
        uint32_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
        csa(twosA, lv[0], lv[0], x[0], x[1]);
        csa(twosB, lv[0], lv[0], x[2], x[3]);
        csa(foursA, lv[1], lv[1], twosA, twosB);
        csa(twosA, lv[0], lv[0], x[4], x[5]);
        csa(twosB, lv[0], lv[0], x[6], x[7]);
        csa(foursB, lv[1], lv[1], twosA, twosB);
        csa(eightsA, lv[2], lv[2], foursA, foursB);
        csa(twosA, lv[0], lv[0], x[8], x[9]);
        csa(twosB, lv[0], lv[0], x[10], x[11]);
        csa(foursA, lv[1], lv[1], twosA, twosB);
        csa(twosA, lv[0], lv[0], x[12], x[13]);
        csa(twosB, lv[0], lv[0], x[14], x[15]);
        csa(foursB, lv[1], lv[1], twosA, twosB);
        csa(eightsB, lv[2], lv[2], foursA, foursB);
        csa(sixteens, lv[3], lv[3], eightsA, eightsB);
        uint32_t c = sixteens;
#pragma unroll
        for (int l = 4; l < L; l++) {
            uint32_t t = lv[l] & c;
            lv[l] ^= c;
            c = t;
        }
    } else {
        uint32_t twosA, twosB, foursA, foursB, eights;
        csa(twosA, lv[0], lv[0], x[0], x[1]);
        csa(twosB, lv[0], lv[0], x[2], x[3]);
        csa(foursA, lv[1], lv[1], twosA, twosB);
        csa(twosA, lv[0], lv[0], x[4], x[5]);
        csa(twosB, lv[0], lv[0], x[6], x[7]);
        csa(foursB, lv[1], lv[1], twosA, twosB);
        csa(eights, lv[2], lv[2], foursA, foursB);
        uint32_t c = eights;
#pragma unroll
        for (int l = 3; l < L; l++) {
            uint32_t t = lv[l] & c;
            lv[l] ^= c;
            c = t;
        }
    }
}

// Bit mask of the documents whose vertical count is >= mn (mn < 2^L).
template <int L>
__device__ __forceinline__ uint32_t ge_mask(const uint32_t (&lv)[L], uint32_t mn) {
    uint32_t gt = 0u, eq = FULL;
#pragma unroll
    for (int l = L - 1; l >= 0; l--) {
        uint32_t mb = ((mn >> l) & 1u) ? FULL : 0u;
        gt |= eq & lv[l] & ~mb;
        eq &= ~(lv[l] ^ mb);
    }
    return gt | eq;
}

template <int L>
__device__ __forceinline__ uint32_t count_of(const uint32_t (&lv)[L], uint32_t bit) {
    uint32_t s = 0;
#pragma unroll
    for (int l = 0; l < L; l++) s |= ((lv[l] >> bit) & 1u) << l;
    return s;
}

__device__ __forceinline__ uint4 ld_row(const uint8_t *p) {
    return __ldcg(reinterpret_cast<const uint4 *>(p));
}

// Accumulate the terms [t0, t1) of one query for one 16-byte column.
// ridx: row indices of hash 0 for this (query, block); hash i at + i * tcap.
template <int L, int G>
__device__ __forceinline__ void accumulate(uint32_t (&lv)[4][L], const uint8_t *colbase, uint32_t rowbytes,
                                           const uint32_t *ridx, uint64_t tcap, uint32_t h, uint32_t t0,
                                           uint32_t t1) {
    for (uint32_t t = t0; t < t1; t += G) {
        uint32_t x[4][G];
        uint32_t row[G];
#pragma unroll
        for (int j = 0; j < G; j += 4) {
            uint4 r = __ldg(reinterpret_cast<const uint4 *>(ridx + t + j));
            row[j] = r.x; row[j + 1] = r.y; row[j + 2] = r.z; row[j + 3] = r.w;
        }
#pragma unroll
        for (int j = 0; j < G; j++) {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (t + j < t1) v = ld_row(colbase + (uint64_t)row[j] * rowbytes);
            x[0][j] = v.x; x[1][j] = v.y; x[2][j] = v.z; x[3][j] = v.w;
        }
        for (uint32_t i = 1; i < h; i++) {
            const uint32_t *ri = ridx + (uint64_t)i * tcap;
#pragma unroll
            for (int j = 0; j < G; j += 4) {
                uint4 r = __ldg(reinterpret_cast<const uint4 *>(ri + t + j));
                row[j] = r.x; row[j + 1] = r.y; row[j + 2] = r.z; row[j + 3] = r.w;
            }
#pragma unroll
            for (int j = 0; j < G; j++) {
                if (t + j < t1) {
                    uint4 v = ld_row(colbase + (uint64_t)row[j] * rowbytes);
                    x[0][j] &= v.x; x[1][j] &= v.y; x[2][j] &= v.z; x[3][j] &= v.w;
                }
            }
        }
#pragma unroll
        for (int w = 0; w < 4; w++) hs_add<L, G>(lv[w], x[w]);
    }
}

// Threshold (Sec. 2.1: score >= ceil(K l)) and hit emission of one lane's 128
// documents after all terms of its query were added.
template <int L>
__device__ __forceinline__ void emit_hits(const GatherArgs &a, const DevBlock &blk, uint32_t col, uint32_t q,
                                          uint32_t ell, const uint32_t (&lv)[4][L]) {
    const uint32_t mn = (uint32_t)(((uint64_t)a.thr[q] * ell + 999u) / 1000u);
    const uint32_t doc0 = col * 8u;
    uint32_t ge[4];
    uint32_t nh = 0;
#pragma unroll
    for (int w = 0; w < 4; w++) {
        uint32_t m = ge_mask<L>(lv[w], mn);
        uint32_t jw = doc0 + 32u * w;
        if (jw >= blk.n_docs) m = 0u;
        else if (blk.n_docs - jw < 32u) m &= (1u << (blk.n_docs - jw)) - 1u;
        ge[w] = m;
        nh += __popc(m);
    }
    if (nh == 0u) return;
    unsigned long long pos = atomicAdd(a.hit_count, (unsigned long long)nh);
    atomicAdd(&a.qcount[q], nh);
#pragma unroll
    for (int w = 0; w < 4; w++) {
        uint32_t m = ge[w];
        while (m) {
            uint32_t bit = __ffs(m) - 1u;
            m &= m - 1u;
            uint32_t score = count_of<L>(lv[w], bit);
            uint32_t id = a.perm[blk.doc_begin + doc0 + 32u * w + bit];
            if (pos < a.hit_cap) {
                a.raw_q[pos] = q;
                a.raw_key[pos] = ((unsigned long long)(~score) << 32) | id;
            }
            pos++;
        }
    }
}

// A split item's counts for the lane's 128 documents (each below 2^16).
template <int L>
__device__ __forceinline__ void write_partials(const GatherArgs &a, const DevBlock &blk, uint32_t col,
                                               uint32_t slot, const uint32_t (&lv)[4][L]) {
    uint16_t *dst = a.partials + (uint64_t)slot * a.n_docs + blk.doc_begin;
    const uint32_t doc0 = col * 8u;
#pragma unroll
    for (int w = 0; w < 4; w++) {
        for (uint32_t bit = 0; bit < 32u; bit++) {
            const uint32_t j = doc0 + 32u * w + bit;
            if (j < blk.n_docs) dst[j] = (uint16_t)count_of<L>(lv[w], bit);
        }
    }
}

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
    if (n == 0u) return;
    emit_hits<L>(a, blk, col, q, ell, lv);
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

// L2 eviction-priority policy: 0 normal, 1 evict first, 2 evict last.
__device__ __forceinline__ uint64_t l2_policy(uint32_t kind) {
    uint64_t p;
    if (kind == 1) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    else if (kind == 2) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    else asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, uint32_t src_bytes, uint64_t pol) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ uint4 ldg_hint(const void *p, uint64_t pol) {
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct W4 {
    uint32_t v[4];
};
__device__ __forceinline__ W4 w4(const uint4 &u) {
    W4 r;
    r.v[0] = u.x; r.v[1] = u.y; r.v[2] = u.z; r.v[3] = u.w;
    return r;
}
// full adder of two words into level LV of all four counters; returns the carry
template <int LV, int L>
__device__ __forceinline__ W4 csa_lv(uint32_t (&lv)[4][L], const W4 &a, const W4 &b) {
    W4 hi;
#pragma unroll
    for (int w = 0; w < 4; w++) csa(hi.v[w], lv[w][LV], lv[w][LV], a.v[w], b.v[w]);
    return hi;
}
template <int FROM, int L>
__device__ __forceinline__ void ripple(uint32_t (&lv)[4][L], W4 c) {
#pragma unroll
    for (int w = 0; w < 4; w++)
#pragma unroll
        for (int l = FROM; l < L; l++) {
            uint32_t t = lv[w][l] & c.v[w];
            lv[w][l] ^= c.v[w];
            c.v[w] = t;
        }
}
// Harley-Seal trees over the rows of one stage (stride 32 uint4 = one per lane):
// 16 rows return the carry of weight 16, 8 rows the carry of weight 8.
template <int L>
__device__ __forceinline__ W4 hs16_stage(uint32_t (&lv)[4][L], const uint4 *st) {
    W4 tA = csa_lv<0>(lv, w4(st[0 * 32]), w4(st[1 * 32]));
    W4 tB = csa_lv<0>(lv, w4(st[2 * 32]), w4(st[3 * 32]));
    W4 fA = csa_lv<1>(lv, tA, tB);
    tA = csa_lv<0>(lv, w4(st[4 * 32]), w4(st[5 * 32]));
    tB = csa_lv<0>(lv, w4(st[6 * 32]), w4(st[7 * 32]));
    W4 fB = csa_lv<1>(lv, tA, tB);
    W4 eA = csa_lv<2>(lv, fA, fB);
    tA = csa_lv<0>(lv, w4(st[8 * 32]), w4(st[9 * 32]));
    tB = csa_lv<0>(lv, w4(st[10 * 32]), w4(st[11 * 32]));
    fA = csa_lv<1>(lv, tA, tB);
    tA = csa_lv<0>(lv, w4(st[12 * 32]), w4(st[13 * 32]));
    tB = csa_lv<0>(lv, w4(st[14 * 32]), w4(st[15 * 32]));
    fB = csa_lv<1>(lv, tA, tB);
    W4 eB = csa_lv<2>(lv, fA, fB);
    return csa_lv<3>(lv, eA, eB);
}
template <int L>
__device__ __forceinline__ W4 hs8_stage(uint32_t (&lv)[4][L], const uint4 *st) {
    W4 tA = csa_lv<0>(lv, w4(st[0 * 32]), w4(st[1 * 32]));
    W4 tB = csa_lv<0>(lv, w4(st[2 * 32]), w4(st[3 * 32]));
    W4 fA = csa_lv<1>(lv, tA, tB);
    tA = csa_lv<0>(lv, w4(st[4 * 32]), w4(st[5 * 32]));
    tB = csa_lv<0>(lv, w4(st[6 * 32]), w4(st[7 * 32]));
    W4 fB = csa_lv<1>(lv, tA, tB);
    return csa_lv<2>(lv, fA, fB);
}

// Carries of weight 2^LV0 from consecutive stages, paired by two more levels of
// full adders: only every fourth stage ripples into the upper counter levels.
// Value held = counters + 2^LV0 * p0 (if h0) + 2^(LV0+1) * p1 (if h1).
template <int LV0, int L>
struct CarryPairs {
    W4 p0, p1;
    bool h0 = false, h1 = false;
    __device__ __forceinline__ void add(uint32_t (&lv)[4][L], const W4 &c) {
        if (!h0) { p0 = c; h0 = true; return; }
        h0 = false;
        const W4 c1 = csa_lv<LV0>(lv, p0, c);
        if (!h1) { p1 = c1; h1 = true; return; }
        h1 = false;
        ripple<LV0 + 2, L>(lv, csa_lv<LV0 + 1>(lv, p1, c1));
    }
    __device__ __forceinline__ void flush(uint32_t (&lv)[4][L]) {
        if (h0) ripple<LV0, L>(lv, p0);
        if (h1) ripple<LV0 + 1, L>(lv, p1);
        h0 = h1 = false;
    }
};

__device__ __forceinline__ void load_idx(const uint32_t *ridx, uint32_t g, uint32_t ng, uint32_t (&r)[PIPE_G],
                                         uint64_t pol) {
    if (g < ng) {
#pragma unroll
        for (int j = 0; j < PIPE_G; j += 4) {
            uint4 v = ldg_hint(ridx + g * (uint32_t)PIPE_G + j, pol);
            r[j] = v.x; r[j + 1] = v.y; r[j + 2] = v.z; r[j + 3] = v.w;
        }
    }
}

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
        if (it.w == ITEM_WHOLE) {
            if (n) emit_hits<L>(a, blk, col, q, ell, lv);
        } else if (active) {
            write_partials<L>(a, blk, col, it.w, lv);  // every part writes, zeros included
        }
    }
}

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
        if (n) emit_hits<L>(a, blk, col, q, ell, lv);
    }
}

// Every instantiation for H opts in to its ring size (once; engines call this
// when they are created, before any stream capture).
template <int H>
static void pipe_h_prepare() {
    static bool done = false;
    if (done) return;
    constexpr int smem = (int)pipe_h_smem<H>();
    cudaFuncSetAttribute(k_gather_pipe_h<8, 8, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_gather_pipe_h<8, 12, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_gather_pipe_h<8, 16, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_gather_pipe_h<8, 24, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    done = true;
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
    if (a.h == 1) {
        // cp.async pipeline
        switch (lanes_per_query) {
            case 2: launch_pipe_L<2>(a, L, grid, s); break;
            case 4: launch_pipe_L<4>(a, L, grid, s); break;
            default: launch_pipe_L<8>(a, L, grid, s); break;
        }
        return;
    }
    if (lanes_per_query == 8 && a.h >= 2 && a.h <= 4) {  // pipelined, 128-byte slices
        if (a.h == 2) launch_pipe_h<2>(a, L, grid, s);
        else if (a.h == 3) launch_pipe_h<3>(a, L, grid, s);
        else launch_pipe_h<4>(a, L, grid, s);
        return;
    }
    switch (lanes_per_query) {
        case 2: launch_L<2, 8>(a, L, grid, s); break;
        case 4: launch_L<4, 8>(a, L, grid, s); break;
        default: launch_L<8, 8>(a, L, grid, s); break;
    }
}

// Resident CTAs per SM of the batched kernel used for h hashes (persistent grid
// = SMs x this).
int gather_batched_max_blocks_per_sm(uint32_t lanes_per_query, uint32_t h) {
    int nb = 0;
    if (h == 1) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_pipe<8, 12>, PIPE_THREADS, 0);
    } else if (lanes_per_query == 8 && h <= 4) {
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
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_batched<8, 8, 12>, GATHER_THREADS, 0);
    }
    return nb;
}

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
