// Device helpers shared by the gather kernels: bit-sliced counters and their
// carry-save adder trees, threshold and hit emission, partial counts, cp.async
// and L2 eviction-policy wrappers, row-index loads.
#pragma once
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

// Warp-collective reservation of hit slots: every lane of the warp calls it
// with its number of hits nh (0 if it emits none).  Lanes of one query are the
// SEG consecutive lanes of a segment.  One atomic on the global hit counter per
// warp, one on the query's count per segment with hits; returns the lane's
// first slot (an exclusive prefix sum over the warp).
template <int SEG>
__device__ __forceinline__ unsigned long long reserve_hits(unsigned long long *hit_count, uint32_t *qcount,
                                                           uint32_t q, uint32_t nh) {
    static_assert(SEG >= 1 && SEG <= 32 && (SEG & (SEG - 1)) == 0, "segments of a power of two lanes");
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t incl = nh;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, d);
        if ((int)lane >= d) incl += y;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    if (total == 0u) return 0ULL;
    unsigned long long base = 0;
    if (lane == 31u) base = atomicAdd(hit_count, (unsigned long long)total);
    base = __shfl_sync(FULL, base, 31);
    uint32_t seg = nh;
#pragma unroll
    for (int d = 1; d < SEG; d <<= 1) seg += __shfl_xor_sync(FULL, seg, d);
    if ((lane & (SEG - 1)) == 0u && seg) atomicAdd(&qcount[q], seg);
    return base + (incl - nh);
}

// Threshold masks (Sec. 2.1: score >= ceil(K l)) of one lane's 128 documents
// (four words of 32) from its vertical counters; documents past the block's end
// are cleared.  Returns the number of hits.
template <int L>
__device__ __forceinline__ uint32_t threshold_masks(const uint32_t (&lv)[4][L], uint32_t mn, uint32_t doc0,
                                                    uint32_t n_docs, uint32_t (&ge)[4]) {
    uint32_t nh = 0;
#pragma unroll
    for (int w = 0; w < 4; w++) {
        uint32_t m = ge_mask<L>(lv[w], mn);
        const uint32_t jw = doc0 + 32u * w;
        if (jw >= n_docs) m = 0u;
        else if (n_docs - jw < 32u) m &= (1u << (n_docs - jw)) - 1u;
        ge[w] = m;
        nh += __popc(m);
    }
    return nh;
}

// Write a lane's hits from slot pos on: (query, key = (~score << 32) | original id).
template <int L>
__device__ __forceinline__ void write_hits(const uint32_t (&lv)[4][L], const uint32_t (&ge)[4], uint32_t q,
                                           const uint32_t *perm_of_doc0, unsigned long long pos, uint32_t *raw_q,
                                           unsigned long long *raw_key, uint64_t hit_cap) {
#pragma unroll
    for (int w = 0; w < 4; w++) {
        uint32_t m = ge[w];
        while (m) {
            const uint32_t bit = __ffs(m) - 1u;
            m &= m - 1u;
            const uint32_t score = count_of<L>(lv[w], bit);
            const uint32_t id = perm_of_doc0[32u * w + bit];
            if (pos < hit_cap) {
                raw_q[pos] = q;
                raw_key[pos] = ((unsigned long long)(~score) << 32) | id;
            }
            pos++;
        }
    }
}

// Threshold and hit emission of one lane's 128 documents after all terms of its
// query were added (emit false: the lane has nothing to report).  Warp-collective:
// every lane of the warp calls it; the lanes of one query are SEG consecutive lanes.
template <int L, int SEG>
__device__ __forceinline__ void emit_hits(const GatherArgs &a, const DevBlock &blk, uint32_t col, uint32_t q,
                                          uint32_t ell, const uint32_t (&lv)[4][L], bool emit) {
    uint32_t ge[4] = {0u, 0u, 0u, 0u};
    uint32_t nh = 0;
    const uint32_t doc0 = col * 8u;
    if (emit) {
        const uint32_t mn = (uint32_t)(((uint64_t)a.thr[q] * ell + 999u) / 1000u);
        nh = threshold_masks<L>(lv, mn, doc0, blk.n_docs, ge);
    }
    const unsigned long long pos = reserve_hits<SEG>(a.hit_count, a.qcount, q, nh);
    if (nh) write_hits<L>(lv, ge, q, a.perm + blk.doc_begin + doc0, pos, a.raw_q, a.raw_key, a.hit_cap);
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
// Harley-Seal trees over the rows of one stage (rows S uint4 apart; 32 = one
// uint4 per lane): 16 rows return the carry of weight 16, 8 rows of weight 8.
template <int L, int S = 32>
__device__ __forceinline__ W4 hs16_stage(uint32_t (&lv)[4][L], const uint4 *st) {
    W4 tA = csa_lv<0>(lv, w4(st[0 * S]), w4(st[1 * S]));
    W4 tB = csa_lv<0>(lv, w4(st[2 * S]), w4(st[3 * S]));
    W4 fA = csa_lv<1>(lv, tA, tB);
    tA = csa_lv<0>(lv, w4(st[4 * S]), w4(st[5 * S]));
    tB = csa_lv<0>(lv, w4(st[6 * S]), w4(st[7 * S]));
    W4 fB = csa_lv<1>(lv, tA, tB);
    W4 eA = csa_lv<2>(lv, fA, fB);
    tA = csa_lv<0>(lv, w4(st[8 * S]), w4(st[9 * S]));
    tB = csa_lv<0>(lv, w4(st[10 * S]), w4(st[11 * S]));
    fA = csa_lv<1>(lv, tA, tB);
    tA = csa_lv<0>(lv, w4(st[12 * S]), w4(st[13 * S]));
    tB = csa_lv<0>(lv, w4(st[14 * S]), w4(st[15 * S]));
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

// Row indices of group g (G terms) of a term list, 16 bytes at a time.
template <int G>
__device__ __forceinline__ void load_idx(const uint32_t *ridx, uint32_t g, uint32_t ng, uint32_t (&r)[G],
                                         uint64_t pol) {
    if (g < ng) {
#pragma unroll
        for (int j = 0; j < G; j += 4) {
            uint4 v = ldg_hint(ridx + g * (uint32_t)G + j, pol);
            r[j] = v.x; r[j + 1] = v.y; r[j + 2] = v.z; r[j + 3] = v.w;
        }
    }
}

}  // namespace cobs
