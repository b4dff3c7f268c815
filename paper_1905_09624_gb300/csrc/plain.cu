// The plain form (one query per launch after its terms kernel) and the
// threshold of split queries (sum of their parts' counts).
#include <algorithm>

#include "gather_common.cuh"
#include "terms_common.cuh"

namespace cobs {

// ------------------------------------------------------------------ plain
// One query per launch: the AND/ADD of Sec. 2.2 over every distinct term and
// every 128-byte column group of every block, spread over tiles (column group
// g, chunk c of the query's distinct terms).  A CTA runs PLAIN_STREAMS streams
// of 8 lanes; stream s takes the 16-term groups s, s + PLAIN_STREAMS, ... of
// its chunk, each lane one 16-byte column (128 documents): 16 row indices, 16
// rows (AND over the h hashes) loaded into registers, added into bit-sliced
// counters by the carry-save tree.  The streams' counters are summed by
// shuffles and shared memory.  With one chunk the CTA thresholds in place; with
// several each CTA stores its sums, and the last CTA of the column group to take
// the group's ticket (the threadfence reduction pattern: no CTA waits for
// another) adds the chunks, resets the ticket for the next query, thresholds
// (score >= ceil(K l), Sec. 2.1) and emits the hits with one reservation per
// warp.
//
// Two forms.  k_plain_fused (queries of at most one term round): every CTA
// finds the query's distinct terms itself in shared memory -- a set with the
// first window of each term, a scan of the first occurrences for their ranks --
// and hashes the terms of its chunk for its own block; no other kernel runs for
// the query.  Consecutive fused launches are programmatic dependents: a query's
// term phase and gather overlap the previous query's kernel, and only the
// epilogue (tickets, partial sums, hit counters) waits for it.  k_plain_query
// (longer queries): the terms kernel writes the distinct terms' rows, this
// kernel gathers them.

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// a += b for vertical counters (the sum stays below 2^L)
template <int L>
__device__ __forceinline__ void vadd(uint32_t (&a)[4][L], const uint32_t (&b)[4][L]) {
#pragma unroll
    for (int w = 0; w < 4; w++) {
        uint32_t c = 0u;
#pragma unroll
        for (int l = 0; l < L; l++) {
            const uint32_t x = a[w][l], y = b[w][l], u = x ^ y;
            a[w][l] = u ^ c;
            c = (x & y) | (u & c);
        }
    }
}

template <int L>
__device__ __forceinline__ void vadd_lane_xor(uint32_t (&a)[4][L], int d) {
    uint32_t b[4][L];
#pragma unroll
    for (int w = 0; w < 4; w++)
#pragma unroll
        for (int l = 0; l < L; l++) b[w][l] = __shfl_xor_sync(FULL, a[w][l], d);
    vadd<L>(a, b);
}

// Sum of the CTA's streams, left in lanes 0..7 of warp 0 (lane = column of the
// group).  Every thread calls it.
template <int L>
__device__ __forceinline__ void plain_cta_sum(uint32_t (&lv)[4][L], uint32_t *s_red) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    vadd_lane_xor<L>(lv, 8);
    vadd_lane_xor<L>(lv, 16);
    if (warp > 0u && lane < 8u) {
#pragma unroll
        for (int l = 0; l < L; l++)
#pragma unroll
            for (int w = 0; w < 4; w++) s_red[(((warp - 1u) * L + l) * 4u + w) * 8u + lane] = lv[w][l];
    }
    __syncthreads();
    if (warp == 0u && lane < 8u) {
        for (uint32_t wp = 0; wp + 1u < PLAIN_WARPS; wp++) {
            uint32_t b[4][L];
#pragma unroll
            for (int l = 0; l < L; l++)
#pragma unroll
                for (int w = 0; w < 4; w++) b[w][l] = s_red[((wp * L + l) * 4u + w) * 8u + lane];
            vadd<L>(lv, b);
        }
    }
}

// A stream's share of a chunk of n terms: 16-term groups stream, stream +
// PLAIN_STREAMS, ...; row indices of hash i at idx + i * idx_stride (16-byte
// aligned groups; entries past n are never used).
template <int L, bool GLOBAL_IDX>
__device__ __forceinline__ void plain_gather(uint32_t (&lv)[4][L], const uint32_t *idx, uint64_t idx_stride,
                                             uint32_t n, uint32_t h, uint32_t stream, const uint8_t *colbase,
                                             uint32_t rowbytes, bool active) {
#pragma unroll
    for (int w = 0; w < 4; w++)
#pragma unroll
        for (int l = 0; l < L; l++) lv[w][l] = 0u;
    for (uint32_t t0 = stream * 16u; t0 < n; t0 += 16u * PLAIN_STREAMS) {
        uint32_t x[4][16];
        uint32_t r[16];
        for (uint32_t i = 0; i < h; i++) {
            const uint32_t *ri = idx + (uint64_t)i * idx_stride + t0;
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
                const uint4 v = GLOBAL_IDX ? __ldg(reinterpret_cast<const uint4 *>(ri + j))
                                           : *reinterpret_cast<const uint4 *>(ri + j);
                r[j] = v.x; r[j + 1] = v.y; r[j + 2] = v.z; r[j + 3] = v.w;
            }
#pragma unroll
            for (int j = 0; j < 16; j++) {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (active && t0 + j < n) v = ld_row(colbase + (uint64_t)r[j] * rowbytes);
                if (i == 0) {
                    x[0][j] = v.x; x[1][j] = v.y; x[2][j] = v.z; x[3][j] = v.w;
                } else {
                    x[0][j] &= v.x; x[1][j] &= v.y; x[2][j] &= v.z; x[3][j] &= v.w;
                }
            }
        }
#pragma unroll
        for (int w = 0; w < 4; w++) hs_add<L, 16>(lv[w], x[w]);
    }
}

// Epilogue of a tile after its streams were summed (lv in lanes 0..7 of warp 0):
// chunk sums and the column group's ticket, then threshold and hits by the
// group's last tile.  ell = l of the query; has_terms: the tile's chunk holds
// terms.  Every thread calls it.
template <int L>
__device__ __forceinline__ void plain_epilogue(const PlainArgs &a, uint32_t (&lv)[4][L], uint32_t *s_red,
                                               uint32_t *s_last, uint32_t ell, bool has_terms, const DevBlock &blk,
                                               uint32_t col, bool active) {
    const uint32_t g = blockIdx.x, c = blockIdx.y;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (a.n_chunks > 1u) {
        const uint32_t stride = (uint32_t)L * 32u;
        if (warp == 0u && lane < 8u && has_terms) {
            uint32_t *part = a.partials + ((uint64_t)g * a.n_chunks + c) * stride;
#pragma unroll
            for (int l = 0; l < L; l++)
#pragma unroll
                for (int w = 0; w < 4; w++) part[(l * 4 + w) * 8 + lane] = lv[w][l];
        }
        __threadfence();
        __syncthreads();  // every store and the reads of s_red are done
        if (threadIdx.x == 0) *s_last = atomicAdd(&a.tickets[g], 1u) == a.n_chunks - 1u ? 1u : 0u;
        __syncthreads();
        if (!*s_last) return;
        __threadfence();
        // the last tile: the chunks that hold terms, spread over the streams
        const uint32_t used = (ell + a.chunk_terms - 1u) / a.chunk_terms;
        const uint32_t stream = warp * 4u + (lane >> 3);
#pragma unroll
        for (int w = 0; w < 4; w++)
#pragma unroll
            for (int l = 0; l < L; l++) lv[w][l] = 0u;
        for (uint32_t cc = stream; cc < used; cc += PLAIN_STREAMS) {
            const uint32_t *pp = a.partials + ((uint64_t)g * a.n_chunks + cc) * stride + (lane & 7u);
            uint32_t b[4][L];
#pragma unroll
            for (int l = 0; l < L; l++)
#pragma unroll
                for (int w = 0; w < 4; w++) b[w][l] = __ldcg(pp + (l * 4 + w) * 8);
            vadd<L>(lv, b);
        }
        plain_cta_sum<L>(lv, s_red);
        if (threadIdx.x == 0) a.tickets[g] = 0u;  // ready for the next query
    }
    if (warp == 0u) {
        uint32_t ge[4] = {0u, 0u, 0u, 0u};
        uint32_t nh = 0;
        const uint32_t doc0 = col * 8u;
        if (lane < 8u && active) {
            const uint32_t mn = (uint32_t)(((uint64_t)a.thr[a.q] * ell + 999u) / 1000u);
            nh = threshold_masks<L>(lv, mn, doc0, blk.n_docs, ge);
        }
        const unsigned long long pos = reserve_hits<32>(a.hit_count, a.qcount, a.q, nh);
        if (nh) write_hits<L>(lv, ge, a.q, a.perm + blk.doc_begin + doc0, pos, a.raw_q, a.raw_key, a.hit_cap);
    }
}

template <int L>
__global__ void __launch_bounds__(PLAIN_THREADS) k_plain_query(PlainArgs a) {
    __shared__ uint32_t s_red[(PLAIN_WARPS - 1) * L * 4 * 8];
    __shared__ uint32_t s_last;
    const uint32_t g = blockIdx.x, c = blockIdx.y;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t stream = warp * 4u + (lane >> 3);
    const SliceDesc sd = a.groups[g];
    const DevBlock blk = a.blocks[sd.block];
    const uint32_t col = sd.byte_off + (lane & 7u) * 16u;
    const bool active = col < blk.rowbytes;
    griddep_wait();  // the terms kernel's l and row indices are complete from here on
    const uint32_t ell = a.ell[a.q];
    if (ell == 0u) return;  // the same for every CTA of the grid
    const uint32_t t_lo = c * a.chunk_terms;
    const uint32_t n = t_lo >= ell ? 0u : (ell - t_lo < a.chunk_terms ? ell - t_lo : a.chunk_terms);
    // t_lo is a multiple of 16: the chunk's groups lie in the query's term
    // region, which spans a multiple of 16 slots
    const uint32_t *idx = a.rows_idx + (uint64_t)sd.block * a.h * a.tcap + a.term_base[a.q] + t_lo;
    uint32_t lv[4][L];
    plain_gather<L, true>(lv, idx, a.tcap, n, a.h, stream, a.rows + blk.row_offset + col, blk.rowbytes, active);
    plain_cta_sum<L>(lv, s_red);
    plain_epilogue<L>(a, lv, s_red, &s_last, ell, n > 0u, blk, col, active);
}

// Shared memory of the fused kernel for a query of npos windows and a chunk of
// chunk_terms terms: the set (cap codes), each slot's first window (cap), each
// window's slot (npos, 16 bits), the chunk's row indices (h x chunk_terms).
__host__ __device__ __forceinline__ uint32_t fused_rows_offset(uint32_t npos) {
    const uint32_t cap = (uint32_t)set_slots(npos);
    return (cap * 12u + npos * 2u + 15u) & ~15u;
}
__host__ __device__ __forceinline__ uint32_t fused_smem_bytes(uint32_t npos, uint32_t h, uint32_t chunk_terms) {
    return fused_rows_offset(npos) + h * chunk_terms * 4u;
}
constexpr uint16_t WSLOT_NONE = 0xFFFFu;   // window with a byte outside the alphabet
constexpr uint16_t WSLOT_EMPTY = 0xFFFEu;  // the one code the set cannot hold

template <int L>
__global__ void __launch_bounds__(PLAIN_THREADS) k_plain_fused(PlainArgs a) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ __align__(16) uint8_t s_bytes[TERMS_STAGE_BYTES];
    __shared__ uint32_t s_pk[TERMS_PK_WORDS];
    __shared__ uint16_t s_inv[TERMS_PK_WORDS];
    __shared__ uint32_t s_red[(PLAIN_WARPS - 1) * L * 4 * 8];
    __shared__ uint32_t s_wsum[PLAIN_WARPS];
    __shared__ uint32_t s_empty_first, s_last;
    // the next query's launch may start its term phase now; it reaches the
    // tickets, partial sums and hit lists only after this grid has completed
    griddep_launch_dependents();
    const uint32_t g = blockIdx.x, c = blockIdx.y;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t stream = warp * 4u + (lane >> 3);
    const SliceDesc sd = a.groups[g];
    const DevBlock blk = a.blocks[sd.block];
    const uint32_t col = sd.byte_off + (lane & 7u) * 16u;
    const bool active = col < blk.rowbytes;
    const uint64_t off0 = a.offsets[a.q];
    const uint64_t len = a.offsets[a.q + 1] - off0;
    const uint32_t k = a.k;
    const uint32_t npos = len >= k ? (uint32_t)(len - k + 1) : 0u;  // at most TERMS_ROUND (host)
    const uint32_t cap = (uint32_t)set_slots(npos);
    unsigned long long *s_table = reinterpret_cast<unsigned long long *>(s_dyn);
    uint32_t *s_first = reinterpret_cast<uint32_t *>(s_table + cap);
    uint16_t *s_wslot = reinterpret_cast<uint16_t *>(s_first + cap);
    uint32_t *s_rows = reinterpret_cast<uint32_t *>(s_dyn + fused_rows_offset(npos));

    // 1. the query's windows into the set; each slot keeps its first window
    for (uint32_t i = tid; i < cap; i += PLAIN_THREADS) {
        s_table[i] = EMPTY_KEY;
        s_first[i] = 0xFFFFFFFFu;
    }
    if (tid == 0) s_empty_first = 0xFFFFFFFFu;
    const bool dna = a.kind != KIND_BYTES;
    if (npos) stage_round(a.bytes + off0, 0, npos, k, dna, s_bytes, s_pk, s_inv);
    __syncthreads();
    const uint64_t mask = kmer_mask(k);
    for (uint32_t p = tid; p < npos; p += PLAIN_THREADS) {
        uint64_t code = 0;
        bool term = true;
        if (dna) term = packed_kmer(s_pk, s_inv, p, k, a.kind == KIND_DNA_CANONICAL, mask, &code);
        else code = bytes_qgram(s_bytes, p, k);
        uint16_t ws = WSLOT_NONE;
        if (term) {
            if (code == EMPTY_KEY) {
                atomicMin(&s_empty_first, p);
                ws = WSLOT_EMPTY;
            } else {
                const uint32_t slot = set_find_insert(s_table, cap, mix64(code), code);
                atomicMin(&s_first[slot], p);
                ws = (uint16_t)slot;
            }
        }
        s_wslot[p] = ws;
    }
    __syncthreads();
    // 2. ranks of the distinct terms = order of their first windows; thread t
    //    owns windows [t * per, (t + 1) * per)
    auto first_of = [&](uint32_t p) -> bool {
        const uint16_t ws = s_wslot[p];
        if (ws == WSLOT_NONE) return false;
        return ws == WSLOT_EMPTY ? s_empty_first == p : s_first[ws] == p;
    };
    const uint32_t per = (npos + PLAIN_THREADS - 1) / PLAIN_THREADS;
    const uint32_t p0 = tid * per < npos ? tid * per : npos;
    const uint32_t p1 = p0 + per < npos ? p0 + per : npos;
    uint32_t cnt = 0;
    for (uint32_t p = p0; p < p1; p++) cnt += first_of(p) ? 1u : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, d);
        if ((int)lane >= d) incl += y;
    }
    if (lane == 31u) s_wsum[warp] = incl;
    __syncthreads();
    uint32_t rank = incl - cnt, ell = 0;
#pragma unroll
    for (uint32_t w = 0; w < PLAIN_WARPS; w++) {
        if (w < warp) rank += s_wsum[w];
        ell += s_wsum[w];
    }
    if (g == 0 && c == 0 && tid == 0) a.ell[a.q] = ell;
    if (ell == 0u) {  // the same for every CTA of the grid
        griddep_wait();  // so this grid completes after the previous one
        return;
    }
    // 3. rows of the chunk's terms in this CTA's block
    const uint32_t T = a.chunk_terms;
    const uint32_t r_lo = c * T;
    const uint32_t n = r_lo >= ell ? 0u : (ell - r_lo < T ? ell - r_lo : T);
    if (n) {
        for (uint32_t p = p0; p < p1; p++) {
            if (!first_of(p)) continue;
            if (rank >= r_lo && rank < r_lo + n) {
                const uint16_t ws = s_wslot[p];
                const uint64_t code = ws == WSLOT_EMPTY ? EMPTY_KEY : (uint64_t)s_table[ws];
                for (uint32_t i = 0; i < a.h; i++)
                    s_rows[i * T + (rank - r_lo)] = barrett_mod(xxh64_u64(code, i), blk.barrett_m, blk.w);
            }
            rank++;
        }
    }
    __syncthreads();
    // 4. gather, AND, ADD; then the epilogue once the previous query's grid is done
    uint32_t lv[4][L];
    plain_gather<L, false>(lv, s_rows, T, n, a.h, stream, a.rows + blk.row_offset + col, blk.rowbytes, active);
    plain_cta_sum<L>(lv, s_red);
    griddep_wait();
    plain_epilogue<L>(a, lv, s_red, &s_last, ell, n > 0u, blk, col, active);
}

// Launches with programmatic stream serialization: the kernel's CTAs may start
// while the previous kernel of the stream runs; griddepcontrol.wait orders
// everything they read from (or write to) that kernel's results.
template <class K>
static cudaError_t launch_pdl(K kernel, const PlainArgs &a, size_t smem, bool pdl, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.n_groups, a.n_chunks, 1);
    cfg.blockDim = dim3(PLAIN_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

cudaError_t launch_plain_query(const PlainArgs &a, uint32_t L, cudaStream_t s) {
    if (a.n_groups == 0 || a.n_chunks == 0) return cudaSuccess;
    switch (L) {
        case 8: return launch_pdl(k_plain_query<8>, a, 0, true, s);
        case 12: return launch_pdl(k_plain_query<12>, a, 0, true, s);
        case 16: return launch_pdl(k_plain_query<16>, a, 0, true, s);
        default: return launch_pdl(k_plain_query<24>, a, 0, true, s);
    }
}

bool plain_fused_fits(uint64_t npos, uint32_t h) { return npos <= TERMS_ROUND && h <= PLAIN_FUSED_MAX_H; }

cudaError_t launch_plain_fused(const PlainArgs &a, uint32_t npos, bool pdl, cudaStream_t s) {
    if (a.n_groups == 0 || a.n_chunks == 0) return cudaSuccess;
    if (!plain_fused_fits(npos, a.h)) return cudaErrorInvalidValue;
    static PerDeviceOnce once;
    once([] {
        const int most = (int)fused_smem_bytes(TERMS_ROUND, PLAIN_FUSED_MAX_H, TERMS_ROUND);
        cudaFuncSetAttribute(k_plain_fused<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        cudaFuncSetAttribute(k_plain_fused<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    });
    const size_t smem = fused_smem_bytes((uint32_t)npos, a.h, a.chunk_terms);
    // at most TERMS_ROUND windows: fewer than 2^12 terms
    return counter_levels_for((uint32_t)npos) <= 8 ? launch_pdl(k_plain_fused<8>, a, smem, pdl, s)
                                                   : launch_pdl(k_plain_fused<12>, a, smem, pdl, s);
}

uint32_t plain_chunks(uint64_t npos, uint32_t n_groups, uint32_t n_sm, uint32_t max_chunks, uint32_t *chunk_terms) {
    // about four CTAs per SM over the grid; a chunk holds at least one 16-term
    // group per stream
    const uint64_t target = 4ULL * (n_sm ? n_sm : 1);
    uint64_t c = (target + (n_groups ? n_groups : 1) - 1) / (n_groups ? n_groups : 1);
    c = std::min<uint64_t>(c, (npos + 16ULL * PLAIN_STREAMS - 1) / (16ULL * PLAIN_STREAMS));
    c = std::min<uint64_t>(std::max<uint64_t>(c, 1), std::max<uint32_t>(max_chunks, 1u));
    uint64_t ct = (npos + c - 1) / c;
    ct = std::max<uint64_t>((ct + 15) / 16 * 16, 16);
    c = std::max<uint64_t>((npos + ct - 1) / ct, 1);
    *chunk_terms = (uint32_t)ct;
    return (uint32_t)c;
}

uint64_t plain_partial_words(uint32_t n_groups, uint32_t n_chunks) {
    return n_chunks > 1 ? (uint64_t)n_groups * n_chunks * 24u * 32u : 0u;
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


}  // namespace cobs
