// K1: query terms.  For every query (one CTA each): all windows of length q
// (Sec. 2.1), canonical form (Sec. 2.3), the distinct set G_q(P) via an
// open-addressing set, then for every distinct term and every block b and hash
// i < h its row XXH64(term, i) mod w_b (Sec. 2.2), written as a u32 row index.
#include "kernels.cuh"

namespace cobs {

__global__ void __launch_bounds__(TERMS_THREADS) k_query_terms(TermsArgs a) {
    extern __shared__ unsigned long long s_table[];
    __shared__ uint32_t s_ell;
    __shared__ uint32_t s_has_empty;

    const uint32_t q = a.q0 + blockIdx.x;
    const uint64_t off0 = a.offsets[q];
    const uint64_t len = a.offsets[q + 1] - off0;
    const uint32_t k = a.k;
    const uint64_t npos = len >= k ? len - k + 1 : 0;
    const uint32_t cap = (uint32_t)set_slots(npos);
    unsigned long long *table = cap <= TERMS_SMEM_SLOTS ? s_table : a.tables + a.table_base[q];

    for (uint32_t i = threadIdx.x; i < cap; i += blockDim.x) table[i] = EMPTY_KEY;
    if (threadIdx.x == 0) { s_ell = 0; s_has_empty = 0; }
    __syncthreads();

    const uint8_t *src = a.bytes + off0;
    const uint64_t mask = kmer_mask(k);
    const uint64_t base = a.term_base[q];
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t nseg = (npos + TERMS_SEG - 1) / TERMS_SEG;
    // Every thread runs the same number of outer iterations so that the warp-level
    // append below always sees the full warp.
    const uint64_t iters = (nseg + blockDim.x - 1) / blockDim.x;
    for (uint64_t it = 0; it < iters; it++) {
        uint64_t seg = it * blockDim.x + threadIdx.x;
        uint64_t p0 = seg * TERMS_SEG;
        uint64_t p1 = p0 + TERMS_SEG < npos ? p0 + TERMS_SEG : npos;
        Roller r;
        roll_init(r);
        uint64_t ib = p0, ie = p1 > p0 ? p1 + k - 1 : p0;  // bytes feeding windows [p0, p1)
        // One step per byte; the loop count is the same for all lanes of a full
        // segment, and lanes past the end simply push nothing.
        for (uint64_t step = 0; step < TERMS_SEG + 64; step++) {
            uint64_t i = ib + step;
            bool in = i < ie;
            uint64_t code = 0;
            bool term = false;
            if (in) term = roll_push(r, src[i], a.kind, k, mask, &code);
            bool fresh = false;
            uint64_t h0 = 0;
            if (term) {
                h0 = xxh64_u64(code, 0);
                if (code == EMPTY_KEY) fresh = atomicExch(&s_has_empty, 1u) == 0u;
                else fresh = set_insert(table, cap, h0, code);
            }
            // warp-aggregated append of the fresh terms
            uint32_t m = __ballot_sync(0xffffffffu, fresh);
            uint32_t slot0 = 0;
            if (m) {
                if (lane == (uint32_t)(__ffs(m) - 1)) slot0 = atomicAdd(&s_ell, (uint32_t)__popc(m));
                slot0 = __shfl_sync(0xffffffffu, slot0, __ffs(m) - 1);
            }
            if (fresh) {
                uint32_t t = slot0 + __popc(m & ((1u << lane) - 1u));
                for (uint32_t i2 = 0; i2 < a.h; i2++) {
                    uint64_t hv = i2 == 0 ? h0 : xxh64_u64(code, i2);
                    for (uint32_t b = 0; b < a.n_blocks; b++) {
                        DevBlock blk = a.blocks[b];
                        uint32_t row = barrett_mod(hv, blk.barrett_m, blk.w);
                        a.rows_idx[(uint64_t)(b * a.h + i2) * a.tcap + base + t] = row;
                    }
                }
            }
            if (__all_sync(0xffffffffu, !(i + 1 < ie))) break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) a.ell[q] = s_ell;
}

void launch_query_terms(const TermsArgs &a, uint32_t n_queries, cudaStream_t s) {
    if (n_queries == 0) return;
    k_query_terms<<<n_queries, TERMS_THREADS, TERMS_SMEM_SLOTS * sizeof(unsigned long long), s>>>(a);
}

}  // namespace cobs
