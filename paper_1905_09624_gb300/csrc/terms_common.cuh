// Staging of a round of query windows in shared memory (DNA packed 2 bits a
// base with a mask of non-ACGT bytes; byte q-grams as they are), shared by the
// term kernels and the fused plain kernel.
#pragma once
#include "kernels.cuh"

namespace cobs {

constexpr uint32_t TERMS_ROUND = TERMS_THREADS * TERMS_SEG;  // windows per round
constexpr uint32_t TERMS_STAGE_BYTES = TERMS_ROUND + 32;      // + k - 1 <= 31 bytes of overlap
// packed words of a round: data words + 2 read past the last window, rounded up
// so the packing loop runs whole warps (4 bytes per lane, 8 words per warp)
constexpr uint32_t TERMS_PK_WORDS = (((TERMS_STAGE_BYTES + 15) / 16 + 2) * 4 + 31) / 32 * 8;
constexpr uint32_t BP = TERMS_BLOCKS_PER_PASS;

// Bytes of windows [r0, r0 + rn) of a query into shared memory: DNA as packed
// bases and a mask of non-ACGT bytes, bytes as they are.  Every thread of the
// CTA calls it; the caller synchronises before (buffers free) and after.
__device__ __forceinline__ void stage_round(const uint8_t *src, uint64_t r0, uint32_t rn, uint32_t k, bool dna,
                                            uint8_t *s_bytes, uint32_t *s_pk, uint16_t *s_inv) {
    const uint32_t nbytes = rn + k - 1;
    if (dna) {
        // 4 bytes per lane -> 8 bits of bases and 4 mask bits; lanes 4j..4j+3 form word j
        const uint32_t nquads = (((nbytes + 15) / 16 + 2) * 4 + 31) & ~31u;
        for (uint32_t t = threadIdx.x; t < nquads; t += blockDim.x) {
            uint32_t pk = 0, inv = 0;
#pragma unroll
            for (uint32_t j = 0; j < 4; j++) {
                const uint32_t i = 4 * t + j;
                const uint32_t c = i < nbytes ? src[r0 + i] : 0u;
                const bool ok = c == 'A' || c == 'C' || c == 'G' || c == 'T';
                uint32_t b = (c >> 1) & 3u;  // A, C, T, G -> 0, 1, 2, 3
                b ^= b >> 1;                 // -> A 0, C 1, G 2, T 3
                pk = (pk << 2) | (ok ? b : 0u);
                inv = (inv << 1) | (ok ? 0u : 1u);
            }
            const uint32_t sub = 3u - (t & 3u);  // first quad of a word is most significant
            pk <<= 8 * sub;
            inv <<= 4 * sub;
            pk |= __shfl_xor_sync(0xffffffffu, pk, 1);
            inv |= __shfl_xor_sync(0xffffffffu, inv, 1);
            pk |= __shfl_xor_sync(0xffffffffu, pk, 2);
            inv |= __shfl_xor_sync(0xffffffffu, inv, 2);
            if ((t & 3u) == 0u) {
                s_pk[t >> 2] = pk;
                s_inv[t >> 2] = (uint16_t)inv;
            }
        }
    } else {
        for (uint32_t i = threadIdx.x; i < nbytes; i += blockDim.x) s_bytes[i] = src[r0 + i];
    }
}

}  // namespace cobs
