// Device helpers shared by the COBS kernels: term codes, XXH64 of one 8-byte
// term, Barrett reduction, device-side block table.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cobs {

// Term kinds (Sec. 2.1 q-grams, Sec. 2.3 canonical k-mers).
enum : uint32_t { KIND_DNA_CANONICAL = 0, KIND_DNA_FORWARD = 1, KIND_BYTES = 2 };

// Device copy of one block (Sec. 2.2 compact layout): rows of `rowbytes` bytes,
// w rows, documents [doc_begin, doc_begin + n_docs) in sorted order.
struct DevBlock {
    uint64_t row_offset;  // byte offset of row 0
    uint64_t barrett_m;   // floor(2^64 / w) (UINT64_MAX for w == 1)
    uint32_t w;
    uint32_t rowbytes;
    uint32_t n_docs;
    uint32_t doc_begin;
};

// ---------------------------------------------------------------- XXH64
// XXH64 of the 8 little-endian bytes of `v` with `seed`: the xxHash64 algorithm
// for an input shorter than 32 bytes holding exactly one 8-byte lane (xxHash
// specification: init with seed + PRIME5 + length, one lane round, avalanche).
__device__ __forceinline__ uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

__device__ __forceinline__ uint64_t xxh64_u64(uint64_t v, uint64_t seed) {
    const uint64_t PR1 = 0x9E3779B185EBCA87ULL;
    const uint64_t PR2 = 0xC2B2AE3D27D4EB4FULL;
    const uint64_t PR3 = 0x165667B19E3779F9ULL;
    const uint64_t PR4 = 0x85EBCA77C2B2AE63ULL;
    const uint64_t PR5 = 0x27D4EB2F165667C5ULL;
    uint64_t acc = seed + PR5 + 8ULL;
    uint64_t lane = rotl64(v * PR2, 31) * PR1;
    acc ^= lane;
    acc = rotl64(acc, 27) * PR1 + PR4;
    acc ^= acc >> 33;
    acc *= PR2;
    acc ^= acc >> 29;
    acc *= PR3;
    acc ^= acc >> 32;
    return acc;
}

// A 64-bit mixer for hash sets and partitions that only need well-spread bits
// (not the method's hash): the finalizer of MurmurHash3 (A. Appleby, public
// domain), xor-shift / multiply / xor-shift / multiply / xor-shift.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xFF51AFD7ED558CCDULL;
    x ^= x >> 33;
    x *= 0xC4CEB9FE1A85EC53ULL;
    x ^= x >> 33;
    return x;
}

// ------------------------------------------------------------- Barrett
// x mod w by Barrett reduction (P. Barrett, "Implementing the Rivest Shamir and
// Adleman public key encryption algorithm on a standard digital signal processor",
// CRYPTO 1986) with m = floor(2^64 / w): the quotient estimate
// floor(x * m / 2^64) is at most one below floor(x / w), so one conditional
// subtraction finishes.  Used for "one wide hash, then modulo each filter size"
// (Sec. 2.2).
__device__ __forceinline__ uint32_t barrett_mod(uint64_t x, uint64_t m, uint32_t w) {
    uint64_t q = __umul64hi(x, m);
    uint64_t r = x - q * (uint64_t)w;
    return (uint32_t)(r >= w ? r - w : r);
}

__device__ __forceinline__ uint64_t kmer_mask(uint32_t k) { return k >= 32 ? ~0ULL : ((1ULL << (2 * k)) - 1ULL); }

// ------------------------------------------------- packed base streams
// A staged run of DNA bytes packed 16 bases per word: pk holds the 2-bit codes,
// first base most significant; inv marks bytes that are not A, C, G or T (first
// base = most significant bit).  Arrays need ceil(nbytes / 16) + 2 words.
// Cooperative: all threads of the CTA call it; the caller synchronises after.
__device__ __forceinline__ void pack_bases(const uint8_t *s_bytes, uint32_t nbytes, uint32_t *s_pk,
                                           uint16_t *s_inv) {
    const uint32_t nwords = (nbytes + 15) >> 4;
    for (uint32_t t = threadIdx.x; t < nwords + 2; t += blockDim.x) {
        uint32_t pk = 0, inv = 0;
        if (t < nwords) {
#pragma unroll
            for (uint32_t j = 0; j < 16; j++) {
                const uint32_t i = t * 16 + j;
                const uint32_t c = i < nbytes ? s_bytes[i] : 0u;
                const bool ok = c == 'A' || c == 'C' || c == 'G' || c == 'T';
                uint32_t b = (c >> 1) & 3u;  // A, C, T, G -> 0, 1, 2, 3
                b ^= b >> 1;                 // -> A 0, C 1, G 2, T 3
                pk = (pk << 2) | (ok ? b : 0u);
                inv = (inv << 1) | (ok ? 0u : 1u);
            }
        }
        s_pk[t] = pk;
        s_inv[t] = (uint16_t)inv;
    }
}

// The k-mer starting at base p of a packed run (k <= 32): its k bases are the
// top 2k bits of words w, w+1, w+2 shifted by 2o, its validity a shift of the
// mask, its reverse complement a bit reversal of the complemented code with the
// two bits of each base swapped back.  Returns false for a window with a
// non-ACGT byte.
__device__ __forceinline__ bool packed_kmer(const uint32_t *s_pk, const uint16_t *s_inv, uint32_t p, uint32_t k,
                                            bool canonical, uint64_t mask, uint64_t *code) {
    const uint32_t w = p >> 4, o = p & 15u;
    const uint64_t A = ((uint64_t)s_pk[w] << 32) | s_pk[w + 1];
    const uint64_t hi = o ? (A << (2 * o)) | (s_pk[w + 2] >> (32 - 2 * o)) : A;
    const uint64_t fwd = hi >> (64 - 2 * k);
    const uint64_t X = ((uint64_t)s_inv[w] << 32) | ((uint64_t)s_inv[w + 1] << 16) | s_inv[w + 2];
    if (((X << (16 + o)) >> (64 - k)) != 0) return false;
    if (canonical) {
        uint64_t x = __brevll(~(fwd << (64 - 2 * k)));
        x = ((x >> 1) & 0x5555555555555555ULL) | ((x & 0x5555555555555555ULL) << 1);
        const uint64_t rc = x & mask;
        *code = rc < fwd ? rc : fwd;
    } else {
        *code = fwd;
    }
    return true;
}

// The byte q-gram starting at byte p (q <= 8 bytes, little-endian).
__device__ __forceinline__ uint64_t bytes_qgram(const uint8_t *s_bytes, uint32_t p, uint32_t q) {
    uint64_t v = 0;
    for (uint32_t j = 0; j < q; j++) v |= (uint64_t)s_bytes[p + j] << (8 * j);
    return v;
}

// Open-addressing set of 64-bit codes; EMPTY marks a free slot.  The value
// EMPTY itself (possible only for 8-byte q-grams of 0xFF bytes) is tracked by a
// separate flag by the caller.
constexpr uint64_t EMPTY_KEY = 0xFFFFFFFFFFFFFFFFULL;

// Insert `key` into the table of `cap` slots, first probe from hash `h` by
// multiply-shift range reduction (Lemire, "Fast random integer generation in an
// interval", 2019), then linear probing.  Returns true when this call inserted it
// (first occurrence).  Every probe sequence ends: callers size the table at least
// twice the number of insertions, so a free slot always exists.
__device__ __forceinline__ bool set_insert(unsigned long long *table, uint32_t cap, uint64_t h, uint64_t key) {
    uint32_t slot = (uint32_t)(((h >> 32) * (uint64_t)cap) >> 32);
    for (uint32_t probe = 0; probe < cap; probe++) {
        unsigned long long old = atomicCAS(&table[slot], (unsigned long long)EMPTY_KEY, (unsigned long long)key);
        if (old == EMPTY_KEY) return true;
        if (old == key) return false;
        slot = slot + 1u == cap ? 0u : slot + 1u;
    }
    return false;  // unreachable for a correctly sized table
}

// The slot that holds `key` after inserting it (now or by an earlier call), with
// the probe sequence of set_insert.
__device__ __forceinline__ uint32_t set_find_insert(unsigned long long *table, uint32_t cap, uint64_t h,
                                                    uint64_t key) {
    uint32_t slot = (uint32_t)(((h >> 32) * (uint64_t)cap) >> 32);
    for (uint32_t probe = 0; probe < cap; probe++) {
        const unsigned long long old =
            atomicCAS(&table[slot], (unsigned long long)EMPTY_KEY, (unsigned long long)key);
        if (old == EMPTY_KEY || old == key) return slot;
        slot = slot + 1u == cap ? 0u : slot + 1u;
    }
    return 0u;  // unreachable for a correctly sized table
}

// Slots of the distinct-term set for `npos` windows.
__host__ __device__ __forceinline__ uint64_t set_slots(uint64_t npos) { return npos * 2 < 16 ? 16 : npos * 2; }

}  // namespace cobs
