// K3 tail: turn the raw hits (query, key) appended by the gather kernels into
// per-query lists sorted by score descending, then original id ascending
// (Sec. 2.3 "Parallelization": scores of disjoint partitions, then the top scores
// are selected).  Key = (~score << 32) | id, so ascending keys give that order.
#include <algorithm>

#include "kernels.cuh"

namespace cobs {

constexpr uint32_t SCAN_THREADS = 1024;
constexpr uint32_t SCAN_PER = 8;  // rows of SCAN_THREADS queries whose inputs are loaded together
constexpr uint32_t SORT_THREADS = 128;
constexpr uint32_t SORT_SMEM_KEYS = 1024;

// Exclusive scan of the per-query hit counts (one CTA), threshold per query,
// reset of the scatter cursors, and the lists of queries to sort: those with
// more than SORT_SMEM_KEYS hits from the front of big_list, those with 1 to
// SORT_SMEM_KEYS from its back.  The CTA walks the queries in rows of
// SCAN_THREADS, one query per thread (coalesced); the inputs of SCAN_PER rows
// are loaded together first.  Each row is one scan (warp shuffles, then the
// warps' sums) of a 64-bit value that packs the query's hit count above two
// 11-bit flags (large list, small list), so the scan gives the hit offset and
// both list positions at once; running totals carry to the next row.
__global__ void __launch_bounds__(SCAN_THREADS) k_hits_scan(HitsArgs a) {
    constexpr uint32_t NW = SCAN_THREADS / 32;
    constexpr uint32_t FB = 11;  // bits of a row's count of listed queries (at most SCAN_THREADS)
    static_assert(SCAN_THREADS < (1u << FB), "list counts of a row fit their fields");
    constexpr unsigned long long FMASK = (1ULL << FB) - 1ULL;
    __shared__ unsigned long long s_warp[NW];
    __shared__ unsigned long long s_carry, s_big, s_mid;
    const uint32_t n = a.n_queries;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) { s_carry = 0; s_big = 0; s_mid = 0; }
    for (uint32_t t0 = 0; t0 < n; t0 += SCAN_THREADS * SCAN_PER) {
        uint32_t c[SCAN_PER], ms[SCAN_PER];
#pragma unroll
        for (uint32_t i = 0; i < SCAN_PER; i++) {
            const uint32_t q = t0 + i * SCAN_THREADS + threadIdx.x;
            c[i] = q < n ? a.qcount[q] : 0u;
            ms[i] = q < n ? (uint32_t)(((uint64_t)a.thr[q] * a.ell[q] + 999u) / 1000u) : 0u;
        }
#pragma unroll
        for (uint32_t i = 0; i < SCAN_PER; i++) {
            const uint32_t q = t0 + i * SCAN_THREADS + threadIdx.x;
            if (t0 + i * SCAN_THREADS >= n) break;  // the same for every thread
            const bool big = c[i] > SORT_SMEM_KEYS;
            const bool mid = c[i] > 0u && !big;
            const unsigned long long v =
                ((unsigned long long)c[i] << (2 * FB)) | ((unsigned long long)big << FB) | (unsigned long long)mid;
            unsigned long long incl = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, d);
                if ((int)lane >= d) incl += y;
            }
            if (lane == 31u) s_warp[warp] = incl;
            __syncthreads();  // warp sums written; the carries of the previous row final
            if (warp == 0) {
                unsigned long long w = lane < NW ? s_warp[lane] : 0ULL;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xffffffffu, w, d);
                    if ((int)lane >= d) w += y;
                }
                if (lane < NW) s_warp[lane] = w;  // inclusive sums of the warps
            }
            __syncthreads();
            const unsigned long long row_total = s_warp[NW - 1];
            const unsigned long long excl = (warp ? s_warp[warp - 1] : 0ULL) + incl - v;
            if (big) a.big_list[s_big + ((excl >> FB) & FMASK)] = q;
            if (mid) a.big_list[n - 1u - (uint32_t)(s_mid + (excl & FMASK))] = q;
            if (q < n) {
                a.hit_off[q] = s_carry + (excl >> (2 * FB));
                a.qcursor[q] = 0;
                a.min_score[q] = ms[i];
            }
            __syncthreads();  // every thread read the carries and s_warp
            if (threadIdx.x == 0) {
                s_carry += row_total >> (2 * FB);
                s_big += (row_total >> FB) & FMASK;
                s_mid += row_total & FMASK;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.hit_off[n] = s_carry;
        *a.big_count = s_big;
        *a.mid_count = s_mid;
    }
}

// Raw hits of one query arrive in runs (a warp tile emits its query's hits
// together): the lanes of a warp holding the same query reserve their slots
// with one atomic (one atomic per hit serialises on the query's cursor when a
// query has thousands of hits).  Every lane of a warp runs the same iterations.
__global__ void k_hits_scatter(HitsArgs a) {
    const unsigned long long total = *a.hit_count;
    // On overflow the offsets exceed the key buffer: leave it; the host re-runs
    // the batch with a larger capacity.
    if (total > a.hit_cap) return;
    const uint32_t lane = threadIdx.x & 31u;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long w0 = ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
         w0 < total; w0 += warps * 32) {
        const unsigned long long r = w0 + lane;
        const bool act = r < total;
        const uint32_t q = act ? a.raw_q[r] : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xffffffffu, q);
        const uint32_t leader = __ffs(peers) - 1;
        uint32_t first = 0;
        if (act && lane == leader) first = atomicAdd(&a.qcursor[q], (uint32_t)__popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (act) a.keys[a.hit_off[q] + first + __popc(peers & ((1u << lane) - 1u))] = a.raw_key[r];
    }
}

// One merge pass of a bottom-up merge sort of n unique keys: runs of `width`
// are merged pairwise; every key finds its output place by counting the keys
// below it in the partner run (binary search), so all keys move in parallel.
__device__ __forceinline__ void merge_pass(const unsigned long long *A, unsigned long long *B, uint32_t n,
                                           uint32_t width) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t run = i / width;
        const uint32_t pair0 = (run & ~1u) * width;
        const unsigned long long key = A[i];
        uint32_t lo, hi, base, dest;
        if ((run & 1u) == 0u) {
            base = pair0 + width;
            if (base >= n) { B[i] = key; continue; }
            lo = base;
            hi = pair0 + 2 * width < n ? pair0 + 2 * width : n;
            while (lo < hi) {
                uint32_t mid = (lo + hi) >> 1;
                if (A[mid] < key) lo = mid + 1; else hi = mid;
            }
            dest = i + (lo - base);
        } else {
            base = pair0;
            lo = pair0;
            hi = pair0 + width;
            while (lo < hi) {
                uint32_t mid = (lo + hi) >> 1;
                if (A[mid] < key) lo = mid + 1; else hi = mid;
            }
            dest = pair0 + (i - (pair0 + width)) + (lo - base);
        }
        B[dest] = key;
    }
}

__device__ __forceinline__ void unpack(const unsigned long long *src, uint32_t n, uint64_t o, uint32_t *ids,
                                       uint32_t *scores) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        unsigned long long key = src[i];
        ids[o + i] = (uint32_t)key;
        scores[o + i] = ~(uint32_t)(key >> 32);
    }
}

// Ascending sort of one key per lane across a warp (bitonic network, 15
// compare-exchange steps by shuffles); lanes without a key hold ~0.
__device__ __forceinline__ unsigned long long warp_sort32(unsigned long long key) {
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (uint32_t k2 = 2; k2 <= 32; k2 <<= 1) {
#pragma unroll
        for (uint32_t j = k2 >> 1; j > 0; j >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, j);
            const bool up = (lane & k2) == 0u;     // this lane's run ascends
            const bool lower = (lane & j) == 0u;   // this lane is the lower of the pair
            const unsigned long long lo = key < other ? key : other, hi = key < other ? other : key;
            key = lower == up ? lo : hi;
        }
    }
    return key;
}

constexpr uint32_t SORT_WARPS = SORT_THREADS / 32;
constexpr uint32_t NO_QUERY = 0xFFFFFFFFu;

// Queries with 1 to SORT_SMEM_KEYS hits (listed from the back of big_list by
// k_hits_scan), a fixed grid looping over them, one listed query per warp and
// round: up to 32 hits the warp sorts them in registers; larger lists are
// sorted in shared memory by the whole CTA after the round's warp sorts.
__global__ void __launch_bounds__(SORT_THREADS) k_hits_segsort(HitsArgs a) {
    __shared__ unsigned long long sA[SORT_SMEM_KEYS];
    __shared__ unsigned long long sB[SORT_SMEM_KEYS];
    __shared__ uint32_t s_defer[SORT_WARPS];
    unsigned long long total = *a.hit_count;
    if (total > a.hit_cap) return;  // the host re-runs with a larger capacity
    const unsigned long long nmid = *a.mid_count;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (unsigned long long base = (unsigned long long)blockIdx.x * SORT_WARPS; base < nmid;
         base += (unsigned long long)gridDim.x * SORT_WARPS) {
        const unsigned long long k = base + warp;
        uint32_t defer = NO_QUERY;
        if (k < nmid) {
            const uint32_t q = a.big_list[a.n_queries - 1u - (uint32_t)k];
            const uint64_t o = a.hit_off[q];
            const uint32_t n = (uint32_t)(a.hit_off[q + 1] - o);
            if (n <= 32u) {
                const unsigned long long key = warp_sort32(lane < n ? a.keys[o + lane] : ~0ULL);
                if (lane < n) {
                    a.out_ids[o + lane] = (uint32_t)key;
                    a.out_scores[o + lane] = ~(uint32_t)(key >> 32);
                }
            } else {
                defer = q;
            }
        }
        if (lane == 0) s_defer[warp] = defer;
        __syncthreads();
        for (uint32_t w = 0; w < SORT_WARPS; w++) {
            const uint32_t q = s_defer[w];
            if (q == NO_QUERY) continue;  // the same for every thread
            const uint64_t o = a.hit_off[q];
            const uint32_t n = (uint32_t)(a.hit_off[q + 1] - o);
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) sA[i] = a.keys[o + i];
            __syncthreads();
            unsigned long long *src = sA, *dst = sB;
            for (uint32_t wd = 1; wd < n; wd <<= 1) {
                merge_pass(src, dst, n, wd);
                __syncthreads();
                unsigned long long *t = src; src = dst; dst = t;
            }
            unpack(src, n, o, a.out_ids, a.out_scores);
            __syncthreads();  // sA and sB free for the next list
        }
        __syncthreads();  // every warp read s_defer before the next round writes it
    }
}

// Merge-path split of the output diagonal d of merging sorted A[0..na) and
// B[0..nb) (unique keys): the number of A elements among the first d outputs.
__device__ __forceinline__ uint32_t merge_split(const unsigned long long *A, uint32_t na,
                                                const unsigned long long *B, uint32_t nb, uint32_t d) {
    uint32_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] < B[d - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

constexpr uint32_t BIG_SORT_THREADS = 1024;
constexpr uint32_t BIG_SORT_CHUNK = 2048;

// One CTA per query with more than SORT_SMEM_KEYS hits: sort chunks of
// BIG_SORT_CHUNK keys in shared memory, then merge pairs of runs in global
// memory; every thread merges a contiguous range of the output, found by a
// merge-path binary search on its diagonal.
__device__ void sort_big_segment(const HitsArgs &a, uint32_t q, unsigned long long *sA, unsigned long long *sB) {
    const uint64_t o = a.hit_off[q];
    const uint32_t n = (uint32_t)(a.hit_off[q + 1] - o);
    unsigned long long *src = a.keys + o, *dst = a.tmp + o;
    for (uint32_t c0 = 0; c0 < n; c0 += BIG_SORT_CHUNK) {
        const uint32_t m = n - c0 < BIG_SORT_CHUNK ? n - c0 : BIG_SORT_CHUNK;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) sA[i] = src[c0 + i];
        __syncthreads();
        unsigned long long *x = sA, *y = sB;
        for (uint32_t w = 1; w < m; w <<= 1) {
            merge_pass(x, y, m, w);
            __syncthreads();
            unsigned long long *t = x; x = y; y = t;
        }
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) src[c0 + i] = x[i];
    }
    __syncthreads();
    for (uint32_t w = BIG_SORT_CHUNK; w < n; w <<= 1) {
        for (uint32_t p0 = 0; p0 < n; p0 += 2 * w) {
            const uint32_t na = n - p0 < w ? n - p0 : w;
            const uint32_t nb = n - p0 - na < w ? n - p0 - na : w;
            const unsigned long long *A = src + p0, *B = src + p0 + na;
            const uint32_t len = na + nb;
            const uint32_t per = (len + blockDim.x - 1) / blockDim.x;
            const uint32_t d0 = threadIdx.x * per < len ? threadIdx.x * per : len;
            const uint32_t d1 = d0 + per < len ? d0 + per : len;
            if (d0 < d1) {
                uint32_t i = merge_split(A, na, B, nb, d0);
                uint32_t j = d0 - i;
                for (uint32_t d = d0; d < d1; d++) {
                    const bool take_a = j >= nb || (i < na && A[i] < B[j]);
                    dst[p0 + d] = take_a ? A[i++] : B[j++];
                }
            }
        }
        __syncthreads();
        unsigned long long *t = src; src = dst; dst = t;
    }
    unpack(src, n, o, a.out_ids, a.out_scores);
    __syncthreads();
}

// Fixed grid over the list of queries with more than SORT_SMEM_KEYS hits (made
// by k_hits_scan).
__global__ void __launch_bounds__(BIG_SORT_THREADS) k_hits_segsort_big(HitsArgs a) {
    __shared__ unsigned long long sA[BIG_SORT_CHUNK];
    __shared__ unsigned long long sB[BIG_SORT_CHUNK];
    if (*a.hit_count > a.hit_cap) return;
    const unsigned long long nbig = *a.big_count;
    for (unsigned long long i = blockIdx.x; i < nbig; i += gridDim.x) sort_big_segment(a, a.big_list[i], sA, sB);
}

void launch_hits_finalize(const HitsArgs &a, cudaStream_t s) {
    if (a.n_queries == 0) return;
    k_hits_scan<<<1, SCAN_THREADS, 0, s>>>(a);
    k_hits_scatter<<<264, 256, 0, s>>>(a);
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t sort_grid = (uint32_t)std::min<uint64_t>(a.n_queries, (uint64_t)n_sm * 8);
    k_hits_segsort<<<sort_grid, SORT_THREADS, 0, s>>>(a);
    const uint32_t grid = a.n_queries < 304 ? a.n_queries : 304;
    k_hits_segsort_big<<<grid, BIG_SORT_THREADS, 0, s>>>(a);
}

}  // namespace cobs
