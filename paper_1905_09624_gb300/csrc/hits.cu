// K3 tail: turn the raw hits (query, key) appended by the gather kernels into
// per-query lists sorted by score descending, then original id ascending
// (Sec. 2.3 "Parallelization": scores of disjoint partitions, then the top scores
// are selected).  Key = (~score << 32) | id, so ascending keys give that order.
#include "kernels.cuh"

namespace cobs {

constexpr uint32_t SCAN_THREADS = 1024;
constexpr uint32_t SORT_THREADS = 128;
constexpr uint32_t SORT_SMEM_KEYS = 1024;

// Exclusive scan of the per-query hit counts (one CTA), threshold per query,
// reset of the scatter cursors.  The CTA walks the queries in tiles of
// SCAN_THREADS, one query per thread (coalesced), scans each tile by warp
// shuffles and the warps' sums, and carries the running total to the next tile.
__global__ void __launch_bounds__(SCAN_THREADS) k_hits_scan(HitsArgs a) {
    constexpr uint32_t NW = SCAN_THREADS / 32;
    __shared__ unsigned long long s_warp[NW];
    __shared__ unsigned long long s_carry;
    const uint32_t n = a.n_queries;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    for (uint32_t t0 = 0; t0 < n; t0 += SCAN_THREADS) {
        const uint32_t q = t0 + threadIdx.x;
        const uint32_t c = q < n ? a.qcount[q] : 0u;
        unsigned long long incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, d);
            if ((int)lane >= d) incl += y;
        }
        if (lane == 31u) s_warp[warp] = incl;
        __syncthreads();  // warp sums written; s_carry of the previous tile final
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
        const unsigned long long tile_total = s_warp[NW - 1];
        const unsigned long long before = s_carry + (warp ? s_warp[warp - 1] : 0ULL);
        if (q < n) {
            a.hit_off[q] = before + incl - c;
            if (c > SORT_SMEM_KEYS) a.big_list[atomicAdd(a.big_count, 1ULL)] = q;
            a.qcursor[q] = 0;
            a.min_score[q] = (uint32_t)(((uint64_t)a.thr[q] * a.ell[q] + 999u) / 1000u);
        }
        __syncthreads();  // every thread read s_carry and s_warp
        if (threadIdx.x == 0) s_carry += tile_total;
    }
    __syncthreads();
    if (threadIdx.x == 0) a.hit_off[n] = s_carry;
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

// One CTA per query with at most SORT_SMEM_KEYS hits: sort in shared memory.
__global__ void __launch_bounds__(SORT_THREADS) k_hits_segsort(HitsArgs a) {
    __shared__ unsigned long long sA[SORT_SMEM_KEYS];
    __shared__ unsigned long long sB[SORT_SMEM_KEYS];
    const uint32_t q = blockIdx.x;
    unsigned long long total = *a.hit_count;
    if (total > a.hit_cap) return;  // the host re-runs with a larger capacity
    const uint64_t o = a.hit_off[q];
    const uint32_t n = (uint32_t)(a.hit_off[q + 1] - o);
    if (n == 0 || n > SORT_SMEM_KEYS) return;  // larger segments: k_hits_segsort_big
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) sA[i] = a.keys[o + i];
    __syncthreads();
    unsigned long long *src = sA, *dst = sB;
    for (uint32_t w = 1; w < n; w <<= 1) {
        merge_pass(src, dst, n, w);
        __syncthreads();
        unsigned long long *t = src; src = dst; dst = t;
    }
    unpack(src, n, o, a.out_ids, a.out_scores);
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
    k_hits_segsort<<<a.n_queries, SORT_THREADS, 0, s>>>(a);
    const uint32_t grid = a.n_queries < 304 ? a.n_queries : 304;
    k_hits_segsort_big<<<grid, BIG_SORT_THREADS, 0, s>>>(a);
}

}  // namespace cobs
