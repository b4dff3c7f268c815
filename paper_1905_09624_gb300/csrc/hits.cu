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
// reset of the scatter cursors.
__global__ void __launch_bounds__(SCAN_THREADS) k_hits_scan(HitsArgs a) {
    __shared__ unsigned long long s_part[SCAN_THREADS];
    const uint32_t n = a.n_queries;
    const uint32_t per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
    const uint32_t q0 = threadIdx.x * per;
    const uint32_t q1 = q0 + per < n ? q0 + per : n;
    unsigned long long sum = 0;
    for (uint32_t q = q0; q < q1; q++) sum += a.qcount[q];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    for (uint32_t d = 1; d < SCAN_THREADS; d <<= 1) {
        unsigned long long v = threadIdx.x >= d ? s_part[threadIdx.x - d] : 0ULL;
        __syncthreads();
        s_part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = s_part[threadIdx.x] - sum;
    for (uint32_t q = q0; q < q1; q++) {
        a.hit_off[q] = run;
        run += a.qcount[q];
        a.qcursor[q] = 0;
        uint32_t ell = a.ell[q];
        a.min_score[q] = (uint32_t)(((uint64_t)a.thr[q] * ell + 999u) / 1000u);
    }
    if (threadIdx.x == SCAN_THREADS - 1) a.hit_off[n] = s_part[SCAN_THREADS - 1];
}

__global__ void k_hits_scatter(HitsArgs a) {
    const unsigned long long total = *a.hit_count;
    // On overflow the offsets exceed the key buffer: leave it; the host re-runs
    // the batch with a larger capacity.
    if (total > a.hit_cap) return;
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < total;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        uint32_t q = a.raw_q[r];
        unsigned long long pos = a.hit_off[q] + atomicAdd(&a.qcursor[q], 1u);
        a.keys[pos] = a.raw_key[r];
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

// One CTA per query: sort its segment in shared memory when it fits, otherwise in
// place in global memory (ping-pong with the scratch array).
__global__ void __launch_bounds__(SORT_THREADS) k_hits_segsort(HitsArgs a) {
    __shared__ unsigned long long sA[SORT_SMEM_KEYS];
    __shared__ unsigned long long sB[SORT_SMEM_KEYS];
    const uint32_t q = blockIdx.x;
    unsigned long long total = *a.hit_count;
    if (total > a.hit_cap) return;  // the host re-runs with a larger capacity
    const uint64_t o = a.hit_off[q];
    const uint32_t n = (uint32_t)(a.hit_off[q + 1] - o);
    if (n == 0) return;
    if (n <= SORT_SMEM_KEYS) {
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) sA[i] = a.keys[o + i];
        __syncthreads();
        unsigned long long *src = sA, *dst = sB;
        for (uint32_t w = 1; w < n; w <<= 1) {
            merge_pass(src, dst, n, w);
            __syncthreads();
            unsigned long long *t = src; src = dst; dst = t;
        }
        unpack(src, n, o, a.out_ids, a.out_scores);
        return;
    }
    unsigned long long *src = a.keys + o, *dst = a.tmp + o;
    for (uint32_t w = 1; w < n; w <<= 1) {
        merge_pass(src, dst, n, w);
        __syncthreads();
        unsigned long long *t = src; src = dst; dst = t;
    }
    unpack(src, n, o, a.out_ids, a.out_scores);
}

void launch_hits_finalize(const HitsArgs &a, cudaStream_t s) {
    if (a.n_queries == 0) return;
    k_hits_scan<<<1, SCAN_THREADS, 0, s>>>(a);
    k_hits_scatter<<<264, 256, 0, s>>>(a);
    k_hits_segsort<<<a.n_queries, SORT_THREADS, 0, s>>>(a);
}

}  // namespace cobs
