// Measurement and test entry points that the paper has no counterpart for:
// the L2 read-bandwidth probe (the ceiling of a gather whose rows are reused
// through L2) and a direct check of the device modulo (Barrett reduction) that
// every row index goes through.
#include "host_internal.h"

using namespace cobs;

namespace {

// Every thread reads 16-byte pieces of the buffer, PROBE_UNROLL at a time, L2
// only (ld.global.cg: no L1 allocation), folding them into one word so the loads
// stay live; the grid strides over the buffer `reps` times.
constexpr int PROBE_THREADS = 256;
#ifndef COBS_PROBE_UNROLL
#define COBS_PROBE_UNROLL 8
#endif
constexpr int PROBE_UNROLL = COBS_PROBE_UNROLL;  // loads in flight per thread

// a volatile L2 load: every pass really reads the buffer again
__device__ __forceinline__ uint4 ld_cg_volatile(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];\n" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_l2_read(const uint4 *buf, uint64_t n16, uint32_t reps,
                                                                 unsigned long long *sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (uint32_t r = 0; r < reps; r++) {
        uint64_t i = tid;
        for (; i + (PROBE_UNROLL - 1) * stride < n16; i += PROBE_UNROLL * stride) {
            uint4 v[PROBE_UNROLL];
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; u++) v[u] = ld_cg_volatile(buf + i + u * stride);
#pragma unroll
            for (int u = 0; u < PROBE_UNROLL; u++) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
        for (; i < n16; i += stride) {
            const uint4 v = ld_cg_volatile(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
        acc = acc * 0x9E3779B1u + r;  // a new dependence per pass
    }
    if (acc == 0x5A5A5A5Au) atomicAdd(sink, 1ULL);  // practically never taken; keeps the loads
}

__global__ void k_debug_barrett(const uint64_t *x, uint64_t n, uint64_t m, uint32_t w, uint32_t *out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = barrett_mod(x[i], m, w);
}

}  // namespace

extern "C" cobs_status cobs_probe_l2_read(const void *buf_dev, uint64_t bytes, uint32_t reps, uint32_t ctas_per_sm,
                                          void *sink_dev, void *stream) {
    if (!buf_dev || !sink_dev || bytes < 16 || reps == 0) return set_error(COBS_ERR_ARG, "probe: bad arguments");
    if (((uintptr_t)buf_dev & 15u) != 0) return set_error(COBS_ERR_ARG, "probe: buffer not 16-byte aligned");
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(COBS_ERR_CUDA, "probe: %s", cudaGetErrorString(e));
    const uint32_t grid = (uint32_t)n_sm * (ctas_per_sm ? ctas_per_sm : 8u);
    k_probe_l2_read<<<grid, PROBE_THREADS, 0, (cudaStream_t)stream>>>(
        static_cast<const uint4 *>(buf_dev), bytes / 16, reps, static_cast<unsigned long long *>(sink_dev));
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(COBS_ERR_CUDA, "probe launch: %s", cudaGetErrorString(e));
    return COBS_OK;
}

extern "C" cobs_status cobs_debug_barrett_mod(const uint64_t *x_dev, uint64_t n, uint64_t w, uint32_t *out_dev,
                                              void *stream) {
    if ((n && (!x_dev || !out_dev)) || w == 0 || w > 0xFFFFFFFFULL)
        return set_error(COBS_ERR_ARG, "barrett check: w must be 1..2^32 - 1");
    if (n == 0) return COBS_OK;
    const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 4096);
    k_debug_barrett<<<(uint32_t)blocks, 256, 0, (cudaStream_t)stream>>>(x_dev, n, barrett_m_of(w), (uint32_t)w,
                                                                        out_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(COBS_ERR_CUDA, "barrett check: %s", cudaGetErrorString(e));
    return COBS_OK;
}
