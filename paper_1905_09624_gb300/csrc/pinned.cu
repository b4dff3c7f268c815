// Pinned host memory, optionally bound to one NUMA node (Linux mbind on an
// anonymous mapping, then cudaHostRegister).  A streamed index's rows are read
// by the device's copy engine every batch, so they sit on the host node
// nearest the device (cudaDevAttrHostNumaId) where the system reports one.
#include <sys/mman.h>
#include <sys/syscall.h>
#include <unistd.h>

#include "host_internal.h"

namespace cobs {

void PinBuf::release() {
    if (p) {
        if (mapped) {
            cudaHostUnregister(p);
            munmap(p, mapped);
        } else {
            cudaFreeHost(p);
        }
    }
    p = nullptr;
    bytes = 0;
    mapped = 0;
    node = -1;
}

cudaError_t PinBuf::ensure_on_node(size_t n, int numa_node) {
    if (numa_node < 0) return ensure(n);
    if (n == 0) n = 16;
    if (n <= bytes) return cudaSuccess;
    release();
    if (alloc_injected_failure()) return cudaErrorMemoryAllocation;
    const size_t page = (size_t)sysconf(_SC_PAGESIZE);
    const size_t len = (n + page - 1) / page * page;
    void *m = mmap(nullptr, len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (m == MAP_FAILED) return cudaErrorMemoryAllocation;
    // MPOL_BIND (2) to the one node; the pages are placed there when first touched
    constexpr int MPOL_BIND_MODE = 2;
    unsigned long mask[16] = {0};
    const int maxnode = (int)(sizeof(mask) * 8);
    if (numa_node >= maxnode) {
        munmap(m, len);
        return ensure(n);
    }
    mask[numa_node / (8 * sizeof(unsigned long))] |= 1UL << (numa_node % (8 * sizeof(unsigned long)));
    if (syscall(SYS_mbind, m, len, MPOL_BIND_MODE, mask, (unsigned long)maxnode, 0UL) != 0) {
        munmap(m, len);
        return ensure(n);  // no NUMA policy on this system: the CUDA allocator's pages
    }
    const cudaError_t e = cudaHostRegister(m, len, cudaHostRegisterDefault);
    if (e != cudaSuccess) {
        munmap(m, len);
        return e;
    }
    p = m;
    bytes = n;
    mapped = len;
    node = numa_node;
    return cudaSuccess;
}

}  // namespace cobs
